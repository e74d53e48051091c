"""Runs under the bounds-checked library (STK_LIBRARY=.../libstokes_gb300_check.so,
started by tests/test_gpu_bounds.py): the operator, both V-cycles, P1..P5 and
FP64 / mixed solves on small and odd-shaped grids, every boundary mix, with
the two-colour kernels and the single-block coarse kernel on every level,
and the same on stacked 2D batches, then prints the number of out-of-range
indices the kernels met (JSON)."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np
import torch

from paper_1308_4605_gb300 import stokes as S
from paper_1308_4605_gb300 import workloads as wl

P, W, F = 0, 1, 2
CASES = [
    (2, (4, 4), (P, P, P, P)), (2, (2, 8), (W, W, P, P)), (2, (16, 4), (W, F, F, W)),
    (2, (64, 32), (F, W, W, F)), (3, (2, 2, 2), (P,) * 6), (3, (4, 2, 8), (W,) * 6),
    (3, (8, 8, 4), (W, W, P, P, F, F)), (3, (16, 32, 8), (F, W, P, P, W, W)),
    (3, (32, 16, 64), (P, P, W, F, W, W)),
]

STACKED = [((4, 4), (P, P, P, P)), ((2, 8), (W, W, P, P)), ((16, 4), (W, F, F, W)),
           ((64, 32), (F, W, W, F))]


def main():
    dev = torch.device("cuda", 0)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    out = {"library": S.LIB_PATH, "cases": []}
    n0, _, _ = S.stk_bounds_violations(reset=True)
    S.stk_bounds_selftest()
    out["selftest"] = S.stk_bounds_violations(reset=True)
    for dim, n, bc in CASES:
        theta = 0.0 if all(b != P for b in bc[:2 * dim]) else 1.0
        pr = wl.generic(dim, n, bc, theta=theta, rho_contrast=10.0, mu_contrast=30.0, seed=3,
                        precond=2 if theta == 0.0 else 1)
        sv = S.StokesSolver(dim, pr.n[:dim], pr.bc[:2 * dim], pr.h)
        sv.set_coefficients(t(pr.rho), t(pr.mu), pr.theta)
        bu, bp = [t(x) for x in pr.b_u], t(pr.b_p)
        nlev = 1
        m = min(pr.n[:dim])
        while m > 2:
            m //= 2
            nlev += 1
        rec = {"dim": dim, "n": n, "bc": bc}
        for prec in (0, 1):
            # last: every level in the thread-block-cluster kernel
            for lc, pl, cl in ((nlev, nlev, None), (nlev, 0, None), (0, 0, None), (nlev, nlev, 0)):
                S.stk_set_schedule(sv.handle, prec, lc, 128, pl, None, cl)
                y_u, y_p = sv.apply_operator(bu, bp)
                for which in (1, 2, 3, 4, 5):
                    sv.apply_preconditioner(which, bu, bp, precision=prec)
                xu, xp, info = sv.solve(bu, bp, precond=pr.precond, precision=prec, maxit=400)
                rec[f"p{prec}_lc{lc}_pl{pl}_cl{cl}"] = [info["iterations"], info["true_residual"]]
        torch.cuda.synchronize()
        sv.close()
        out["cases"].append(rec)
    # stacked 2D batches (three instances of each grid along a third axis)
    for n, bc in STACKED:
        prs = [wl.generic(2, n, bc, theta=1.0, rho_contrast=10.0, mu_contrast=30.0 + 20 * i, seed=5 + i)
               for i in range(3)]
        pr = prs[0]
        sv = S.StokesSolver(2, pr.n[:2], pr.bc[:4], pr.h, count=3)
        stack = lambda arrs, shape: t(np.stack(arrs)).reshape(shape)
        sv.set_coefficients(stack([q.rho for q in prs], sv.cell_shape()),
                            stack([q.mu for q in prs], sv.cell_shape()), pr.theta)
        bu = [stack([q.b_u[a] for q in prs], sv.face_shape(a)) for a in range(2)]
        bp = stack([q.b_p for q in prs], sv.cell_shape())
        nlev = 1
        m = min(pr.n[:2])
        while m > 2:
            m //= 2
            nlev += 1
        rec = {"dim": 2, "n": n, "bc": bc, "stacked": 3}
        for prec in (0, 1):
            for lc, pl in ((nlev, nlev), (nlev, 0), (0, 0)):
                S.stk_set_schedule(sv.handle, prec, lc, 128, pl)
                sv.apply_operator(bu, bp)
                for which in (1, 2, 3, 4, 5):
                    sv.apply_preconditioner(which, bu, bp, precision=prec)
                xu, xp, info = sv.solve(bu, bp, precond=1, precision=prec, maxit=400)
                rec[f"p{prec}_lc{lc}_pl{pl}"] = [info["iterations"], info["true_residual"]]
        torch.cuda.synchronize()
        sv.close()
        out["cases"].append(rec)
    out["violations"] = S.stk_bounds_violations(reset=False)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
