"""Many independent 2D Stokes systems of mixed sizes, solved together.

`StackedBatch` groups the problems by grid (cells, boundary conditions,
spacing and theta), keeps one stacked handle per group (stk_create_stacked:
the group's instances along a third array axis, one launch of every kernel
for all of them) and solves every group in one stk_solve_batched call, each
group advancing at its own pace.  Each instance's solution is the one its
own handle would give (include/stokes.h).  Argument marshalling only: the
arrays are stacked and unstacked with torch on the device.
"""
from __future__ import annotations

from . import stokes as S


class StackedBatch:
    """problems: a sequence of dicts with keys n (nx, ny), bc (4 codes), h,
    theta, rho and mu (CUDA float64 tensors of shape (ny, nx) or (1, ny, nx)).
    Problems with the same n, bc, h and theta share one stacked handle."""

    def __init__(self, problems, tune=False):
        import torch
        self.count = len(problems)
        groups = {}
        for i, p in enumerate(problems):
            key = (tuple(int(v) for v in p["n"]), tuple(int(v) for v in p["bc"]), float(p["h"]),
                   float(p["theta"]))
            groups.setdefault(key, []).append(i)
        self.groups = []
        for (n, bc, h, theta), idx in groups.items():
            sv = S.StokesSolver(2, n, bc, h, count=len(idx))
            rho = torch.stack([problems[i]["rho"].reshape(sv.cell_shape()[1:]) for i in idx])
            mu = torch.stack([problems[i]["mu"].reshape(sv.cell_shape()[1:]) for i in idx])
            sv.set_coefficients(rho.contiguous(), mu.contiguous(), theta)
            if tune:
                from . import tuning
                tuning.tune(sv, S.STK_FP64)
                tuning.tune(sv, S.STK_MIXED)
            self.groups.append((idx, sv))

    def close(self):
        for _, sv in self.groups:
            sv.close()
        self.groups = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, b_us, b_ps, x_us=None, x_ps=None, **params):
        """b_us[i]: the two face arrays of problem i, b_ps[i] its cell array
        (x_us / x_ps: initial guesses, zero if None).  Keyword arguments set
        stk_solver_params fields (precond, precision, rtol, maxit, ...).
        Returns (x_us, x_ps, infos) in the order of the problems; infos[i]
        is problem i's record (stk_stack_info)."""
        import torch
        p = S.stk_default_params()
        for k, v in params.items():
            setattr(p, k, v)
        hs, bu, bp, xu, xp = [], [], [], [], []
        for idx, sv in self.groups:
            fs = [sv.face_shape(a) for a in range(2)]
            bu.append([torch.stack([b_us[i][a].reshape(fs[a][1:]) for i in idx]).contiguous() for a in range(2)])
            bp.append(torch.stack([b_ps[i].reshape(sv.cell_shape()[1:]) for i in idx]).contiguous())
            if x_us is None:
                gu, gp = sv.zeros(bp[-1].device)
            else:
                gu = [torch.stack([x_us[i][a].reshape(fs[a][1:]) for i in idx]).contiguous() for a in range(2)]
                gp = torch.stack([x_ps[i].reshape(sv.cell_shape()[1:]) for i in idx]).contiguous()
            xu.append(gu)
            xp.append(gp)
            hs.append(sv.handle)
        S.stk_solve_batched(hs, p, bu, bp, xu, xp)
        out_u, out_p, infos = [None] * self.count, [None] * self.count, [None] * self.count
        for g, (idx, sv) in enumerate(self.groups):
            for k, i in enumerate(idx):
                out_u[i] = [xu[g][a][k] for a in range(2)]
                out_p[i] = xp[g][k]
                infos[i] = sv.instance_info(k)
        return out_u, out_p, infos


def problem_dict(pr, device="cuda"):
    """A workloads.Problem (2D) as the dict StackedBatch takes."""
    import numpy as np
    import torch
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(device)
    return {"n": pr.n[:2], "bc": pr.bc[:4], "h": pr.h, "theta": pr.theta, "rho": t(pr.rho), "mu": t(pr.mu)}


__all__ = ["StackedBatch", "problem_dict"]
