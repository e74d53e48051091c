"""Full-size workloads in the benchmark's launch configuration (autotuned
schedules, FP64 and mixed forms) against independent oracle solutions.

The oracle solves the same seeded systems M x = b (Eq. Saddle_sys) with its
own GMRES(10) and V-cycle preconditioner to a true residual of 1e-13,
measured with the assembled sparse M (oracle/reference_solve.py), in a pool
of spawned worker processes that runs while the GPU solves.  Each GPU
solution must match it to 1e-8 relative L2 in velocity and in mean-free
pressure, and its residual b - M x, evaluated over every row by the
point-by-point oracle stencils (oracle/pointwise.py), must be below
1e-10 ||b||:
  * 3D 128^3 periodic unsteady (P1), FP64 and mixed;
  * every instance of the 64-instance batched workload (2D {64..512}^2
    periodic, P1, mixed), solved in one stk_solve_batched call, once with one
    handle per instance and once as the benchmark's stacked batches (one
    stacked handle per grid size, FP64 and mixed);
  * the steady no-slip adjoint workload's forward solve (P2) at 128^3, FP64
    and mixed (the oracle's sparse matrices at 256^3 outgrow the host; the
    256^3 solves are checked by the full residual alone).
"""
import multiprocessing as mp
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import direct, pointwise
from oracle import reference_solve as rs
from oracle.grid import Grid
from paper_1308_4605_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1308_4605_gb300 import stokes
    return stokes


@pytest.fixture(scope="module")
def oracle(S):
    """Oracle solutions, computed by spawned workers (no CUDA in them):
    {"c3": AsyncResult, "c5": AsyncResult, "c4": [AsyncResult per instance]}."""
    ctx = mp.get_context("spawn")
    workers = max(2, min((os.cpu_count() or 4) - 2, 12))
    pool = ctx.Pool(processes=workers)
    jobs = {"c3": pool.apply_async(rs.solve_workload, ("c3", 128)),
            "c5": pool.apply_async(rs.solve_workload, ("c5", 128))}
    sizes = wl.config_c4_sizes()
    order = sorted(range(len(sizes)), key=lambda i: -sizes[i])     # largest first
    c4 = {i: pool.apply_async(rs.solve_workload, ("c4", sizes[i], i)) for i in order}
    jobs["c4"] = [c4[i] for i in range(len(sizes))]
    pool.close()
    yield jobs
    pool.terminate()
    pool.join()


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(DEV)


def _pack(pr, x_u, x_p):
    g = Grid(pr.dim, pr.n, pr.h, pr.bc)
    return g, g.pack([a.cpu().numpy() for a in x_u], x_p.cpu().numpy())


def _full_residual(g, pr, x, chunk=1 << 22):
    """||b - M x|| / ||b|| over every unknown, M applied point by point."""
    b = g.pack(pr.b_u, pr.b_p)
    b[~g.active] = 0.0
    act = np.flatnonzero(g.active)
    ss = 0.0
    for s in range(0, len(act), chunk):
        sel = act[s:s + chunk]
        r = b[sel] - pointwise.rows(g, x, pr.rho, pr.mu, pr.theta, sel)
        ss += float(r @ r)
    return np.sqrt(ss) / np.linalg.norm(b)


def _compare(g, pr, x, ref):
    xr, info = ref
    assert info["true_residual"] <= 1e-12, info
    eu, ep = direct.relative_error(g, x, xr)
    assert eu <= 1e-8 and ep <= 1e-8, (eu, ep)
    res = _full_residual(g, pr, x)
    assert res <= 1.0001e-10, res
    return eu, ep, res


def _solve(S, pr, precision):
    from paper_1308_4605_gb300 import tuning
    sv = S.StokesSolver(pr.dim, pr.n[:pr.dim], pr.bc[:2 * pr.dim], pr.h)
    sv.set_coefficients(_t(pr.rho), _t(pr.mu), pr.theta)
    tuning.tune(sv, precision)
    x_u, x_p, info = sv.solve([_t(x) for x in pr.b_u], _t(pr.b_p), precond=pr.precond,
                              precision=precision, maxit=3000)
    sv.close()
    assert info["converged"] and info["true_residual"] <= 1e-10, info
    return x_u, x_p


@pytest.mark.parametrize("cfg", ["c3", "c5"])
def test_full_size_solves_match_oracle(S, oracle, cfg):
    pr = wl.config_c3(128) if cfg == "c3" else wl.config_c5(128)
    sols = [_solve(S, pr, precision) for precision in (0, 1)]
    ref = oracle[cfg].get(timeout=1800)
    for x_u, x_p in sols:
        g, x = _pack(pr, x_u, x_p)
        _compare(g, pr, x, ref)


def test_full_batched_workload_matches_oracle(S, oracle):
    """The 64-instance batched workload (2D {64..512}^2), solved in one
    stk_solve_batched call in the mixed form."""
    from paper_1308_4605_gb300 import tuning
    sizes = wl.config_c4_sizes()
    prs, svs, bus, bps, xus, xps = [], [], [], [], [], []
    for i, n in enumerate(sizes):
        pr = wl.config_c4_instance(i, n)
        sv = S.StokesSolver(2, pr.n[:2], pr.bc[:4], pr.h)
        sv.set_coefficients(_t(pr.rho), _t(pr.mu), pr.theta)
        tuning.tune(sv, 1)
        xu, xp = sv.zeros()
        prs.append(pr); svs.append(sv)
        bus.append([_t(x) for x in pr.b_u]); bps.append(_t(pr.b_p)); xus.append(xu); xps.append(xp)
    p = S.stk_default_params()
    p.precision = 1
    infos = S.stk_solve_batched([s.handle for s in svs], p, bus, bps, xus, xps)
    for sv in svs:
        sv.close()
    for i, (pr, info) in enumerate(zip(prs, infos)):
        assert info["converged"] and info["true_residual"] <= 1e-10, (i, info)
    for i, pr in enumerate(prs):
        g, x = _pack(pr, xus[i], xps[i])
        _compare(g, pr, x, oracle["c4"][i].get(timeout=1800))


@pytest.mark.parametrize("precision", [0, 1])
def test_full_batched_workload_stacked_matches_oracle(S, oracle, precision):
    """The same 64 instances as four stacked handles (16 x 64^2, 23 x 128^2,
    11 x 256^2, 14 x 512^2) solved in one stk_solve_batched call, the form
    the benchmark times."""
    from paper_1308_4605_gb300 import tuning
    sizes = wl.config_c4_sizes()
    prs = [wl.config_c4_instance(i, n) for i, n in enumerate(sizes)]
    groups = []
    for n in sorted(set(sizes)):
        idx = [i for i, s in enumerate(sizes) if s == n]
        p0 = prs[idx[0]]
        sv = S.StokesSolver(2, p0.n[:2], p0.bc[:4], p0.h, count=len(idx))
        stk = lambda arrs, shape: _t(np.stack(arrs)).reshape(shape)
        sv.set_coefficients(stk([prs[i].rho for i in idx], sv.cell_shape()),
                            stk([prs[i].mu for i in idx], sv.cell_shape()), p0.theta)
        tuning.tune(sv, precision)
        bu = [stk([prs[i].b_u[a] for i in idx], sv.face_shape(a)) for a in range(2)]
        bp = stk([prs[i].b_p for i in idx], sv.cell_shape())
        xu, xp = sv.zeros()
        groups.append((idx, sv, bu, bp, xu, xp))
    p = S.stk_default_params()
    p.precision = precision
    p.maxit = 3000
    S.stk_solve_batched([gr[1].handle for gr in groups], p, [gr[2] for gr in groups],
                        [gr[3] for gr in groups], [gr[4] for gr in groups], [gr[5] for gr in groups])
    recs = {}
    for idx, sv, _, _, _, _ in groups:
        for k, i in enumerate(idx):
            recs[i] = sv.instance_info(k)
        sv.close()
    for i in range(len(sizes)):
        assert recs[i]["converged"] and recs[i]["true_residual"] <= 1e-10, (i, recs[i])
    for idx, _, _, _, xu, xp in groups:
        for k, i in enumerate(idx):
            g, x = _pack(prs[i], [v[k] for v in xu], xp[k])
            _compare(g, prs[i], x, oracle["c4"][i].get(timeout=1800))


@pytest.mark.parametrize("precision", [0, 1])
def test_256_cubed_adjoint_workload_full_residual(S, precision):
    """The 256^3 steady no-slip workload (the adjoint throughput size): the
    residual over all 67M unknowns, evaluated by the oracle's point-by-point
    stencils, is below 1e-10 ||b||."""
    pr = wl.config_c5(256)
    x_u, x_p = _solve(S, pr, precision)
    g, x = _pack(pr, x_u, x_p)
    assert _full_residual(g, pr, x) <= 1.0001e-10
