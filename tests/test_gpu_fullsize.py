"""Full-size workloads in the benchmark's launch configuration (autotuned
schedules, FP64 and mixed forms): the solutions are checked on sampled rows
of M x - b that the oracle evaluates point by point (oracle/pointwise.py):
every sampled |b - M x| must lie below 1e-10 ||b||, which the 2-norm bound
||b - M x|| <= 1e-10 ||b|| implies for each row."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import pointwise
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


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(DEV)


def _check_rows(pr, x_u, x_p, nsample, seed):
    g = Grid(pr.dim, pr.n, pr.h, pr.bc)
    x = g.pack([a.cpu().numpy() for a in x_u], x_p.cpu().numpy())
    b = g.pack(pr.b_u, pr.b_p)
    b[~g.active] = 0.0
    act = np.flatnonzero(g.active)
    sel = np.random.default_rng(seed).choice(act, size=min(nsample, len(act)), replace=False)
    r = b[sel] - pointwise.rows(g, x, pr.rho, pr.mu, pr.theta, sel)
    bound = 1.0001e-10 * np.linalg.norm(b)
    assert np.abs(r).max() <= bound, (np.abs(r).max(), bound)
    return np.abs(r).max() / np.linalg.norm(b)


@pytest.mark.parametrize("cfg", ["c3_128", "c5_256"])
def test_full_size_solves_on_sampled_rows(S, cfg):
    from paper_1308_4605_gb300 import tuning
    pr = wl.config_c3(128) if cfg == "c3_128" else wl.config_c5(256)
    sv = S.StokesSolver(pr.dim, pr.n[:pr.dim], pr.bc[:2 * pr.dim], pr.h)
    sv.set_coefficients(_t(pr.rho), _t(pr.mu), pr.theta)
    bu = [_t(x) for x in pr.b_u]
    bp = _t(pr.b_p)
    for precision in (0, 1):
        tuning.tune(sv, precision)
        x_u, x_p, info = sv.solve(bu, bp, precond=pr.precond, precision=precision, maxit=3000)
        assert info["converged"] and info["true_residual"] <= 1e-10
        _check_rows(pr, x_u, x_p, 20000, 100 + precision)
    sv.close()


def test_full_batched_workload_on_sampled_rows(S):
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
    for i, (pr, info) in enumerate(zip(prs, infos)):
        assert info["converged"] and info["true_residual"] <= 1e-10, (i, info)
        _check_rows(pr, xus[i], xps[i], 2000, 200 + i)
    for sv in svs:
        sv.close()
