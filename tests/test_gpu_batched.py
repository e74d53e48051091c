"""Batched solve (stk_solve_batched): many independent systems of uneven
sizes solved together.  Each instance's arithmetic is that of a single
stk_solve (same kernels, same order), so results must be bitwise equal to
the single solves; two instances are also checked against the oracle's
exact solution (1e-8, residual 1e-10)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import assemble as asm
from oracle import direct
from oracle.grid import Grid, PERIODIC, NOSLIP, FREESLIP
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


def _problems():
    prs = [wl.config_c4_instance(i, n) for i, n in enumerate([64, 128, 64, 256])]
    prs.append(wl.generic(3, (16, 16, 8), (NOSLIP,) * 6, theta=0.0, mu_contrast=50.0, seed=41, precond=2))
    prs.append(wl.bubble(2, 64, 100.0, 100.0))
    return prs


@pytest.mark.parametrize("precision", [0, 1])
def test_batched_equals_single_solves(S, precision):
    prs = _problems()
    solvers, bus, bps, xus, xps = [], [], [], [], []
    for pr in prs:
        sv = S.StokesSolver(pr.dim, pr.n[:pr.dim], pr.bc[:2 * pr.dim], pr.h)
        sv.set_coefficients(_t(pr.rho), _t(pr.mu), pr.theta)
        solvers.append(sv)
        bus.append([_t(x) for x in pr.b_u])
        bps.append(_t(pr.b_p))
        xu, xp = sv.zeros()
        xus.append(xu)
        xps.append(xp)
    p = S.stk_default_params()
    p.precision = precision
    p.precond = 1
    infos = S.stk_solve_batched([sv.handle for sv in solvers], p, bus, bps, xus, xps)
    torch.cuda.synchronize()
    assert all(i["converged"] for i in infos), infos
    for k, (pr, sv) in enumerate(zip(prs, solvers)):
        xu1, xp1, info1 = sv.solve(bus[k], bps[k], precond=1, precision=precision)
        assert info1["iterations"] == infos[k]["iterations"]
        assert all(torch.equal(a, b) for a, b in zip(xu1, xus[k])) and torch.equal(xp1, xps[k])
    for k in (0, 4):
        pr = prs[k]
        g = Grid(pr.dim, pr.n, pr.h, pr.bc)
        M = asm.stokes_from_fields(g, pr.rho, pr.mu, pr.theta)
        b = g.pack(pr.b_u, pr.b_p)
        x = g.pack([v.cpu().numpy() for v in xus[k]], xps[k].cpu().numpy())
        assert np.linalg.norm(b - M @ x) <= 1.0001e-10 * np.linalg.norm(b)
        assert max(direct.relative_error(g, x, direct.solve(g, M, b))) <= 1e-8
    for sv in solvers:
        sv.close()


def test_batched_rejects_duplicate_handles(S):
    pr = wl.config_c4_instance(0, 64)
    sv = S.StokesSolver(2, pr.n[:2], pr.bc[:4], pr.h)
    sv.set_coefficients(_t(pr.rho), _t(pr.mu), pr.theta)
    bu = [_t(x) for x in pr.b_u]
    bp = _t(pr.b_p)
    xu, xp = sv.zeros()
    with pytest.raises(S.StokesError):
        S.stk_solve_batched([sv.handle, sv.handle], S.stk_default_params(), [bu, bu], [bp, bp], [xu, xu], [xp, xp])
    sv.close()


def test_schedules_change_timing_not_results(S, tmp_path):
    """Every multigrid schedule (coarse-kernel level, colour block size) gives
    bitwise the same solution; the autotuner picks one and caches it."""
    from paper_1308_4605_gb300 import tuning
    pr = wl.config_c4_instance(5, 128)
    sv = S.StokesSolver(2, pr.n[:2], pr.bc[:4], pr.h)
    sv.set_coefficients(_t(pr.rho), _t(pr.mu), pr.theta)
    bu = [_t(x) for x in pr.b_u]
    bp = _t(pr.b_p)
    ref = None
    nlev = 7                      # 128, 64, ..., 2
    for prec in (0, 1):
        ref = None
        for lc, th in ((nlev, 256), (0, 256), (2, 128), (3, 512), (4, 64)):
            S.stk_set_schedule(sv.handle, prec, lc, th)
            xu, xp, info = sv.solve(bu, bp, precision=prec)
            assert info["converged"]
            if ref is None:
                ref = (xu, xp, info["iterations"])
            else:
                assert info["iterations"] == ref[2]
                assert all(torch.equal(a, b) for a, b in zip(xu, ref[0])) and torch.equal(xp, ref[1])
        path = str(tmp_path / "sched.json")
        sc = tuning.tune(sv, prec, path)
        assert 0 <= sc["coarse_level"] <= nlev and sc["threads"] in (128, 256, 512)
        assert tuning.tune(sv, prec, path) == sc          # cache hit
        assert S.stk_get_schedule(sv.handle, prec) == sc
    sv.close()
