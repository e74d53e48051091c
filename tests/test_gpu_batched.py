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
    """Every multigrid schedule (coarse-kernel level, two-colour level, colour
    block size) gives bitwise the same solution (FP64 with the whole V-cycle
    in the coarse kernel: the same up to rounding); the autotuner picks one
    and caches it."""
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
        for lc, th, pl in ((nlev, 256, nlev), (0, 256, 0), (2, 128, 0), (3, 512, 1), (4, 64, 4),
                           (nlev, 128, 0), (5, 256, 2)):
            S.stk_set_schedule(sv.handle, prec, lc, th, pl)
            xu, xp, info = sv.solve(bu, bp, precision=prec)
            assert info["converged"]
            if ref is None:
                ref = (xu, xp, info["iterations"])
            elif prec == 0 and lc == 0:
                # the whole V-cycle in the single-block kernel evaluates the
                # finest FP64 residual point by point instead of through the
                # stresses: equal up to rounding
                assert abs(info["iterations"] - ref[2]) <= 1
                for a, b in zip(list(xu) + [xp], list(ref[0]) + [ref[1]]):
                    assert float((a - b).abs().max()) <= 1e-9 * float(b.abs().max())
            else:
                assert info["iterations"] == ref[2]
                assert all(torch.equal(a, b) for a, b in zip(xu, ref[0])) and torch.equal(xp, ref[1])
        path = str(tmp_path / "sched.json")
        sc = tuning.tune(sv, prec, path)
        assert 0 <= sc["coarse_level"] <= nlev and sc["threads"] in (128, 256, 512)
        assert 0 <= sc["pair_level"] <= sc["coarse_level"]
        assert tuning.tune(sv, prec, path) == sc          # cache hit
        assert S.stk_get_schedule(sv.handle, prec) == sc
    sv.close()


@pytest.mark.parametrize("n,bc", [((64, 32, 16), (0,) * 6), ((32, 16, 16), (1, 1, 2, 1, 0, 0)),
                                  ((16, 32, 64), (1, 1, 0, 0, 2, 1)), ((128, 16, 32), (0,) * 6)])
def test_two_colour_sweeps_equal_per_colour_3d(S, n, bc):
    """3D: V-cycles and solves (FP64 and mixed) with the two-colour kernels
    (columns marching along z) on every grid level equal, bitwise, those with
    one launch per colour (periodic, and mixed no-slip / free-slip / periodic
    boundaries whose face arrays are not multiples of the column; several
    columns along x and several z ranges per column)."""
    theta = 1.0 if bc[0] == 0 else 0.0
    pr = wl.generic(3, n, bc, theta=theta, seed=41, precond=1 if theta else 2)
    sv = S.StokesSolver(3, pr.n, pr.bc, pr.h)
    sv.set_coefficients(_t(pr.rho), _t(pr.mu), pr.theta)
    g = Grid(3, pr.n, pr.h, pr.bc)
    rng = np.random.default_rng(4)
    ru, rp = g.unpack(rng.standard_normal(g.size) * g.active)
    ru = [_t(x) for x in ru]
    rp = _t(rp - rp.mean())
    bu = [_t(x) for x in pr.b_u]
    bp = _t(pr.b_p)
    sched = {p: S.stk_get_schedule(sv.handle, p) for p in (0, 1)}
    out = []
    for paired in (True, False):
        for p in (0, 1):
            sc = sched[p]
            S.stk_set_schedule(sv.handle, p, sc["coarse_level"], sc["threads"],
                               0 if paired else sc["coarse_level"])
        xu = [torch.zeros_like(x) for x in ru]
        xp = torch.zeros_like(rp)
        S.stk_velocity_vcycle(sv.handle, ru, xu)
        S.stk_pressure_vcycle(sv.handle, rp, xp)
        torch.cuda.synchronize()
        res = [xu, xp]
        for prec in (0, 1):
            su, sp, info = sv.solve(bu, bp, precision=prec, precond=pr.precond)
            assert info["converged"]
            res += [su, sp]
        out.append(res)
    for a, b in zip(out[0], out[1]):
        if isinstance(a, list):
            assert all(torch.equal(x, y) for x, y in zip(a, b))
        else:
            assert torch.equal(a, b)
    sv.close()


def test_two_colour_sweeps_equal_per_colour_3d_bulk(S):
    """The same with the bulk-viscosity stress form (mixed solve, two-colour
    kernels from the finest level)."""
    pr = wl.generic(3, (32, 32, 16), (1, 1, 0, 0, 2, 2), theta=1.0, seed=43, precond=1)
    sv = S.StokesSolver(3, pr.n, pr.bc, pr.h)
    sv.set_coefficients(_t(pr.rho), _t(pr.mu), pr.theta)
    gam = torch.full(sv.cell_shape(), 0.7, dtype=torch.float64, device=DEV)
    sv.set_bulk_viscosity(gam)
    bu = [_t(x) for x in pr.b_u]
    bp = _t(pr.b_p)
    out = []
    for paired in (True, False):
        sc = S.stk_get_schedule(sv.handle, 1)
        S.stk_set_schedule(sv.handle, 1, sc["coarse_level"], sc["threads"], 0 if paired else sc["coarse_level"])
        su, sp, info = sv.solve(bu, bp, precision=1, precond=1)
        assert info["converged"]
        out.append([*su, sp])
    assert all(torch.equal(a, b) for a, b in zip(out[0], out[1]))
    sv.close()


def test_coefficient_updates_keep_graphs_valid(S):
    """set_coefficients keeps the captured preconditioner graphs unless theta
    switches between zero and non-zero (they read coefficients and theta
    from device memory): a solve after new coefficients and a new theta must
    equal, bitwise, the same solve on a fresh handle."""
    pr = wl.config_c1(32)
    pr2 = wl.generic(2, (32, 32), (0,) * 4, theta=0.5, rho_contrast=5.0, mu_contrast=30.0, seed=77)
    bu = [_t(x) for x in pr.b_u]
    bp = _t(pr.b_p)
    sv = S.StokesSolver(2, pr.n[:2], pr.bc[:4], pr.h)
    for prec in (0, 1):
        sv.set_coefficients(_t(pr.rho), _t(pr.mu), pr.theta)
        sv.solve(bu, bp, precision=prec)
        for rho, mu, theta in ((pr2.rho, pr2.mu, 0.5), (pr.rho, pr.mu, 2.0), (pr2.rho, pr2.mu, 0.5)):
            sv.set_coefficients(_t(rho), _t(mu), theta)
            xu, xp, info = sv.solve(bu, bp, precision=prec)
            fresh = S.StokesSolver(2, pr.n[:2], pr.bc[:4], pr.h)
            fresh.set_coefficients(_t(rho), _t(mu), theta)
            fu, fp, finfo = fresh.solve(bu, bp, precision=prec)
            fresh.close()
            assert info["converged"] and info["iterations"] == finfo["iterations"]
            assert all(torch.equal(a, b) for a, b in zip(xu, fu)) and torch.equal(xp, fp)
    sv.close()
    # theta switching to zero and back (walls: steady flow is admissible)
    pw = wl.generic(2, (32, 32), (1,) * 4, theta=1.0, seed=78, precond=2)
    sv = S.StokesSolver(2, pw.n[:2], pw.bc[:4], pw.h)
    bu = [_t(x) for x in pw.b_u]
    bp = _t(pw.b_p)
    for theta in (1.0, 0.0, 3.0, 0.0):
        sv.set_coefficients(_t(pw.rho), _t(pw.mu), theta)
        xu, xp, info = sv.solve(bu, bp, precond=2)
        fresh = S.StokesSolver(2, pw.n[:2], pw.bc[:4], pw.h)
        fresh.set_coefficients(_t(pw.rho), _t(pw.mu), theta)
        fu, fp, _ = fresh.solve(bu, bp, precond=2)
        fresh.close()
        assert info["converged"]
        assert all(torch.equal(a, b) for a, b in zip(xu, fu)) and torch.equal(xp, fp)
    sv.close()
