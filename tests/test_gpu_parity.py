"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances (FP64 everywhere unless stated):
  * the operator and the transfer of data are a few roundings apart from the
    oracle's sparse products: elementwise |y - y_ref| <= 1e-12 max|y_ref|;
  * a V-cycle or a preconditioner is a fixed sequence of O(100) stencil
    sweeps whose rounding differs from the oracle's sparse row products:
    relative max error <= 1e-10;
  * solves stop at ||b - M x|| <= 1e-10 ||b||; the solution must match the
    oracle's exact discrete solution to <= 1e-8 relative L2 in velocity and
    in mean-free pressure;
  * the mixed form (FP32 preconditioner inside FP64 flexible GMRES) meets the
    same residual and error bounds, because the outer iteration works on the
    FP64 true residual.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import assemble as asm
from oracle import direct, krylov
from oracle import multigrid as mg
from oracle.grid import Grid, PERIODIC, NOSLIP, FREESLIP
from oracle.precond import Preconditioner
from paper_1308_4605_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1308_4605_gb300 import stokes
    return stokes


DEV = "cuda"


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(DEV)


def _split(g, x):
    u, p = g.unpack(x)
    return [_t(v) for v in u], _t(p)


def _join(g, u, p):
    return g.pack([v.cpu().numpy() for v in u], p.cpu().numpy())


def _make(S, pr):
    solver = S.StokesSolver(pr.dim, pr.n[:pr.dim], pr.bc[:2 * pr.dim], pr.h)
    solver.set_coefficients(_t(pr.rho), _t(pr.mu), pr.theta)
    return solver


CASES = [
    (2, (16, 8), (PERIODIC,) * 4, 1.0),
    (2, (8, 16), (NOSLIP,) * 4, 0.0),
    (2, (16, 16), (FREESLIP, NOSLIP, PERIODIC, PERIODIC), 2.0),
    (2, (32, 8), (NOSLIP, FREESLIP, FREESLIP, NOSLIP), 0.5),
    (3, (8, 8, 8), (PERIODIC,) * 6, 1.0),
    (3, (8, 4, 16), (NOSLIP,) * 6, 0.0),
    (3, (8, 8, 4), (NOSLIP, NOSLIP, PERIODIC, PERIODIC, FREESLIP, FREESLIP), 1.0),
    # above 4096 cells: the finer levels run as grid-wide kernels, the rest in
    # the single-block coarse-level kernel
    (2, (128, 64), (NOSLIP, FREESLIP, PERIODIC, PERIODIC), 1.0),
    (3, (32, 16, 16), (PERIODIC, PERIODIC, NOSLIP, NOSLIP, FREESLIP, NOSLIP), 0.5),
]


def _problem(dim, n, bc, theta, seed=0):
    return wl.generic(dim, n, bc, theta=theta, rho_contrast=10.0, mu_contrast=30.0, seed=seed)


@pytest.mark.parametrize("dim,n,bc,theta", CASES)
def test_operator_matches_oracle(S, dim, n, bc, theta):
    pr = _problem(dim, n, bc, theta)
    g = Grid(dim, pr.n, pr.h, pr.bc)
    M = asm.stokes_from_fields(g, pr.rho, pr.mu, pr.theta)
    u, p = wl.random_face_vector(g.n, g.bc, dim, 5)
    x = g.pack(u, p)
    x[~g.active] = 0.0
    solver = _make(S, pr)
    y_u, y_p = solver.apply_operator(*_split(g, x))
    y = _join(g, y_u, y_p)
    ref = M @ x
    assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max()
    assert np.all(y[~g.active] == 0.0)
    solver.close()


@pytest.mark.parametrize("dim,n,bc,theta", CASES)
def test_vcycles_match_oracle(S, dim, n, bc, theta):
    pr = _problem(dim, n, bc, theta, seed=3)
    g = Grid(dim, pr.n, pr.h, pr.bc)
    coef = asm.fine_coefficients(g, pr.rho, pr.mu, pr.theta)
    levels = mg.build_hierarchy(g, coef)
    rng = np.random.default_rng(9)
    r = rng.standard_normal(g.size) * g.active
    ref_u = mg.vcycle_velocity(levels, r[:g.nvel])
    rp = r[g.nvel:] - r[g.nvel:].mean()
    ref_p = mg.vcycle_pressure(levels, rp)
    solver = _make(S, pr)
    r_u, _ = _split(g, r)
    x_u, x_p = solver.zeros()
    S.stk_velocity_vcycle(solver.handle, r_u, x_u)
    xp = torch.zeros_like(x_p)
    S.stk_pressure_vcycle(solver.handle, _t(rp.reshape(g.cell_shape())), xp)
    got_u = _join(g, x_u, xp)[:g.nvel]
    got_p = xp.cpu().numpy().ravel()
    assert np.abs(got_u - ref_u).max() <= 1e-10 * np.abs(ref_u).max()
    assert np.abs(got_p - ref_p).max() <= 1e-10 * np.abs(ref_p).max()
    solver.close()


@pytest.mark.parametrize("which", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("dim,n,bc,theta", [CASES[0], CASES[1], CASES[4], CASES[6], CASES[7], CASES[8]])
def test_preconditioners_match_oracle(S, which, dim, n, bc, theta):
    pr = _problem(dim, n, bc, theta, seed=4)
    g = Grid(dim, pr.n, pr.h, pr.bc)
    P = Preconditioner(g, pr.rho, pr.mu, pr.theta, which)
    rng = np.random.default_rng(11)
    b = rng.standard_normal(g.size) * g.active
    ref = P(b)
    solver = _make(S, pr)
    x_u, x_p = solver.apply_preconditioner(which, *_split(g, b))
    got = _join(g, x_u, x_p)
    assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()
    solver.close()


@pytest.mark.parametrize("which", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("dim,n,bc,theta", [CASES[3], CASES[7], CASES[8]])
def test_repeated_cycle_preconditioners_match_oracle(S, which, dim, n, bc, theta):
    """Two velocity and three pressure V-cycles per subsolve (Sec. 4.1.2):
    FP64 to 1e-10 of the oracle; the FP32 form (inputs rounded to FP32,
    FP32 hierarchy) to 1e-4, the accuracy of FP32 multigrid."""
    pr = _problem(dim, n, bc, theta, seed=5)
    g = Grid(dim, pr.n, pr.h, pr.bc)
    P = Preconditioner(g, pr.rho, pr.mu, pr.theta, which, cycles_u=2, cycles_p=3)
    rng = np.random.default_rng(12)
    b = rng.standard_normal(g.size) * g.active
    ref = P(b)
    solver = _make(S, pr)
    for precision, tol in ((0, 1e-10), (1, 1e-4)):
        x_u, x_p = solver.apply_preconditioner(which, *_split(g, b), precision=precision,
                                               vcycles_u=2, vcycles_p=3)
        got = _join(g, x_u, x_p)
        assert np.abs(got - ref).max() <= tol * np.abs(ref).max(), (precision, np.abs(got - ref).max())
    solver.close()


@pytest.mark.parametrize("ncoarse", [8, 3])
@pytest.mark.parametrize("dim,n,bc,theta", [CASES[1], CASES[4], CASES[7], CASES[8]])
def test_coarse_solve_sweep_counts_match_oracle(S, ncoarse, dim, n, bc, theta):
    """The coarsest-level solve (App. C) with the default 8 sweeps, which the
    library applies as the precomputed matrix of those sweeps, and with
    another count, which it sweeps, both match the oracle's sweeps: FP64 to
    1e-10, FP32 to 1e-4."""
    pr = _problem(dim, n, bc, theta, seed=6)
    g = Grid(dim, pr.n, pr.h, pr.bc)
    P = Preconditioner(g, pr.rho, pr.mu, pr.theta, 1, ncoarse=ncoarse)
    rng = np.random.default_rng(13)
    b = rng.standard_normal(g.size) * g.active
    ref = P(b)
    solver = _make(S, pr)
    for precision, tol in ((0, 1e-10), (1, 1e-4)):
        x_u, x_p = solver.apply_preconditioner(1, *_split(g, b), precision=precision, ncoarse=ncoarse)
        got = _join(g, x_u, x_p)
        assert np.abs(got - ref).max() <= tol * np.abs(ref).max(), (precision, np.abs(got - ref).max())
    solver.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_solve_with_repeated_cycles(S, precision):
    """GMRES with two V-cycles per subsolve on the 32^2 periodic workload:
    same discrete solution, iteration count within 2 of the oracle's GMRES
    with the same preconditioner."""
    pr = wl.config_c1(32)
    g = Grid(2, pr.n, pr.h, pr.bc)
    M = asm.stokes_from_fields(g, pr.rho, pr.mu, pr.theta)
    b = g.pack(pr.b_u, pr.b_p)
    xd = direct.solve(g, M, b)
    P = Preconditioner(g, pr.rho, pr.mu, pr.theta, 1, cycles_u=2, cycles_p=2)
    _, oinfo = krylov.gmres(lambda v: M @ v, P, b, rtol=1e-10, flexible=bool(precision))
    solver = _make(S, pr)
    x_u, x_p, info = solver.solve(*_split(g, b), precision=precision, vcycles_u=2, vcycles_p=2)
    assert info["converged"]
    assert abs(info["iterations"] - oinfo["iterations"]) <= 2, (info, oinfo)
    # P1 with 2 + 2 cycles: d * 2 + 2 = 6 scalar V-cycles per application
    assert info["scalar_vcycles"] % 6 == 0 and info["scalar_vcycles"] >= 6 * info["iterations"]
    x = _join(g, x_u, x_p)
    assert np.linalg.norm(b - M @ x) / np.linalg.norm(b) <= 1.0001e-10
    eu, ep = direct.relative_error(g, x, xd)
    assert eu <= 1e-8 and ep <= 1e-8
    solver.close()


def _solve_and_check(S, pr, precision, which=None, rtol=1e-10, tol=1e-8):
    g = Grid(pr.dim, pr.n, pr.h, pr.bc)
    M = asm.stokes_from_fields(g, pr.rho, pr.mu, pr.theta)
    b = g.pack(pr.b_u, pr.b_p)
    xd = direct.solve(g, M, b)
    solver = _make(S, pr)
    b_u, b_p = _split(g, b)
    x_u, x_p, info = solver.solve(b_u, b_p, precond=which or pr.precond, rtol=rtol,
                                  precision=precision, maxit=2000)
    assert info["converged"], info
    x = _join(g, x_u, x_p)
    res = np.linalg.norm(b - M @ x) / np.linalg.norm(b)
    assert res <= rtol * 1.0001, res
    eu, ep = direct.relative_error(g, x, xd)
    assert eu <= tol and ep <= tol, (eu, ep, info)
    solver.close()
    return info


@pytest.mark.parametrize("precision", [0, 1])
def test_solve_32x32_periodic_unsteady(S, precision):
    """The 32^2 periodic unsteady workload, P1, GMRES(10)."""
    pr = wl.config_c1(32)
    info = _solve_and_check(S, pr, precision)
    g = Grid(2, pr.n, pr.h, pr.bc)
    M = asm.stokes_from_fields(g, pr.rho, pr.mu, pr.theta)
    P = Preconditioner(g, pr.rho, pr.mu, pr.theta, 1)
    _, oinfo = krylov.gmres(lambda v: M @ v, P, g.pack(pr.b_u, pr.b_p), rtol=1e-10,
                            flexible=bool(precision))
    assert abs(info["iterations"] - oinfo["iterations"]) <= 2, (info, oinfo)


@pytest.mark.parametrize("which", [1, 2, 3, 5])
@pytest.mark.parametrize("precision", [0, 1])
def test_solve_bubble_2d(S, which, precision):
    """The paper's bubble problem (Eq. varcoeff_def), r = 100, steady, 64^2."""
    pr = wl.bubble(2, 64, 100.0, 100.0)
    _solve_and_check(S, pr, precision, which)


@pytest.mark.parametrize("precision", [0, 1])
def test_solve_bubble_2d_256(S, precision):
    """Bubble r = 100 at 256^2: four levels run as grid-wide kernels."""
    pr = wl.bubble(2, 256, 100.0, 100.0)
    _solve_and_check(S, pr, precision, 1)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("cfg", ["c3", "c5", "c4"])
def test_solve_reduced_configs(S, cfg, precision):
    """Reduced-size versions of the 3D periodic unsteady, the 3D steady no-slip
    and the batched-instance workloads (same generators)."""
    if cfg == "c3":
        pr = wl.config_c3(16)
    elif cfg == "c5":
        pr = wl.config_c5(16)
    else:
        pr = wl.config_c4_instance(3, 64)
    _solve_and_check(S, pr, precision)


def test_errors(S):
    with pytest.raises(S.StokesError) as e:
        S.stk_create(2, (12, 16), 1.0, (0, 0, 0, 0))
    assert e.value.code == S.STK_ERR_SIZE
    with pytest.raises(S.StokesError):
        S.stk_create(2, (16, 16), 1.0, (0, 1, 0, 0))
    solver = S.StokesSolver(2, (16, 16), (1, 1, 1, 1))
    b_u, b_p = solver.zeros()
    with pytest.raises(S.StokesError) as e:
        solver.solve(b_u, b_p)
    assert e.value.code == S.STK_ERR_STATE
    rho = torch.ones(solver.cell_shape(), dtype=torch.float64, device=DEV)
    mu = rho.clone()
    mu[0, 3, 3] = float("nan")
    with pytest.raises(S.StokesError) as e:
        solver.set_coefficients(rho, mu, 1.0)
    assert e.value.code == S.STK_ERR_NONFINITE
    mu[0, 3, 3] = -1.0
    with pytest.raises(S.StokesError) as e:
        solver.set_coefficients(rho, mu, 1.0)
    assert e.value.code == S.STK_ERR_ARG
    mu[0, 3, 3] = 1.0
    solver.set_coefficients(rho, mu, 1.0)
    # zero right-hand side: x = 0, converged
    x_u, x_p, info = solver.solve(b_u, b_p)
    assert info["converged"] and float(x_p.abs().max()) == 0.0
    # maxit = 1 on a random right-hand side: not converged, reported
    b_u[0].normal_()
    b_u[0][0, :, 0] = 0
    b_u[0][0, :, -1] = 0
    x_u, x_p, info = solver.solve(b_u, b_p, maxit=1)
    assert not info["converged"] and info["status"] == S.STK_ERR_NOT_CONVERGED
    solver.close()


def test_deterministic(S):
    """Fixed-order reductions: two solves give bitwise identical results."""
    pr = wl.config_c1(32)
    g = Grid(2, pr.n, pr.h, pr.bc)
    solver = _make(S, pr)
    b_u, b_p = _split(g, g.pack(pr.b_u, pr.b_p))
    x1 = solver.solve(b_u, b_p, precond=1)
    x2 = solver.solve(b_u, b_p, precond=1)
    assert all(torch.equal(a, b) for a, b in zip(x1[0], x2[0])) and torch.equal(x1[1], x2[1])
    solver.close()
