"""The bulk-viscosity stress form on the GPU (stk_set_bulk_viscosity)
against the oracle: operator, V-cycles, P1..P5 and solves of compressible
(g != 0) problems; switching the term off restores the plain form."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import assemble as asm
from oracle import direct
from oracle import multigrid as mg
from oracle.grid import Grid, PERIODIC, NOSLIP, FREESLIP
from oracle.precond import Preconditioner
from paper_1308_4605_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
DEV = "cuda"

CASES = [
    (2, (16, 8), (PERIODIC,) * 4, 1.0),
    (2, (32, 8), (NOSLIP, FREESLIP, FREESLIP, NOSLIP), 0.0),
    (3, (8, 8, 4), (NOSLIP, NOSLIP, PERIODIC, PERIODIC, FREESLIP, FREESLIP), 1.0),
    (2, (128, 64), (NOSLIP, FREESLIP, PERIODIC, PERIODIC), 1.0),
    (3, (32, 16, 16), (PERIODIC, PERIODIC, NOSLIP, NOSLIP, FREESLIP, NOSLIP), 0.5),
]


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1308_4605_gb300 import stokes
    return stokes


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(DEV)


def _split(g, x):
    u, p = g.unpack(x)
    return [_t(v) for v in u], _t(p)


def _join(g, u, p):
    return g.pack([v.cpu().numpy() for v in u], p.cpu().numpy())


def _problem(dim, n, bc, theta, seed):
    pr = wl.generic(dim, n, bc, theta=theta, rho_contrast=10.0, mu_contrast=30.0, seed=seed)
    rng = np.random.default_rng(seed + 100)
    gamma = np.exp(rng.standard_normal(pr.mu.shape)) * 2.0
    return pr, gamma


def _make(S, pr, gamma):
    sv = S.StokesSolver(pr.dim, pr.n[:pr.dim], pr.bc[:2 * pr.dim], pr.h)
    sv.set_coefficients(_t(pr.rho), _t(pr.mu), pr.theta)
    sv.set_bulk_viscosity(_t(gamma))
    return sv


@pytest.mark.parametrize("dim,n,bc,theta", CASES)
def test_bulk_operator_and_vcycles_match_oracle(S, dim, n, bc, theta):
    pr, gamma = _problem(dim, n, bc, theta, 71)
    g = Grid(dim, pr.n, pr.h, pr.bc)
    M = asm.stokes_from_fields(g, pr.rho, pr.mu, pr.theta, gamma=gamma)
    rng = np.random.default_rng(3)
    x = rng.standard_normal(g.size) * g.active
    sv = _make(S, pr, gamma)
    y = _join(g, *sv.apply_operator(*_split(g, x)))
    ref = M @ x
    assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max()
    coef = asm.fine_coefficients(g, pr.rho, pr.mu, pr.theta, gamma)
    levels = mg.build_hierarchy(g, coef)
    ref_u = mg.vcycle_velocity(levels, x[:g.nvel])
    r_u, _ = _split(g, x)
    x_u, x_p = sv.zeros()
    S.stk_velocity_vcycle(sv.handle, r_u, x_u)
    got_u = _join(g, x_u, x_p)[:g.nvel]
    assert np.abs(got_u - ref_u).max() <= 1e-10 * np.abs(ref_u).max()
    sv.close()


@pytest.mark.parametrize("which", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("dim,n,bc,theta", [CASES[0], CASES[2], CASES[3]])
def test_bulk_preconditioners_match_oracle(S, which, dim, n, bc, theta):
    pr, gamma = _problem(dim, n, bc, theta, 72)
    g = Grid(dim, pr.n, pr.h, pr.bc)
    P = Preconditioner(g, pr.rho, pr.mu, pr.theta, which, gamma=gamma)
    rng = np.random.default_rng(5)
    b = rng.standard_normal(g.size) * g.active
    ref = P(b)
    sv = _make(S, pr, gamma)
    got = _join(g, *sv.apply_preconditioner(which, *_split(g, b)))
    assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()
    sv.close()


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("dim,n,bc,theta", [CASES[1], CASES[3], CASES[4]])
def test_bulk_solve_compressible(S, precision, dim, n, bc, theta):
    """A compressible problem (b_p = -g with g != 0, mean-free): the GPU solve
    reaches 1e-10 and the oracle's direct solution to 1e-8."""
    pr, gamma = _problem(dim, n, bc, theta, 73)
    g = Grid(dim, pr.n, pr.h, pr.bc)
    M = asm.stokes_from_fields(g, pr.rho, pr.mu, pr.theta, gamma=gamma)
    b = g.pack(pr.b_u, pr.b_p)
    xd = direct.solve(g, M, b)
    sv = _make(S, pr, gamma)
    x_u, x_p, info = sv.solve(*_split(g, b), precision=precision, precond=1 if theta else 2,
                              maxit=2000)
    assert info["converged"]
    x = _join(g, x_u, x_p)
    assert np.linalg.norm(b - M @ x) / np.linalg.norm(b) <= 1.0001e-10
    assert max(direct.relative_error(g, x, xd)) <= 1e-8
    sv.close()


def test_bulk_switch_off_restores_plain_form(S):
    """After set_bulk_viscosity(None) the solves are bitwise those of a
    handle that never had the bulk term; the gradient is refused while it is
    on; negative gamma is rejected."""
    pr, gamma = _problem(2, (32, 32), (PERIODIC,) * 4, 1.0, 74)
    g = Grid(2, pr.n, pr.h, pr.bc)
    b = g.pack(pr.b_u, pr.b_p)
    plain = S.StokesSolver(2, pr.n[:2], pr.bc[:4], pr.h)
    plain.set_coefficients(_t(pr.rho), _t(pr.mu), pr.theta)
    ref_u, ref_p, _ = plain.solve(*_split(g, b))
    sv = _make(S, pr, gamma)
    bu, bp = _split(g, b)
    sv.solve(bu, bp)
    with pytest.raises(S.StokesError):
        d = torch.empty_like(_t(pr.mu))
        S.stk_gradient(sv.handle, ref_u, ref_u, d, d.clone())
    with pytest.raises(S.StokesError):
        sv.set_bulk_viscosity(_t(-gamma))
    sv.set_bulk_viscosity(None)
    x_u, x_p, _ = sv.solve(bu, bp)
    assert all(torch.equal(a, c) for a, c in zip(x_u, ref_u)) and torch.equal(x_p, ref_p)
    sv.close()
    plain.close()
