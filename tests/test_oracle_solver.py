"""Pins of the oracle's preconditioners (Sec. 2, App. B) and GMRES (Sec. 3.2,
Sec. 4) against the exact-subsolver identities and the direct solve."""
import numpy as np
import pytest

from oracle import assemble as asm
from oracle import direct, krylov
from oracle.grid import Grid, PERIODIC, NOSLIP, FREESLIP
from oracle.precond import Preconditioner
from paper_1308_4605_gb300 import workloads as wl


def _operator_matrix(fn, g):
    """Dense matrix of a linear map on the active unknowns (pressure mean
    removed from inputs)."""
    act = np.flatnonzero(g.active)
    cols = []
    for k in act:
        e = np.zeros(g.size)
        e[k] = 1.0
        cols.append(fn(e)[act])
    return np.array(cols).T


def _proj(g):
    """Projector on the active unknowns that removes the pressure mean."""
    act = np.flatnonzero(g.active)
    n = len(act)
    Pm = np.eye(n)
    pc = act >= g.cell_offset
    Pm[np.ix_(pc, pc)] -= 1.0 / pc.sum()
    return Pm


def _preconditioned(g, rho, mu, theta, which):
    M = asm.stokes_from_fields(g, rho, mu, theta)
    P = Preconditioner(g, rho, mu, theta, which, exact=True)
    T = _operator_matrix(lambda v: P(M @ v), g)
    Pm = _proj(g)
    return Pm @ T @ Pm, Pm


@pytest.mark.parametrize("dim,n", [(2, (8, 8)), (3, (4, 4, 4))])
def test_P1_exact_for_periodic_constant_coefficients(dim, n):
    """App. B: with exact subsolvers and constant coefficients on a periodic
    grid, P1^{-1} M = I."""
    g = Grid(dim, n, 1.0, (PERIODIC,) * 6)
    one = np.ones(g.cell_shape())
    T, Pm = _preconditioned(g, 1.3 * one, 0.7 * one, 2.0, 1)
    assert np.abs(T - Pm).max() < 1e-10


@pytest.mark.parametrize("which", [2, 3])
def test_P2_P3_square_to_identity_periodic(which):
    """Constant-coefficient periodic, exact subsolvers: S~^{-1} S = I, so
    (P^{-1} M - I)^2 = 0 for P2 and P3 (App. B)."""
    g = Grid(2, (8, 8), 1.0, (PERIODIC,) * 6)
    one = np.ones(g.cell_shape())
    T, Pm = _preconditioned(g, 1.3 * one, 0.7 * one, 2.0, which)
    E = T - Pm
    assert np.abs(E @ E).max() < 1e-9
    assert np.abs(E).max() > 1e-3          # not the identity itself


@pytest.mark.parametrize("bc", [(NOSLIP,) * 4, (FREESLIP, NOSLIP, PERIODIC, PERIODIC)])
def test_inviscid_identities_with_walls(bc):
    """Inviscid limit (L_mu = 0), variable density, any boundary: P1^{-1}M = I,
    (P2^{-1}M - I)^2 = 0, (P3^{-1}M - I)^2 = 0 (App. B), P5^{-1} M = I (its only
    approximation is S~, exact here, Sec. 2.4) and for the block-diagonal P4
    with the "-" sign of Sec. 4.2.1, (T - I)(T^2 - T + I) = 0: an eigenvalue
    other than 1 solves lambda (lambda - 1) = -1 when S~ = S."""
    g = Grid(2, (8, 8), 1.0, bc)
    rng = np.random.default_rng(1)
    rho = np.exp(0.5 * rng.standard_normal(g.cell_shape()))
    mu = np.zeros(g.cell_shape())
    I = None
    for which in (1, 2, 3, 4, 5):
        T, Pm = _preconditioned(g, rho, mu, 1.7, which)
        E = T - Pm
        if which in (1, 5):
            assert np.abs(E).max() < 1e-10
        elif which in (2, 3):
            assert np.abs(E @ E).max() < 1e-9
        else:
            assert np.abs(E @ (T @ T - T + Pm)).max() < 1e-9


def test_gmres_iteration_counts_with_exact_subsolvers():
    """Sec. 4.1.2 / App. B: GMRES converges in 1 iteration with P1 and 2 with
    P2, P3 for constant-coefficient periodic problems and exact subsolvers."""
    g = Grid(2, (16, 16), 1.0, (PERIODIC,) * 6)
    one = np.ones(g.cell_shape())
    rho, mu, theta = 1.0 * one, 1.0 * one, 1.0
    M = asm.stokes_from_fields(g, rho, mu, theta)
    u, p = wl.random_face_vector(g.n, g.bc, 2, 3)
    b = M @ g.pack(u, p - p.mean())
    for which, expect in ((1, 1), (2, 2), (3, 2)):
        P = Preconditioner(g, rho, mu, theta, which, exact=True)
        x, info = krylov.gmres(lambda v: M @ v, P, b, rtol=1e-10)
        assert info["converged"]
        assert info["iterations"] == expect, (which, info)


@pytest.mark.parametrize("which", [1, 2, 3, 4, 5])
def test_multigrid_preconditioners_are_linear(which):
    """GMRES needs a fixed linear preconditioner (Sec. 4, App. C)."""
    g = Grid(2, (16, 8), 1.0, (NOSLIP, NOSLIP, PERIODIC, PERIODIC))
    rng = np.random.default_rng(4)
    rho = np.exp(rng.standard_normal(g.cell_shape()))
    mu = np.exp(rng.standard_normal(g.cell_shape()))
    P = Preconditioner(g, rho, mu, 1.0, which)
    a = rng.standard_normal(g.size) * g.active
    b = rng.standard_normal(g.size) * g.active
    lhs = P(3.0 * a - b)
    rhs = 3.0 * P(a) - P(b)
    assert np.abs(lhs - rhs).max() < 1e-12 * np.abs(rhs).max()


@pytest.mark.parametrize("which", [1, 2, 3, 5])
def test_gmres_matches_direct_solve_c1(which):
    """The 32^2 periodic unsteady workload: GMRES(10) with one V-cycle per
    subsolve reaches 1e-10 and agrees with the exact discrete solution."""
    pr = wl.config_c1(32)
    g = Grid(2, pr.n, pr.h, pr.bc)
    M = asm.stokes_from_fields(g, pr.rho, pr.mu, pr.theta)
    b = g.pack(pr.b_u, pr.b_p)
    P = Preconditioner(g, pr.rho, pr.mu, pr.theta, which)
    x, info = krylov.gmres(lambda v: M @ v, P, b, rtol=1e-10)
    assert info["converged"] and info["iterations"] < 60
    xd = direct.solve(g, M, b)
    assert max(direct.relative_error(g, x, xd)) < 1e-8


@pytest.mark.parametrize("which", [1, 2])
def test_fgmres_matches_direct_solve_3d(which):
    pr = wl.generic(3, (8, 8, 8), (NOSLIP,) * 6, theta=0.0 if which == 2 else 1.0,
                    rho_contrast=10.0, mu_contrast=100.0, seed=11, precond=which)
    g = Grid(3, pr.n, pr.h, pr.bc)
    M = asm.stokes_from_fields(g, pr.rho, pr.mu, pr.theta)
    b = g.pack(pr.b_u, pr.b_p)
    P = Preconditioner(g, pr.rho, pr.mu, pr.theta, which)
    xd = direct.solve(g, M, b)
    for flexible in (False, True):
        x, info = krylov.gmres(lambda v: M @ v, P, b, rtol=1e-10, flexible=flexible)
        assert info["converged"]
        assert max(direct.relative_error(g, x, xd)) < 1e-8


def test_workload_generators():
    pr = wl.config_c1(32)
    assert np.isclose(pr.rho.max() / pr.rho.min(), 10.0)
    assert np.isclose(pr.mu.max() / pr.mu.min(), 10.0)
    assert np.isclose(np.sqrt(pr.mu.max() * pr.mu.min()), 1.0)
    assert abs(pr.b_p.mean()) < 1e-15
    pr2 = wl.config_c2(64)
    assert set(np.unique(pr2.mu)) <= {1.0, 1e4}
    disks = pr2.meta["disks"]
    assert len(disks) == 20
    for i in range(20):
        for j in range(i):
            (x1, y1, r1), (x2, y2, r2) = disks[i], disks[j]
            assert (x1 - x2) ** 2 + (y1 - y2) ** 2 > (r1 + r2) ** 2
    assert pr2.b_u[0][0, :, 0].max() == 0.0 and pr2.b_u[1][0, -1, :].max() == 0.0
    f3 = wl.smooth_field_3d((8, 8, 8), 1.0, 6)
    assert f3.shape == (8, 8, 8) and np.isfinite(f3).all()
    sizes = wl.config_c4_sizes()
    assert len(sizes) == 64 and set(sizes) <= {64, 128, 256, 512}


@pytest.mark.parametrize("bc,theta", [((NOSLIP, NOSLIP, FREESLIP, NOSLIP), 1.0),
                                      ((PERIODIC,) * 4, 2.0),
                                      ((NOSLIP,) * 4, 0.0)])
@pytest.mark.parametrize("which", [1, 2, 3, 4, 5])
def test_repeated_cycles_tend_to_exact_subsolvers(bc, theta, which):
    """Sec. 4.1.2: with many V-cycles per subsolve the preconditioner becomes
    the exact-subsolver one (App. B), and the subsolve error falls
    geometrically with the number of cycles (each V-cycle reduces the
    residual by about ten, Sec. 4.1.1)."""
    g = Grid(2, (16, 16), 1.0, bc)
    rng = np.random.default_rng(6)
    rho = np.exp(0.5 * rng.standard_normal(g.cell_shape()))
    mu = np.exp(0.5 * rng.standard_normal(g.cell_shape()))
    b = rng.standard_normal(g.size) * g.active
    b[g.nvel:] -= b[g.nvel:].mean()
    ex = Preconditioner(g, rho, mu, theta, which, exact=True)(b)
    many = Preconditioner(g, rho, mu, theta, which, cycles_u=40, cycles_p=40)(b)
    assert np.abs(many - ex).max() <= 1e-9 * np.abs(ex).max()
    # subsolve errors for 1, 2, 3 cycles
    P = Preconditioner(g, rho, mu, theta, which)
    Pe = Preconditioner(g, rho, mu, theta, which, exact=True)
    r_u = b[:g.nvel]
    r_p = b[g.nvel:]
    eu = Pe.velocity_solve(r_u)
    ep = Pe.poisson_solve(r_p)
    du, dp = [], []
    for c in (1, 2, 3):
        P.cycles_u = P.cycles_p = c
        du.append(np.linalg.norm(P.velocity_solve(r_u) - eu))
        x = P.poisson_solve(r_p)
        dp.append(np.linalg.norm((x - x.mean()) - (ep - ep.mean())))
    for d in (du, dp):
        assert d[1] <= 0.25 * d[0] and d[2] <= 0.25 * d[1], d


def test_repeated_cycles_gmres_converges_to_direct():
    """GMRES with two V-cycles per subsolve reaches the same discrete
    solution with fewer iterations than with one."""
    pr = wl.config_c1(32)
    g = Grid(2, pr.n, pr.h, pr.bc)
    M = asm.stokes_from_fields(g, pr.rho, pr.mu, pr.theta)
    b = g.pack(pr.b_u, pr.b_p)
    xd = direct.solve(g, M, b)
    its = []
    for c in (1, 2):
        P = Preconditioner(g, pr.rho, pr.mu, pr.theta, 1, cycles_u=c, cycles_p=c)
        x, info = krylov.gmres(lambda v: M @ v, P, b, rtol=1e-10)
        assert info["converged"]
        assert max(direct.relative_error(g, x, xd)) < 1e-8
        its.append(info["iterations"])
    assert its[1] <= its[0]


@pytest.mark.parametrize("name,n,i", [("c1", 32, None), ("c3", 16, None), ("c5", 16, None),
                                      ("c4", 64, 3)])
def test_reference_solve_matches_direct_solve(name, n, i):
    """The tight-tolerance GMRES solve used for full-size parity reaches
    1e-13 and equals the exact discrete solution to 1e-11 on the workloads'
    generators at reduced size."""
    from oracle import reference_solve as rs
    x, info = rs.solve_workload(name, n, i)
    assert info["converged"] and info["true_residual"] <= 1e-13
    pr = {"c1": lambda: wl.config_c1(n), "c3": lambda: wl.config_c3(n),
          "c5": lambda: wl.config_c5(n), "c4": lambda: wl.config_c4_instance(i, n)}[name]()
    g = Grid(pr.dim, pr.n, pr.h, pr.bc)
    M = asm.stokes_from_fields(g, pr.rho, pr.mu, pr.theta)
    b = g.pack(pr.b_u, pr.b_p)
    b[~g.active] = 0.0
    xd = direct.solve(g, M, b)
    assert max(direct.relative_error(g, x, xd)) < 1e-11
    assert abs(x[g.cell_offset:].mean()) < 1e-14 * np.abs(x[g.cell_offset:]).max()
