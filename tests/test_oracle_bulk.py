"""Pins of the bulk-viscosity form of the viscous operator (Sec. 2:
tau = mu (grad u + grad u^T) + (gamma - 2/3 mu)(div u) I, Schur
approximation Eq. Schur_app_bulk, App. A)."""
import numpy as np
import pytest

from oracle import assemble as asm
from oracle import direct
from oracle.grid import Grid, PERIODIC, NOSLIP, FREESLIP
from oracle.precond import Preconditioner

CASES = [(2, (8, 4), (PERIODIC,) * 4), (2, (8, 8), (NOSLIP, FREESLIP, PERIODIC, PERIODIC)),
         (2, (4, 8), (NOSLIP,) * 4), (3, (4, 4, 4), (NOSLIP, NOSLIP, PERIODIC, PERIODIC, FREESLIP, NOSLIP))]


def _fields(g, seed):
    rng = np.random.default_rng(seed)
    return tuple(np.exp(rng.standard_normal(g.cell_shape())) for _ in range(3))


def _L(g, mu, gamma):
    c = asm.fine_coefficients(g, np.ones(g.cell_shape()), mu, 0.0, gamma)
    return (asm.viscous(g, c["mu_c"], c["mu_e"]) + asm.bulk_viscous(g, c["lam_c"])).toarray()


@pytest.mark.parametrize("dim,n,bc", CASES)
def test_bulk_operator_symmetric_negative_semidefinite(dim, n, bc):
    """G diag(lam) D is symmetric (D = -G^*) and the total viscous operator
    stays negative semidefinite for gamma >= 0 (the dissipation
    2 mu |eps|^2 - 2/3 mu (div u)^2 + gamma (div u)^2 >= 0)."""
    g = Grid(dim, n, 0.5, bc)
    rho, mu, gamma = _fields(g, 1)
    act = np.flatnonzero(g.active[:g.nvel])
    L = _L(g, mu, gamma)[np.ix_(act, act)]
    assert np.abs(L - L.T).max() <= 1e-12 * np.abs(L).max()
    ev = np.linalg.eigvalsh(0.5 * (L + L.T))
    assert ev.max() <= 1e-10 * np.abs(ev).max()
    # gamma = 0 (lam = -2/3 mu) too
    L0 = _L(g, mu, 0.0 * gamma)[np.ix_(act, act)]
    assert np.linalg.eigvalsh(0.5 * (L0 + L0.T)).max() <= 1e-10 * np.abs(L0).max()
    # M stays symmetric (M = M^*, Sec. 2), so the adjoint solve is a forward solve
    M = asm.stokes_from_fields(g, rho, mu, 1.0, gamma=gamma)
    Ma = M[g.active][:, g.active].toarray()
    assert np.abs(Ma - Ma.T).max() <= 1e-12 * np.abs(Ma).max()


@pytest.mark.parametrize("dim,n,bc", CASES)
def test_bulk_term_vanishes_on_divergence_free_fields(dim, n, bc):
    g = Grid(dim, n, 0.5, bc)
    rho, mu, gamma = _fields(g, 2)
    M = asm.stokes_from_fields(g, rho, mu, 1.0)
    rng = np.random.default_rng(3)
    b = rng.standard_normal(g.size) * g.active
    b[g.nvel:] = 0.0
    u = direct.solve(g, M, b)[:g.nvel]           # D u = 0
    c = asm.fine_coefficients(g, rho, mu, 1.0, gamma)
    B = asm.bulk_viscous(g, c["lam_c"])
    assert np.abs(B @ u).max() <= 1e-10 * np.abs(asm.viscous(g, c["mu_c"], c["mu_e"]) @ u).max()


@pytest.mark.parametrize("dim,n", [(2, (8, 8)), (3, (4, 4, 4))])
def test_schur_complement_with_bulk_viscosity_periodic(dim, n):
    """App. A with bulk viscosity: (D L^{-1} G)^{-1} = 4/3 mu0 + gamma0 on
    every non-constant pressure mode of a constant-coefficient periodic grid,
    and P1 with exact subsolvers inverts M (App. B)."""
    g = Grid(dim, n, 1.0, (PERIODIC,) * 6)
    mu0, gamma0 = 0.8, 1.7
    one = np.ones(g.cell_shape())
    L = _L(g, mu0 * one, gamma0 * one)
    D, G = asm.divergence(g).toarray(), asm.gradient(g).toarray()
    Sc = D @ np.linalg.pinv(L, rcond=1e-10) @ G
    ev = np.sort(np.linalg.eigvalsh(0.5 * (Sc + Sc.T)))
    assert abs(ev[0]) < 1e-10
    assert np.allclose(ev[1:], 1.0 / (4.0 / 3.0 * mu0 + gamma0), rtol=1e-10)
    # P1^{-1} M = I on the active unknowns with the pressure mean removed
    M = asm.stokes_from_fields(g, 1.3 * one, mu0 * one, 2.0, gamma=gamma0 * one)
    P = Preconditioner(g, 1.3 * one, mu0 * one, 2.0, 1, exact=True, gamma=gamma0 * one)
    rng = np.random.default_rng(4)
    for _ in range(3):
        x = rng.standard_normal(g.size) * g.active
        x[g.nvel:] -= x[g.nvel:].mean()
        y = P(M @ x)
        assert np.abs(y - x).max() <= 1e-10 * np.abs(x).max()


def _mms(bc_kind):
    sympy = pytest.importorskip("sympy")
    x, y = sympy.symbols("x y")
    pi = sympy.pi
    if bc_kind == "periodic":
        u = sympy.sin(2 * pi * x) * sympy.cos(2 * pi * y)
        v = sympy.cos(2 * pi * x) * sympy.sin(4 * pi * y) * sympy.Rational(1, 2)
        p = sympy.cos(2 * pi * x) * sympy.cos(2 * pi * y)
        mu = 1 + sympy.Rational(1, 2) * sympy.sin(2 * pi * x) * sympy.sin(2 * pi * y)
        gam = 2 + sympy.cos(2 * pi * y) * sympy.sin(2 * pi * x)
        rho = 1 + sympy.Rational(3, 10) * sympy.cos(2 * pi * x)
    else:
        u = sympy.sin(pi * x) ** 2 * sympy.sin(2 * pi * y)
        v = sympy.sin(2 * pi * x) * sympy.sin(pi * y) ** 2 * sympy.Rational(1, 3)
        p = sympy.cos(pi * x) * sympy.cos(pi * y)
        mu = 1 + sympy.Rational(1, 2) * x * y
        gam = 1 + x * x
        rho = 1 + sympy.Rational(3, 10) * x
    theta = 1
    dv = sympy.diff(u, x) + sympy.diff(v, y)
    lam = gam - sympy.Rational(2, 3) * mu
    fx = 2 * sympy.diff(mu * sympy.diff(u, x), x) + sympy.diff(mu * (sympy.diff(u, y) + sympy.diff(v, x)), y) \
        + sympy.diff(lam * dv, x)
    fy = 2 * sympy.diff(mu * sympy.diff(v, y), y) + sympy.diff(mu * (sympy.diff(v, x) + sympy.diff(u, y)), x) \
        + sympy.diff(lam * dv, y)
    f1 = theta * rho * u - fx + sympy.diff(p, x)
    f2 = theta * rho * v - fy + sympy.diff(p, y)
    fns = {k: sympy.lambdify((x, y), e, "numpy") for k, e in
           dict(u=u, v=v, p=p, mu=mu, gam=gam, rho=rho, f1=f1, f2=f2, g=dv).items()}
    return fns, theta


@pytest.mark.parametrize("bc_kind", ["periodic", "noslip"])
def test_bulk_manufactured_solution_second_order(bc_kind):
    """A compressible (div u = g != 0) manufactured solution with variable
    rho, mu and gamma converges at second order (Sec. 3.1 discretisation of
    the bulk-viscosity stress)."""
    fns, theta = _mms(bc_kind)
    bc = (PERIODIC,) * 4 if bc_kind == "periodic" else (NOSLIP,) * 4
    errs = []
    for n in (16, 32, 64):
        h = 1.0 / n
        g = Grid(2, (n, n), h, bc)
        xc = (np.arange(n) + 0.5) * h
        Xc, Yc = np.meshgrid(xc, xc)
        Xu, Yu = np.meshgrid(np.arange(g.face_ext[0][0]) * h, xc)
        Xv, Yv = np.meshgrid(xc, np.arange(g.face_ext[1][1]) * h)
        F = lambda k, X, Y: fns[k](X, Y) + 0 * X
        M = asm.stokes_from_fields(g, F("rho", Xc, Yc)[None], F("mu", Xc, Yc)[None], theta,
                                   gamma=F("gam", Xc, Yc)[None])
        gg = F("g", Xc, Yc)
        b = g.pack([F("f1", Xu, Yu)[None], F("f2", Xv, Yv)[None]], -(gg - gg.mean())[None])
        b[~g.active] = 0.0
        xs = direct.solve(g, M, b)
        ue = g.pack([F("u", Xu, Yu)[None], F("v", Xv, Yv)[None]], F("p", Xc, Yc)[None])
        ue[~g.active] = 0.0
        errs.append(direct.relative_error(g, xs, ue))
    errs = np.array(errs)
    order = np.log2(errs[:-1] / errs[1:])
    assert (order > 1.8).all(), (errs, order)
