"""Pins of the oracle's discrete operators against what Sec. 3.1, App. A and
App. B of the paper fix."""
import itertools

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import assemble as asm
from oracle import direct, fourier
from oracle.grid import Grid, PERIODIC, NOSLIP, FREESLIP
from paper_1308_4605_gb300 import workloads as wl

BCS_2D = [(PERIODIC,) * 4, (NOSLIP,) * 4, (FREESLIP,) * 4, (NOSLIP, FREESLIP, PERIODIC, PERIODIC),
          (PERIODIC, PERIODIC, FREESLIP, NOSLIP), (NOSLIP, NOSLIP, FREESLIP, FREESLIP)]
BCS_3D = [(PERIODIC,) * 6, (NOSLIP,) * 6, (FREESLIP,) * 6, (NOSLIP, NOSLIP, PERIODIC, PERIODIC, FREESLIP, NOSLIP)]
CASES = [(2, (8, 4), bc) for bc in BCS_2D] + [(3, (4, 4, 8), bc) for bc in BCS_3D]


def _fields(g, seed):
    rng = np.random.default_rng(seed)
    return (np.exp(rng.standard_normal(g.cell_shape())),
            np.exp(rng.standard_normal(g.cell_shape())))


@pytest.mark.parametrize("dim,n,bc", CASES)
def test_divergence_is_minus_gradient_transpose(dim, n, bc):
    """D = -G^* for periodic, no-slip and free-slip boundaries (Sec. 3.1)."""
    g = Grid(dim, n, 0.5, bc)
    D, G = asm.divergence(g), asm.gradient(g)
    assert abs(D + G.T).max() == 0.0


@pytest.mark.parametrize("dim,n,bc", CASES)
def test_DG_is_standard_laplacian(dim, n, bc):
    """D G = L_p, the 5-point (2D) / 7-point (3D) Laplacian (Sec. 3.1), written
    here point by point with no flux through walls."""
    g = Grid(dim, n, 0.5, bc)
    DG = (asm.divergence(g) @ asm.gradient(g)).toarray()
    ref = np.zeros((g.ncell, g.ncell))
    h2 = g.h ** 2
    for c in itertools.product(*[range(g.n[a]) for a in range(3)]):
        row = int(g.cell_id([np.array(c[0]), np.array(c[1]), np.array(c[2])], offset=False))
        for a in range(dim):
            for s in (-1, 1):
                nb = list(c)
                nb[a] += s
                if not g.periodic[a] and not (0 <= nb[a] < g.n[a]):
                    continue
                col = int(g.cell_id([np.array(v) for v in nb], offset=False))
                ref[row, col] += 1.0 / h2
                ref[row, row] -= 1.0 / h2
    assert np.abs(DG - ref).max() < 1e-12


@pytest.mark.parametrize("dim,n,bc", CASES)
def test_viscous_operator_symmetric_negative_semidefinite(dim, n, bc):
    g = Grid(dim, n, 1.0, bc)
    rho, mu = _fields(g, 3)
    c = asm.fine_coefficients(g, rho, mu, 1.0)
    L = asm.viscous(g, c["mu_c"], c["mu_e"])
    assert abs(L - L.T).max() <= 1e-14 * abs(L).max()
    va = g.active[:g.nvel]
    ev = np.linalg.eigvalsh(L[va][:, va].toarray())
    assert ev.max() <= 1e-12 * abs(ev).max()
    M = asm.stokes_operator(g, c)
    assert abs(M - M.T).max() <= 1e-14 * abs(M).max()      # M = M^* (Sec. 2)


def _div_free_velocity(g, seed):
    """u = curl psi with psi on nodes (2D); psi = 0 on walls so that u . n = 0."""
    rng = np.random.default_rng(seed)
    ext = g.edge_ext(0, 1)
    psi = rng.standard_normal((1, ext[1], ext[0]))
    if not g.periodic[0]:
        psi[:, :, 0] = psi[:, :, -1] = 0.0
    if not g.periodic[1]:
        psi[:, 0, :] = psi[:, -1, :] = 0.0
    h = g.h
    u = np.zeros(g.face_shape(0))
    v = np.zeros(g.face_shape(1))
    for j in range(g.n[1]):
        for i in range(g.face_ext[0][0]):
            u[0, j, i] = (psi[0, (j + 1) % ext[1], i] - psi[0, j, i]) / h
    for j in range(g.face_ext[1][1]):
        for i in range(g.n[0]):
            v[0, j, i] = -(psi[0, j, (i + 1) % ext[0]] - psi[0, j, i]) / h
    return g.pack([u, v], np.zeros(g.cell_shape()))[:g.nvel]


@pytest.mark.parametrize("bc", BCS_2D)
def test_constant_viscosity_stress_form_reduces_to_laplacian(bc):
    """For constant mu0 and D u = 0, L_mu u = mu0 L u (Sec. 3.1)."""
    g = Grid(2, (8, 8), 1.0, bc)
    mu0 = 1.7
    one = np.ones(g.cell_shape())
    c = asm.fine_coefficients(g, one, mu0 * one, 0.0)
    u = _div_free_velocity(g, 4)
    assert np.abs(asm.divergence(g) @ u).max() < 1e-12
    Ls = asm.viscous(g, c["mu_c"], c["mu_e"], "stress")
    Ll = asm.viscous(g, c["mu_c"], c["mu_e"], "laplacian")
    assert np.abs(Ls @ u - Ll @ u).max() < 1e-12 * np.abs(Ll @ u).max()


@pytest.mark.parametrize("dim,n", [(2, (8, 8)), (3, (4, 4, 4))])
def test_schur_complement_constant_viscosity_periodic(dim, n):
    """App. A: (D L_mu^{-1} G)^{-1} = 2 mu0 (stress form) and mu0 (Laplacian
    form) on every non-constant pressure mode of a periodic grid."""
    g = Grid(dim, n, 1.0, (PERIODIC,) * 6)
    mu0 = 0.8
    one = np.ones(g.cell_shape())
    c = asm.fine_coefficients(g, one, mu0 * one, 0.0)
    D, G = asm.divergence(g).toarray(), asm.gradient(g).toarray()
    for form, expect in (("stress", 2 * mu0), ("laplacian", mu0)):
        L = asm.viscous(g, c["mu_c"], c["mu_e"], form).toarray()
        S = D @ np.linalg.pinv(L, rcond=1e-10) @ G
        ev = np.sort(np.linalg.eigvalsh(0.5 * (S + S.T)))
        assert abs(ev[0]) < 1e-10
        assert np.allclose(ev[1:], 1.0 / expect, rtol=1e-10)
        sym = fourier.schur_symbol(g, mu0, form)
        assert np.nanmax(np.abs(sym - expect)) < 1e-12


@pytest.mark.parametrize("dim,n,theta", [(2, (16, 8), 1.5), (3, (8, 4, 8), 0.7), (2, (8, 8), 0.0)])
def test_fourier_closed_form_matches_direct_solve(dim, n, theta):
    """Constant coefficients on a periodic grid: the mode-by-mode solve of
    App. A equals the sparse direct solve of the assembled M."""
    g = Grid(dim, n, 0.5, (PERIODIC,) * 6)
    rho0, mu0 = 2.0, 3.0
    one = np.ones(g.cell_shape())
    M = asm.stokes_from_fields(g, rho0 * one, mu0 * one, theta)
    u, p = wl.random_face_vector(g.n, g.bc, dim, 1)
    p -= p.mean()
    if theta == 0.0:
        u = [x - x.mean() for x in u]      # steady periodic: velocity fixed up to a constant
    b = M @ g.pack(u, p)
    xf = fourier.solve_periodic(g, rho0, mu0, theta, b)
    if theta == 0.0:
        assert np.abs(M @ xf - b).max() < 1e-11 * np.abs(b).max()
        return
    xd = direct.solve(g, M, b)
    assert np.abs(xf - xd).max() < 1e-11 * np.abs(xd).max()


@pytest.mark.parametrize("dim,n,bc", [(2, (8, 8), (NOSLIP,) * 4), (2, (16, 8), (PERIODIC, PERIODIC, NOSLIP, FREESLIP)),
                                      (3, (4, 4, 4), (NOSLIP,) * 6)])
def test_direct_solve_recovers_random_solution(dim, n, bc):
    """Sec. 4: random x, b = M x; the solve returns x (pressure up to a constant)."""
    g = Grid(dim, n, 1.0, bc)
    rho, mu = _fields(g, 7)
    M = asm.stokes_from_fields(g, rho, mu, 1.0)
    u, p = wl.random_face_vector(g.n, g.bc, dim, 2)
    x = g.pack(u, p - p.mean())
    b = M @ x
    xs = direct.solve(g, M, b, dense=True)
    xsp = direct.solve(g, M, b, dense=False)
    assert max(direct.relative_error(g, xs, x)) < 1e-11
    assert max(direct.relative_error(g, xsp, x)) < 1e-11


@pytest.mark.slow
def test_eigenvalues_32x32_no_slip():
    """App. B.1 on 32^2 cells with four no-slip walls, steady, mu = 1:
    N_dof = 3008; M has exactly 1024 eigenvalues <= 0; the Schur complement
    S = D L^{-1} G (Laplacian form) has spectrum in {0} u (0, 1] with one zero
    and at most 2(nx-1) + 2(ny-1) = 124 non-unit eigenvalues; with the stress
    form and S~^{-1} = 2 mu the count of non-unit eigenvalues is the same ~4%."""
    g = Grid(2, (32, 32), 1.0, (NOSLIP,) * 4)
    one = np.ones(g.cell_shape())
    c = asm.fine_coefficients(g, one, one, 0.0)
    M = asm.stokes_operator(g, c)
    act = g.active
    assert act.sum() == 3008
    ev = np.linalg.eigvalsh(M[act][:, act].toarray())
    assert (ev <= 1e-10).sum() == 1024
    assert (ev < -1e-10).sum() == 1023
    va = act[:g.nvel]
    G = asm.gradient(g)[va].toarray()
    D = asm.divergence(g)[:, va].toarray()
    for form, fac in (("laplacian", 1.0), ("stress", 2.0)):
        A = asm.velocity_operator(g, c, form)[va][:, va].toarray()
        S = -D @ np.linalg.solve(A, G)
        lam = np.sort(np.linalg.eigvals(fac * S).real)
        assert (np.abs(lam) < 1e-10).sum() == 1
        assert (np.abs(lam - 1.0) > 1e-8).sum() <= 124
        assert lam.max() <= 1.0 + 1e-10
        assert lam[1] > 0.2          # bounded away from zero (inf-sup)


def _mms_case(bc_kind):
    sympy = pytest.importorskip("sympy")
    x, y = sympy.symbols("x y")
    pi = sympy.pi
    if bc_kind == "periodic":
        u = sympy.sin(2 * pi * x) * sympy.cos(2 * pi * y)
        v = sympy.cos(2 * pi * x) * sympy.sin(4 * pi * y) * sympy.Rational(1, 2)
        p = sympy.cos(2 * pi * x) * sympy.cos(2 * pi * y)
        mu = 1 + sympy.Rational(1, 2) * sympy.sin(2 * pi * x) * sympy.sin(2 * pi * y)
        rho = 1 + sympy.Rational(3, 10) * sympy.cos(2 * pi * x)
    else:
        u = sympy.sin(pi * x) ** 2 * sympy.sin(2 * pi * y)
        v = -sympy.sin(2 * pi * x) * sympy.sin(pi * y) ** 2 * sympy.Rational(1, 2)
        p = sympy.cos(pi * x) * sympy.cos(pi * y)
        mu = 1 + sympy.Rational(1, 2) * x * y
        rho = 1 + sympy.Rational(3, 10) * x
    theta = 1
    # div mu (grad u + grad u^T), Eq. div_stress
    fx = 2 * sympy.diff(mu * sympy.diff(u, x), x) + sympy.diff(mu * (sympy.diff(u, y) + sympy.diff(v, x)), y)
    fy = 2 * sympy.diff(mu * sympy.diff(v, y), y) + sympy.diff(mu * (sympy.diff(v, x) + sympy.diff(u, y)), x)
    f1 = theta * rho * u - fx + sympy.diff(p, x)
    f2 = theta * rho * v - fy + sympy.diff(p, y)
    gdiv = sympy.diff(u, x) + sympy.diff(v, y)
    lam = {k: sympy.lambdify((x, y), e, "numpy") for k, e in
           dict(u=u, v=v, p=p, mu=mu, rho=rho, f1=f1, f2=f2, g=gdiv).items()}
    return lam, theta


@pytest.mark.parametrize("bc_kind", ["periodic", "noslip"])
def test_manufactured_solution_second_order(bc_kind):
    """The discretisation is globally second-order accurate (Sec. 3.1)."""
    lam, theta = _mms_case(bc_kind)
    bc = (PERIODIC,) * 4 if bc_kind == "periodic" else (NOSLIP,) * 4
    errs = []
    for n in (16, 32, 64):
        h = 1.0 / n
        g = Grid(2, (n, n), h, bc)
        xc = (np.arange(n) + 0.5) * h
        Xc, Yc = np.meshgrid(xc, xc)
        xf = np.arange(g.face_ext[0][0]) * h
        Xu, Yu = np.meshgrid(xf, xc)
        Xv, Yv = np.meshgrid(xc, np.arange(g.face_ext[1][1]) * h)
        rho = lam["rho"](Xc, Yc) + 0 * Xc
        mu = lam["mu"](Xc, Yc) + 0 * Xc
        M = asm.stokes_from_fields(g, rho[None], mu[None], theta)
        f1 = lam["f1"](Xu, Yu) + 0 * Xu
        f2 = lam["f2"](Xv, Yv) + 0 * Xv
        gg = lam["g"](Xc, Yc) + 0 * Xc
        b = g.pack([f1[None], f2[None]], -(gg - gg.mean())[None])
        b[~g.active] = 0.0
        x = direct.solve(g, M, b)
        ue = g.pack([lam["u"](Xu, Yu)[None] + 0 * Xu, lam["v"](Xv, Yv)[None] + 0 * Xv],
                    (lam["p"](Xc, Yc) + 0 * Xc)[None])
        ue[~g.active] = 0.0
        errs.append(direct.relative_error(g, x, ue))
    errs = np.array(errs)
    order = np.log2(errs[:-1] / errs[1:])
    assert (order > 1.8).all(), (errs, order)
