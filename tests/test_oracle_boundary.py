"""Pins of the oracle's boundary terms for inhomogeneous velocity boundary
conditions (Sec. 3.2): exact Couette and through-flow solutions in 2D and
3D, and second-order convergence of a manufactured solution with non-zero
wall values."""
import numpy as np
import pytest

from oracle import assemble as asm
from oracle import boundary as bd
from oracle import direct
from oracle.grid import Grid, PERIODIC, NOSLIP, FREESLIP


def _wall_vector(g, fn):
    """Packed velocity vector with fn(a, x, y, z) at the wall faces."""
    u = np.zeros(g.nvel)
    h = g.h
    for a in range(g.dim):
        if g.periodic[a]:
            continue
        idx = g.face_positions(a)
        X = [(idx[c] + (0.0 if c == a else 0.5)) * h for c in range(3)]
        wall = (idx[a] == 0) | (idx[a] == g.n[a])
        st = g.offsets[a] + g._flat(g.face_ext[a], [v[wall] for v in idx])
        u[st] = fn(a, *(v[wall] for v in X))
    return u


def _tangential(g, fn):
    """tan[(d, side, a)] from fn(a, x, y, z) on the no-slip walls."""
    out = {}
    h = g.h
    for d in range(g.dim):
        if g.periodic[d]:
            continue
        for side in (0, 1):
            if g.bc[2 * d + side] != NOSLIP:
                continue
            for a in range(g.dim):
                if a == d:
                    continue
                ext = list(g.face_ext[a])
                ext[d] = 1
                k, j, i = np.meshgrid(np.arange(ext[2]), np.arange(ext[1]), np.arange(ext[0]), indexing="ij")
                pos = [i, j, k]
                X = [(pos[c] + (0.0 if c == a else 0.5)) * h for c in range(3)]
                X[d] = np.full(i.shape, 0.0 if side == 0 else g.n[d] * h)
                out[(d, side, a)] = fn(a, *X).reshape(-1)
    return out


@pytest.mark.parametrize("dim", [2, 3])
def test_couette_flow_is_exactly_linear(dim):
    """Walls normal to the last axis, the upper one moving with U0 along x:
    the steady solution is u_x = U0 z / L exactly (the one-sided wall
    derivative is exact for linear profiles), other components and the
    pressure gradient zero."""
    n = (8, 4) if dim == 2 else (4, 4, 8)
    d = dim - 1
    bc = [PERIODIC] * 6
    bc[2 * d] = bc[2 * d + 1] = NOSLIP
    g = Grid(dim, n, 0.25, bc)
    mu = np.full(g.cell_shape(), 1.7)
    coef = asm.fine_coefficients(g, np.ones(g.cell_shape()), mu, 0.0)
    M = asm.stokes_operator(g, coef)
    L = g.n[d] * g.h
    U0 = 0.8
    tan = _tangential(g, lambda a, x, y, z: (U0 if a == 0 else 0.0) * ((y if d == 1 else z) > 0))
    c = bd.boundary_terms(g, coef, np.zeros(g.nvel), tan)
    x = direct.solve(g, M, -c)
    idx = g.face_positions(0)
    zc = (idx[d] + 0.5) * g.h
    ux = x[:int(np.prod(g.face_ext[0]))]
    assert np.abs(ux - U0 * zc / L).max() <= 1e-12
    assert np.abs(x[int(np.prod(g.face_ext[0])):g.nvel]).max() <= 1e-12
    p = x[g.nvel:]
    assert np.abs(p - p.mean()).max() <= 1e-11


@pytest.mark.parametrize("dim", [2, 3])
def test_uniform_through_flow_is_exact(dim):
    """Inflow and outflow walls normal to x with normal velocity U0, the
    other axes periodic, variable mu and rho, steady: u = (U0, 0, 0) and a
    constant pressure solve the inhomogeneous problem exactly."""
    n = (8, 4) if dim == 2 else (8, 4, 4)
    bc = [PERIODIC] * 6
    bc[0] = bc[1] = NOSLIP
    g = Grid(dim, n, 0.5, bc)
    rng = np.random.default_rng(3)
    mu = np.exp(rng.standard_normal(g.cell_shape()))
    rho = np.exp(rng.standard_normal(g.cell_shape()))
    coef = asm.fine_coefficients(g, rho, mu, 0.0)
    M = asm.stokes_operator(g, coef)
    U0 = 1.3
    uw = _wall_vector(g, lambda a, x, y, z: U0 if a == 0 else 0.0)
    c = bd.boundary_terms(g, coef, uw, {})
    x = direct.solve(g, M, -c)
    ux = x[:int(np.prod(g.face_ext[0]))]
    interior = g.active[:int(np.prod(g.face_ext[0]))]
    assert np.abs(ux[interior] - U0).max() <= 1e-12
    assert np.abs(x[int(np.prod(g.face_ext[0])):g.nvel]).max() <= 1e-12


def test_inhomogeneous_manufactured_solution_second_order():
    """u, v that do not vanish on the walls (normal and tangential wall values
    from the exact solution), variable rho, mu and gamma: second-order
    convergence of the inhomogeneous problem."""
    sympy = pytest.importorskip("sympy")
    x, y = sympy.symbols("x y")
    pi = sympy.pi
    u = sympy.cos(pi * x) * sympy.sin(pi * y) + x
    v = sympy.sin(pi * x) * sympy.cos(2 * pi * y) - y * y
    p = sympy.sin(pi * x) * sympy.sin(pi * y)
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
    F = {k: sympy.lambdify((x, y), e, "numpy") for k, e in
         dict(u=u, v=v, p=p, mu=mu, gam=gam, rho=rho, g=dv,
              f1=theta * rho * u - fx + sympy.diff(p, x), f2=theta * rho * v - fy + sympy.diff(p, y)).items()}
    E = lambda k, X, Y: F[k](X, Y) + 0 * X
    bc = (NOSLIP,) * 4
    errs = []
    for n in (16, 32, 64):
        h = 1.0 / n
        g = Grid(2, (n, n), h, bc)
        xc = (np.arange(n) + 0.5) * h
        Xc, Yc = np.meshgrid(xc, xc)
        Xu, Yu = np.meshgrid(np.arange(g.face_ext[0][0]) * h, xc)
        Xv, Yv = np.meshgrid(xc, np.arange(g.face_ext[1][1]) * h)
        coef = asm.fine_coefficients(g, E("rho", Xc, Yc)[None], E("mu", Xc, Yc)[None], theta,
                                     E("gam", Xc, Yc)[None])
        M = asm.stokes_operator(g, coef)
        ue = g.pack([E("u", Xu, Yu)[None], E("v", Xv, Yv)[None]], E("p", Xc, Yc)[None])
        uw = ue[:g.nvel].copy()
        tan = _tangential(g, lambda a, X, Y, Z: E("u" if a == 0 else "v", X, Y))
        c = bd.boundary_terms(g, coef, uw, tan)
        gg = E("g", Xc, Yc)
        b = g.pack([E("f1", Xu, Yu)[None], E("f2", Xv, Yv)[None]], -gg[None])
        b = b - c
        b[~g.active] = 0.0
        b[g.nvel:] -= b[g.nvel:].mean()      # compatibility (net wall flux = integral of g) up to O(h^2)
        xs = direct.solve(g, M, b)
        ue[~g.active] = 0.0
        errs.append(direct.relative_error(g, xs, ue))
    errs = np.array(errs)
    order = np.log2(errs[:-1] / errs[1:])
    assert (order > 1.8).all(), (errs, order)
