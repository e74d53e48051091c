"""Inhomogeneous velocity boundary conditions on the GPU
(stk_subtract_boundary_terms) against the oracle's boundary terms, and
solves of problems with moving walls and through-flow."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import assemble as asm
from oracle import boundary as bd
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


def _random_data(g, rng):
    uw = rng.standard_normal(g.nvel) * (~g.active[:g.nvel])
    tan = {}
    for d in range(g.dim):
        if g.periodic[d]:
            continue
        for side in (0, 1):
            if g.bc[2 * d + side] != NOSLIP:
                continue
            for a in range(g.dim):
                if a != d:
                    ext = [g.face_ext[a][c] for c in range(3) if c != d]
                    tan[(d, side, a)] = rng.standard_normal(ext[0] * ext[1])
    return uw, tan


@pytest.mark.parametrize("dim,n,bc,bulk", [
    (2, (16, 8), (NOSLIP, NOSLIP, NOSLIP, NOSLIP), False),
    (2, (8, 16), (NOSLIP, FREESLIP, PERIODIC, PERIODIC), True),
    (3, (8, 4, 8), (NOSLIP, NOSLIP, FREESLIP, NOSLIP, PERIODIC, PERIODIC), False),
    (3, (4, 8, 8), (NOSLIP,) * 6, True),
])
def test_boundary_terms_match_oracle(S, dim, n, bc, bulk):
    pr = wl.generic(dim, n, bc, theta=0.7, seed=81)
    g = Grid(dim, pr.n, pr.h, pr.bc)
    rng = np.random.default_rng(5)
    gamma = np.exp(rng.standard_normal(pr.mu.shape)) if bulk else None
    coef = asm.fine_coefficients(g, pr.rho, pr.mu, pr.theta, gamma)
    uw, tan = _random_data(g, rng)
    ref = -bd.boundary_terms(g, coef, uw, tan)
    sv = S.StokesSolver(dim, pr.n[:dim], pr.bc[:2 * dim], pr.h)
    sv.set_coefficients(_t(pr.rho), _t(pr.mu), pr.theta)
    if bulk:
        sv.set_bulk_viscosity(_t(gamma))
    b_u, b_p = sv.zeros()
    wu, _ = g.unpack(np.concatenate([uw, np.zeros(g.ncell)]))
    sv.subtract_boundary_terms(b_u, b_p, u_wall=[_t(x) for x in wu],
                               u_tan={k: _t(v) for k, v in tan.items()})
    got = g.pack([x.cpu().numpy() for x in b_u], b_p.cpu().numpy())
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()
    sv.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_lid_driven_cavity_and_through_flow(S, precision):
    """A lid-driven cavity (top wall moving, walls all around, variable mu,
    steady) and a channel with a parabolic inflow / outflow profile: GPU
    solves of M x = b - c equal the oracle's direct solves to 1e-8."""
    n = 32
    g = Grid(2, (n, n), 1.0 / n, (NOSLIP,) * 4)
    pr = wl.generic(2, (n, n), (NOSLIP,) * 4, theta=0.0, mu_contrast=20.0, seed=82, h=1.0 / n)
    coef = asm.fine_coefficients(g, pr.rho, pr.mu, 0.0)
    M = asm.stokes_operator(g, coef)
    xf = np.arange(g.face_ext[0][0]) * g.h
    yc = (np.arange(n) + 0.5) * g.h
    cases = {
        "cavity": (np.zeros(g.nvel), {(1, 1, 0): np.sin(np.pi * xf) ** 2}),
        "channel": None,
    }
    # channel: inflow u = 4 y (1 - y) on x = 0 and the same outflow on x = 1
    uw = np.zeros(g.nvel)
    idx = g.face_positions(0)
    prof = 4.0 * ((idx[1] + 0.5) * g.h) * (1.0 - (idx[1] + 0.5) * g.h)
    wall = (idx[0] == 0) | (idx[0] == n)
    uw[:len(idx[0])][wall] = prof[wall]
    cases["channel"] = (uw, {})
    sv = S.StokesSolver(2, (n, n), (NOSLIP,) * 4, g.h)
    sv.set_coefficients(_t(pr.rho), _t(pr.mu), 0.0)
    for name, (uw, tan) in cases.items():
        c = bd.boundary_terms(g, coef, uw, tan)
        b = -c
        xd = direct.solve(g, M, b)
        b_u, b_p = sv.zeros()
        wu, _ = g.unpack(np.concatenate([uw, np.zeros(g.ncell)]))
        sv.subtract_boundary_terms(b_u, b_p, u_wall=[_t(x) for x in wu],
                                   u_tan={k: _t(v) for k, v in tan.items()})
        x_u, x_p, info = sv.solve(b_u, b_p, precond=2, precision=precision, maxit=2000)
        assert info["converged"], (name, info)
        x = g.pack([a.cpu().numpy() for a in x_u], x_p.cpu().numpy())
        assert max(direct.relative_error(g, x, xd)) <= 1e-8, name
    sv.close()
