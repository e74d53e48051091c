"""Pins of the oracle's adjoint gradient: brute-force derivatives of the
assembled operator (M is affine in mu and rho) and central finite differences
of the loss through direct solves."""
import numpy as np
import pytest

from oracle import assemble as asm
from oracle import direct, gradient
from oracle.grid import Grid, PERIODIC, NOSLIP, FREESLIP
from paper_1308_4605_gb300 import workloads as wl

CASES = [(2, (4, 4), (NOSLIP,) * 4), (2, (8, 4), (PERIODIC, PERIODIC, FREESLIP, NOSLIP)),
         (3, (4, 4, 4), (NOSLIP,) * 6), (3, (4, 2, 4), (PERIODIC, PERIODIC, NOSLIP, FREESLIP, FREESLIP, NOSLIP))]


@pytest.mark.parametrize("dim,n,bc", CASES)
def test_viscosity_gradient_is_the_derivative(dim, n, bc):
    """lambda^T L_mu u is linear in mu: its derivative in mu_c is
    lambda^T L_mu(e_c) u, with L_mu(e_c) assembled for the unit field."""
    g = Grid(dim, n, 1.0, bc)
    rng = np.random.default_rng(2)
    mu = np.exp(rng.standard_normal(g.cell_shape()))
    u = rng.standard_normal(g.nvel) * g.active[:g.nvel]
    lam = rng.standard_normal(g.nvel) * g.active[:g.nvel]
    got = gradient.viscosity_gradient(g, mu, u, lam)
    ref = np.zeros(g.ncell)
    for c in range(g.ncell):
        e = np.zeros(g.ncell)
        e[c] = 1.0
        L = asm.viscous(g, e.reshape(g.cell_shape()), asm.edge_viscosity(g, e))
        ref[c] = lam @ (L @ u)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("dim,n,bc", CASES)
def test_density_gradient_is_the_derivative(dim, n, bc):
    g = Grid(dim, n, 1.0, bc)
    rng = np.random.default_rng(3)
    u = rng.standard_normal(g.nvel) * g.active[:g.nvel]
    lam = rng.standard_normal(g.nvel) * g.active[:g.nvel]
    theta = 1.7
    got = gradient.density_gradient(g, theta, u, lam)
    ref = np.zeros(g.ncell)
    for c in range(g.ncell):
        e = np.zeros(g.ncell)
        e[c] = 1.0
        rf = np.concatenate([x.ravel() for x in asm.face_density(g, e.reshape(g.cell_shape()))])
        ref[c] = -theta * lam @ (rf * u)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("dim,n,bc,theta", [(2, (8, 8), (NOSLIP,) * 4, 0.0),
                                            (3, (4, 4, 4), (PERIODIC,) * 6, 1.0),
                                            (2, (8, 8), (FREESLIP, NOSLIP, PERIODIC, PERIODIC), 0.5)])
def test_gradient_matches_finite_differences(dim, n, bc, theta):
    """L = 1/2 ||u - u_t||^2: central differences along random directions in
    log mu and rho agree with the adjoint gradient to 1e-6."""
    pr = wl.generic(dim, n, bc, theta=theta, rho_contrast=5.0, mu_contrast=20.0, seed=21)
    g = Grid(dim, pr.n, pr.h, pr.bc)
    b = g.pack(pr.b_u, pr.b_p)
    rng = np.random.default_rng(5)
    u_t = rng.standard_normal(g.nvel) * g.active[:g.nvel]
    solve = lambda M, r: direct.solve(g, M, r, dense=True)
    L, glogmu, grho, _, _ = gradient.loss_and_gradient(g, pr.rho, pr.mu, theta, b, u_t, solve)
    eps = 1e-5

    def loss(rho, mu):
        return gradient.loss_and_gradient(g, rho, mu, theta, b, u_t, solve)[0]

    for k in range(3):
        d = rng.standard_normal(g.cell_shape())
        d /= np.linalg.norm(d)
        fd = (loss(pr.rho, pr.mu * np.exp(eps * d)) - loss(pr.rho, pr.mu * np.exp(-eps * d))) / (2 * eps)
        assert abs(fd - glogmu @ d.ravel()) <= 1e-6 * abs(fd) + 1e-12 * abs(L)
        if theta != 0.0:
            fd = (loss(pr.rho + eps * d, pr.mu) - loss(pr.rho - eps * d, pr.mu)) / (2 * eps)
            assert abs(fd - grho @ d.ravel()) <= 1e-6 * abs(fd) + 1e-12 * abs(L)
