"""Pins of the oracle's backward-Euler time loop (Sec. 2, Eq. Stokes_eqn):
energy decay, the exact decay factor of a Fourier mode, and the steady
limit."""
import numpy as np
import pytest

from oracle import assemble as asm
from oracle import direct, timeloop
from oracle.grid import Grid, PERIODIC, NOSLIP, FREESLIP


def _fields(g, seed, s=0.5):
    rng = np.random.default_rng(seed)
    return (np.exp(s * rng.standard_normal(g.cell_shape())),
            np.exp(s * rng.standard_normal(g.cell_shape())), rng)


@pytest.mark.parametrize("bc", [(NOSLIP, NOSLIP, FREESLIP, NOSLIP), (PERIODIC,) * 4])
def test_energy_never_grows(bc):
    """Unforced, divergence-free: <rho_f u^{n+1}, u^{n+1}> <= <rho_f u^n, u^n>
    (multiply the momentum equation by u^{n+1}: the pressure term vanishes,
    -<L_mu u, u> >= 0)."""
    g = Grid(2, (16, 16), 1.0, bc)
    rho, mu, rng = _fields(g, 3)
    # a divergence-free start: the velocity of a steady solve (D u = 0)
    M0 = asm.stokes_from_fields(g, rho, mu, 1.0)
    b = rng.standard_normal(g.size) * g.active
    b[g.nvel:] = 0.0
    u0 = direct.solve(g, M0, b)[:g.nvel]
    D = asm.divergence(g)
    assert np.abs(D @ u0).max() < 1e-10 * np.abs(u0).max()
    rf = timeloop.face_density_vector(g, rho)
    E = [rf @ (u0 * u0)]
    for x in timeloop.backward_euler(g, rho, mu, 0.5, u0, 8):
        u = x[:g.nvel]
        E.append(rf @ (u * u))
    assert all(E[i + 1] <= E[i] * (1 + 1e-13) for i in range(len(E) - 1)), E
    assert E[-1] < 0.9 * E[0]


@pytest.mark.parametrize("k", [1, 3])
def test_fourier_mode_decay_factor(k):
    """Constant rho0, mu0 on a periodic n x n grid: u = (sin(2 pi k y / L), 0)
    is divergence-free with p = 0, and each step divides it by
    1 + dt mu0 lambda_h / rho0, lambda_h = (4/h^2) sin^2(pi k / n)."""
    n, h, rho0, mu0, dt = 16, 0.5, 2.0, 0.7, 0.3
    g = Grid(2, (n, n), h, (PERIODIC,) * 4)
    rho = np.full(g.cell_shape(), rho0)
    mu = np.full(g.cell_shape(), mu0)
    L = n * h
    y = (np.arange(n) + 0.5) * h
    ux = np.repeat(np.sin(2 * np.pi * k * y / L)[:, None], n, axis=1)   # (j, i)
    u0 = g.pack([ux, np.zeros((n, n))], np.zeros(g.ncell))[:g.nvel]
    lam = 4.0 / h ** 2 * np.sin(np.pi * k / n) ** 2
    fac = 1.0 / (1.0 + dt * mu0 * lam / rho0)
    xs = timeloop.backward_euler(g, rho, mu, dt, u0, 3)
    for s, x in enumerate(xs, start=1):
        assert np.abs(x[:g.nvel] - fac ** s * u0).max() <= 1e-12
        p = x[g.nvel:]
        assert np.abs(p - p.mean()).max() <= 1e-12


def test_steady_limit():
    """With time-independent forcing and divergence source the steps
    converge to the steady solution (theta = 0), pressure included."""
    g = Grid(2, (8, 8), 1.0, (NOSLIP,) * 4)
    rho, mu, rng = _fields(g, 5)
    f = rng.standard_normal(g.nvel) * g.active[:g.nvel]
    bp = rng.standard_normal(g.ncell)
    bp -= bp.mean()
    xs = timeloop.backward_euler(g, rho, mu, 50.0, np.zeros(g.nvel), 60, f=f, b_p=bp)
    Ms = asm.stokes_from_fields(g, rho, mu, 0.0)
    xsteady = direct.solve(g, Ms, np.concatenate([f, bp]))
    eu, ep = direct.relative_error(g, xs[-1], xsteady)
    assert eu <= 1e-8 and ep <= 1e-8, (eu, ep)
