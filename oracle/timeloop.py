"""Backward-Euler time stepping (Sec. 2, Eq. Stokes_eqn) with direct solves.

Test infrastructure: only tests and the benchmark's CPU baseline use it.

Step n -> n+1: M(theta = 1/dt) x = (theta rho_f u^n + f, b_p) with rho_f the
face densities (mean of the two adjacent cells, Sec. 3.1), zero on wall
faces; x^{n+1} = the exact discrete solution (direct.solve).

Parity: pinned (tests/test_oracle_timeloop.py: the kinetic energy
1/2 sum rho_f u^2 of unforced divergence-free flow never grows; a
divergence-free Fourier mode of constant-coefficient periodic flow decays
by exactly 1/(1 + dt mu lambda_h / rho) per step, lambda_h the eigenvalue of
the discrete Laplacian; with steady forcing the steps converge to the
steady solution).
"""
from __future__ import annotations

import numpy as np

from . import assemble as asm
from . import direct
from .grid import Grid


def face_density_vector(grid: Grid, rho):
    return np.concatenate([np.asarray(r).ravel() for r in asm.face_density(grid, rho)])


def backward_euler(grid: Grid, rho, mu, dt, u0, nsteps, f=None, b_p=None):
    """u0: packed velocity (length nvel).  Returns the list of packed Stokes
    vectors x^1..x^nsteps."""
    theta = 1.0 / dt
    M = asm.stokes_from_fields(grid, rho, mu, theta)
    rf = face_density_vector(grid, rho)
    act = grid.active[:grid.nvel]
    u = np.asarray(u0, dtype=np.float64).copy()
    bp = np.zeros(grid.ncell) if b_p is None else np.asarray(b_p, dtype=np.float64).ravel()
    out = []
    for n in range(1, nsteps + 1):
        fn = f(n) if callable(f) else (np.zeros(grid.nvel) if f is None else f)
        b_u = (theta * rf * u + fn) * act
        x = direct.solve(grid, M, np.concatenate([b_u, bp]))
        u = x[:grid.nvel]
        out.append(x)
    return out
