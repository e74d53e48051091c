"""Fourier closed forms for constant coefficients on a periodic grid, App. A.

Test infrastructure: see the package docstring.

On an all-periodic grid with constant rho0, mu0 every operator of Sec. 3.1 is
diagonalised by the discrete Fourier transform taken over the storage index
of each array.  With w_a = exp(2 pi i m_a / n_a) for mode m:
  (D_a u)_c = (u_a[c+e_a] - u_a[c]) / h        -> d_a = (w_a - 1) / h
  (G_a p)_f = (p[f] - p[f-e_a]) / h            -> g_a = (1 - 1/w_a) / h
  du_a/dx_b on the edge sharing the face index -> g_b
  d/dx_b of an edge stress at the face         -> d_b
so the stress-form viscous symbol is
  (L u)_a = mu0 [ 2 d_a g_a u_a + sum_{b != a} d_b (g_b u_a + g_a u_b) ]
and the (d+1) x (d+1) system [[theta rho0 - L, g], [-d^T, 0]] is solved mode by
mode.  The mean mode carries u = f / (theta rho0) and p = 0.

Parity: this module is itself the closed-form pin of the assembled operator
(tests compare it with the sparse direct solve) and of the Schur symbol
L_S = 2 mu0 (stress form) / mu0 (Laplacian form), App. A.
"""
from __future__ import annotations

import numpy as np

from .grid import Grid


def _symbols(grid: Grid):
    d = grid.dim
    shape = grid.cell_shape()
    ws = []
    for a in range(d):
        m = np.arange(grid.n[a])
        w = np.exp(2j * np.pi * m / grid.n[a])
        sh = [1, 1, 1]
        sh[2 - a] = grid.n[a]
        ws.append(np.broadcast_to(w.reshape(sh), shape))
    h = grid.h
    dsym = [(w - 1.0) / h for w in ws]
    gsym = [(1.0 - 1.0 / w) / h for w in ws]
    return dsym, gsym


def viscous_symbol(grid: Grid, mu0, form="stress"):
    """(..., d, d) symbol of L_mu."""
    dsym, gsym = _symbols(grid)
    d = grid.dim
    shape = grid.cell_shape()
    Lh = np.zeros(shape + (d, d), dtype=complex)
    nf = 2.0 if form == "stress" else 1.0
    for a in range(d):
        Lh[..., a, a] += nf * mu0 * dsym[a] * gsym[a]
        for b in range(d):
            if b == a:
                continue
            Lh[..., a, a] += mu0 * dsym[b] * gsym[b]
            if form == "stress":
                Lh[..., a, b] += mu0 * dsym[b] * gsym[a]
    return Lh


def solve_periodic(grid: Grid, rho0, mu0, theta, b, form="stress"):
    """x with M x = b for constant rho0, mu0 on an all-periodic grid."""
    assert all(grid.periodic[a] for a in range(grid.dim))
    d = grid.dim
    u, p = grid.unpack(b)
    fh = [np.fft.fftn(u[a]) for a in range(d)]
    gh = np.fft.fftn(p)
    dsym, gsym = _symbols(grid)
    Lh = viscous_symbol(grid, mu0, form)
    shape = grid.cell_shape()
    K = np.zeros(shape + (d + 1, d + 1), dtype=complex)
    for a in range(d):
        for c in range(d):
            K[..., a, c] = -Lh[..., a, c]
        K[..., a, a] += theta * rho0
        K[..., a, d] = gsym[a]
        K[..., d, a] = -dsym[a]
    rhs = np.stack(fh + [gh], axis=-1)
    zero = (0,) * 3
    K[zero] = np.eye(d + 1)
    if theta * rho0 != 0.0:
        K[zero][:d, :d] *= theta * rho0
    sol = np.linalg.solve(K, rhs[..., None])[..., 0]
    sol[zero][d] = 0.0
    ux = [np.real(np.fft.ifftn(sol[..., a])) for a in range(d)]
    px = np.real(np.fft.ifftn(sol[..., d]))
    px -= px.mean()
    return grid.pack(ux, px)


def schur_symbol(grid: Grid, mu0, form="stress"):
    """L_S = (d^T L^{-1} g)^{-1} on every non-zero mode (App. A, Eq. Fourier_Schur)."""
    dsym, gsym = _symbols(grid)
    d = grid.dim
    Lh = viscous_symbol(grid, mu0, form)
    shape = grid.cell_shape()
    zero = (0,) * 3
    Lh[zero] = np.eye(d)
    g = np.stack(gsym, axis=-1)[..., None]
    Dv = np.stack(dsym, axis=-1)[..., None, :]
    S = (Dv @ np.linalg.solve(Lh, g))[..., 0, 0]
    S[zero] = np.nan
    return 1.0 / S
