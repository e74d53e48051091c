"""Adjoint gradient of a velocity loss with respect to the cell viscosity and
density (the differentiation form built on Sec. 2 and Sec. 3.1).

Test infrastructure: see the package docstring.

For a loss L(x) of the solution x = (u, p) of M(mu, rho) x = b, the adjoint
lambda solves M^T lambda = dL/dx.  M is symmetric (Sec. 2: D = -G^*), so the
adjoint solve is a forward solve.  Because M is affine in mu and in rho,

    dL/dmu_c  = -lambda^T (dM/dmu_c) x  =  lambda_u^T (dL_mu/dmu_c) u
    dL/drho_c = -lambda^T (dM/drho_c) x = -theta lambda_u^T (d rho_f/drho_c) u

with L_mu the stress-form viscous operator, whose cell viscosities enter the
normal stresses directly and whose edge viscosities are the mean of the
in-domain neighbouring cells (Sec. 3.1); rho_f is the mean of the two cells
beside a face.  `viscosity_gradient` evaluates the first line with the
assembled operators of assemble.py,
    lambda^T L_mu u = sum_a 2 mu_c (G_a^T lambda)(D_a u)
                      + sum_pairs (E mu)_e m_e (T^T lambda)_e (S u)_e,
i.e. d/dmu = 2 sum_a (G_a^T lambda) (D_a u) + sum_pairs E^T[(T^T lambda) m (S u)],
where E averages cell values onto edges.

Parity: pinned (brute-force derivative lambda^T L_mu(e_c) u cell by cell,
central finite differences of the loss through direct solves).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import assemble as asm
from .grid import Grid


def edge_average_matrix(grid: Grid, a, b):
    """E (nedge x ncell): the (a, b) edge value is the mean of the in-domain
    cells around the edge (Sec. 3.1)."""
    idx = grid.edge_positions(a, b)
    row = grid.edge_id(a, b, idx)
    cols, rows, cnt = [], [], np.zeros(idx[0].shape)
    for da in (-1, 0):
        for db in (-1, 0):
            cid = grid.cell_id(asm._shift(asm._shift(idx, a, da), b, db), offset=False)
            ok = cid >= 0
            cnt += ok
            rows.append(row[ok])
            cols.append(cid[ok])
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    w = 1.0 / cnt[rows]
    nedge = int(np.prod(grid.edge_ext(a, b)))
    return sp.coo_matrix((w, (rows, cols)), shape=(nedge, grid.ncell)).tocsr()


def viscosity_gradient(grid: Grid, mu, u, lam):
    """d(lambda_u^T L_mu u)/d mu_c for every cell (u, lam: velocity parts of
    full storage vectors)."""
    mu = np.asarray(mu, dtype=np.float64).ravel()
    Dp = asm.divergence_parts(grid)
    Gp = asm.gradient_parts(grid)
    g = np.zeros(grid.ncell)
    for a in range(grid.dim):
        g += 2.0 * (Gp[a].T @ lam) * (Dp[a] @ u)
    for a in range(grid.dim):
        for b in range(a + 1, grid.dim):
            idx = grid.edge_positions(a, b)
            m = asm._edge_mask(grid, a, b, idx)
            S = asm._edge_rate(grid, a, b) + asm._edge_rate(grid, b, a)
            T = asm._edge_flux_divergence(grid, a, b) + asm._edge_flux_divergence(grid, b, a)
            E = edge_average_matrix(grid, a, b)
            g += E.T @ ((T.T @ lam) * m * (S @ u))
    return g


def density_gradient(grid: Grid, theta, u, lam):
    """-theta lambda_u^T (d rho_f / d rho_c) u for every cell."""
    g = np.zeros(grid.ncell)
    for a in range(grid.dim):
        idx = grid.face_positions(a)
        fid = grid.face_id(a, idx)
        ok = fid >= 0
        prod = np.zeros(fid.shape)
        prod[ok] = lam[fid[ok]] * u[fid[ok]]
        for d in (-1, 0):
            cid = grid.cell_id(asm._shift(idx, a, d), offset=False)
            sel = ok & (cid >= 0)
            np.add.at(g, cid[sel], -0.5 * theta * prod[sel])
    return g


def loss_and_gradient(grid: Grid, rho, mu, theta, b, u_target, solve):
    """L = 1/2 ||u - u_target||^2 over the unknown faces, with u from
    M x = b (solve(M, rhs) returns the exact solution), and its gradients
    with respect to log mu and rho by one adjoint solve."""
    M = asm.stokes_from_fields(grid, rho, mu, theta)
    x = solve(M, b)
    u = x[:grid.nvel]
    r = (u - u_target) * grid.active[:grid.nvel]
    L = 0.5 * float(r @ r)
    rhs = np.zeros(grid.size)
    rhs[:grid.nvel] = r
    lam = solve(M, rhs)
    gmu = viscosity_gradient(grid, mu, u, lam[:grid.nvel])
    grho = density_gradient(grid, theta, u, lam[:grid.nvel])
    return L, np.asarray(mu).ravel() * gmu, grho, x, lam
