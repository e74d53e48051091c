"""Sparse assembly of the staggered Stokes operators, Sec. 2 and Sec. 3.1.

Test infrastructure: see the package docstring.

Every matrix is built entry by entry from the difference formulas of Sec. 3.1
(vectorised over all faces, cells or edges at once), as scipy.sparse CSR
matrices over the storage vectors of ``grid.Grid``.  Wall faces are never
unknowns: their rows and columns are empty.

  D      (ncell x nvel)  divergence, (Du)_c = sum_a (u_a[c+e_a] - u_a[c])/h
  G      (nvel x ncell)  gradient, (G_a p)_f = (p[f] - p[f-e_a])/h
  L_mu   (nvel x nvel)   stress-form viscous operator, Eq. div_stress:
                         x-momentum = d/dx(2 mu du/dx) + d/dy(mu (du/dy + dv/dx)) ...
                         normal stresses 2 mu_c du_a/dx_a at cell centres,
                         shear stresses mu_e (du_a/dx_b + du_b/dx_a) at nodes (2D)
                         or edges (3D)
  A      = diag(theta rho_f) - L_mu                         (Sec. 2, Eq. Saddle_sys)
  M      = [[A, G], [-D, 0]]                                (Eq. Saddle_sys)
  L_rho  = D diag(1/rho_f) G  (density-weighted Poisson operator, Sec. 2)

Readings where Sec. 3.1 is not explicit (each is pinned by a test):
  * a shear stress on a wall edge takes the one-sided derivative
    (u_first - 0)/(h/2) of the tangential velocity and a zero normal-velocity
    derivative along the wall (no-slip); on a free-slip wall the shear stress
    is zero; an edge on two walls touches only wall faces and is unused;
  * mu on a wall edge is the mean of the in-domain cells around it.

Parity: pinned (D = -G^T, DG = 5/7-point Laplacian, L_mu symmetric negative
semidefinite, constant-mu reduction to the Laplacian on divergence-free
fields, Fourier symbol of App. A, eigenvalue counts of App. B.1, second-order
manufactured-solution convergence).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .grid import Grid, PERIODIC, NOSLIP, FREESLIP


class _Triplets:
    def __init__(self):
        self.r, self.c, self.v = [], [], []

    def add(self, rows, cols, vals):
        rows, cols, vals = np.broadcast_arrays(np.asarray(rows), np.asarray(cols),
                                               np.asarray(vals, dtype=np.float64))
        keep = (rows >= 0) & (cols >= 0)
        self.r.append(rows[keep].ravel())
        self.c.append(cols[keep].ravel())
        self.v.append(vals[keep].ravel())

    def matrix(self, shape):
        if not self.r:
            return sp.csr_matrix(shape)
        r = np.concatenate(self.r)
        c = np.concatenate(self.c)
        v = np.concatenate(self.v)
        return sp.coo_matrix((v, (r, c)), shape=shape).tocsr()


def _shift(idx, axis, delta):
    out = list(idx)
    out[axis] = idx[axis] + delta
    return out


# ----------------------------------------------------------------- coefficients
def face_density(grid: Grid, rho):
    """rho_f = (rho[left cell] + rho[right cell]) / 2 on every unknown face
    (Sec. 3.1); wall faces 0.  Returns a list of face arrays."""
    rho = np.asarray(rho, dtype=np.float64).ravel()
    out = []
    for a in range(grid.dim):
        idx = grid.face_positions(a)
        fid = grid.face_id(a, idx)
        lo = grid.cell_id(_shift(idx, a, -1), offset=False)
        hi = grid.cell_id(idx, offset=False)
        val = np.zeros(fid.shape)
        ok = fid >= 0
        val[ok] = 0.5 * (rho[lo[ok]] + rho[hi[ok]])
        out.append(val.reshape(grid.face_shape(a)))
    return out


def edge_viscosity(grid: Grid, mu):
    """mu on (a, b) edges (nodes in 2D): the mean of the four neighbouring
    cell values (Sec. 3.1); on a wall edge, the mean of the in-domain ones."""
    mu = np.asarray(mu, dtype=np.float64).ravel()
    out = {}
    for a in range(grid.dim):
        for b in range(a + 1, grid.dim):
            idx = grid.edge_positions(a, b)
            acc = np.zeros(idx[0].shape)
            cnt = np.zeros(idx[0].shape)
            for da in (-1, 0):
                for db in (-1, 0):
                    cid = grid.cell_id(_shift(_shift(idx, a, da), b, db), offset=False)
                    ok = cid >= 0
                    acc[ok] += mu[cid[ok]]
                    cnt[ok] += 1
            out[(a, b)] = (acc / np.maximum(cnt, 1)).reshape(grid.np_shape(grid.edge_ext(a, b)))
    return out


def fine_coefficients(grid: Grid, rho, mu, theta, gamma=None):
    """Coefficients of the finest level: alpha_f = theta rho_f, beta_f = 1/rho_f
    on faces, mu at cells and at edges; with a bulk viscosity gamma (Sec. 2:
    tau = mu (grad u + grad u^T) + (gamma - 2/3 mu)(div u) I) also
    lam_c = gamma - 2/3 mu at cells."""
    rho_f = face_density(grid, rho)
    alpha = [theta * r for r in rho_f]
    beta = [np.where(r > 0, 1.0 / np.where(r > 0, r, 1.0), 0.0) for r in rho_f]
    mu_c = np.asarray(mu, dtype=np.float64).reshape(grid.cell_shape()).copy()
    out = {"alpha": alpha, "beta": beta, "mu_c": mu_c, "mu_e": edge_viscosity(grid, mu)}
    if gamma is not None:
        out["lam_c"] = np.asarray(gamma, dtype=np.float64).reshape(grid.cell_shape()) - 2.0 / 3.0 * mu_c
    return out


# -------------------------------------------------------------------- operators
def divergence_parts(grid: Grid):
    """D_a (ncell x nvel): (D_a u)_c = (u_a[c + e_a] - u_a[c]) / h."""
    h = grid.h
    idx = grid.cell_positions()
    row = grid.cell_id(idx, offset=False)
    parts = []
    for a in range(grid.dim):
        t = _Triplets()
        t.add(row, grid.face_id(a, _shift(idx, a, 1)), 1.0 / h)
        t.add(row, grid.face_id(a, idx), -1.0 / h)
        parts.append(t.matrix((grid.ncell, grid.nvel)))
    return parts


def divergence(grid: Grid):
    return sum(divergence_parts(grid)).tocsr()


def gradient_parts(grid: Grid):
    """G_a (nvel x ncell): (G_a p)_f = (p[cell f] - p[cell f - e_a]) / h on
    every unknown a-face f."""
    h = grid.h
    parts = []
    for a in range(grid.dim):
        idx = grid.face_positions(a)
        row = grid.face_id(a, idx)
        t = _Triplets()
        t.add(row, grid.cell_id(idx, offset=False), 1.0 / h)
        t.add(row, grid.cell_id(_shift(idx, a, -1), offset=False), -1.0 / h)
        parts.append(t.matrix((grid.nvel, grid.ncell)))
    return parts


def gradient(grid: Grid):
    return sum(gradient_parts(grid)).tocsr()


def _edge_mask(grid: Grid, a, b, idx):
    """1 where the shear stress on the edge is live, 0 on free-slip walls and
    on edges lying on two walls."""
    m = np.ones(idx[0].shape)
    wall_a = grid.on_wall(a, idx[a])
    wall_b = grid.on_wall(b, idx[b])
    m[wall_a & wall_b] = 0.0
    for c in (a, b):
        if grid.periodic[c]:
            continue
        lo_free = grid.bc[2 * c] == FREESLIP
        hi_free = grid.bc[2 * c + 1] == FREESLIP
        if lo_free:
            m[idx[c] == 0] = 0.0
        if hi_free:
            m[idx[c] == grid.n[c]] = 0.0
    return m


def _edge_rate(grid: Grid, a, b):
    """S (nedge x nvel): du_a/dx_b on the (a, b) edges (edge array of the
    unordered pair).  Interior: (u_a[.., i_b] - u_a[.., i_b - 1]) / h.  On a
    b-wall with no-slip: one-sided (u_a[first] - 0)/(h/2).  On an a-wall the
    a-faces are wall faces (u_a = 0), so the row is empty."""
    h = grid.h
    lo, hi = min(a, b), max(a, b)
    idx = grid.edge_positions(lo, hi)
    row = grid.edge_id(lo, hi, idx)
    t = _Triplets()
    wall_a = grid.on_wall(a, idx[a])
    interior = ~wall_a & ~grid.on_wall(b, idx[b])
    sel = np.flatnonzero(interior)
    ii = [v[sel] for v in idx]
    t.add(row[sel], grid.face_id(a, ii), 1.0 / h)
    t.add(row[sel], grid.face_id(a, _shift(ii, b, -1)), -1.0 / h)
    if not grid.periodic[b]:
        if grid.bc[2 * b] == NOSLIP:
            sel = np.flatnonzero(~wall_a & (idx[b] == 0))
            ii = [v[sel] for v in idx]
            t.add(row[sel], grid.face_id(a, ii), 2.0 / h)
        if grid.bc[2 * b + 1] == NOSLIP:
            sel = np.flatnonzero(~wall_a & (idx[b] == grid.n[b]))
            ii = [v[sel] for v in idx]
            t.add(row[sel], grid.face_id(a, _shift(ii, b, -1)), -2.0 / h)
    nedge = int(np.prod(grid.edge_ext(lo, hi)))
    return t.matrix((nedge, grid.nvel))


def _edge_flux_divergence(grid: Grid, a, b):
    """T (nvel x nedge): d/dx_b of an edge stress at a-faces,
    (tau[.., i_b + 1] - tau[.., i_b]) / h."""
    h = grid.h
    lo, hi = min(a, b), max(a, b)
    idx = grid.face_positions(a)
    row = grid.face_id(a, idx)
    t = _Triplets()
    t.add(row, grid.edge_id(lo, hi, _shift(idx, b, 1)), 1.0 / h)
    t.add(row, grid.edge_id(lo, hi, idx), -1.0 / h)
    nedge = int(np.prod(grid.edge_ext(lo, hi)))
    return t.matrix((grid.nvel, nedge))


def viscous(grid: Grid, mu_c, mu_e, form="stress"):
    """L_mu (nvel x nvel), Eq. div_stress (form='stress') or the Laplacian form
    sum_b d/dx_b(mu du_a/dx_b) (form='laplacian', Sec. 3.1)."""
    Dp = divergence_parts(grid)
    Gp = gradient_parts(grid)
    cfac = 2.0 if form == "stress" else 1.0
    Wc = sp.diags(cfac * np.asarray(mu_c, dtype=np.float64).ravel())
    L = sp.csr_matrix((grid.nvel, grid.nvel))
    for a in range(grid.dim):
        L = L + Gp[a] @ Wc @ Dp[a]
    for a in range(grid.dim):
        for b in range(a + 1, grid.dim):
            idx = grid.edge_positions(a, b)
            We = sp.diags(np.asarray(mu_e[(a, b)], dtype=np.float64).ravel()
                          * _edge_mask(grid, a, b, idx))
            S_ab = _edge_rate(grid, a, b)     # du_a/dx_b
            S_ba = _edge_rate(grid, b, a)     # du_b/dx_a
            T_ab = _edge_flux_divergence(grid, a, b)
            T_ba = _edge_flux_divergence(grid, b, a)
            if form == "stress":
                L = L + (T_ab + T_ba) @ We @ (S_ab + S_ba)
            else:
                L = L + T_ab @ We @ S_ab + T_ba @ We @ S_ba
    return L.tocsr()


def bulk_viscous(grid: Grid, lam_c):
    """The bulk part of the viscous operator, grad (lam div u) = G diag(lam) D:
    on the a-face between cells c-e_a and c it is
    (lam_c (D u)_c - lam_{c-e_a} (D u)_{c-e_a}) / h (Sec. 2, bulk-viscosity
    stress; D u vanishes identically on divergence-free fields)."""
    return (gradient(grid) @ sp.diags(np.asarray(lam_c, dtype=np.float64).ravel())
            @ divergence(grid)).tocsr()


def velocity_operator(grid: Grid, coef, form="stress"):
    """A = diag(alpha) - L_mu (Sec. 2), L_mu including the bulk part when
    the coefficients carry lam_c."""
    alpha = np.concatenate([np.asarray(x).ravel() for x in coef["alpha"]])
    A = sp.diags(alpha) - viscous(grid, coef["mu_c"], coef["mu_e"], form)
    if coef.get("lam_c") is not None:
        A = A - bulk_viscous(grid, coef["lam_c"])
    return A.tocsr()


def poisson_operator(grid: Grid, beta):
    """L_rho = D diag(beta) G, beta = 1/rho_f on the finest level (Sec. 2)."""
    b = np.concatenate([np.asarray(x).ravel() for x in beta])
    return (divergence(grid) @ sp.diags(b) @ gradient(grid)).tocsr()


def stokes_operator(grid: Grid, coef, form="stress"):
    """M = [[A, G], [-D, 0]] over the full storage vector (Eq. Saddle_sys)."""
    A = velocity_operator(grid, coef, form)
    G = gradient(grid)
    D = divergence(grid)
    Z = sp.csr_matrix((grid.ncell, grid.ncell))
    return sp.bmat([[A, G], [-D, Z]], format="csr")


def stokes_from_fields(grid: Grid, rho, mu, theta, form="stress", gamma=None):
    return stokes_operator(grid, fine_coefficients(grid, rho, mu, theta, gamma), form)


def pressure_nullspace(grid: Grid):
    """Constant pressure is in the null space of M when no face carries a
    prescribed non-zero normal flux, i.e. always for periodic, no-slip and
    free-slip boundaries (Sec. 3.2)."""
    return True
