"""Inhomogeneous velocity boundary conditions: the boundary terms of the
affine operator (Sec. 3.2: the viscous stencils next to a wall use the
prescribed boundary values; the Krylov solver is applied to the homogeneous
problem after these terms are subtracted from the right-hand side).

Test infrastructure: only tests use it.

Boundary data:
  * normal velocity on every wall face (the a-faces at i_a = 0 and n_a of a
    non-periodic axis a), given in a packed velocity vector whose wall
    entries hold it (other entries ignored);
  * tangential velocity on no-slip walls: tan[(d, side, a)] for the wall of
    axis d (side 0 low, 1 high) and a component a != d, an array over the
    a-face positions with axis d removed (numpy order, x fastest).  Free-slip
    walls carry no tangential data (zero shear stress).

Full operator with boundary data u_w, U:  M x + c  with
  c_p = -D_w u_w                              (continuity: -D u)
  c_u = -L_w(u_w, U)                          (momentum: alpha u - L u + G p)
where D_w holds the wall-face columns of the divergence and L_w the affine
part of the viscous operator: the normal stresses 2 mu (D u) (and
lam (D u) with bulk viscosity) of the cells next to a wall, and the edge
stresses mu_e (du_a/dx_b + du_b/dx_a) on wall edges, whose wall-normal
derivative of a tangential component is one-sided, (u_first - U)/(h/2), and
whose along-wall derivative of the normal component uses the wall values.

Parity: pinned (tests/test_oracle_boundary.py: Couette flow between moving
walls is exactly linear; a uniform through-flow with prescribed normal
velocities is exact; a manufactured solution with non-zero wall values
converges at second order).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import assemble as asm
from .grid import Grid, NOSLIP


def _wall_storage(grid: Grid, a, idx):
    return grid.offsets[a] + grid._flat(grid.face_ext[a], idx)


def wall_divergence(grid: Grid):
    """D_w (ncell x nvel): the wall-face terms of (D u)_c = sum_a
    (u_a[c + e_a] - u_a[c]) / h, i.e. -u/h from a wall face on the low side
    of a cell and +u/h from one on its high side."""
    h = grid.h
    rows, cols, vals = [], [], []
    for a in range(grid.dim):
        if grid.periodic[a]:
            continue
        idx = grid.face_positions(a)
        for side, sel in ((0, idx[a] == 0), (1, idx[a] == grid.n[a])):
            ii = [v[sel] for v in idx]
            cell = [v.copy() for v in ii]
            if side == 1:
                cell[a] = cell[a] - 1
            rows.append(grid.cell_id(cell, offset=False))
            cols.append(_wall_storage(grid, a, ii))
            vals.append(np.full(len(ii[0]), (-1.0 if side == 0 else 1.0) / h))
    if not rows:
        return sp.csr_matrix((grid.ncell, grid.nvel))
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(grid.ncell, grid.nvel))


def boundary_terms(grid: Grid, coef, u_wall, tan=None):
    """The boundary terms c (packed Stokes vector, wall entries 0)."""
    h = grid.h
    tan = tan or {}
    uw = np.asarray(u_wall, dtype=np.float64)
    Dw = wall_divergence(grid)
    duw = Dw @ uw                                        # wall part of D u at cells
    Gp = asm.gradient_parts(grid)
    mu_c = np.asarray(coef["mu_c"], dtype=np.float64).ravel()
    L = np.zeros(grid.nvel)
    # normal stresses of the cells next to a wall: 2 mu_c (du_a/dx_a)
    for a in range(grid.dim):
        if grid.periodic[a]:
            continue
        Dwa = wall_divergence_component(grid, a)
        L += Gp[a] @ (2.0 * mu_c * (Dwa @ uw))
    if coef.get("lam_c") is not None:                    # grad (lam div u)
        L += asm.gradient(grid) @ (np.asarray(coef["lam_c"]).ravel() * duw)
    # edge stresses on wall edges
    for p in range(grid.dim):
        for q in range(p + 1, grid.dim):
            idx = grid.edge_positions(p, q)
            mue = np.asarray(coef["mu_e"][(p, q)], dtype=np.float64).ravel() \
                * asm._edge_mask(grid, p, q, idx)
            stress = np.zeros(len(idx[0]))
            for d, a in ((q, p), (p, q)):                # wall normal d, tangential component a
                if grid.periodic[d]:
                    continue
                for side, wall_i in ((0, 0), (1, grid.n[d])):
                    on = idx[d] == wall_i
                    if not on.any():
                        continue
                    ii = [v[on] for v in idx]
                    # along-wall derivative of the normal velocity: d-faces on the wall
                    lo = [v.copy() for v in ii]
                    lo[a] = lo[a] - 1
                    if grid.periodic[a]:
                        lo[a] = lo[a] % grid.n[a]
                    hi_v = np.zeros(len(ii[0]))
                    lo_v = np.zeros(len(ii[0]))
                    inb = ii[a] < grid.face_ext[d][a]
                    hi_v[inb] = uw[_wall_storage(grid, d, [v[inb] for v in ii])]
                    okl = lo[a] >= 0
                    lo_v[okl] = uw[_wall_storage(grid, d, [v[okl] for v in lo])]
                    rate = (hi_v - lo_v) / h
                    # wall-normal derivative of the tangential velocity: one-sided
                    if grid.bc[2 * d + side] == NOSLIP and (d, side, a) in tan:
                        U = np.asarray(tan[(d, side, a)], dtype=np.float64)
                        ext = list(grid.face_ext[a])
                        pos = [ii[c] for c in range(3) if c != d]
                        ext2 = [ext[c] for c in range(3) if c != d]
                        flat = pos[1] * ext2[0] + pos[0]
                        rate = rate + (2.0 / h if side == 1 else -2.0 / h) * U.ravel()[flat]
                    stress[np.flatnonzero(on)] += rate
            stress *= mue
            L += asm._edge_flux_divergence(grid, p, q) @ stress
            L += asm._edge_flux_divergence(grid, q, p) @ stress
    c = np.zeros(grid.size)
    c[:grid.nvel] = -L
    c[grid.nvel:] = -duw
    c[~grid.active] = 0.0
    return c


def wall_divergence_component(grid: Grid, a):
    """The a-component part of wall_divergence."""
    D = wall_divergence(grid).tocoo()
    lo, hi = grid.offsets[a], grid.offsets[a] + int(np.prod(grid.face_ext[a]))
    keep = (D.col >= lo) & (D.col < hi)
    return sp.csr_matrix((D.data[keep], (D.row[keep], D.col[keep])), shape=D.shape)
