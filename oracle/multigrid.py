"""Geometric multigrid subsolvers, App. C.

Test infrastructure: see the package docstring.

Two V-cycles, each with a zero initial guess (Sec. 3.2):
  * the staggered velocity solver for  alpha phi - div beta[grad phi + grad phi^T] = r
    (A = theta rho - L_mu with the level's coefficients);
  * the cell-centred solver for  div beta grad phi = r  (L_rho).
Residual formulation, coarsening by 2 until the smallest axis has 2 cells;
`nu` multicolour Gauss-Seidel sweeps before and after the coarse correction
(2 in the paper, Sec. 4.1.1) and `ncoarse` sweeps on the coarsest level
(8, App. C).  One Gauss-Seidel sweep relaxes, in order, red-x, black-x,
red-y, black-y[, red-z, black-z] for the velocity and red, black for the
pressure; each colour applies phi += D^{-1} (r - L phi) on its points
(omega = 1).  A point (i, j, k) is red when i + j + k is even.

Coarse coefficients (App. C): face alpha (and face beta of the Poisson
operator) = mean of the overlying fine faces; cell mu = mean of the 2^d fine
cells; node mu (2D) by injection; edge mu (3D) = mean of the two overlying
fine edges.  Restriction: cell mean; 6-point (2D) / 12-point (3D) face
stencil.  Prolongation: cell injection; face interpolation that is linear
(3/4, 1/4) across the transverse cells and, for fine faces between coarse
faces, the mean of the two coarse faces.

Readings where App. C is silent (stated here, pinned by tests):
  * the printed prolongation covers even transverse indices; odd ones use
    the mirror image (3/4 on the own coarse cell, 1/4 on the next one);
  * a transverse neighbour across a wall is a ghost equal to -phi (no-slip:
    linear to zero on the wall) or +phi (free-slip);
  * the 3D restriction weights are 1/8 on the four coincident fine faces and
    1/16 on the eight neighbouring ones (the 2D weights 1/4, 1/8 extended);
  * the Poisson solver coarsens beta like alpha.

Parity: pinned (brute-force per-point Gauss-Seidel on tiny grids, transfer
operators on constants and linears, coarse coefficients worked out by hand
on 4^2 and 4^3 grids with distinct cell values, the V-cycle rates of
Sec. 4.1.1 on constant coefficients: tenfold per pressure cycle, tenfold in
the first velocity cycles and 1e11-1e12 over twelve, the velocity cycle's
later rate of 0.10-0.15 recorded as a departure from the paper).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import assemble as asm
from .grid import Grid, PERIODIC, NOSLIP, FREESLIP


def _ravel_index(ext, idx):
    return (idx[2] * ext[1] + idx[1]) * ext[0] + idx[0]


def _gather(arr, ext, idx):
    return np.asarray(arr).ravel()[_ravel_index(ext, idx)]


# --------------------------------------------------------- coarse coefficients
def coarse_coefficients(gf: Grid, cf, gc: Grid):
    d = gf.dim
    out = {"alpha": [], "beta": [], "mu_c": None, "mu_e": {}}
    for key in ("alpha", "beta"):
        for a in range(d):
            idx = gc.face_positions(a)
            acc = np.zeros(idx[0].shape)
            trans = [b for b in range(d) if b != a]
            cnt = 0
            for t in np.ndindex(*([2] * len(trans))):
                fi = [2 * v if c < d else v for c, v in enumerate(idx)]
                for tb, b in zip(t, trans):
                    fi[b] = fi[b] + tb
                acc += _gather(cf[key][a], gf.face_ext[a], fi)
                cnt += 1
            out[key].append((acc / cnt).reshape(gc.face_shape(a)))
    idx = gc.cell_positions()
    acc = np.zeros(idx[0].shape)
    cnt = 0
    for t in np.ndindex(*([2] * d)):
        fi = [2 * idx[c] + (t[c] if c < d else 0) if c < d else idx[c] for c in range(3)]
        acc += _gather(cf["mu_c"], gf.n, fi)
        cnt += 1
    out["mu_c"] = (acc / cnt).reshape(gc.cell_shape())
    if cf.get("lam_c") is not None:    # bulk term: cell average, like mu_c
        acc = np.zeros(idx[0].shape)
        for t in np.ndindex(*([2] * d)):
            fi = [2 * idx[c] + (t[c] if c < d else 0) if c < d else idx[c] for c in range(3)]
            acc += _gather(cf["lam_c"], gf.n, fi)
        out["lam_c"] = (acc / cnt).reshape(gc.cell_shape())
    for (a, b), arr in cf["mu_e"].items():
        idx = gc.edge_positions(a, b)
        fext = gf.edge_ext(a, b)
        if d == 2:
            fi = [2 * idx[0], 2 * idx[1], idx[2]]
            val = _gather(arr, fext, fi)
        else:
            c = 3 - a - b
            val = np.zeros(idx[0].shape)
            for t in (0, 1):
                fi = [2 * idx[0], 2 * idx[1], 2 * idx[2]]
                fi[c] += t
                val += 0.5 * _gather(arr, fext, fi)
        out["mu_e"][(a, b)] = val.reshape(gc.np_shape(gc.edge_ext(a, b)))
    return out


# ------------------------------------------------------------ transfer operators
def face_restriction(gf: Grid, gc: Grid):
    """R (nvel_c x nvel_f): 1/4 (2D) or 1/8 (3D) on the coincident fine faces,
    1/8 (2D) or 1/16 (3D) on the neighbouring fine faces."""
    d = gf.dim
    t = asm._Triplets()
    for a in range(d):
        idx = gc.face_positions(a)
        row = gc.face_id(a, idx)
        trans = [b for b in range(d) if b != a]
        for s in (-1, 0, 1):
            wa = 0.5 if s == 0 else 0.25
            for tt in np.ndindex(*([2] * len(trans))):
                fi = [2 * idx[c] if c < d else idx[c] for c in range(3)]
                fi[a] = fi[a] + s
                for tb, b in zip(tt, trans):
                    fi[b] = fi[b] + tb
                w = wa * 0.5 ** len(trans)
                t.add(row, gf.face_id(a, fi), w)
    return t.matrix((gc.nvel, gf.nvel))


def _transverse_weights(gc: Grid, b, j):
    """Coarse-cell weights (list of (index array, weight array)) for fine
    cell index j along transverse axis b: 3/4 on J = j//2 and 1/4 on the
    nearer neighbour; a neighbour beyond a wall folds onto J with sign -1
    (no-slip) or +1 (free-slip)."""
    J = j // 2
    nb = np.where(j % 2 == 0, J - 1, J + 1)
    w_own = np.full(j.shape, 0.75)
    w_nb = np.full(j.shape, 0.25)
    if not gc.periodic[b]:
        lo_sign = -1.0 if gc.bc[2 * b] == NOSLIP else 1.0
        hi_sign = -1.0 if gc.bc[2 * b + 1] == NOSLIP else 1.0
        below = nb < 0
        above = nb >= gc.n[b]
        w_own = w_own + np.where(below, 0.25 * lo_sign, 0.0) + np.where(above, 0.25 * hi_sign, 0.0)
        w_nb = np.where(below | above, 0.0, w_nb)
        nb = np.where(below | above, J, nb)
    return [(J, w_own), (nb, w_nb)]


def face_prolongation(gf: Grid, gc: Grid):
    d = gf.dim
    t = asm._Triplets()
    for a in range(d):
        idx = gf.face_positions(a)
        row = gf.face_id(a, idx)
        ia = idx[a]
        along = [(ia // 2, np.where(ia % 2 == 0, 1.0, 0.5)),
                 ((ia + 1) // 2, np.where(ia % 2 == 0, 0.0, 0.5))]
        trans = [b for b in range(d) if b != a]
        tw = [_transverse_weights(gc, b, idx[b]) for b in trans]
        for ca, wa in along:
            for combo in np.ndindex(*([2] * len(trans))):
                ci = [None, None, idx[2]]
                ci[a] = ca
                w = wa.copy()
                for k, b in enumerate(trans):
                    jb, wb = tw[k][combo[k]]
                    ci[b] = jb
                    w = w * wb
                if d == 2:
                    ci[2] = idx[2]
                t.add(row, gc.face_id(a, ci), w)
    return t.matrix((gf.nvel, gc.nvel))


def cell_restriction(gf: Grid, gc: Grid):
    d = gf.dim
    t = asm._Triplets()
    idx = gc.cell_positions()
    row = gc.cell_id(idx, offset=False)
    for tt in np.ndindex(*([2] * d)):
        fi = [2 * idx[c] + tt[c] if c < d else idx[c] for c in range(3)]
        t.add(row, gf.cell_id(fi, offset=False), 1.0 / 2 ** d)
    return t.matrix((gc.ncell, gf.ncell))


def cell_prolongation(gf: Grid, gc: Grid):
    d = gf.dim
    t = asm._Triplets()
    idx = gf.cell_positions()
    row = gf.cell_id(idx, offset=False)
    ci = [idx[c] // 2 if c < d else idx[c] for c in range(3)]
    t.add(row, gc.cell_id(ci, offset=False), 1.0)
    return t.matrix((gf.ncell, gc.ncell))


# ---------------------------------------------------------------------- levels
class Level:
    def __init__(self, grid: Grid, coef):
        self.grid = grid
        self.coef = coef
        self.A = asm.velocity_operator(grid, coef)
        self.Lrho = asm.poisson_operator(grid, coef["beta"])
        self.dA = self.A.diagonal()
        self.dL = self.Lrho.diagonal()
        self.vel_colours = []
        for a in range(grid.dim):
            idx = grid.face_positions(a)
            fid = grid.face_id(a, idx)
            par = (idx[0] + idx[1] + idx[2]) % 2
            for colour in (0, 1):
                rows = fid[(par == colour) & (fid >= 0)]
                self.vel_colours.append((rows, self.A[rows]))
        idx = grid.cell_positions()
        cid = grid.cell_id(idx, offset=False)
        par = (idx[0] + idx[1] + idx[2]) % 2
        self.cell_colours = []
        for colour in (0, 1):
            rows = cid[par == colour]
            self.cell_colours.append((rows, self.Lrho[rows]))
        self.R = self.P = self.Rc = self.Pc = None


def n_levels(grid: Grid):
    m = min(grid.n[a] for a in range(grid.dim))
    L = 1
    while m > 2:
        m //= 2
        L += 1
    return L


def build_hierarchy(grid: Grid, coef):
    levels = [Level(grid, coef)]
    g, c = grid, coef
    for _ in range(n_levels(grid) - 1):
        gc = g.coarsen()
        cc = coarse_coefficients(g, c, gc)
        lev = levels[-1]
        lev.R = face_restriction(g, gc)
        lev.P = face_prolongation(g, gc)
        lev.Rc = cell_restriction(g, gc)
        lev.Pc = cell_prolongation(g, gc)
        levels.append(Level(gc, cc))
        g, c = gc, cc
    return levels


# ------------------------------------------------------------------- smoothers
def gs_velocity(lev: Level, phi, r, sweeps):
    for _ in range(sweeps):
        for rows, Arows in lev.vel_colours:
            phi[rows] += (r[rows] - Arows @ phi) / lev.dA[rows]
    return phi


def gs_pressure(lev: Level, phi, r, sweeps):
    for _ in range(sweeps):
        for rows, Lrows in lev.cell_colours:
            phi[rows] += (r[rows] - Lrows @ phi) / lev.dL[rows]
    return phi


def vcycle_velocity(levels, r, l=0, nu=2, ncoarse=8):
    """One V-cycle for A phi = r with phi = 0 initially (App. C)."""
    lev = levels[l]
    phi = np.zeros_like(r)
    if l == len(levels) - 1:
        return gs_velocity(lev, phi, r, ncoarse)
    gs_velocity(lev, phi, r, nu)
    res = r - lev.A @ phi
    e = vcycle_velocity(levels, lev.R @ res, l + 1, nu, ncoarse)
    phi += lev.P @ e
    return gs_velocity(lev, phi, r, nu)


def vcycle_pressure(levels, r, l=0, nu=2, ncoarse=8):
    """One V-cycle for L_rho phi = r with phi = 0 initially (App. C)."""
    lev = levels[l]
    phi = np.zeros_like(r)
    if l == len(levels) - 1:
        return gs_pressure(lev, phi, r, ncoarse)
    gs_pressure(lev, phi, r, nu)
    res = r - lev.Lrho @ phi
    e = vcycle_pressure(levels, lev.Rc @ res, l + 1, nu, ncoarse)
    phi += lev.Pc @ e
    return gs_pressure(lev, phi, r, nu)
