"""Rows of M x evaluated point by point (Sec. 3.1 stencils), for checking
solutions of grids too large to assemble.

Test infrastructure: only tests use it.

For an unknown a-face at position q (between cells q - e_a and q):
  (M x)_q = alpha_q u_a(q) - (L_mu u)_a(q) + (p(q) - p(q - e_a)) / h,
  alpha_q = theta (rho(q) + rho(q - e_a)) / 2,
  (L_mu u)_a(q) = (tau_aa(q) - tau_aa(q - e_a)) / h
                  + sum_{b != a} (tau_ab(edge q + e_b) - tau_ab(edge q)) / h,
  tau_aa(c) = 2 mu_c (u_a(c + e_a) - u_a(c)) / h,
  tau_ab(e) = mu_e (du_a/dx_b + du_b/dx_a) at the edge, mu_e the mean of the
  in-domain cells around it; on a no-slip b-wall du_a/dx_b is one-sided,
  (u_first - 0)/(h/2); on a free-slip wall, and on edges lying on two walls,
  tau_ab = 0; wall faces hold zero velocity.
For a cell c: (M x)_c = -(D u)_c = -sum_a (u_a(c + e_a) - u_a(c)) / h.

Parity: pinned (tests/test_oracle_pointwise.py: equal to the assembled M on
every boundary mix, 2D and 3D).
"""
from __future__ import annotations

import numpy as np

from .grid import Grid, FREESLIP, NOSLIP


class Fields:
    """Random access to the packed vector and the cell fields of a grid."""

    def __init__(self, grid: Grid, x, rho, mu, theta):
        self.g = grid
        self.x = np.asarray(x, dtype=np.float64)
        self.rho = np.asarray(rho, dtype=np.float64).ravel()
        self.mu = np.asarray(mu, dtype=np.float64).ravel()
        self.theta = float(theta)

    def u(self, a, pos):
        """u_a at integer positions pos (3 arrays, may step past a periodic
        seam or onto / beyond a wall: zero there)."""
        g = self.g
        pos = [np.asarray(v).copy() for v in pos]
        ok = np.ones(pos[0].shape, dtype=bool)
        for c in range(3):
            if g.periodic[c]:
                pos[c] = pos[c] % g.n[c]
            else:
                hi = g.n[c] if c == a else g.n[c] - 1
                ok &= (pos[c] >= 0) & (pos[c] <= hi)
                if c == a:
                    ok &= (pos[c] > 0) & (pos[c] < g.n[c])     # wall faces are zero
        safe = [np.where(ok, pos[c], 0) for c in range(3)]
        flat = g.offsets[a] + g._flat(g.face_ext[a], safe)
        return np.where(ok, self.x[flat], 0.0)

    def cell(self, arr, pos):
        """(value, inside) of a cell array at positions pos."""
        g = self.g
        pos = [np.asarray(v).copy() for v in pos]
        ok = np.ones(pos[0].shape, dtype=bool)
        for c in range(3):
            if g.periodic[c]:
                pos[c] = pos[c] % g.n[c]
            else:
                ok &= (pos[c] >= 0) & (pos[c] < g.n[c])
        safe = [np.where(ok, pos[c], 0) for c in range(3)]
        return np.where(ok, arr[g._flat(g.n, safe)], 0.0), ok

    def p(self, pos):
        return self.cell(self.x[self.g.nvel:], pos)[0]


def _shift(pos, c, d):
    out = [np.asarray(v).copy() for v in pos]
    out[c] = out[c] + d
    return out


def _edge_stress(F: Fields, a, b, e):
    """tau_ab at the (a, b) edges whose a- and b-coordinates are e[a] h and
    e[b] h (third coordinate at the cell centre)."""
    g, h = F.g, F.g.h
    on_lo = (~np.asarray(g.periodic[b])) & (e[b] == 0)
    on_hi = (~np.asarray(g.periodic[b])) & (e[b] == g.n[b])
    wall_a = (~np.asarray(g.periodic[a])) & ((e[a] == 0) | (e[a] == g.n[a]))
    # du_a/dx_b
    up = F.u(a, e)
    dn = F.u(a, _shift(e, b, -1))
    dab = (up - dn) / h
    if not g.periodic[b]:
        dab = np.where(on_lo, up / (0.5 * h), dab)
        dab = np.where(on_hi, -dn / (0.5 * h), dab)
    # du_b/dx_a (b-faces at b-index e_b; zero on a b-wall)
    dba = (F.u(b, e) - F.u(b, _shift(e, a, -1))) / h
    # mu at the edge: mean of the in-domain cells around it
    acc = np.zeros(e[0].shape)
    cnt = np.zeros(e[0].shape)
    for da in (-1, 0):
        for db in (-1, 0):
            v, ok = F.cell(F.mu, _shift(_shift(e, a, da), b, db))
            acc += v
            cnt += ok
    mue = acc / np.maximum(cnt, 1)
    live = ~(wall_a & (on_lo | on_hi))
    if not g.periodic[b]:
        if g.bc[2 * b] == FREESLIP:
            live &= ~on_lo
        if g.bc[2 * b + 1] == FREESLIP:
            live &= ~on_hi
    if not g.periodic[a]:
        if g.bc[2 * a] == FREESLIP:
            live &= ~(e[a] == 0)
        if g.bc[2 * a + 1] == FREESLIP:
            live &= ~(e[a] == g.n[a])
    return np.where(live, mue * (dab + dba), 0.0)


def rows(grid: Grid, x, rho, mu, theta, sel):
    """(M x)[sel] for storage indices sel of unknowns (faces or cells)."""
    F = Fields(grid, x, rho, mu, theta)
    g, h = grid, grid.h
    sel = np.asarray(sel)
    out = np.zeros(sel.shape)
    cell = sel >= g.nvel
    if cell.any():
        t = sel[cell] - g.nvel
        pos = _unflat(t, g.n)
        div = np.zeros(t.shape)
        for a in range(g.dim):
            div += (F.u(a, _shift(pos, a, 1)) - F.u(a, pos)) / h
        out[cell] = -div
    for a in range(g.dim):
        lo = g.offsets[a]
        hi = lo + int(np.prod(g.face_ext[a]))
        m = (sel >= lo) & (sel < hi)
        if not m.any():
            continue
        q = _unflat(sel[m] - lo, g.face_ext[a])
        qm = _shift(q, a, -1)
        rho_f = 0.5 * (F.cell(F.rho, q)[0] + F.cell(F.rho, qm)[0])
        ua = F.u(a, q)
        tau_hi = 2.0 * F.cell(F.mu, q)[0] * (F.u(a, _shift(q, a, 1)) - ua) / h
        tau_lo = 2.0 * F.cell(F.mu, qm)[0] * (ua - F.u(a, qm)) / h
        L = (tau_hi - tau_lo) / h
        for b in range(g.dim):
            if b != a:
                L += (_edge_stress(F, a, b, _shift(q, b, 1)) - _edge_stress(F, a, b, q)) / h
        grad = (F.p(q) - F.p(qm)) / h
        out[m] = theta * rho_f * ua - L + grad
    return out


def _unflat(t, ext):
    t = np.asarray(t)
    i = t % ext[0]
    r = t // ext[0]
    j = r % ext[1]
    k = r // ext[1]
    return [i, j, k]
