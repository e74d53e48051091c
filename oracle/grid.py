"""Index maps of the staggered (MAC) grid, Sec. 3.1.

Test infrastructure: see the package docstring.

Positions use integer storage indices.  Cell (i, j, k) has its centre at
((i+1/2)h, (j+1/2)h, (k+1/2)h).  The a-component face with index (i, j, k)
lies on the low-a side of cell (i, j, k): its a-coordinate is i_a*h.  The
(a, b) edge (a node in 2D) with index (i, j, k) has a-coordinate i_a*h,
b-coordinate i_b*h and sits at the cell centre along the third axis.

Storage vector ("full" vector): the face arrays of components x, y[, z]
followed by the cell array, each flattened with x fastest.  Faces that lie on
a wall are kept in storage as zeros; they are not unknowns.  ``active`` marks
the unknowns.
"""
from __future__ import annotations

import numpy as np

PERIODIC, NOSLIP, FREESLIP = 0, 1, 2


class Grid:
    def __init__(self, dim, n, h=1.0, bc=None):
        n = list(n) + [1] * (3 - len(n))
        self.dim = int(dim)
        self.n = tuple(int(v) for v in n)
        if bc is None:
            bc = (PERIODIC,) * 6
        bc = list(bc) + [PERIODIC] * (6 - len(bc))
        for a in range(self.dim, 3):
            bc[2 * a] = bc[2 * a + 1] = PERIODIC
        for a in range(3):
            if (bc[2 * a] == PERIODIC) != (bc[2 * a + 1] == PERIODIC):
                raise ValueError("periodic must be set on both sides of an axis")
        self.bc = tuple(bc)
        self.periodic = tuple(bc[2 * a] == PERIODIC for a in range(3))
        self.h = float(h)
        # extents (x, y, z) of each array family
        self.face_ext = []
        for a in range(3):
            e = list(self.n)
            if not self.periodic[a]:
                e[a] += 1
            self.face_ext.append(tuple(e))
        self.offsets = []
        off = 0
        for a in range(self.dim):
            self.offsets.append(off)
            off += int(np.prod(self.face_ext[a]))
        self.cell_offset = off
        self.ncell = int(np.prod(self.n))
        self.size = off + self.ncell
        self.nvel = off
        self.active = np.ones(self.size, dtype=bool)
        for a in range(self.dim):
            if not self.periodic[a]:
                idx = self.face_positions(a)
                wall = (idx[a] == 0) | (idx[a] == self.n[a])
                self.active[self.offsets[a] + np.flatnonzero(wall.ravel())] = False

    # ------------------------------------------------------------------ shapes
    @staticmethod
    def np_shape(ext):
        return (ext[2], ext[1], ext[0])

    def face_shape(self, a):
        return self.np_shape(self.face_ext[a])

    def cell_shape(self):
        return self.np_shape(self.n)

    def edge_ext(self, a, b):
        e = list(self.n)
        for c in (a, b):
            if not self.periodic[c]:
                e[c] += 1
        return tuple(e)

    # --------------------------------------------------------------- positions
    @staticmethod
    def _positions(ext):
        k, j, i = np.meshgrid(np.arange(ext[2]), np.arange(ext[1]), np.arange(ext[0]),
                              indexing="ij")
        return [i.ravel(), j.ravel(), k.ravel()]

    def face_positions(self, a):
        return self._positions(self.face_ext[a])

    def cell_positions(self):
        return self._positions(self.n)

    def edge_positions(self, a, b):
        return self._positions(self.edge_ext(a, b))

    # ----------------------------------------------------------------- lookups
    def _flat(self, ext, idx):
        return (idx[2] * ext[1] + idx[1]) * ext[0] + idx[0]

    def face_id(self, a, idx):
        """Storage index of a-face at integer position idx (3 arrays), periodic
        wrap applied; -1 where the face is outside the domain or on a wall."""
        idx = [np.asarray(v).copy() for v in idx]
        ok = np.ones(idx[0].shape, dtype=bool)
        for c in range(3):
            if self.periodic[c]:
                idx[c] = idx[c] % self.n[c]
            else:
                hi = self.n[c] if c == a else self.n[c] - 1
                ok &= (idx[c] >= 0) & (idx[c] <= hi)
                if c == a:
                    ok &= (idx[c] > 0) & (idx[c] < self.n[c])
        ext = self.face_ext[a]
        safe = [np.where(ok, idx[c], 0) for c in range(3)]
        return np.where(ok, self.offsets[a] + self._flat(ext, safe), -1)

    def cell_id(self, idx, offset=True):
        """Storage index of cell idx (periodic wrap), -1 outside the domain."""
        idx = [np.asarray(v).copy() for v in idx]
        ok = np.ones(idx[0].shape, dtype=bool)
        for c in range(3):
            if self.periodic[c]:
                idx[c] = idx[c] % self.n[c]
            else:
                ok &= (idx[c] >= 0) & (idx[c] < self.n[c])
        safe = [np.where(ok, idx[c], 0) for c in range(3)]
        base = self.cell_offset if offset else 0
        return np.where(ok, base + self._flat(self.n, safe), -1)

    def edge_id(self, a, b, idx):
        """Index into the (a, b) edge array (no offset), -1 outside."""
        idx = [np.asarray(v).copy() for v in idx]
        ext = self.edge_ext(a, b)
        ok = np.ones(idx[0].shape, dtype=bool)
        for c in range(3):
            if self.periodic[c]:
                idx[c] = idx[c] % self.n[c]
            else:
                ok &= (idx[c] >= 0) & (idx[c] < ext[c])
        safe = [np.where(ok, idx[c], 0) for c in range(3)]
        return np.where(ok, self._flat(ext, safe), -1)

    def on_wall(self, c, pos):
        """True where face-position pos along axis c lies on a wall."""
        if self.periodic[c]:
            return np.zeros(np.shape(pos), dtype=bool)
        return (pos == 0) | (pos == self.n[c])

    # ------------------------------------------------------------ conversions
    def pack(self, u, p):
        """Face arrays + cell array -> full storage vector."""
        parts = [np.asarray(u[a], dtype=np.float64).reshape(-1) for a in range(self.dim)]
        parts.append(np.asarray(p, dtype=np.float64).reshape(-1))
        return np.concatenate(parts)

    def unpack(self, x):
        u = []
        for a in range(self.dim):
            sz = int(np.prod(self.face_ext[a]))
            u.append(x[self.offsets[a]:self.offsets[a] + sz].reshape(self.face_shape(a)))
        p = x[self.cell_offset:].reshape(self.cell_shape())
        return u, p

    def coarsen(self):
        return Grid(self.dim, [self.n[a] // 2 if a < self.dim else 1 for a in range(3)],
                    2.0 * self.h, self.bc)

    def velocity_mask(self):
        m = np.zeros(self.size, dtype=bool)
        m[:self.cell_offset] = True
        return m
