"""The exact solution of the discrete system M x = b (Eq. Saddle_sys).

Test infrastructure: see the package docstring.

The pressure is determined up to a constant for periodic, no-slip and
free-slip boundaries (Sec. 3.2).  The solve removes that freedom by fixing
the pressure of cell 0 (its row and column are dropped: for a compatible b
the dropped equation, -sum_c (D u)_c = 0, holds automatically) and then
shifts p to mean zero.  Dense LU for small systems, SuperLU otherwise.
A constant-velocity null space (steady flow on an all-periodic grid) is not
supported.

Parity: pinned (b = M x_true recovers x_true; agreement with the Fourier
closed form and between the dense and sparse paths).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .grid import Grid


def solve(grid: Grid, M, b, dense=None):
    act = grid.active.copy()
    act[grid.cell_offset] = False          # pin p at cell 0
    idx = np.flatnonzero(act)
    Ma = M[idx][:, idx]
    ba = b[idx]
    if dense is None:
        dense = len(idx) <= 6000
    if dense:
        xa = sla.solve(Ma.toarray(), ba)
    else:
        xa = spla.spsolve(Ma.tocsc(), ba)
    x = np.zeros(grid.size)
    x[idx] = xa
    p = x[grid.cell_offset:]
    p -= p.mean()
    return x


def relative_error(grid: Grid, x, x_ref):
    """(||u - u_ref|| / ||u_ref||, ||p' - p'_ref|| / ||p'_ref||), p' = p - mean(p)."""
    u, ur = x[:grid.nvel], x_ref[:grid.nvel]
    p = x[grid.nvel:] - x[grid.nvel:].mean()
    pr = x_ref[grid.nvel:] - x_ref[grid.nvel:].mean()
    eu = np.linalg.norm(u - ur) / max(np.linalg.norm(ur), 1e-300)
    ep = np.linalg.norm(p - pr) / max(np.linalg.norm(pr), 1e-300)
    return eu, ep
