"""The point-by-point rows of M x equal the assembled operator (both written
from Sec. 3.1), for every boundary mix in 2D and 3D."""
import numpy as np
import pytest

from oracle import assemble as asm
from oracle import pointwise
from oracle.grid import Grid, PERIODIC, NOSLIP, FREESLIP

BCS_2D = [(PERIODIC,) * 4, (NOSLIP,) * 4, (FREESLIP,) * 4, (NOSLIP, FREESLIP, PERIODIC, PERIODIC),
          (PERIODIC, PERIODIC, FREESLIP, NOSLIP), (NOSLIP, NOSLIP, FREESLIP, FREESLIP)]
BCS_3D = [(PERIODIC,) * 6, (NOSLIP,) * 6, (FREESLIP,) * 6, (NOSLIP, NOSLIP, PERIODIC, PERIODIC, FREESLIP, NOSLIP)]


@pytest.mark.parametrize("dim,n,bc", [(2, (8, 4), b) for b in BCS_2D] + [(3, (4, 4, 8), b) for b in BCS_3D])
def test_pointwise_rows_equal_assembled_operator(dim, n, bc):
    g = Grid(dim, n, 0.5, bc)
    rng = np.random.default_rng(7)
    rho = np.exp(rng.standard_normal(g.cell_shape()))
    mu = np.exp(rng.standard_normal(g.cell_shape()))
    x = rng.standard_normal(g.size) * g.active
    M = asm.stokes_from_fields(g, rho, mu, 1.3)
    ref = M @ x
    sel = np.flatnonzero(g.active)
    got = pointwise.rows(g, x, rho, mu, 1.3, sel)
    assert np.abs(got - ref[sel]).max() <= 1e-13 * np.abs(ref).max()
