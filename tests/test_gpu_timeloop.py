"""Backward-Euler time stepping on the GPU (stk_backward_euler_rhs and
timeloop.backward_euler) against the oracle's time loop with direct solves."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import direct, timeloop as otl
from oracle.grid import Grid, PERIODIC, NOSLIP, FREESLIP
from paper_1308_4605_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1308_4605_gb300 import stokes
    return stokes


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(DEV)


@pytest.mark.parametrize("dim,n,bc", [(2, (32, 16), (NOSLIP, NOSLIP, FREESLIP, NOSLIP)),
                                      (3, (8, 8, 8), (PERIODIC,) * 6)])
def test_backward_euler_rhs_kernel(S, dim, n, bc):
    pr = wl.generic(dim, n, bc, theta=2.5, seed=61)
    g = Grid(dim, pr.n, pr.h, pr.bc)
    sv = S.StokesSolver(dim, pr.n[:dim], pr.bc[:2 * dim], pr.h)
    sv.set_coefficients(_t(pr.rho), _t(pr.mu), 2.5)
    rng = np.random.default_rng(2)
    u = rng.standard_normal(g.nvel) * g.active[:g.nvel]
    f = rng.standard_normal(g.nvel)          # wall entries must be ignored
    uu, _ = g.unpack(np.concatenate([u, np.zeros(g.ncell)]))
    ff, _ = g.unpack(np.concatenate([f, np.zeros(g.ncell)]))
    b = [torch.empty_like(_t(x)) for x in uu]
    S.stk_backward_euler_rhs(sv.handle, [_t(x) for x in uu], [_t(x) for x in ff], b)
    got = g.pack([x.cpu().numpy() for x in b], np.zeros(g.ncell))[:g.nvel]
    rf = otl.face_density_vector(g, pr.rho)
    ref = (2.5 * rf * u + f) * g.active[:g.nvel]
    assert np.abs(got - ref).max() <= 1e-14 * np.abs(ref).max()
    # no forcing
    S.stk_backward_euler_rhs(sv.handle, [_t(x) for x in uu], None, b)
    got = g.pack([x.cpu().numpy() for x in b], np.zeros(g.ncell))[:g.nvel]
    assert np.abs(got - 2.5 * rf * u * g.active[:g.nvel]).max() <= 1e-14 * np.abs(ref).max()
    sv.close()


@pytest.mark.parametrize("dim,n,bc,precision", [
    (2, (32, 32), (PERIODIC,) * 4, 0),
    (2, (32, 16), (NOSLIP, NOSLIP, FREESLIP, NOSLIP), 1),
    (3, (16, 16, 8), (NOSLIP,) * 6, 0),
])
def test_time_loop_matches_oracle(S, dim, n, bc, precision):
    """Five backward-Euler steps with forcing and a divergence source: the
    GPU loop (solves to 1e-12, warm started) equals the oracle's direct
    solves to 1e-8 at every step; warm starts need fewer iterations than
    cold ones."""
    from paper_1308_4605_gb300 import timeloop
    pr = wl.generic(dim, n, bc, theta=1.0, rho_contrast=10.0, mu_contrast=30.0, seed=62)
    g = Grid(dim, pr.n, pr.h, pr.bc)
    rng = np.random.default_rng(8)
    u0 = rng.standard_normal(g.nvel) * g.active[:g.nvel]
    f = np.concatenate([x.ravel() for x in pr.b_u])
    dt = 0.7
    ref = otl.backward_euler(g, pr.rho, pr.mu, dt, u0, 5, f=f, b_p=pr.b_p)
    sv = S.StokesSolver(dim, pr.n[:dim], pr.bc[:2 * dim], pr.h)
    uu, _ = g.unpack(np.concatenate([u0, np.zeros(g.ncell)]))
    args = (sv, _t(pr.rho), _t(pr.mu), dt, [_t(x) for x in uu])
    kw = dict(f=[_t(x) for x in pr.b_u], b_p=_t(pr.b_p), rtol=1e-12, precision=precision,
              precond=1, maxit=2000)
    u, p, infos = timeloop.backward_euler(*args, 5, **kw)
    x = g.pack([a.cpu().numpy() for a in u], p.cpu().numpy())
    eu, ep = direct.relative_error(g, x, ref[-1])
    assert eu <= 1e-8 and ep <= 1e-8, (eu, ep)
    # every step, by running the loop one step longer each time
    for s in (1, 3):
        u, p, _ = timeloop.backward_euler(*args, s, **kw)
        x = g.pack([a.cpu().numpy() for a in u], p.cpu().numpy())
        assert max(direct.relative_error(g, x, ref[s - 1])) <= 1e-8
    _, _, cold = timeloop.backward_euler(*args, 5, warm=False, **kw)
    assert sum(i["iterations"] for i in infos[1:]) < sum(i["iterations"] for i in cold[1:])
    sv.close()
