"""The persistent multi-block V-cycle (schedule field grid_level) and the
thread-block-cluster V-cycle (cluster_level): the middle levels run as one
cooperative launch with grid-wide barriers, or as one cluster with hardware
cluster barriers, between stages instead of one kernel per colour and
transfer.  Its stages are the
same per-point functions in the same order, so V-cycles and solves equal,
bitwise, those of the per-level kernels; inside a solve it is part of the
cycle graph.  Every barrier wait is bounded: with a budget of zero cycles the
first wait runs out, the solve returns STK_ERR_TIMEOUT without faulting or
hanging, and the handle then solves normally again."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.grid import Grid
from paper_1308_4605_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
DEV = "cuda"
P, W, F = 0, 1, 2


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1308_4605_gb300 import stokes
    return stokes


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(DEV)


def _nlev(n):
    m, k = min(n), 1
    while m > 2:
        m //= 2
        k += 1
    return k


CASES = [(2, (128, 64), (W, F, P, P)), (3, (32, 32, 16), (P,) * 6),
         (3, (64, 32, 32), (W, W, P, P, F, W))]


@pytest.mark.parametrize("dim,n,bc", CASES)
def test_grid_kernel_equals_per_level_kernels(S, dim, n, bc):
    theta = 1.0 if bc[0] == P else 0.0
    pr = wl.generic(dim, n, bc, theta=theta, seed=21, precond=1 if theta else 2)
    sv = S.StokesSolver(dim, pr.n[:dim], pr.bc[:2 * dim], pr.h)
    sv.set_coefficients(_t(pr.rho), _t(pr.mu), pr.theta)
    g = Grid(dim, pr.n, pr.h, pr.bc)
    rng = np.random.default_rng(4)
    ru, rp = g.unpack(rng.standard_normal(g.size) * g.active)
    ru = [_t(x) for x in ru]
    rp = _t(rp - rp.mean())
    bu, bp = [_t(x) for x in pr.b_u], _t(pr.b_p)
    nl = _nlev(n)
    out = {}
    for prec in (0, 1):
        # per-level kernels down to level 3, block kernel below; then the
        # grid kernel (gl) or the cluster kernel (cl) from level 1 or 2 down
        # to the block kernel
        for lc, gl, cl in ((3, 3, 3), (3, 1, 3), (3, 2, 3), (nl, 1, nl), (3, 3, 1), (3, 3, 2),
                           (nl, nl, 1)):
            S.stk_set_schedule(sv.handle, prec, lc, 256, lc, gl, cl)
            res = []
            if prec == 0:
                xu = [torch.zeros_like(x) for x in ru]
                xp = torch.zeros_like(rp)
                S.stk_velocity_vcycle(sv.handle, ru, xu)
                S.stk_pressure_vcycle(sv.handle, rp, xp)
                res += xu + [xp]
            su, sp, info = sv.solve(bu, bp, precision=prec, precond=pr.precond)
            assert info["converged"], info
            assert S.stk_graphs_in_use(sv.handle) == 1
            res += list(su) + [sp, info["iterations"]]
            out[(prec, lc, gl, cl)] = res
    sv.close()
    for prec in (0, 1):
        ref = out[(prec, 3, 3, 3)]
        for key, res in out.items():
            if key[0] != prec:
                continue
            assert res[-1] == ref[-1], key
            for a, b in zip(res[:-1], ref[:-1]):
                assert torch.equal(a, b), key


def test_bounded_wait_runs_out_without_fault(S):
    pr = wl.config_c3(32)
    sv = S.StokesSolver(3, pr.n, pr.bc, pr.h)
    sv.set_coefficients(_t(pr.rho), _t(pr.mu), pr.theta)
    bu, bp = [_t(x) for x in pr.b_u], _t(pr.b_p)
    S.stk_set_schedule(sv.handle, 0, 3, 256, 3, 1)
    _, _, ref = sv.solve(bu, bp)
    assert ref["converged"]
    S.stk_set_wait_budget(sv.handle, 0)
    with pytest.raises(S.StokesError) as e:
        sv.solve(bu, bp)
    assert e.value.code == S.STK_ERR_TIMEOUT
    assert S.stk_wait_status(sv.handle, reset=True) == S.STK_ERR_TIMEOUT
    assert S.stk_wait_status(sv.handle) == S.STK_OK
    S.stk_set_wait_budget(sv.handle, 2_000_000_000)
    xu, xp, info = sv.solve(bu, bp)
    assert info["converged"] and info["iterations"] == ref["iterations"]
    sv.close()
