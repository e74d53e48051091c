"""GMRES with its least-squares problem on the device (Sec. 3.2): every
cycle runs as one CUDA graph whose phases (the stopping test, the first
basis vector, each Arnoldi step, the update of x) are gated by conditional
nodes that the Givens kernel sets; with profiling on, the host gates the
same phases itself.  Both orders of the same kernels give bitwise equal
solutions, and the residual history agrees with the info record."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.grid import PERIODIC, NOSLIP, FREESLIP
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


PROBLEMS = [
    lambda: wl.config_c1(32),
    lambda: wl.generic(3, (16, 16, 8), (NOSLIP,) * 6, theta=0.0, mu_contrast=50.0, seed=41, precond=2),
    lambda: wl.generic(2, (64, 32), (FREESLIP, NOSLIP, PERIODIC, PERIODIC), theta=1.0, seed=5, precond=3),
]


@pytest.mark.parametrize("k", range(len(PROBLEMS)))
@pytest.mark.parametrize("precision", [0, 1])
def test_graph_gated_cycles_equal_host_gated(S, k, precision):
    pr = PROBLEMS[k]()
    sv = S.StokesSolver(pr.dim, pr.n[:pr.dim], pr.bc[:2 * pr.dim], pr.h)
    sv.set_coefficients(_t(pr.rho), _t(pr.mu), pr.theta)
    bu, bp = [_t(x) for x in pr.b_u], _t(pr.b_p)
    out = []
    # graph-gated, host-gated (profiling), graph-gated again, graphs off
    for prof, graphs in ((0, 1), (1, 1), (0, 1), (0, 0)):
        S.stk_profile(sv.handle, prof)
        S.stk_set_graphs(sv.handle, graphs)
        xu, xp, info = sv.solve(bu, bp, precond=pr.precond, precision=precision, restart=7)
        assert info["converged"], info
        out.append(([a.cpu().numpy() for a in xu], xp.cpu().numpy(), info))
    S.stk_profile(sv.handle, 0)
    S.stk_set_graphs(sv.handle, 1)
    sv.close()
    for xu, xp, info in out[1:]:
        assert info["iterations"] == out[0][2]["iterations"]
        assert info["restarts"] == out[0][2]["restarts"]
        assert all(np.array_equal(a, b) for a, b in zip(xu, out[0][0]))
        assert np.array_equal(xp, out[0][1])


@pytest.mark.parametrize("precision", [0, 1])
def test_residual_history(S, precision):
    pr = wl.config_c1(32)
    sv = S.StokesSolver(2, pr.n[:2], pr.bc[:4], pr.h)
    sv.set_coefficients(_t(pr.rho), _t(pr.mu), pr.theta)
    xu, xp, info = sv.solve([_t(x) for x in pr.b_u], _t(pr.b_p), precision=precision, restart=5)
    true = S.stk_solve_history(sv.handle, 0)
    est = S.stk_solve_history(sv.handle, 1)
    sv.close()
    assert info["converged"] and info["restarts"] >= 2
    # one true residual per cycle start plus the final one
    assert len(true) == info["restarts"] + 1
    assert true[0] == pytest.approx(1.0, rel=1e-14)        # x0 = 0
    assert true[-1] == info["true_residual"] <= 1e-10
    assert all(t > 1e-10 for t in true[:-1])
    assert len(est) == info["iterations"]
    assert est[-1] == pytest.approx(info["est_residual"], rel=1e-14)
    if precision == 1:   # the flexible estimate is the true residual at cycle ends
        ends = np.cumsum([5] * (len(true) - 1))
        ends[-1] = len(est)
        for c, e in enumerate(ends):
            if true[c + 1] > 1e-7:   # above the rounding floor of the true residual
                assert est[e - 1] == pytest.approx(true[c + 1], rel=1e-6)


def test_zero_rhs_and_maxit(S):
    pr = wl.config_c1(16)
    sv = S.StokesSolver(2, pr.n[:2], pr.bc[:4], pr.h)
    sv.set_coefficients(_t(pr.rho), _t(pr.mu), pr.theta)
    zu = [torch.zeros_like(_t(x)) for x in pr.b_u]
    xu, xp, info = sv.solve(zu, torch.zeros_like(_t(pr.b_p)))
    assert info["converged"] and info["iterations"] == 0
    assert all(float(a.abs().max()) == 0.0 for a in xu)
    xu, xp, info = sv.solve([_t(x) for x in pr.b_u], _t(pr.b_p), maxit=3)
    assert not info["converged"] and info["iterations"] == 3
    assert info["status"] == S.STK_ERR_NOT_CONVERGED
    sv.close()


def test_widening_is_bitwise_the_conversion_instruction(S):
    """stk_widen (integer construction of the binary64 encoding, used for the
    FP32 preconditioner outputs of the flexible solve) equals the hardware
    conversion bit for bit: random bit patterns plus zeros, subnormals, the
    extreme normals, infinities and NaN."""
    rng = np.random.default_rng(12)
    bits = rng.integers(0, 2 ** 32, size=1 << 20, dtype=np.uint64).astype(np.uint32)
    special = np.array([0x00000000, 0x80000000, 0x00000001, 0x807fffff, 0x00800000, 0x7f7fffff,
                        0xff7fffff, 0x7f800000, 0xff800000, 0x7fc00000, 0x3f800000, 0xbf800001],
                       dtype=np.uint32)
    bits = np.concatenate([bits, special])
    x = torch.from_numpy(bits.view(np.float32).copy()).to(DEV)
    y = torch.empty(x.numel(), dtype=torch.float64, device=DEV)
    S.stk_widen(x, y)
    ref = x.double()
    yb, rb = y.cpu().numpy().view(np.uint64), ref.cpu().numpy().view(np.uint64)
    nan = np.isnan(ref.cpu().numpy())
    assert np.array_equal(yb[~nan], rb[~nan])
    assert np.isnan(y.cpu().numpy()[nan]).all()
