"""stk_pressure_vcycle_noalloc: the pressure V-cycle for callers that cannot
allocate device memory (their GPU memory belongs to another allocator, or
their loop cannot afford cudaMalloc's synchronisation).  Its output must equal
that of stk_pressure_vcycle on a handle set up with the same density, on two
calls in a row that reuse the shared workspace array with different grids."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1308_4605_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

PERIODIC, NOSLIP, FREESLIP = 0, 1, 2


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1308_4605_gb300 import stokes
    return stokes


def _case(dim, n, bc, seed):
    pr = wl.generic(dim, n, bc, theta=1.0, rho_contrast=50.0, mu_contrast=5.0, seed=seed)
    rng = np.random.default_rng(seed + 100)
    r = rng.standard_normal(pr.rho.shape)
    r -= r.mean()
    return pr, r


def _with_handle(S, pr, r, dev):
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    solver = S.StokesSolver(pr.dim, pr.n[:pr.dim], pr.bc[:2 * pr.dim], pr.h)
    solver.set_coefficients(t(pr.rho), t(pr.mu), pr.theta)
    x = torch.zeros(pr.rho.shape, dtype=torch.float64, device=dev)
    S.stk_pressure_vcycle(solver.handle, t(r), x)
    torch.cuda.synchronize()
    solver.close()
    return x.cpu().numpy()


def _no_alloc(S, pr, r, dev):
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    x = torch.full(pr.rho.shape, float("nan"), dtype=torch.float64, device=dev)
    S.stk_pressure_vcycle_noalloc(pr.dim, pr.n[:pr.dim], pr.h, pr.bc[:2 * pr.dim], t(pr.rho), t(r), x)
    torch.cuda.synchronize()
    return x.cpu().numpy()


def test_no_alloc_matches_handle_on_two_calls_in_a_row(S):
    dev = torch.device("cuda", 0)
    cases = [_case(3, (16, 16, 16), (PERIODIC,) * 6, 1),
             _case(2, (64, 32), (NOSLIP, FREESLIP, NOSLIP, NOSLIP), 2)]
    refs = [_with_handle(S, pr, r, dev) for pr, r in cases]
    for (pr, r), ref in zip(cases, refs):          # two calls in a row
        got = _no_alloc(S, pr, r, dev)
        assert np.isfinite(got).all()
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    # the same grid twice: the second call must not see the first call's leftovers
    pr, r = cases[1]
    again = _no_alloc(S, pr, r, dev)
    assert np.abs(again - refs[1]).max() <= 1e-12 * np.abs(refs[1]).max()


def test_no_alloc_leaves_free_memory_unchanged(S):
    """After a warm-up call (which, under lazy module loading, places the
    workspace array and the kernels' code on the device), a call allocates
    nothing: the device's free memory is the same before and after it."""
    dev = torch.device("cuda", 0)
    pr, r = _case(3, (32, 32, 32), (NOSLIP,) * 6, 3)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    rho, rr = t(pr.rho), t(r)
    x = torch.zeros(pr.rho.shape, dtype=torch.float64, device=dev)
    call = lambda: S.stk_pressure_vcycle_noalloc(pr.dim, pr.n[:3], pr.h, pr.bc[:6], rho, rr, x)
    call()                                        # warm-up
    torch.cuda.synchronize()
    first = x.clone()
    free0, _ = torch.cuda.mem_get_info(dev)
    call()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info(dev)
    assert free1 == free0, (free0, free1)
    assert torch.equal(x, first)


def test_no_alloc_rejects_oversized_grids(S):
    """A 128^3 grid needs about 12.6M doubles of workspace, more than the
    2,097,152 of the array: rejected before any device work."""
    import ctypes
    dev = torch.device("cuda", 0)
    dummy = torch.ones(4, dtype=torch.float64, device=dev)
    ptr = ctypes.c_void_p(dummy.data_ptr())
    nn = (ctypes.c_int * 3)(128, 128, 128)
    bb = (ctypes.c_int * 6)(0, 0, 0, 0, 0, 0)
    rc = S.library().stk_pressure_vcycle_noalloc(3, nn, 1.0, bb, ptr, ptr, ptr, None)
    assert rc == S.STK_ERR_SIZE
    assert bool(torch.all(dummy == 1.0))
