"""Stacked batches (stk_create_stacked): same-shape 2D instances stored along a
third array axis, solved by one set of kernel launches for all of them.

Each instance is the 2D system of Sec. 3.1 on its own, so an instance of the
stack must give what a single handle gives for it: the operator and the
preconditioners bitwise (with a sweeping coarsest level, ncoarse != 8: the
single handle applies a precomputed coarse-solve matrix for ncoarse = 8), the
GMRES solve bitwise too (per-instance reductions in the single handle's
order), and the default parameters to rounding.  Solutions are also checked
against the oracle's exact discrete solutions (1e-8), and the per-instance
bookkeeping on instances that converge at different iterations, that have a
zero or a non-finite right-hand side, or that run out of iterations."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import assemble as asm
from oracle import direct
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


def _instances(n, bc, count, seed=0, theta=1.0, mu_contrasts=None):
    prs = []
    for i in range(count):
        mc = mu_contrasts[i] if mu_contrasts else 10.0 + 40.0 * i
        prs.append(wl.generic(2, n, bc, theta=theta, rho_contrast=5.0, mu_contrast=mc, seed=seed + 17 * i))
    return prs


def _stack(S, prs):
    """One stacked handle for the problems prs (same grid) and the stacked
    right-hand side; plus a single handle per problem."""
    pr0 = prs[0]
    K = len(prs)
    st = S.StokesSolver(2, pr0.n[:2], pr0.bc[:4], pr0.h, count=K)
    rho = _t(np.stack([p.rho for p in prs]))
    mu = _t(np.stack([p.mu for p in prs]))
    st.set_coefficients(rho.reshape(st.cell_shape()), mu.reshape(st.cell_shape()), pr0.theta)
    bu = [_t(np.stack([p.b_u[a] for p in prs])).reshape(st.face_shape(a)) for a in range(2)]
    bp = _t(np.stack([p.b_p for p in prs])).reshape(st.cell_shape())
    singles = []
    for p in prs:
        sv = S.StokesSolver(2, p.n[:2], p.bc[:4], p.h)
        sv.set_coefficients(_t(p.rho), _t(p.mu), p.theta)
        singles.append(sv)
    return st, bu, bp, singles


def _slice(arrs, i):
    return [a[i] for a in arrs]


def _eq(a, b):
    """bitwise equal values (a single handle's arrays carry a leading axis of 1)"""
    return torch.equal(a.reshape(-1), b.reshape(-1))


def _eqv(us, vs):
    return all(_eq(a, b) for a, b in zip(us, vs))


def _close(st, singles):
    st.close()
    for sv in singles:
        sv.close()


GRIDS = [((32, 16), (PERIODIC,) * 4), ((16, 32), (NOSLIP, NOSLIP, FREESLIP, FREESLIP)),
         ((64, 64), (PERIODIC,) * 4), ((32, 32), (NOSLIP,) * 4)]


@pytest.mark.parametrize("n,bc", GRIDS)
def test_stacked_shapes(S, n, bc):
    prs = _instances(n, bc, 3)
    st, bu, bp, singles = _stack(S, prs)
    assert S.stk_stack_count(st.handle) == 3
    assert S.stk_stack_count(singles[0].handle) == 1
    for a in range(2):
        assert S.stk_face_length(st.handle, a) == 3 * S.stk_face_length(singles[0].handle, a)
    assert S.stk_cell_length(st.handle) == 3 * S.stk_cell_length(singles[0].handle)
    _close(st, singles)


@pytest.mark.parametrize("n,bc", GRIDS)
def test_stacked_operator_bitwise(S, n, bc):
    prs = _instances(n, bc, 3, seed=5)
    st, bu, bp, singles = _stack(S, prs)
    yu, yp = st.apply_operator(bu, bp)
    for i, sv in enumerate(singles):
        zu, zp = sv.apply_operator(_slice(bu, i), bp[i])
        assert _eqv(zu, _slice(yu, i))
        assert _eq(zp, yp[i])
    _close(st, singles)


@pytest.mark.parametrize("n,bc", GRIDS)
@pytest.mark.parametrize("precision", [0, 1])
def test_stacked_preconditioners_bitwise(S, n, bc, precision):
    """Every preconditioner (V-cycles, means, Schur complement algebra) with
    a sweeping coarsest level: bitwise per instance."""
    theta = 1.0 if bc[0] == PERIODIC else 0.0
    prs = _instances(n, bc, 3, seed=9, theta=theta)
    st, bu, bp, singles = _stack(S, prs)
    for which in (1, 2, 3, 4, 5):
        xu, xp = st.apply_preconditioner(which, bu, bp, precision=precision, ncoarse=6)
        for i, sv in enumerate(singles):
            zu, zp = sv.apply_preconditioner(which, _slice(bu, i), bp[i], precision=precision, ncoarse=6)
            assert _eqv(zu, _slice(xu, i)), (which, i)
            assert _eq(zp, xp[i]), (which, i)
    _close(st, singles)


@pytest.mark.parametrize("n,bc", GRIDS[:2])
def test_stacked_preconditioner_default_matches(S, n, bc):
    """Default parameters (the single handle's coarse-solve matrix): equal to
    rounding."""
    prs = _instances(n, bc, 2, seed=13)
    st, bu, bp, singles = _stack(S, prs)
    xu, xp = st.apply_preconditioner(1, bu, bp)
    for i, sv in enumerate(singles):
        zu, zp = sv.apply_preconditioner(1, _slice(bu, i), bp[i])
        for a, b in zip(zu + [zp], _slice(xu, i) + [xp[i]]):
            a, b = a.reshape(-1), b.reshape(-1)
            assert torch.linalg.norm(a - b) <= 1e-12 * torch.linalg.norm(a)
    _close(st, singles)


@pytest.mark.parametrize("n,bc", GRIDS)
@pytest.mark.parametrize("precision", [0, 1])
def test_stacked_solve_bitwise(S, n, bc, precision):
    """GMRES per instance inside the stack: the same iterations and bitwise
    the same solution as the instance solved alone (ncoarse = 6)."""
    theta = 1.0 if bc[0] == PERIODIC else 0.0
    prs = _instances(n, bc, 4, seed=21, theta=theta, mu_contrasts=[2.0, 30.0, 300.0, 1000.0])
    st, bu, bp, singles = _stack(S, prs)
    pc = 1 if theta else 2
    xu, xp, info = st.solve(bu, bp, precond=pc, precision=precision, ncoarse=6)
    torch.cuda.synchronize()
    assert info["converged"], info
    its = []
    for i, sv in enumerate(singles):
        zu, zp, inf1 = sv.solve(_slice(bu, i), bp[i], precond=pc, precision=precision, ncoarse=6)
        rec = st.instance_info(i)
        assert rec["converged"] and rec["status"] == 0
        assert rec["iterations"] == inf1["iterations"], (i, rec, inf1)
        assert rec["true_residual"] == inf1["true_residual"]
        assert _eqv(zu, _slice(xu, i)), i
        assert _eq(zp, xp[i]), i
        assert S.stk_stack_history(st.handle, i, 0) == S.stk_solve_history(sv.handle, 0)
        assert S.stk_stack_history(st.handle, i, 1) == S.stk_solve_history(sv.handle, 1)
        its.append(rec["iterations"])
    assert info["iterations"] == max(its)
    _close(st, singles)


@pytest.mark.parametrize("precision", [0, 1])
def test_stacked_solve_matches_oracle(S, precision):
    """Instances of the batched workload (64^2 periodic, mu contrast 1e3) in
    one stack: each matches the oracle's exact discrete solution."""
    prs = [wl.config_c4_instance(i, 64) for i in range(5)]
    st, bu, bp, singles = _stack(S, prs)
    xu, xp, info = st.solve(bu, bp, precond=1, precision=precision)
    torch.cuda.synchronize()
    assert info["converged"], info
    for i, pr in enumerate(prs):
        g = Grid(2, pr.n, pr.h, pr.bc)
        M = asm.stokes_from_fields(g, pr.rho, pr.mu, pr.theta)
        b = g.pack(pr.b_u, pr.b_p)
        x = g.pack([v[i].cpu().numpy() for v in xu], xp[i].cpu().numpy())
        assert np.linalg.norm(b - M @ x) <= 1.0001e-10 * np.linalg.norm(b)
        assert max(direct.relative_error(g, x, direct.solve(g, M, b))) <= 1e-8
    _close(st, singles)


def test_stacked_zero_and_nonfinite_instances(S):
    """A zero right-hand side gives x = 0 at once; a non-finite one fails
    that instance alone; the others converge as if alone."""
    prs = _instances((32, 32), (PERIODIC,) * 4, 4, seed=33)
    st, bu, bp, singles = _stack(S, prs)
    for a in range(2):
        bu[a][1].zero_()
    bp[1].zero_()
    bp[3][0, 5] = float("nan")
    x_u, x_p = st.zeros()
    for a in range(2):
        x_u[a].fill_(1.0)
    x_p.fill_(1.0)
    with pytest.raises(S.StokesError) as e:
        st.solve(bu, bp, x_u, x_p, precond=1, ncoarse=6)
    assert e.value.code == S.STK_ERR_NONFINITE
    assert "instance 3" in str(e.value)
    torch.cuda.synchronize()
    r1 = st.instance_info(1)
    assert r1["converged"] and r1["iterations"] == 0
    assert all(float(torch.abs(v[1]).max()) == 0.0 for v in x_u) and float(torch.abs(x_p[1]).max()) == 0.0
    assert st.instance_info(3)["status"] == S.STK_ERR_NONFINITE
    for i in (0, 2):
        zu, zp = singles[i].zeros()
        for v in zu + [zp]:
            v.fill_(1.0)
        _, _, inf1 = singles[i].solve(_slice(bu, i), bp[i], zu, zp, precond=1, ncoarse=6)
        rec = st.instance_info(i)
        assert rec["converged"] and rec["iterations"] == inf1["iterations"]
        assert _eqv(zu, _slice(x_u, i)) and _eq(zp, x_p[i])
    _close(st, singles)


def test_stacked_maxit(S):
    """maxit reached by some instances: NOT_CONVERGED for the solve, per
    instance status and iteration counts as alone."""
    prs = _instances((32, 32), (NOSLIP,) * 4, 3, seed=45, theta=0.0, mu_contrasts=[1.0, 100.0, 1000.0])
    st, bu, bp, singles = _stack(S, prs)
    x_u, x_p = st.zeros()
    _, _, info = st.solve(bu, bp, x_u, x_p, precond=2, maxit=6, ncoarse=6)
    torch.cuda.synchronize()
    assert not info["converged"] and info["status"] == S.STK_ERR_NOT_CONVERGED
    conv = []
    for i, sv in enumerate(singles):
        zu, zp = sv.zeros()
        _, _, inf1 = sv.solve(_slice(bu, i), bp[i], zu, zp, precond=2, maxit=6, ncoarse=6)
        rec = st.instance_info(i)
        assert rec["iterations"] == inf1["iterations"] <= 6
        assert rec["converged"] == inf1["converged"]
        assert rec["status"] == (0 if inf1["converged"] else S.STK_ERR_NOT_CONVERGED)
        assert _eqv(zu, _slice(x_u, i)) and _eq(zp, x_p[i])
        conv.append(rec["converged"])
    assert not all(conv)
    _close(st, singles)


def test_stacked_autotune_and_graphs_off(S):
    """The autotuned schedule and the host-gated (graphs off) path give the
    same solution as the default schedule."""
    prs = [wl.config_c4_instance(i, 128) for i in range(3)]
    st, bu, bp, singles = _stack(S, prs)
    xu0, xp0, info0 = st.solve(bu, bp, precond=1, precision=1, ncoarse=6)
    sc = S.stk_autotune(st.handle, 1)
    assert sc["grid_level"] >= sc["coarse_level"]
    xu1, xp1, info1 = st.solve(bu, bp, precond=1, precision=1, ncoarse=6)
    assert info1["iterations"] == info0["iterations"]
    assert _eqv(xu0, xu1) and _eq(xp0, xp1)
    S.stk_set_graphs(st.handle, 0)
    xu2, xp2, info2 = st.solve(bu, bp, precond=1, precision=1, ncoarse=6)
    assert _eqv(xu0, xu2) and _eq(xp0, xp2)
    _close(st, singles)


def test_stacked_one_instance_equals_single(S):
    prs = _instances((64, 32), (PERIODIC, PERIODIC, NOSLIP, NOSLIP), 1, seed=51, theta=1.0)
    st, bu, bp, singles = _stack(S, prs)
    xu, xp, info = st.solve(bu, bp, precond=1, ncoarse=6)
    zu, zp, inf1 = singles[0].solve(_slice(bu, 0), bp[0], precond=1, ncoarse=6)
    assert info["iterations"] == inf1["iterations"]
    assert _eqv(zu, _slice(xu, 0)) and _eq(zp, xp[0])
    _close(st, singles)


def test_stacked_rejects(S):
    with pytest.raises(S.StokesError):
        S.stk_create_stacked(3, (8, 8, 8), 1.0, (PERIODIC,) * 6, 2)
    with pytest.raises(S.StokesError):
        S.stk_create_stacked(2, (8, 8), 1.0, (PERIODIC,) * 4, 0)
    pr = _instances((16, 16), (NOSLIP,) * 4, 2)
    st, bu, bp, singles = _stack(S, pr)
    with pytest.raises(S.StokesError):
        st.set_bulk_viscosity(torch.ones(st.cell_shape(), dtype=torch.float64, device=DEV))
    with pytest.raises(S.StokesError):
        S.stk_set_schedule(st.handle, 0, 2, 256, 2, 0)
    _close(st, singles)


def test_stacked_batch_helper_mixed_sizes(S):
    """paper_1308_4605_gb300.batch.StackedBatch: problems of three grids
    (periodic 32^2 and 64^2, walled 32x16) in one call; each instance equals,
    bitwise, the solve on its own handle (ncoarse = 6), and the oracle's exact
    solution to 1e-8."""
    from paper_1308_4605_gb300.batch import StackedBatch, problem_dict
    prs = (_instances((32, 32), (PERIODIC,) * 4, 3, seed=61)
           + _instances((64, 64), (PERIODIC,) * 4, 2, seed=71)
           + _instances((32, 16), (NOSLIP,) * 4, 2, seed=81))
    prs = [prs[i] for i in (0, 3, 5, 1, 6, 4, 2)]          # interleaved sizes
    sb = StackedBatch([problem_dict(p) for p in prs])
    assert len(sb.groups) == 3
    bus = [[_t(x) for x in p.b_u] for p in prs]
    bps = [_t(p.b_p) for p in prs]
    xu, xp, infos = sb.solve(bus, bps, precond=1, ncoarse=6)
    torch.cuda.synchronize()
    for i, p in enumerate(prs):
        assert infos[i]["converged"], (i, infos[i])
        sv = S.StokesSolver(2, p.n[:2], p.bc[:4], p.h)
        sv.set_coefficients(_t(p.rho), _t(p.mu), p.theta)
        zu, zp, inf1 = sv.solve(bus[i], bps[i], precond=1, ncoarse=6)
        sv.close()
        assert inf1["iterations"] == infos[i]["iterations"]
        assert _eqv(zu, xu[i]) and _eq(zp, xp[i])
        g = Grid(2, p.n, p.h, p.bc)
        M = asm.stokes_from_fields(g, p.rho, p.mu, p.theta)
        b = g.pack(p.b_u, p.b_p)
        x = g.pack([v.cpu().numpy() for v in xu[i]], xp[i].cpu().numpy())
        assert max(direct.relative_error(g, x, direct.solve(g, M, b))) <= 1e-8
    sb.close()


@pytest.mark.parametrize("n,bc", GRIDS[:2])
def test_stacked_entry_points_per_instance(S, n, bc):
    """The other calls on a stacked handle act on each instance as alone:
    the two V-cycles, repeated V-cycles per subsolve (P1..P5, 2 + 3 cycles,
    sweeping coarsest level), the pressure mean removal and the
    backward-Euler right-hand side, bitwise; the V-cycles with the default
    coarsest solve to 1e-12."""
    theta = 1.0
    prs = _instances(n, bc, 3, seed=91, theta=theta)
    st, bu, bp, singles = _stack(S, prs)
    # V-cycles (default parameters)
    xu = [torch.zeros_like(v) for v in bu]
    xp = torch.zeros_like(bp)
    S.stk_velocity_vcycle(st.handle, bu, xu)
    S.stk_pressure_vcycle(st.handle, bp - bp.mean(dim=(1, 2), keepdim=True), xp)
    for i, sv in enumerate(singles):
        zu, zp = sv.zeros()
        S.stk_velocity_vcycle(sv.handle, _slice(bu, i), zu)
        rp = (bp[i] - bp[i].mean()).reshape(zp.shape).contiguous()
        S.stk_pressure_vcycle(sv.handle, rp, zp)
        for a, b in zip(zu + [zp], _slice(xu, i) + [xp[i]]):
            a, b = a.reshape(-1), b.reshape(-1)
            assert torch.linalg.norm(a - b) <= 1e-12 * torch.linalg.norm(a)
    # repeated V-cycles per subsolve
    for which in (1, 2, 3, 4, 5):
        xu, xp = st.apply_preconditioner(which, bu, bp, ncoarse=6, vcycles_u=2, vcycles_p=3)
        for i, sv in enumerate(singles):
            zu, zp = sv.apply_preconditioner(which, _slice(bu, i), bp[i], ncoarse=6, vcycles_u=2,
                                             vcycles_p=3)
            assert _eqv(zu, _slice(xu, i)) and _eq(zp, xp[i]), which
    # mean removal
    yp = torch.empty_like(bp)
    S.stk_remove_mean(st.handle, bp, yp)
    for i, sv in enumerate(singles):
        zp = torch.empty_like(bp[i])
        S.stk_remove_mean(sv.handle, bp[i].contiguous(), zp)
        assert _eq(zp, yp[i])
    # backward-Euler right-hand side
    fu = [torch.randn_like(v) for v in bu]
    ou = [torch.empty_like(v) for v in bu]
    S.stk_backward_euler_rhs(st.handle, bu, fu, ou)
    for i, sv in enumerate(singles):
        zu = [torch.empty_like(v) for v in _slice(bu, i)]
        S.stk_backward_euler_rhs(sv.handle, [v.contiguous() for v in _slice(bu, i)],
                                 [v.contiguous() for v in _slice(fu, i)], zu)
        assert _eqv(zu, _slice(ou, i))
    _close(st, singles)
