"""Adjoint gradient on the GPU (stk_gradient and the autograd wrapper) against
the oracle's gradient and central finite differences.

Tolerances: the gradient kernel is pure FP64 arithmetic on given (u, lambda):
1e-12 relative to the oracle's sparse-matrix evaluation.  End-to-end
gradients (GPU solves to 1e-12) must match the oracle's (direct solves) and
central differences to 1e-6 relative, the bound of the differentiation form."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import direct, gradient
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


@pytest.mark.parametrize("dim,n,bc,theta", [
    (2, (16, 8), (NOSLIP,) * 4, 1.3),
    (2, (8, 16), (PERIODIC, PERIODIC, FREESLIP, NOSLIP), 0.0),
    (3, (8, 8, 4), (NOSLIP, FREESLIP, PERIODIC, PERIODIC, NOSLIP, NOSLIP), 0.7),
    (3, (8, 8, 8), (PERIODIC,) * 6, 1.0),
])
def test_gradient_kernel_matches_oracle(S, dim, n, bc, theta):
    pr = wl.generic(dim, n, bc, theta=theta, seed=31)
    g = Grid(dim, pr.n, pr.h, pr.bc)
    rng = np.random.default_rng(7)
    u = rng.standard_normal(g.size) * g.active
    lam = rng.standard_normal(g.size) * g.active
    ref_mu = pr.mu.ravel() * gradient.viscosity_gradient(g, pr.mu, u[:g.nvel], lam[:g.nvel])
    ref_rho = gradient.density_gradient(g, theta, u[:g.nvel], lam[:g.nvel])
    solver = S.StokesSolver(dim, pr.n[:dim], pr.bc[:2 * dim], pr.h)
    solver.set_coefficients(_t(pr.rho), _t(pr.mu), theta)
    uu, _ = g.unpack(u)
    ll, _ = g.unpack(lam)
    dmu = torch.empty(g.cell_shape(), dtype=torch.float64, device=DEV)
    drho = torch.empty_like(dmu)
    S.stk_gradient(solver.handle, [_t(x) for x in uu], [_t(x) for x in ll], dmu, drho)
    assert np.abs(dmu.cpu().numpy().ravel() - ref_mu).max() <= 1e-12 * np.abs(ref_mu).max()
    if theta != 0.0:
        assert np.abs(drho.cpu().numpy().ravel() - ref_rho).max() <= 1e-12 * np.abs(ref_rho).max()
    else:
        assert float(drho.abs().max()) == 0.0
    solver.close()


def _loss_setup(S, pr, seed):
    from paper_1308_4605_gb300 import adjoint
    g = Grid(pr.dim, pr.n, pr.h, pr.bc)
    solver = S.StokesSolver(pr.dim, pr.n[:pr.dim], pr.bc[:2 * pr.dim], pr.h)
    rng = np.random.default_rng(seed)
    u_t = rng.standard_normal(g.nvel) * g.active[:g.nvel]
    ut, _ = g.unpack(np.concatenate([u_t, np.zeros(g.ncell)]))
    ut = [_t(x) for x in ut]
    b_u = [_t(x) for x in pr.b_u]
    b_p = _t(pr.b_p)

    def loss(log_mu, rho, rtol=1e-12, precision=0):
        out = adjoint.stokes_solve(solver, log_mu, rho, pr.theta, b_u, b_p, precond=pr.precond,
                                   rtol=rtol, precision=precision, maxit=4000)
        return 0.5 * sum(((o - t) ** 2).sum() for o, t in zip(out[:pr.dim], ut))

    return g, solver, u_t, loss


@pytest.mark.parametrize("cfg,precision", [("c5", 0), ("c5", 1), ("c1", 0)])
def test_autograd_matches_oracle_gradient(S, cfg, precision):
    """Gradients w.r.t. log mu and rho from one forward and one adjoint solve
    equal the oracle's (direct solves) to 1e-6."""
    pr = wl.config_c5(16) if cfg == "c5" else wl.config_c1(32)
    g, solver, u_t, loss = _loss_setup(S, pr, 3)
    log_mu = _t(np.log(pr.mu)).requires_grad_(True)
    rho = _t(pr.rho).requires_grad_(True)
    L = loss(log_mu, rho, precision=precision)
    L.backward()
    b = g.pack(pr.b_u, pr.b_p)
    Lr, glogmu, grho, _, _ = gradient.loss_and_gradient(
        g, pr.rho, pr.mu, pr.theta, b, u_t, lambda M, r: direct.solve(g, M, r))
    assert abs(float(L.detach()) - Lr) <= 1e-8 * abs(Lr)
    gm = log_mu.grad.cpu().numpy().ravel()
    assert np.linalg.norm(gm - glogmu) <= 1e-6 * np.linalg.norm(glogmu)
    if pr.theta != 0.0:
        gr = rho.grad.cpu().numpy().ravel()
        assert np.linalg.norm(gr - grho) <= 1e-6 * np.linalg.norm(grho)
    solver.close()


def test_adjoint_64_finite_differences(S):
    """The 64^3 no-slip steady adjoint workload: loss 1/2 ||u - u_target||^2
    with u_target the solution for a second seeded viscosity field; the
    gradient w.r.t. log mu is checked by central differences along 16 seeded
    directions (eps = 1e-4, solves to 1e-12).  The directions are seeded
    smooth fields (|k| <= 4 Fourier modes, unit norm) like the log-viscosity
    itself: along white noise the directional derivative is ~sqrt(N) smaller
    than |grad L| and the difference quotient measures solver round-off."""
    from paper_1308_4605_gb300 import adjoint
    pr = wl.config_c5(64)
    prt = wl.config_c5(64, target=True)
    solver = S.StokesSolver(3, pr.n, pr.bc, pr.h)
    b_u = [_t(x) for x in pr.b_u]
    b_p = _t(pr.b_p)
    with torch.no_grad():
        ut = adjoint.stokes_solve(solver, _t(np.log(prt.mu)), _t(prt.rho), 0.0, b_u, b_p,
                                  precond=2, rtol=1e-12, maxit=4000)[:3]
        ut = [x.clone() for x in ut]

    def loss(log_mu, rtol=1e-12):
        out = adjoint.stokes_solve(solver, log_mu, _t(pr.rho), 0.0, b_u, b_p, precond=2,
                                   rtol=rtol, maxit=4000)
        return 0.5 * sum(((o - t) ** 2).sum() for o, t in zip(out[:3], ut))

    lm = _t(np.log(pr.mu)).requires_grad_(True)
    L = loss(lm, rtol=1e-12)
    L.backward()
    grad = lm.grad.detach()
    eps = 1e-4
    worst = 0.0
    with torch.no_grad():
        for k in range(16):
            d = _t(wl.smooth_field_3d(pr.n, pr.h, 500 + k, kmax=4))
            d /= torch.linalg.norm(d)
            fd = (float(loss(lm + eps * d)) - float(loss(lm - eps * d))) / (2 * eps)
            an = float((grad * d).sum())
            worst = max(worst, abs(fd - an) / abs(fd))
    assert worst <= 1e-6, worst
    solver.close()


@pytest.mark.parametrize("dim,n,bc,theta", [
    (2, (32, 16), (NOSLIP, NOSLIP, FREESLIP, NOSLIP), 0.7),
    (3, (16, 16, 8), (PERIODIC, PERIODIC, NOSLIP, NOSLIP, FREESLIP, FREESLIP), 1.0),
])
def test_adjoint_identity(S, dim, n, bc, theta):
    """<y, M x> = <M y, x> for the GPU operator (M is its own adjoint, so the
    adjoint solve is a forward solve), on random x, y with zero wall faces."""
    pr = wl.generic(dim, n, bc, theta=theta, seed=51)
    g = Grid(dim, pr.n, pr.h, pr.bc)
    sv = S.StokesSolver(dim, pr.n[:dim], pr.bc[:2 * dim], pr.h)
    sv.set_coefficients(_t(pr.rho), _t(pr.mu), theta)
    rng = np.random.default_rng(9)
    x = rng.standard_normal(g.size) * g.active
    y = rng.standard_normal(g.size) * g.active
    xu, xp = g.unpack(x)
    yu, yp = g.unpack(y)
    Mxu, Mxp = sv.apply_operator([_t(a) for a in xu], _t(xp))
    Myu, Myp = sv.apply_operator([_t(a) for a in yu], _t(yp))
    Mx = g.pack([a.cpu().numpy() for a in Mxu], Mxp.cpu().numpy())
    My = g.pack([a.cpu().numpy() for a in Myu], Myp.cpu().numpy())
    lhs, rhs = float(y @ Mx), float(My @ x)
    scale = np.linalg.norm(y) * np.linalg.norm(Mx)
    assert abs(lhs - rhs) <= 1e-13 * scale
    sv.close()


def test_gradient_taylor_remainder(S):
    """Taylor test of the autograd gradient on the 16^3 no-slip workload:
    |L(m + eps d) - L(m) - eps <grad L, d>| falls as eps^2 (ratio about 4
    per halving of eps) while the first-order remainder falls as eps."""
    pr = wl.config_c5(16)
    g, solver, u_t, loss = _loss_setup(S, pr, 12)
    lm = _t(np.log(pr.mu)).requires_grad_(True)
    rho = _t(pr.rho)
    L0 = loss(lm, rho)
    L0.backward()
    grad = lm.grad.detach()
    d = _t(wl.smooth_field_3d(pr.n, pr.h, 901, kmax=4))
    d /= torch.linalg.norm(d)
    slope = float((grad * d).sum())
    rem2, rem1 = [], []
    with torch.no_grad():
        for eps in (0.04, 0.02, 0.01, 0.005):
            Le = float(loss(lm + eps * d, rho))
            rem1.append(abs(Le - float(L0)))
            rem2.append(abs(Le - float(L0) - eps * slope))
    r1 = [rem1[i] / rem1[i + 1] for i in range(3)]
    r2 = [rem2[i] / rem2[i + 1] for i in range(3)]
    assert all(1.7 <= r <= 2.3 for r in r1), r1
    assert all(3.4 <= r <= 4.6 for r in r2), r2
    solver.close()


@pytest.mark.parametrize("n,inplace", [((16, 8), False), ((64, 64), True), ((32, 16, 8), False)])
def test_remove_mean(S, n, inplace):
    """stk_remove_mean: y = x - mean(x) on a cell array (the projection the
    adjoint applies to the pressure part of its right-hand side)."""
    dim = len(n)
    solver = S.StokesSolver(dim, n, (PERIODIC,) * (2 * dim), 1.0)
    one = torch.ones(solver.cell_shape(), dtype=torch.float64, device=DEV)
    solver.set_coefficients(one, one, 1.0)
    x = np.random.default_rng(3).standard_normal(solver.cell_shape()) + 2.5
    xt = _t(x)
    y = xt if inplace else torch.empty_like(xt)
    S.stk_remove_mean(solver.handle, xt, y)
    ref = x - x.mean()
    got = y.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()
    assert abs(got.mean()) <= 1e-14 * np.abs(got).max() * 10
    solver.close()
