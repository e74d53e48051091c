"""The 2D steady workload with sharp inclusions (20 disks of mu = 1e4 in
mu = 1, no-slip walls, P2) on the oracle's side: the App. C velocity V-cycle
(rediscretised coarse operators with averaged / injected coefficients,
Sec. 4.1.1) diverges on the sharp jumps, and GMRES(10) with one V-cycle per
subsolve stalls far above the 1e-10 target.  The paper claims robustness
only for contrasts of 1e2-1e3 with jumps smoothed over a few cells (Sec. 4,
Eq. varcoeff_def); these tests record, with the oracle alone, that the
library's C2 stall is the method's and not a fault of the CUDA path."""
import numpy as np
import pytest

from oracle import assemble as asm
from oracle import krylov
from oracle import multigrid as mg
from oracle.grid import Grid
from oracle.precond import Preconditioner
from paper_1308_4605_gb300 import workloads as wl


def _vcycle_rates(pr, cycles=8):
    g = Grid(pr.dim, pr.n, pr.h, pr.bc)
    levels = mg.build_hierarchy(g, asm.fine_coefficients(g, pr.rho, pr.mu, pr.theta))
    A = levels[0].A
    r = np.random.default_rng(5).standard_normal(g.nvel) * g.active[:g.nvel]
    x = np.zeros_like(r)
    res = [np.linalg.norm(r)]
    for _ in range(cycles):
        x = x + mg.vcycle_velocity(levels, r - A @ x)
        res.append(np.linalg.norm(r - A @ x))
    res = np.array(res)
    return res[1:] / res[:-1]


@pytest.mark.parametrize("n", [64, 128])
def test_velocity_vcycle_diverges_on_sharp_inclusions(n):
    rates = _vcycle_rates(wl.config_c2(n))
    # after the first two cycles every cycle amplifies the residual
    # (x2.0-2.6 per cycle at 64^2, x3.7-7.4 at 128^2)
    assert rates[2:].min() > 1.5, rates
    assert np.prod(rates) > 1.0, rates


@pytest.mark.parametrize("n", [64, 128])
def test_velocity_vcycle_stagnates_on_smoothed_inclusions(n):
    """The tanh-smoothed variant (jump width h) converges, but the rate
    approaches one (0.95-0.99 per cycle)."""
    rates = _vcycle_rates(wl.config_c2(n, smooth=True))
    assert rates.max() < 1.0, rates
    assert rates[-3:].min() > 0.9, rates


@pytest.mark.parametrize("n,maxit", [(64, 100), (128, 50)])
def test_p2_gmres_stalls_on_sharp_inclusions(n, maxit):
    """P2-GMRES(10), one V-cycle per subsolve: the true relative residual
    never falls below 1 (it rises to 10^1.3-10^1.9 and stays there)."""
    pr = wl.config_c2(n)
    g = Grid(pr.dim, pr.n, pr.h, pr.bc)
    M = asm.stokes_operator(g, asm.fine_coefficients(g, pr.rho, pr.mu, pr.theta))
    P = Preconditioner(g, pr.rho, pr.mu, pr.theta, which=2)
    b = g.pack(pr.b_u, pr.b_p)
    b[~g.active] = 0.0
    _, info = krylov.gmres(lambda v: M @ v, P.apply, b, rtol=1e-10, m=10, maxit=maxit)
    assert info["iterations"] == maxit and not info["converged"]
    assert min(info["true_residual"][1:]) > 1.0, info["true_residual"]
