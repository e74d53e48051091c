"""Tight-tolerance solves of the seeded workloads, for full-size parity.

Test infrastructure: see the package docstring.

At sizes where a direct solve of M x = b (Eq. Saddle_sys) is out of reach
(3D 128^3, the 512^2 instances of the batched workload) the exact discrete
solution is approximated by the oracle's own restarted GMRES(10) (Sec. 3.2)
with the workload's block preconditioner (P1 or P2, one V-cycle per subsolve,
App. C), run until the true residual, computed with the assembled sparse M
of Sec. 3.1, is below 1e-13 ||b||.  The error of that iterate is at most
cond(M) times 1e-13, five orders below the 1e-8 the library's solutions are
compared at.  The pressure is returned with zero mean.

Parity: pinned (tests/test_oracle_solver.py: equal to the direct solve to
1e-11 on the workloads' generators at reduced size).
"""
from __future__ import annotations

import numpy as np

from . import assemble as asm
from . import krylov
from .grid import Grid
from .precond import Preconditioner


def solve_problem(pr, rtol=1e-13, maxit=600, m=10):
    """x (packed storage vector, mean-free pressure) and the GMRES info of the
    problem ``pr`` (a workloads.Problem)."""
    g = Grid(pr.dim, pr.n, pr.h, pr.bc)
    coef = asm.fine_coefficients(g, pr.rho, pr.mu, pr.theta)
    M = asm.stokes_operator(g, coef)
    P = Preconditioner(g, pr.rho, pr.mu, pr.theta, which=pr.precond)
    b = g.pack(pr.b_u, pr.b_p)
    b[~g.active] = 0.0
    x, info = krylov.gmres(lambda v: M @ v, P.apply, b, rtol=rtol, m=m, maxit=maxit)
    x[g.cell_offset:] -= x[g.cell_offset:].mean()
    res = np.linalg.norm(b - M @ x) / np.linalg.norm(b)
    return x, {"iterations": info["iterations"], "true_residual": float(res),
               "converged": bool(res <= rtol)}


def solve_workload(name, n, i=None, rtol=1e-13):
    """The seeded workload by name ("c1", "c3", "c4" (instance i), "c5")
    at size n, solved by ``solve_problem``; picklable for process pools."""
    from paper_1308_4605_gb300 import workloads as wl
    if name == "c1":
        pr = wl.config_c1(n)
    elif name == "c3":
        pr = wl.config_c3(n)
    elif name == "c4":
        pr = wl.config_c4_instance(i, n)
    elif name == "c5":
        pr = wl.config_c5(n)
    else:
        raise ValueError(name)
    return solve_problem(pr, rtol=rtol)
