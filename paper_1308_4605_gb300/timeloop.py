"""Backward-Euler time stepping of the variable-coefficient Stokes equations
(Sec. 2, Eq. Stokes_eqn) with the library's coupled solver.

Step n -> n+1 solves
    rho (u^{n+1} - u^n)/dt + G p^{n+1} - L_mu u^{n+1} = f^{n+1},
    -D u^{n+1} = b_p                    (b_p = -g^{n+1}),
that is M x = (b_u, b_p) with theta = 1/dt and b_u = (rho_f/dt) u^n + f^{n+1}
formed on the GPU by stk_backward_euler_rhs.  Each solve starts from the
previous step's solution (warm start).  All arithmetic runs in the CUDA
library; this module only orders the calls and copies buffers.
"""
from __future__ import annotations

import torch

from . import stokes as S


def backward_euler(solver, rho, mu, dt, u0, nsteps, f=None, b_p=None, p0=None, warm=True,
                   **opts):
    """Advance u0 (list of face arrays) by nsteps steps of size dt on
    `solver` (a stokes.StokesSolver).  f: face arrays of the forcing, or a
    callable n -> face arrays for step n (1-based), or None; b_p: the
    pressure right-hand side -g (cell array) or None for g = 0.  opts go to
    StokesSolver.solve.  Returns (u, p, infos)."""
    solver.set_coefficients(rho, mu, 1.0 / dt)
    dev = u0[0].device
    u = [x.clone() for x in u0]
    zu, zp = solver.zeros(dev)
    p = p0.clone() if p0 is not None else zp
    bp = b_p if b_p is not None else torch.zeros_like(zp)
    b_u = [torch.empty_like(x) for x in u]
    infos = []
    for n in range(1, nsteps + 1):
        fn = f(n) if callable(f) else f
        S.stk_backward_euler_rhs(solver.handle, u, fn, b_u)
        if warm:
            x_u = [x.clone() for x in u]
            x_p = p.clone()
        else:
            x_u, x_p = solver.zeros(dev)
        x_u, x_p, info = solver.solve(b_u, bp, x_u, x_p, **opts)
        if not info["converged"]:
            raise S.StokesError(S.STK_ERR_NOT_CONVERGED, f"time step {n}: {info}")
        u, p = x_u, x_p
        infos.append(info)
    return u, p, infos
