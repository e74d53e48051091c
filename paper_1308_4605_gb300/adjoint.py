"""Differentiable Stokes solve: torch.autograd.Function around libstokes_gb300.

forward:  set the coefficients (mu = exp(log_mu), rho, theta) and solve
          M x = b with the library's GMRES; only the solution x is kept for
          the backward pass (no Krylov basis is stored).
backward: one adjoint solve M^T lambda = (dL/du, dL/dp) with the same solver
          (M is symmetric: D = -G^*, L_mu symmetric, Sec. 2), then the
          library's gradient kernel (stk_gradient) forms dL/dlog(mu) and
          dL/drho at cell centres from u and lambda; dL/db = lambda.

All arithmetic runs in the CUDA library; this module only orders the calls.
"""
from __future__ import annotations

import torch

from . import stokes as S


class _StokesSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, log_mu, rho, solver, theta, b_p, opts, *b_u):
        mu = torch.exp(log_mu)
        solver.set_coefficients(rho.contiguous(), mu.contiguous(), theta)
        x_u, x_p, info = solver.solve([b.contiguous() for b in b_u], b_p.contiguous(), **opts)
        if not info["converged"]:
            raise S.StokesError(S.STK_ERR_NOT_CONVERGED, f"forward solve: {info}")
        ctx.solver, ctx.theta, ctx.opts = solver, theta, opts
        ctx.info = info
        ctx.save_for_backward(log_mu, rho, *x_u)
        return tuple(x_u) + (x_p,)

    @staticmethod
    def backward(ctx, *grads):
        log_mu, rho, *x_u = ctx.saved_tensors
        solver = ctx.solver
        dim = solver.dim
        mu = torch.exp(log_mu)
        solver.set_coefficients(rho.contiguous(), mu.contiguous(), ctx.theta)
        g_u = [g.contiguous() if g is not None else torch.zeros_like(x_u[a])
               for a, g in enumerate(grads[:dim])]
        g_p = torch.zeros(solver.cell_shape(), dtype=torch.float64, device=log_mu.device)
        if grads[dim] is not None:
            # the pressure part of the adjoint right-hand side, projected onto
            # mean-zero vectors (the pressure null space) by the library
            S.stk_remove_mean(solver.handle, grads[dim].contiguous(), g_p)
        lam_u, lam_p, info = solver.solve(g_u, g_p, **ctx.opts)
        if not info["converged"]:
            raise S.StokesError(S.STK_ERR_NOT_CONVERGED, f"adjoint solve: {info}")
        dlogmu = torch.empty_like(log_mu)
        drho = torch.empty_like(rho)
        S.stk_gradient(solver.handle, x_u, lam_u, dlogmu, drho)
        return (dlogmu, drho, None, None, lam_p, None, *lam_u)


def stokes_solve(solver, log_mu, rho, theta, b_u, b_p, **opts):
    """Differentiable solve of M(exp(log_mu), rho, theta) x = b on `solver`
    (a stokes.StokesSolver).  Returns the velocity face arrays and the
    pressure.  opts go to StokesSolver.solve (precond, rtol, precision...)."""
    return _StokesSolve.apply(log_mu, rho, solver, float(theta), b_p, dict(opts), *b_u)
