"""Block Schur-complement preconditioners P1..P5, Sec. 2.1-2.4.

Test infrastructure: see the package docstring.

Notation: x* = A~^{-1} b_u (velocity V-cycle, zero guess), L~_rho^{-1} (pressure
V-cycle, zero guess), Schur complement inverse approximation
S~^{-1} = -theta L~_rho^{-1} + 2 mu  (Eq. Schur_app_varDen_varVis; mu is the
diagonal of cell viscosities), rho^{-1} the diagonal of inverse face densities.

  P1 (Eq. P1_practical):     x* = A~^{-1} b_u;  b_c = D x* + b_p;  phi = L~^{-1} b_c;
                             x_u = x* - rho^{-1} G phi;  x_p = theta phi - 2 mu b_c
  P2 (Eq. CC_Pre_lower):     x_u = x*;  x_p = -S~^{-1} (D x* + b_p)
  P3 (Eq. CC_Pre_upper):     x_p = -S~^{-1} b_p;  x_u = A~^{-1} (b_u - G x_p)
  P4 (Eq. CC_Pre_diagonal):  x_u = A~^{-1} b_u;  x_p = -S~^{-1} b_p
  P5 (Sec. 2.4, Uzawa-like): x* = A~^{-1} b_u;  x_p = -S~^{-1} (D x* + b_p);
                             x_u = one more V-cycle for A x = b_u - G x_p
                             started from x*
With theta = 0 the Poisson solve drops out of S~^{-1} (Sec. 2.2).

Subsolvers with more than one multigrid cycle (Sec. 4.1.2 studies the
number of V-cycles per application of the preconditioner): the velocity
subsolve with c_u cycles is x = V(r), then c_u - 1 times x = x + V(r - A x)
(multigrid as a stationary iteration); the pressure subsolve projects r onto
mean-zero vectors, phi = V(r), then c_p - 1 times phi = phi + V(res) with
res = r - L_rho phi projected onto mean-zero vectors.  As c grows both tend
to the exact subsolves (pinned).

Readings (stated, pinned by the exact-subsolver identities of App. B):
  * the pressure null space (constant p) is handled by removing the mean of
    every right-hand side handed to the Poisson solver and the mean of x_p;
  * the V-cycle of P5 started from x* is applied in residual-correction form,
    x* + V(b_u - G x_p - A x*), which equals a V-cycle from initial guess x*
    in exact arithmetic because every smoothing step is a stationary linear
    iteration.

Parity: pinned (with exact subsolvers: P1^{-1} M = I on constant-coefficient
periodic grids and for inviscid flow with walls; (P2^{-1}M - I)^2 = 0 and
(P3^{-1}M - I)^2 = 0 for inviscid flow; P5^{-1} M = I for inviscid flow;
linearity of every preconditioner built from V-cycles).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import assemble as asm
from . import multigrid as mg
from .grid import Grid


class Preconditioner:
    def __init__(self, grid: Grid, rho, mu, theta, which=1, exact=False, nu=2, ncoarse=8,
                 cycles_u=1, cycles_p=1, gamma=None):
        self.grid = grid
        self.theta = float(theta)
        self.which = int(which)
        self.exact = exact
        self.nu, self.ncoarse = nu, ncoarse
        self.cycles_u, self.cycles_p = int(cycles_u), int(cycles_p)
        self.coef = asm.fine_coefficients(grid, rho, mu, theta, gamma)
        self.mu = np.asarray(mu, dtype=np.float64).ravel()
        # the local-viscosity Schur factor: 2 mu (Eq. Schur_app_varDen_varVis),
        # gamma + 4/3 mu = 2 mu + lam with bulk viscosity (Eq. Schur_app_bulk)
        self.kappa = 2.0 * self.mu
        if gamma is not None:
            self.kappa = 2.0 * self.mu + self.coef["lam_c"].ravel()
        self.inv_rho_f = np.concatenate([np.asarray(b).ravel() for b in self.coef["beta"]])
        self.D = asm.divergence(grid)
        self.G = asm.gradient(grid)
        self.A = asm.velocity_operator(grid, self.coef)
        if exact:
            va = grid.active[:grid.nvel]
            self._va = va
            Aa = self.A[va][:, va].toarray()
            self._A_lu = sla.lu_factor(Aa)
            L = asm.poisson_operator(grid, self.coef["beta"]).toarray()
            self._L_pinv = np.linalg.pinv(L, rcond=1e-10)
        else:
            self.levels = mg.build_hierarchy(grid, self.coef)

    # subsolvers ------------------------------------------------------------
    def velocity_solve(self, r):
        if self.exact:
            out = np.zeros_like(r)
            out[self._va] = sla.lu_solve(self._A_lu, r[self._va])
            return out
        x = mg.vcycle_velocity(self.levels, r, 0, self.nu, self.ncoarse)
        for _ in range(self.cycles_u - 1):
            x = x + mg.vcycle_velocity(self.levels, r - self.A @ x, 0, self.nu, self.ncoarse)
        return x

    def poisson_solve(self, r):
        r = r - r.mean()
        if self.exact:
            return self._L_pinv @ r
        phi = mg.vcycle_pressure(self.levels, r, 0, self.nu, self.ncoarse)
        for _ in range(self.cycles_p - 1):
            res = r - self.levels[0].Lrho @ phi
            res = res - res.mean()
            phi = phi + mg.vcycle_pressure(self.levels, res, 0, self.nu, self.ncoarse)
        return phi

    def neg_schur_inverse(self, r):
        """-S~^{-1} r = theta L~^{-1} r - kappa r, kappa = 2 mu (or
        gamma + 4/3 mu with bulk viscosity)."""
        out = -self.kappa * r
        if self.theta != 0.0:
            out = out + self.theta * self.poisson_solve(r)
        return out

    # application ------------------------------------------------------------
    def apply(self, b):
        g = self.grid
        b_u, b_p = b[:g.nvel], b[g.nvel:]
        w = self.which
        if w == 1:
            xs = self.velocity_solve(b_u)
            bc = self.D @ xs + b_p
            phi = self.poisson_solve(bc)
            x_u = xs - self.inv_rho_f * (self.G @ phi)
            x_p = self.theta * phi - self.kappa * bc
        elif w == 2:
            x_u = self.velocity_solve(b_u)
            x_p = self.neg_schur_inverse(self.D @ x_u + b_p)
        elif w == 3:
            x_p = self.neg_schur_inverse(b_p)
            x_u = self.velocity_solve(b_u - self.G @ x_p)
        elif w == 4:
            x_u = self.velocity_solve(b_u)
            x_p = self.neg_schur_inverse(b_p)
        elif w == 5:
            xs = self.velocity_solve(b_u)
            x_p = self.neg_schur_inverse(self.D @ xs + b_p)
            x_u = xs + self.velocity_solve(b_u - self.G @ x_p - self.A @ xs)
        else:
            raise ValueError("preconditioner must be 1..5")
        x_p = x_p - x_p.mean()
        return np.concatenate([x_u, x_p])

    __call__ = apply
