"""Restarted GMRES(m), Sec. 3.2 and Sec. 4.

Test infrastructure: see the package docstring.

``gmres``: left-preconditioned GMRES(m) on P^{-1} M x = P^{-1} b (Sec. 3.2),
textbook Arnoldi with modified Gram-Schmidt, Givens rotations and the
(m+1) x m Hessenberg least-squares problem (Saad).  ``fgmres``: the flexible,
right-preconditioned variant (Sec. 4) that stores Z_j = P^{-1} v_j and
updates x with Z y.

Stopping rule (a reading: the paper allows either residual, Sec. 3.2): the
solve ends when the true residual satisfies ||b - M x|| <= rtol ||b||; it is
computed at the start of every cycle.  Inside a cycle the Arnoldi residual
estimate is compared with a target: for the flexible variant the estimate is
the true residual and the target is rtol ||b||; for the left-preconditioned
variant the estimate is the preconditioned residual and the target is its
value at the start of the cycle times rtol ||b|| / ||b - M x||, i.e. the
cycle asks of the preconditioned residual the reduction the true residual
still needs.  The iteration count is the number of Arnoldi steps
(applications of M).

Parity: pinned (iteration counts 1 (P1) and 2 (P2, P3) with exact subsolvers,
App. B; convergence to the direct solution).
"""
from __future__ import annotations

import numpy as np


def _givens(a, b):
    if b == 0.0:
        return 1.0, 0.0
    r = np.hypot(a, b)
    return a / r, b / r


def _arnoldi_cycle(Mv, Pv, r0, m, tol_abs, flexible, it_left):
    beta = np.linalg.norm(r0)
    V = [r0 / beta]
    Z = []
    H = np.zeros((m + 1, m))
    cs, sn = np.zeros(m), np.zeros(m)
    g = np.zeros(m + 1)
    g[0] = beta
    k = 0
    for j in range(min(m, it_left)):
        if flexible:
            z = Pv(V[j])
            Z.append(z)
            w = Mv(z)
        else:
            w = Pv(Mv(V[j]))
        for i in range(j + 1):
            H[i, j] = np.dot(w, V[i])
            w = w - H[i, j] * V[i]
        H[j + 1, j] = np.linalg.norm(w)
        V.append(w / H[j + 1, j] if H[j + 1, j] > 0 else w)
        for i in range(j):
            t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
            H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
            H[i, j] = t
        cs[j], sn[j] = _givens(H[j, j], H[j + 1, j])
        H[j, j] = cs[j] * H[j, j] + sn[j] * H[j + 1, j]
        H[j + 1, j] = 0.0
        g[j + 1] = -sn[j] * g[j]
        g[j] = cs[j] * g[j]
        k = j + 1
        if abs(g[j + 1]) <= tol_abs or H[j, j] == 0.0:
            break
    y = np.zeros(k)
    for i in range(k - 1, -1, -1):
        y[i] = (g[i] - H[i, i + 1:k] @ y[i + 1:k]) / H[i, i]
    basis = Z if flexible else V
    dx = np.zeros_like(r0)
    for i in range(k):
        dx += y[i] * basis[i]
    return dx, k, abs(g[k])


def gmres(Mv, Pv, b, x0=None, rtol=1e-10, m=10, maxit=2000, flexible=False):
    """Solve M x = b.  Mv(x) = M x, Pv(r) = P^{-1} r.  Returns (x, info)."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    bnorm = np.linalg.norm(b)
    info = {"iterations": 0, "restarts": 0, "true_residual": [], "est_residual": []}
    if bnorm == 0.0:
        info["converged"] = True
        return np.zeros_like(b), info
    while True:
        r = b - Mv(x)
        rnorm = np.linalg.norm(r)
        rel = rnorm / bnorm
        info["true_residual"].append(rel)
        if rel <= rtol or info["iterations"] >= maxit:
            break
        if flexible:
            r0 = r
            target = rtol * bnorm
        else:
            r0 = Pv(r)
            target = np.linalg.norm(r0) * (rtol * bnorm / rnorm)
        dx, k, est = _arnoldi_cycle(Mv, Pv, r0, m, target, flexible,
                                    maxit - info["iterations"])
        x = x + dx
        info["iterations"] += k
        info["restarts"] += 1
        info["est_residual"].append(est)
    info["converged"] = info["true_residual"][-1] <= rtol
    return x, info


def fgmres(Mv, Pv, b, x0=None, rtol=1e-10, m=10, maxit=2000):
    return gmres(Mv, Pv, b, x0, rtol, m, maxit, flexible=True)
