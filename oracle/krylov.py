"""Oracle Krylov solver: textbook restarted GMRES(m) with right preconditioning.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper solves the subdomain problems (Section 3.2) and the interface
system (Eq. 8) with GMRES.  This is the standard algorithm (Arnoldi with
modified Gram-Schmidt, Givens rotations on the Hessenberg matrix, least-squares
update at the end of each cycle), right-preconditioned so that the residual it
monitors is the true residual of the unpreconditioned system.
"""
from __future__ import annotations

import numpy as np


def gmres(matvec, b, *, precond=None, tol=1e-8, restart=60, maxiter=1000, x0=None,
          atol=0.0):
    """Solve A x = b.  Returns (x, n_iterations, residual_history).

    Stops when ||b - A x|| <= max(tol * ||b||, atol) (estimated by the Givens
    recurrence, exact in exact arithmetic) or after maxiter inner steps.
    """
    b = np.asarray(b, np.complex128)
    n = b.shape[0]
    x = np.zeros(n, np.complex128) if x0 is None else np.array(x0, np.complex128)
    M = (lambda v: v) if precond is None else precond
    bnorm = np.linalg.norm(b)
    hist = []
    if bnorm == 0.0:
        return x, 0, [0.0]
    target = max(tol * bnorm, atol)
    it = 0
    r = b - matvec(x) if x0 is not None else b.copy()
    beta = np.linalg.norm(r)
    hist.append(beta / bnorm)
    while beta > target and it < maxiter:
        m = min(restart, maxiter - it)
        V = np.zeros((m + 1, n), np.complex128)
        Z = np.zeros((m, n), np.complex128)
        H = np.zeros((m + 1, m), np.complex128)
        cs = np.zeros(m)
        sn = np.zeros(m, np.complex128)
        g = np.zeros(m + 1, np.complex128)
        V[0] = r / beta
        g[0] = beta
        k_used = 0
        for j in range(m):
            Z[j] = M(V[j])
            w = matvec(Z[j])
            for i in range(j + 1):                      # modified Gram-Schmidt
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):                          # previous rotations
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            # new rotation G = [[c, s], [-conj(s), c]] (c real) zeroing H[j+1, j]
            a, c = H[j, j], H[j + 1, j]
            d = np.sqrt(abs(a) ** 2 + abs(c) ** 2)
            if d == 0:
                cs[j], sn[j] = 1.0, 0.0
            elif abs(a) == 0:
                cs[j], sn[j] = 0.0, 1.0
            else:
                cs[j] = abs(a) / d
                sn[j] = (a / abs(a)) * np.conj(c) / d
            H[j, j] = cs[j] * H[j, j] + sn[j] * H[j + 1, j]
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            k_used = j + 1
            hist.append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) <= target or it >= maxiter:
                break
        y = np.zeros(k_used, np.complex128)
        for i in range(k_used - 1, -1, -1):             # back substitution
            y[i] = (g[i] - H[i, i + 1:k_used] @ y[i + 1:k_used]) / H[i, i]
        x = x + y @ Z[:k_used]
        r = b - matvec(x)
        beta = np.linalg.norm(r)
        hist[-1] = beta / bnorm
    return x, it, hist
