"""Right-preconditioned restarted GMRES with the oracle's operator and preconditioner.

ORACLE -- test infrastructure only (see ``oracle/__init__``).

Section 4: inside the Arnoldi iteration the matrix (H - E* S) of Eq. FM-lin is
inverted by preconditioned GMRES with the tensor-trick preconditioner.  This is
the textbook algorithm (Arnoldi with modified Gram-Schmidt, Givens rotations,
restart from the true residual), written plainly in NumPy; the preconditioned
directions are kept (flexible form) so that x = x0 + Z y.
"""
from __future__ import annotations

import time

import numpy as np


def fgmres(matvec, precond, b, tol=1e-12, m=30, max_iters=1000, x0=None, max_seconds=None):
    """Solve A x = b.  Returns (x, info) with info = {iters, resid, seconds}."""
    t0 = time.perf_counter()
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    bnorm = np.linalg.norm(b)
    r = b - matvec(x)
    beta = np.linalg.norm(r)
    iters = 0
    while beta > tol * bnorm and iters < max_iters:
        V = [r / beta]
        Z = []
        Hm = np.zeros((m + 1, m))
        g = np.zeros(m + 1)
        g[0] = beta
        cs, sn = np.zeros(m), np.zeros(m)
        j = 0
        for j in range(m):
            Z.append(precond(V[j]))
            w = matvec(Z[j])
            for i in range(j + 1):  # modified Gram-Schmidt
                Hm[i, j] = V[i] @ w
                w = w - Hm[i, j] * V[i]
            hn = np.linalg.norm(w)
            Hm[j + 1, j] = hn
            for i in range(j):  # earlier rotations
                t = cs[i] * Hm[i, j] + sn[i] * Hm[i + 1, j]
                Hm[i + 1, j] = -sn[i] * Hm[i, j] + cs[i] * Hm[i + 1, j]
                Hm[i, j] = t
            rr = np.hypot(Hm[j, j], Hm[j + 1, j])
            cs[j], sn[j] = Hm[j, j] / rr, Hm[j + 1, j] / rr
            Hm[j, j], Hm[j + 1, j] = rr, 0.0
            g[j + 1], g[j] = -sn[j] * g[j], cs[j] * g[j]
            iters += 1
            done = abs(g[j + 1]) <= tol * bnorm or iters >= max_iters
            if max_seconds is not None and time.perf_counter() - t0 > max_seconds:
                done = True
            if done:
                break
            V.append(w / hn)
        k = j + 1
        y = np.linalg.solve(np.triu(Hm[:k, :k]), g[:k])
        x = x + np.stack(Z[:k], axis=1) @ y
        r = b - matvec(x)
        beta = np.linalg.norm(r)
        if max_seconds is not None and time.perf_counter() - t0 > max_seconds:
            break
    return x, {"iters": iters, "resid": beta / bnorm, "seconds": time.perf_counter() - t0}
