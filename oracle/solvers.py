"""Direct solves and shift-invert eigenvalues of H c = E S c (oracle).

ORACLE -- test infrastructure only (see ``oracle/__init__``).

* ``solve``: (H - E S) x = b by sparse LU (SuperLU through SciPy) plus one
  step of iterative refinement in float64.
* ``eigs_near``: the eigenvalues nearest a shift E* by Arnoldi on the
  shift-invert operator (H - E* S)^{-1} S, backed by the same sparse LU.  Its
  eigenvalues theta are those of S (H - E* S)^{-1} in Eq. FM-lin, and
  E = E* + 1/theta.
* ``eigs_dense``: brute-force dense generalized eigenvalues for tiny grids.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse.linalg as spla


def lu(H, S, E):
    A = (H - E * S).tocsc()
    return spla.splu(A, permc_spec="COLAMD")


def solve(H, S, E, b, factor=None):
    f = factor or lu(H, S, E)
    x = f.solve(b)
    r = b - (H @ x - E * (S @ x))
    return x + f.solve(r)


def eigs_near(H, S, shift, k, factor=None, tol=1e-13, ncv=None, v0=None):
    """k eigenpairs of H c = E S c nearest ``shift``; returns (E sorted by |E - shift|, vectors)."""
    f = factor or lu(H, S, shift)
    N = H.shape[0]
    op = spla.LinearOperator((N, N), matvec=lambda v: f.solve(S @ v), dtype=np.float64)
    ncv = ncv or max(2 * k + 1, 20)
    theta, vec = spla.eigs(op, k=k, which="LM", tol=tol, ncv=ncv, v0=v0)
    E = shift + 1.0 / theta
    order = np.argsort(np.abs(E - shift))
    return E[order], vec[:, order]


def eigs_dense(H, S):
    """All generalized eigenvalues of the dense pencil (H, S)."""
    return sla.eig(H.toarray(), S.toarray(), right=False)


def residual(H, S, E, c):
    c = np.real_if_close(c)
    return np.linalg.norm(H @ c - E * (S @ c)) / np.linalg.norm(S @ c)
