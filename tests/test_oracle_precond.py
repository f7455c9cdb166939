"""Pins for the oracle's tensor-trick preconditioner: the WW-scale and MDA
identities, the z eigen-relations of the Appendix, and L^{-1} L = I."""
import numpy as np
import pytest

from fm_inputs import workload
from oracle import physics as ph
from oracle.precond import Preconditioner, decompose, g_at_one
from oracle.system import FMSystem


def _real_pencil(n, rng):
    Q = rng.standard_normal((n, n))
    A1 = Q @ np.diag(np.arange(1.0, n + 1)) @ np.linalg.inv(Q)
    A2 = np.eye(n) + 0.1 * rng.standard_normal((n, n))
    return A1 @ A2, A2


def test_ww_scale_and_mda():
    """Eq. WW-scale and Eq. MDA: (A1 x B1 + A2 x B2)^{-1} = (W_A x W_B)(L_A x L_B + I)^{-1}(W-bar_A x W-bar_B)."""
    rng = np.random.default_rng(11)
    A1, A2 = _real_pencil(5, rng)
    B1, B2 = _real_pencil(4, rng)
    WbA, WA, lA = decompose(A1, A2)
    WbB, WB, lB = decompose(B1, B2)
    assert np.allclose(WbA @ A1 @ WA, np.diag(lA), atol=1e-10)
    assert np.allclose(WbA @ A2 @ WA, np.eye(5), atol=1e-10)
    # Eq. MDA needs A2 (x) B2 -> I (x) I after scaling, which holds for A2 = B2-scaled forms
    M = np.kron(A1, B1) + np.kron(A2, B2)
    inv = np.kron(WA, WB) @ np.diag(1.0 / (np.kron(lA, lB) + 1.0)) @ np.kron(WbA, WbB)
    assert np.allclose(inv @ M, np.eye(20), atol=1e-9)


def test_g_at_one_matches_legendre():
    """g_l^{M'}(1) from Eq. g-def with the associated Legendre functions (Condon-Shortley phase)."""
    from scipy.special import lpmv
    from math import factorial
    z = 1 - 1e-7
    for l in range(0, 5):
        for Mp in range(0, l + 1):
            nrm = np.sqrt((2 * l + 1) / 2 * factorial(l - Mp) / factorial(l + Mp))
            val = nrm * lpmv(Mp, l, z) / (1 - z * z) ** (Mp / 2)
            assert abs(val - g_at_one(l, Mp)) < 1e-5 * max(1, abs(val))


@pytest.mark.parametrize("Mp", [0, 1, 2])
def test_z_eigen_relations(Mp):
    """Appendix: for modes representable by cubics, Lambda~ = -l(l+1) exactly (Eq. g-ev), and the
    off-diagonal products W-bar D^{M'+-} W equal Lambda^{M'+-} (Eq. prop-eq) in that block."""
    wl = workload("he_l0_24x24x8", J=3, nint=(2, 2, 6), R=(8.0, 8.0))
    s = FMSystem(wl)
    P = Preconditioner(s, -2.9)
    C = P.comp[1]
    g = s.g[1]
    z = g.az.pts
    Sz, D1z = g.az.mat(0), g.az.mat(1)
    iM = s.Mps.index(Mp)
    assert np.allclose(C["Lz"][iM][:4], [-(Mp + l) * (Mp + l + 1) for l in range(4)], atol=1e-9)
    Dp = -(1 - z * z)[:, None] * D1z + (2 * (Mp + 1) * z)[:, None] * Sz
    X = C["Wzb"][iM] @ Dp @ C["Wz"][iM + 1]
    for k in range(1, 4):
        assert abs(X[k, k - 1] + ph.lam(Mp + k, Mp)) < 1e-8
    Y = C["Wzb"][iM + 1] @ (-D1z) @ C["Wz"][iM]
    for k in range(0, 3):
        assert abs(Y[k, k + 1] - ph.lam(Mp + 1 + k, -(Mp + 1))) < 1e-8


@pytest.mark.parametrize("J,tau,basis", [(0, 1, 0), (1, 1, 0), (2, 1, 0), (2, -1, 0), (0, 1, 1), (2, 1, 1)])
def test_preconditioner_inverts_its_operator(J, tau, basis):
    """L^{-1} (Eq. prec-2, step by step) times the densely built approximate operator L = I."""
    wl = workload("he_l0_24x24x8", J=J, tau=tau, nint=(3, 4, 3), R=(10.0, 12.0), basis=basis)
    s = FMSystem(wl)
    P = Preconditioner(s, -2.9)
    rng = np.random.default_rng(12)
    for a in s.comps:
        g = s.g[a]
        L = P.dense_L(a)
        v = rng.standard_normal(g.csize)
        full = np.zeros(s.N)
        full[s.off[a]:s.off[a] + g.csize] = L @ v
        back = P.apply(full)[s.off[a]:s.off[a] + g.csize]
        # rounding amplified by the condition of L (1e3 cubic; 1e8 quintic, whose second-derivative
        # functions scale as h^2); an index or layout error gives O(1)
        bound = max(1e-12, np.finfo(float).eps * np.linalg.cond(L))
        assert np.linalg.norm(back - v) < bound * np.linalg.norm(v)


@pytest.mark.parametrize("J,tau,basis", [(0, 1, 0), (1, -1, 0), (0, 1, 1)])
def test_computed_z_gives_exact_inverse(J, tau, basis):
    """With the computed z eigenvalues (n_M = 1) the approximation is exact: L^{-1} L_FM-fin = I."""
    wl = workload("he_l0_24x24x8", J=J, tau=tau, nint=(3, 3, 3), R=(10.0, 12.0), basis=basis)
    s = FMSystem(wl)
    P = Preconditioner(s, -2.7, z_eigs="computed")
    for a in s.comps:
        g = s.g[a]
        L = P.dense_L_fmfin(a)
        kappa = np.linalg.cond(L)
        assert np.allclose(P.dense_L(a), L, atol=max(1e-10, 1e-15 * kappa) * np.abs(L).max())
        v = np.random.default_rng(13).standard_normal(g.csize)
        full = np.zeros(s.N)
        full[s.off[a]:s.off[a] + g.csize] = L @ v
        bound = max(1e-12, np.finfo(float).eps * kappa)
        assert np.linalg.norm(P.apply(full)[s.off[a]:s.off[a] + g.csize] - v) < bound * np.linalg.norm(v)


def test_oracle_fgmres_matches_sparse_lu():
    """The oracle's preconditioned GMRES reaches the sparse-LU solution of (H - E S) x = b."""
    from oracle import solvers
    from oracle.krylov import fgmres
    wl = workload("he_l0_24x24x8", nint=(6, 7, 4), R=(18.0, 16.0))
    s = FMSystem(wl)
    H, S = s.H(), s.S()
    E = -2.6
    P = Preconditioner(s, E)
    b = np.random.default_rng(14).standard_normal(s.N)
    x, info = fgmres(lambda v: H @ v - E * (S @ v), P.apply, b, tol=1e-12, m=40)
    ref = solvers.solve(H, S, E, b)
    assert info["resid"] < 1e-12
    assert np.linalg.norm(x - ref) < 1e-9 * np.linalg.norm(ref)
    assert info["iters"] < 100  # the preconditioner is effective (unpreconditioned GMRES stalls)


def test_complex_pairs_real_basis():
    """M' = 3 z pencil on 8 sin-mapped intervals has complex pairs: the real basis keeps
    W-bar A2 W = I, W-bar A1 W block diagonal with the pairs' 2x2 rotation-scaling blocks,
    and the low (cubic-representable) modes exact."""
    from oracle.precond import decompose_pairs
    wl = workload("he_l0_24x24x8", J=3, nint=(2, 2, 8), R=(8.0, 8.0))
    s = FMSystem(wl)
    g = s.g[1]
    z = g.az.pts
    Sz, D1z, D2z = g.az.mat(0), g.az.mat(1), g.az.mat(2)
    Mp = 3
    Dz = (1 - z * z)[:, None] * D2z - (2 * (Mp + 1) * z)[:, None] * D1z - Mp * (Mp + 1) * Sz
    Wb, W, lr, kinds = decompose_pairs(Dz, Sz, 2 * g.az.basis.N)
    assert kinds.count(1) == kinds.count(2) >= 1
    assert np.allclose(Wb @ Sz @ W, np.eye(g.nz), atol=1e-10)
    T = Wb @ Dz @ W
    for l, kd in enumerate(kinds):
        if kd == 0:
            assert abs(T[l, l] - lr[l]) < 1e-8 * abs(lr).max()
        elif kd == 1:
            blk = T[l:l + 2, l:l + 2]
            assert abs(blk[0, 0] - blk[1, 1]) < 1e-8 * abs(lr).max() and abs(blk[0, 1] + blk[1, 0]) < 1e-8 * abs(lr).max()
    off = T - np.diag(np.diag(T))
    for l, kd in enumerate(kinds):
        if kd == 1:
            off[l, l + 1] = off[l + 1, l] = 0
    assert np.abs(off).max() < 1e-8 * abs(lr).max()
    assert np.allclose(lr[:4], [-(Mp + l) * (Mp + l + 1) for l in range(4)], atol=1e-9)
    P = Preconditioner(s, -0.3)  # builds with the pairs and still inverts its own operator
    L = P.dense_L(1)
    v = np.random.default_rng(15).standard_normal(g.csize)
    full = np.zeros(s.N)
    full[:g.csize] = L @ v
    assert np.linalg.norm(P.apply(full)[:g.csize] - v) < 1e-11 * np.linalg.norm(v)
