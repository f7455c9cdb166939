"""Tensor-trick preconditioner L^{-1} of Eq. prec-2, as Section 3.2 builds it (oracle).

ORACLE -- test infrastructure only (see ``oracle/__init__``).

For one solved component alpha:

1. z: (W-bar_z^{M'}, W_z^{M'}, Lambda~_z^{M'}) = D(D_z^{M'}, S_z) for every M'
   (Eq. z-dec), eigenpairs sorted by descending eigenvalue; Lambda~ is then
   replaced by diag(-l(l+1)), l = M', ..., M' + n_z - 1 (Eq. prop-eq).
2. x: (W-bar_x^l, W_x^l, Lambda_x^l) = D(-D_x + l(l+1) X_r2 S_x + V_a S_x, S_x)
   for l = M0, ..., J + n_z - 1.
3. y: (W-bar_y^{l i}, W_y^{l i}, Lambda_y^{l i}) =
   D(-D_y + V^_a S_y - E* S_y + (Lambda_x^l)_{ii} S_y, Y_r2 S_y)  (Eq. ops).
4. L0: for every (l, i_x, i_y) a tridiagonal system along M' (the rows with
   equal remainders modulo (n_z - 1) n_x n_y) with diagonal
   (Lambda_y^{l i})_{jj} + J(J+1) - 2M'^2 + l(l+1) and off-diagonals
   lambda-hat^{J,M'} (Lambda_z^{M'+})_{l-M'+1, l-M'} (to M'+1) and
   -lambda-hat^{J,-M'} (Lambda_z^{M'-})_{l-M'+1, l-M'+2} (to M'-1).
5. L^{-1} v = W_z W_x W_y P (L~0)^{-1} P W-bar_y W-bar_x W-bar_z v.

D(A1, A2) is computed with LAPACK (scipy.linalg.eig, left and right
eigenvectors) and scaled so that W-bar A1 W = Lambda and W-bar A2 W = I
(Eq. WW-scale).

Readings:
* z eigenvectors are normalised so that the spline function of column l
  equals g_l^{M'}(1) (Appendix, Eq. g-def, with the Condon-Shortley phase of
  the associated Legendre functions): the off-diagonal replacements
  Lambda_z^{M'+-} of Eq. prop-eq hold for that normalisation.
* ``z_eigs="computed"`` keeps Lambda~_z (allowed only with n_M = 1); then
  L_alpha = L exactly, the left-hand operator of Eq. FM-fin.
* A z pencil with complex-conjugate pairs (high modes of M' >= 2-3) is
  represented by a real basis: see ``decompose_pairs``.
* The y pencils of step 3 may have complex-conjugate pairs (their top modes on
  coarse grids, notably with the quintic basis): they are then kept complex,
  as the paper computes in complex arithmetic (Section 4), and the component's
  stages run in complex arithmetic; the result is real up to rounding and its
  real part is returned.  A complex x pencil is rejected.
"""
from __future__ import annotations

from math import factorial

import numpy as np
import scipy.linalg as sla

from . import physics as ph


class ComplexSpectrum(RuntimeError):
    pass


def decompose(A1, A2, order="ascending", allow_complex=False):
    """(W-bar, W, lambda) with W-bar A1 W = diag(lambda), W-bar A2 W = I (Eq. WW-scale).

    LAPACK's left eigenvectors satisfy vl^H A1 = lambda vl^H A2; W-bar's rows are vl^H scaled by
    1 / (vl^H A2 w).  A complex spectrum raises ComplexSpectrum unless ``allow_complex``, which keeps
    the complex eigenpairs (sorted by real part, then imaginary part)."""
    lam, VL, VR = sla.eig(A1, A2, left=True, right=True)
    cplx = np.max(np.abs(lam.imag)) > 1e-10 * np.max(np.abs(lam))
    if cplx and not allow_complex:
        raise ComplexSpectrum("complex 1D spectrum")
    key = lam.real if order == "ascending" else -lam.real
    idx = np.lexsort((lam.imag, key))
    if cplx:
        lam, VL, VR = lam[idx], VL[:, idx], VR[:, idx]
    else:
        lam, VL, VR = lam.real[idx], VL[:, idx].real, VR[:, idx].real
    W = VR
    scale = np.einsum("ki,kl,li->i", VL.conj(), A2, W)  # vl_i^H A2 w_i
    Wbar = (VL.conj() / scale[None, :]).T
    return Wbar, W, lam


def decompose_pairs(A1, A2, top):
    """D(A1, A2) for a pencil with complex-conjugate pairs, as a real basis (reading).

    Columns in descending order of the real part; a pair contributes the real and imaginary
    parts of the eigenvector of its member with positive imaginary part, with the phase chosen
    so that coefficient ``top`` (the value at z = 1) is real and positive.  W-bar = (A2 W)^{-1},
    so W-bar A2 W = I and W-bar A1 W is block diagonal (2x2 blocks for the pairs).
    Returns (W-bar, W, real parts, kinds) with kind 0 = real, 1 / 2 = real / imaginary part.
    """
    lam, VR = sla.eig(A1, A2)
    cx = np.abs(lam.imag) > 1e-10 * np.max(np.abs(lam))
    idx = [i for i in range(len(lam)) if (not cx[i]) or lam[i].imag > 0]
    idx.sort(key=lambda i: -lam[i].real)
    cols, lr, kinds = [], [], []
    for i in idx:
        if not cx[i]:
            cols.append(VR[:, i].real)
            lr.append(lam[i].real)
            kinds.append(0)
        else:
            w = VR[:, i]
            w = w * np.conj(w[top]) / abs(w[top])
            cols += [w.real, w.imag]
            lr += [lam[i].real, lam[i].real]
            kinds += [1, 2]
    W = np.stack(cols, axis=1)
    return np.linalg.inv(A2 @ W), W, np.array(lr), kinds


def g_at_one(l, Mp):
    """g_l^{M'}(1) of Eq. g-def (Condon-Shortley phase)."""
    nrm = np.sqrt((2 * l + 1) / 2.0 * factorial(l - Mp) / factorial(l + Mp))
    return nrm * (-1.0) ** Mp * factorial(l + Mp) / (2 ** Mp * factorial(Mp) * factorial(l - Mp))


class Preconditioner:
    def __init__(self, sysm, Estar, z_eigs="replaced"):
        self.s = sysm
        self.Estar = float(Estar)
        self.z_eigs = z_eigs
        if z_eigs == "computed" and sysm.nM != 1:
            raise ValueError("computed z eigenvalues only with n_M = 1")
        self.comp = {a: self._component(a) for a in sysm.comps}

    @staticmethod
    def _mats(g):
        return (g.az.mat(0), g.az.mat(1), g.az.mat(2), g.ax.mat(0), g.ax.mat(2), g.ay.mat(0), g.ay.mat(2))

    def _component(self, a):
        s = self.s
        g = s.g[a]
        z, x, y = g.az.pts, g.ax.pts, g.ay.pts
        Sz, D1z, D2z, Sx, D2x, Sy, D2y = self._mats(g)
        C = {"Wz": [], "Wzb": [], "Lz": [], "Wx": {}, "Wxb": {}, "Lx": {}, "Wy": {}, "Wyb": {}, "Ly": {},
             "complex": False}
        # z decompositions per M' (Eq. z-dec), normalised to g_l^{M'}(1)
        onez = g.az.basis.matrix(np.array([1.0]), 0)[0]
        top = g.az.basis.q * g.az.basis.N  # value function of the node z = 1
        for Mp in s.Mps:
            Dz = (1 - z * z)[:, None] * D2z - (2 * (Mp + 1) * z)[:, None] * D1z - Mp * (Mp + 1) * Sz
            try:
                Wb, W, lz = decompose(Dz, Sz, order="descending")
                kinds = [0] * g.nz
            except ComplexSpectrum:
                if self.z_eigs == "computed":
                    raise
                Wb, W, lz, kinds = decompose_pairs(Dz, Sz, top)
            f1 = onez @ W
            sc = np.empty(g.nz)
            for l in range(g.nz):  # the imaginary-part column of a pair takes its partner's scale
                sc[l] = sc[l - 1] if kinds[l] == 2 else g_at_one(Mp + l, Mp) / f1[l]
            C["Wz"].append(W * sc[None, :])
            C["Wzb"].append(Wb / sc[:, None])
            C["Lz"].append(lz)
        C["ells"] = list(range(s.M0, s.J + g.nz))
        Va = ph.coulomb(s.m, s.Z, a, x)
        Vh = ph.vhat(s.m, s.Z, a, y, g.Ry)
        B = -D2y + (Vh - self.Estar)[:, None] * Sy
        A2y = (1.0 / y ** 2)[:, None] * Sy
        for l in C["ells"]:
            A1 = -D2x + (self._ll1(C, l) / x ** 2)[:, None] * Sx + Va[:, None] * Sx
            Wb, W, lx = decompose(A1, Sx)
            C["Wx"][l], C["Wxb"][l], C["Lx"][l] = W, Wb, lx
            for i in range(g.nx):
                Wb, W, ly = decompose(B + lx[i] * Sy, A2y, allow_complex=True)
                C["Wy"][(l, i)], C["Wyb"][(l, i)], C["Ly"][(l, i)] = W, Wb, ly
                C["complex"] = C["complex"] or np.iscomplexobj(ly)
        return C

    def _ll1(self, C, l):
        """The value l(l+1) of z-mode l (or -Lambda~ for computed z eigenvalues, n_M = 1)."""
        if self.z_eigs == "computed":
            return -C["Lz"][0][l - self.s.M0]
        return l * (l + 1.0)

    # ------------------------------------------------------------------
    def chain(self, g, l):
        """M' indices (into Mps) whose z-mode range M'..M'+n_z-1 contains l."""
        return [iM for iM, Mp in enumerate(self.s.Mps) if Mp <= l <= Mp + g.nz - 1]

    def apply(self, v):
        s = self.s
        v = np.asarray(v, dtype=np.float64)
        out = np.empty_like(v)
        for a in s.comps:
            g = s.g[a]
            lo = s.off[a]
            blk = v[lo:lo + g.csize].reshape(s.nM, g.nz, g.nx, g.ny)
            out[lo:lo + g.csize] = self._apply_comp(a, blk).reshape(-1)
        return out

    def _apply_comp(self, a, v):
        s = self.s
        g = s.g[a]
        C = self.comp[a]
        J = s.J
        if C["complex"]:  # complex y eigenpairs: the stages in complex arithmetic
            v = v.astype(np.complex128)
        t = np.empty_like(v)
        for iM in range(s.nM):  # W-bar_z
            t[iM] = np.einsum("lk,kij->lij", C["Wzb"][iM], v[iM])
        for iM, Mp in enumerate(s.Mps):  # W-bar_x, W-bar_y
            for li in range(g.nz):
                l = Mp + li
                t[iM, li] = C["Wxb"][l] @ t[iM, li]
                for i in range(g.nx):
                    t[iM, li, i] = C["Wyb"][(l, i)] @ t[iM, li, i]
        u = np.empty_like(t)  # (L~0)^{-1}: tridiagonal along M' for every (l, i, j)
        for l in C["ells"]:
            ch = self.chain(g, l)
            n = len(ch)
            for i in range(g.nx):
                ly = C["Ly"][(l, i)]
                A = np.zeros((n, n, g.ny), dtype=np.result_type(ly.dtype, np.float64))
                for r, iM in enumerate(ch):
                    Mp = s.Mps[iM]
                    A[r, r] = ly + J * (J + 1) - 2 * Mp * Mp + self._ll1(C, l)
                    if r + 1 < n:  # to M'+1: lambda-hat^{J,M'} (Lambda_z^{M'+})_{l-M'+1,l-M'} = -lambda^{l,M'}
                        A[r, r + 1] = ph.lam_hat_plus(J, Mp) * (-ph.lam(l, Mp))
                    if r - 1 >= 0:  # to M'-1: -lambda-hat^{J,-M'} (Lambda_z^{M'-})_{l-M'+1,l-M'+2} = lambda^{l,-M'}
                        A[r, r - 1] = -ph.lam_hat_minus(J, Mp) * ph.lam(l, -Mp)
                rhs = np.stack([t[iM, l - s.Mps[iM], i] for iM in ch])
                for j in range(g.ny):
                    sol = np.linalg.solve(A[:, :, j], rhs[:, j])
                    for r, iM in enumerate(ch):
                        u[iM, l - s.Mps[iM], i, j] = sol[r]
        for iM, Mp in enumerate(s.Mps):  # W_y, W_x, W_z
            for li in range(g.nz):
                l = Mp + li
                for i in range(g.nx):
                    u[iM, li, i] = C["Wy"][(l, i)] @ u[iM, li, i]
                u[iM, li] = C["Wx"][l] @ u[iM, li]
        res = np.empty_like(u)
        for iM in range(s.nM):
            res[iM] = np.einsum("kl,lij->kij", C["Wz"][iM], u[iM])
        return res.real if C["complex"] else res

    # ------------------------------------------------------------------
    def dense_L(self, a):
        """The approximate operator L_alpha built densely from its definition (tiny grids).

        L_alpha = W-bar_z^{-1} L^{xy}_alpha W_z^{-1}, with the blocks of L^{xy}
        formed by Kronecker products with Lambda_z^{M'} and Lambda_z^{M'+-}.
        """
        s = self.s
        g = s.g[a]
        C = self.comp[a]
        J = s.J
        x, y = g.ax.pts, g.ay.pts
        _, _, _, Sx, D2x, Sy, D2y = self._mats(g)
        Va = ph.coulomb(s.m, s.Z, a, x)
        Vh = ph.vhat(s.m, s.Z, a, y, g.Ry)
        Xr2, Yr2 = np.diag(1 / x ** 2), np.diag(1 / y ** 2)
        nxy = g.nx * g.ny
        Iz = np.eye(g.nz)
        blocks = {}
        for iM, Mp in enumerate(s.Mps):
            base = (np.kron(Sx, -D2y) + np.kron(-D2x, Sy) + (J * (J + 1) - 2 * Mp * Mp) * np.kron(Sx, Yr2 @ Sy)
                    + np.kron(np.diag(Va) @ Sx, Sy) + np.kron(Sx, np.diag(Vh) @ Sy) - self.Estar * np.kron(Sx, Sy))
            lam_diag = np.array([-self._ll1(C, Mp + k) for k in range(g.nz)])
            blocks[(iM, iM)] = np.kron(Iz, base) - np.kron(np.diag(lam_diag), np.kron(Sx, Yr2 @ Sy) + np.kron(Xr2 @ Sx, Sy))
            if iM + 1 < s.nM:
                Lp = np.zeros((g.nz, g.nz))
                for k in range(1, g.nz):
                    Lp[k, k - 1] = -ph.lam(Mp + k, Mp)
                blocks[(iM, iM + 1)] = ph.lam_hat_plus(J, Mp) * np.kron(Lp, np.kron(Sx, Yr2 @ Sy))
            if iM - 1 >= 0:
                Lm = np.zeros((g.nz, g.nz))
                for k in range(g.nz - 1):
                    Lm[k, k + 1] = ph.lam(Mp + k, -Mp)
                blocks[(iM, iM - 1)] = -ph.lam_hat_minus(J, Mp) * np.kron(Lm, np.kron(Sx, Yr2 @ Sy))
        n = g.nz * nxy
        Lxy = np.zeros((s.nM * n, s.nM * n))
        for (r, c), b in blocks.items():
            Lxy[r * n:(r + 1) * n, c * n:(c + 1) * n] = b
        Wzb_full = sla.block_diag(*[np.kron(Wb, np.eye(nxy)) for Wb in C["Wzb"]])
        Wz_full = sla.block_diag(*[np.kron(W, np.eye(nxy)) for W in C["Wz"]])
        return np.linalg.solve(Wzb_full, np.linalg.solve(Wz_full.T, Lxy.T).T)

    def dense_L_fmfin(self, a):
        """The left-hand operator L of Eq. FM-fin at E = E*, built from the 1D matrices (Section 3.2)."""
        s = self.s
        g = s.g[a]
        J = s.J
        x, y, z = g.ax.pts, g.ay.pts, g.az.pts
        Va = ph.coulomb(s.m, s.Z, a, x)
        Vh = ph.vhat(s.m, s.Z, a, y, g.Ry)
        Xr2, Yr2 = np.diag(1 / x ** 2), np.diag(1 / y ** 2)
        Sz, D1z, D2z, Sx, D2x, Sy, D2y = self._mats(g)
        k3 = lambda A, B, C: np.kron(A, np.kron(B, C))
        n = g.npts
        L = np.zeros((s.nM * n, s.nM * n))
        for iM, Mp in enumerate(s.Mps):
            Dz = (1 - z * z)[:, None] * D2z - (2 * (Mp + 1) * z)[:, None] * D1z - Mp * (Mp + 1) * Sz
            blk = (-k3(Sz, Sx, D2y) - k3(Sz, D2x, Sy) + (J * (J + 1) - 2 * Mp * Mp) * k3(Sz, Sx, Yr2 @ Sy)
                   - k3(Dz, Sx, Yr2 @ Sy) - k3(Dz, Xr2 @ Sx, Sy) + k3(Sz, np.diag(Va) @ Sx, Sy)
                   + k3(Sz, Sx, np.diag(Vh) @ Sy) - self.Estar * k3(Sz, Sx, Sy))
            L[iM * n:(iM + 1) * n, iM * n:(iM + 1) * n] = blk
            if iM + 1 < s.nM:
                Dp = -(1 - z * z)[:, None] * D1z + (2 * (Mp + 1) * z)[:, None] * Sz
                L[iM * n:(iM + 1) * n, (iM + 1) * n:(iM + 2) * n] = ph.lam_hat_plus(J, Mp) * k3(Dp, Sx, Yr2 @ Sy)
            if iM - 1 >= 0:
                L[iM * n:(iM + 1) * n, (iM - 1) * n:iM * n] = -ph.lam_hat_minus(J, Mp) * k3(-D1z, Sx, Yr2 @ Sy)
        return L
