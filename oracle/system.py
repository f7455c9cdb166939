"""Collocation matrices H and S of the 3D Faddeev-Merkuriev equations (oracle).

ORACLE -- test infrastructure only (see ``oracle/__init__``).

H is the discretised operator of Eq. FM-pre with its right-hand side moved to
the left (Eq. FM-lin, E = 0); S has the entries S^k(z) S^i(x) S^j(y) at the
collocation points.  Every entry is formed from its definition: the operator
of Eq. FM-pre applied to one product basis function and evaluated at one
collocation point (Section 3.1).  The coupling rows follow Eqs. r-form and
s-rot: the beta-basis evaluated at alpha's collocation points mapped to the
beta Jacobi coordinates.

Unknown ordering (Section 3.2): y fastest, then x, then z, then M', then the
solved component:  index = off[a] + ((iM * nz_a + k) * nx_a + i) * ny_a + j.

Readings of points where the paper is silent or inconsistent:

* Sign of the coupling block.  Eq. FM-6d has -V^(s) sum psi_beta on the right;
  moving it to the left gives +V^(s)_a (...) in H.  (The leading minus on
  F_ab in Eq. r-form describes the right-hand-side operator.)
* The angular ratio (1 - z_b^2)^{M''/2} / (1 - z_a^2)^{M'/2} is evaluated with
  the area identity x_a y_a sin(theta_a) = x_b y_b sin(theta_b) and, for
  M'' < M', with sin(theta_a) = |sin w| y_b / (|s| x_a); both are exact
  rewritings of the quotient.
* Points rotated outside the source box contribute zero (Dirichlet extension).
* Coupling rows: in the Merkuriev split a row carries the coupling only where
  chi_a(x, y) > vs_cut (the same rule on every side; default 1e-20).
* One spline grid serves every solved component unless a per-component grid
  is given (the paper's runs use per-component boxes, Section 4).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import physics as ph
from .splines import Axis

MERKURIEV, NO_SPLIT, SCHRODINGER = 0, 1, 2


class Grid:
    """Spline axes of one solved component (Section 3.1 notation (n_x, n_y, n_z), (R_x, R_y))."""

    def __init__(self, nint, R, maps, nM, basis=0):
        nix, niy, niz = nint
        self.Rx, self.Ry = float(R[0]), float(R[1])
        self.ax = Axis(maps[0], nix, 0.0, self.Rx, dirichlet=True, basis=basis)
        self.ay = Axis(maps[1], niy, 0.0, self.Ry, dirichlet=True, basis=basis)
        self.az = Axis(maps[2], niz, -1.0, 1.0, dirichlet=False, basis=basis)
        self.nx, self.ny, self.nz = self.ax.n, self.ay.n, self.az.n
        self.npts = self.nz * self.nx * self.ny
        self.csize = nM * self.npts

    def coords(self, pts):
        pts = np.asarray(pts, dtype=np.int64)
        k, rem = np.divmod(pts, self.nx * self.ny)
        i, j = np.divmod(rem, self.ny)
        return k, i, j, self.az.pts[k], self.ax.pts[i], self.ay.pts[j]


class FMSystem:
    def __init__(self, wl):
        self.wl = dict(wl)
        self.m = np.array(wl["mass"], dtype=np.float64)
        self.Z = np.array(wl["charge"], dtype=np.float64)
        self.J, self.tau, self.p = int(wl["J"]), int(wl["tau"]), int(wl["p"])
        self.mode = int(wl["mode"])
        self.nu, self.x0, self.y0 = float(wl["nu"]), float(wl["x0"]), float(wl["y0"])
        self.vs_cut = float(wl.get("vs_cut", 0.0))
        self.M0 = (1 - self.tau) // 2
        self.nM = self.J - self.M0 + 1
        if self.nM <= 0:
            raise ValueError("no admissible M' for this (J, tau)")
        self.Mps = list(range(self.M0, self.J + 1))
        if self.mode == SCHRODINGER:
            self.comps = [1]
        elif int(wl["identical_pair"]) == 12:
            self.comps = [1, 3]
        else:
            self.comps = [1, 2, 3]
        grids = wl.get("grids") or {}
        self.g = {}
        off = 0
        self.off = {}
        for a in self.comps:
            nint = grids.get(a, {}).get("nint", wl["nint"])
            R = grids.get(a, {}).get("R", wl["R"])
            mx, my, mz = wl["maps"]
            g = Grid(nint, R, (mx, my, mz), self.nM, int(wl.get("basis", 0)))
            self.g[a] = g
            self.off[a] = off
            off += g.csize
        self.N = off
        self.mu_pair, self.mu_rel = ph.reduced_masses(self.m)

    # ------------------------------------------------------------------
    def sources(self, alpha):
        """Coupling sources of component alpha: (beta, source component, z sign, symmetry factor?).

        With particles 1, 2 identical only alpha = 1, 3 are solved and
        psi_2(x, y, z) = p (-1)^{M'} psi_1(x, y, -z) (Eq. 2-sym-part).
        """
        if self.mode == SCHRODINGER:
            return []
        out = []
        for beta in (1, 2, 3):
            if beta == alpha:
                continue
            if beta in self.comps:
                out.append((beta, beta, 1.0, False))
            else:  # beta = 2 with the identical pair (1, 2)
                out.append((beta, 1, -1.0, True))
        return out

    def point_coords(self, a, pts):
        return self.g[a].coords(pts)

    def W(self, alpha, x, y, z):
        """Left-hand potential of Eq. FM-pre: V_a(x) + sum_{b != a} V^(l)_b(x_b, y_b)."""
        tot = ph.coulomb(self.m, self.Z, alpha, x)
        for beta in (1, 2, 3):
            if beta == alpha:
                continue
            c, s = ph.rotation_cs(self.m, beta, alpha)
            xb, yb, _ = ph.rotate_xyz(c, s, x, y, z)
            if self.mode == SCHRODINGER:
                tot = tot + ph.coulomb(self.m, self.Z, beta, xb)
            else:
                _, vl = ph.split_potential(self.m, self.Z, beta, xb, yb, self.mode, self.nu, self.x0, self.y0)
                tot = tot + vl
        return tot

    def vs(self, alpha, x, y):
        vs, _ = ph.split_potential(self.m, self.Z, alpha, x, y, self.mode, self.nu, self.x0, self.y0)
        return vs

    def coupling_active(self, alpha, x, y):
        if self.mode == NO_SPLIT:
            return np.ones(np.broadcast(x, y).shape, dtype=bool)
        return ph.cutoff_chi(x, y, self.nu, self.x0, self.y0) > self.vs_cut

    # ------------------------------------------------------------------
    def _cols(self, a_label, iM, cz, cx, cy):
        g = self.g[a_label]
        base = self.off[a_label] + iM * g.npts
        c = base + (cz[:, :, None, None] * g.nx + cx[:, None, :, None]) * g.ny + cy[:, None, None, :]
        bad = (cz[:, :, None, None] < 0) | (cx[:, None, :, None] < 0) | (cy[:, None, None, :] < 0)
        return np.where(bad, -1, c)

    @staticmethod
    def _outer(fz, fx, fy):
        return fz[:, :, None, None] * fx[:, None, :, None] * fy[:, None, None, :]

    def local_entries(self, a_label, iM, pts):
        """COO entries of rows (a, M', pts) of the alpha-diagonal part of H (Eq. FM-pre left side, E = 0)."""
        J, Mp = self.J, self.Mps[iM]
        g = self.g[a_label]
        k, i, j, z, x, y = g.coords(pts)
        cz, Sz = g.az.basis.local(z, 0)
        _, D1z = g.az.basis.local(z, 1)
        _, D2z = g.az.basis.local(z, 2)
        cx, Sx = g.ax.basis.local(x, 0)
        _, D2x = g.ax.basis.local(x, 2)
        cy, Sy = g.ay.basis.local(y, 0)
        _, D2y = g.ay.basis.local(y, 2)
        q = 1.0 / x ** 2 + 1.0 / y ** 2
        Cc = q * Mp * (Mp + 1) + (J * (J + 1) - 2 * Mp * Mp) / y ** 2 + self.W(a_label, x, y, z)
        zfac = (-q * (1 - z * z))[:, None] * D2z + (2 * (Mp + 1) * z * q)[:, None] * D1z + Cc[:, None] * Sz
        vals = -self._outer(Sz, Sx, D2y) - self._outer(Sz, D2x, Sy) + self._outer(zfac, Sx, Sy)
        rows = self.off[a_label] + iM * g.npts + np.asarray(pts)
        blocks = [(iM, vals)]
        if iM + 1 < self.nM:  # T-hat^+ couples to psi-hat_{M'+1}
            f = (ph.lam_hat_plus(J, Mp) / y ** 2)[:, None] * (-(1 - z * z)[:, None] * D1z + (2 * (Mp + 1) * z)[:, None] * Sz)
            blocks.append((iM + 1, self._outer(f, Sx, Sy)))
        if iM - 1 >= 0:  # T-hat^- couples to psi-hat_{M'-1}
            f = (ph.lam_hat_minus(J, Mp) / y ** 2)[:, None] * D1z
            blocks.append((iM - 1, self._outer(f, Sx, Sy)))
        R, C, V = [], [], []
        for jM, v in blocks:
            cols = self._cols(a_label, jM, cz, cx, cy)
            ok = cols >= 0
            R.append(np.broadcast_to(rows[:, None, None, None], cols.shape)[ok])
            C.append(cols[ok])
            V.append(v[ok])
        return np.concatenate(R), np.concatenate(C), np.concatenate(V)

    def coupling_weight(self, alpha, beta, iM, iMpp, x, y, z, xb, yb, w, s):
        """V^(s)_a * (x y)/(x_b y_b) * angular factor of Eq. FM-pre for M' -> M''.

        Angular factor: (1 - z_b^2)^{M''/2} / (1 - z^2)^{M'/2} times
        (-1)^{M''-M'} 2/sqrt(2+2 delta_{M''0}) F^{J tau}_{M'' M'}(0, w, 0), with the
        area identity (1 - z_b^2)^{1/2} = rho (1 - z^2)^{1/2}, rho = x y / (x_b y_b).
        """
        J, tau = self.J, self.tau
        Mp, Mpp = self.Mps[iM], self.Mps[iMpp]
        rho = x * y / (xb * yb)
        sin_t = np.sqrt(np.clip(1.0 - z * z, 0.0, None))
        if Mpp >= Mp:
            ang = sin_t ** (Mpp - Mp) * ph.coupling_K(J, tau, Mp, Mpp, w)
        else:
            kk = Mp - Mpp
            sgn = 1.0 if (beta, alpha) in ((1, 2), (2, 3), (3, 1)) else -1.0
            ang = (abs(s) * x / yb) ** kk * sgn ** kk * ph.coupling_K_over_sin(J, tau, Mp, Mpp, w, kk)
        return self.vs(alpha, x, y) * rho * rho ** Mpp * ang

    def coupling_entries(self, a_label, iM, pts):
        """COO entries of rows (a, M', pts) of the coupling part of H (+V^(s) sum_b ..., reading of Eq. FM-6d)."""
        pts = np.asarray(pts, dtype=np.int64)
        k, i, j, z, x, y = self.point_coords(a_label, pts)
        act = self.coupling_active(a_label, x, y)
        pts, z, x, y = pts[act], z[act], x[act], y[act]
        R, C, V = [np.zeros(0, np.int64)], [np.zeros(0, np.int64)], [np.zeros(0)]
        rows = self.off[a_label] + iM * self.g[a_label].npts + pts
        for beta, src, zsign, sym in self.sources(a_label):
            c, s = ph.rotation_cs(self.m, beta, a_label)
            xb, yb, zb = ph.rotate_xyz(c, s, x, y, z)
            w = ph.w_angle(beta, a_label, c, s, x, y, z, yb)
            gs = self.g[src]
            cz, Sz = gs.az.basis.local(zsign * zb, 0)
            cx, Sx = gs.ax.basis.local(xb, 0)
            cy, Sy = gs.ay.basis.local(yb, 0)
            basis = self._outer(Sz, Sx, Sy)
            for iMpp, Mpp in enumerate(self.Mps):
                wgt = self.coupling_weight(a_label, beta, iM, iMpp, x, y, z, xb, yb, w, s)
                if sym:
                    wgt = wgt * self.p * (-1.0) ** Mpp
                cols = self._cols(src, iMpp, cz, cx, cy)
                ok = cols >= 0
                R.append(np.broadcast_to(rows[:, None, None, None], cols.shape)[ok])
                C.append(cols[ok])
                V.append((wgt[:, None, None, None] * basis)[ok])
        return np.concatenate(R), np.concatenate(C), np.concatenate(V)

    def S_entries(self, a_label, iM, pts):
        g = self.g[a_label]
        k, i, j, z, x, y = g.coords(pts)
        cz, Sz = g.az.basis.local(z, 0)
        cx, Sx = g.ax.basis.local(x, 0)
        cy, Sy = g.ay.basis.local(y, 0)
        rows = self.off[a_label] + iM * g.npts + np.asarray(pts)
        cols = self._cols(a_label, iM, cz, cx, cy)
        v = self._outer(Sz, Sx, Sy)
        ok = cols >= 0
        return np.broadcast_to(rows[:, None, None, None], cols.shape)[ok], cols[ok], v[ok]

    # ------------------------------------------------------------------
    def split_rows(self, rows):
        """Global row indices -> list of (component label, iM, point indices, positions)."""
        rows = np.asarray(rows, dtype=np.int64)
        out = []
        for a in self.comps:
            npts = self.g[a].npts
            for iM in range(self.nM):
                lo = self.off[a] + iM * npts
                sel = np.nonzero((rows >= lo) & (rows < lo + npts))[0]
                if len(sel):
                    out.append((a, iM, rows[sel] - lo, sel))
        return out

    def _assemble(self, fn, rows):
        if rows is None:
            rows = np.arange(self.N)
        rows = np.asarray(rows, dtype=np.int64)
        R, C, V = [], [], []
        for a, iM, pts, _ in self.split_rows(rows):
            for f in fn:
                r, c, v = f(a, iM, pts)
                R.append(r)
                C.append(c)
                V.append(v)
        R, C, V = np.concatenate(R), np.concatenate(C), np.concatenate(V)
        # renumber rows to positions in the requested list
        pos = np.empty(self.N, dtype=np.int64)
        pos[rows] = np.arange(len(rows))
        return sp.csr_matrix((V, (pos[R], C)), shape=(len(rows), self.N))

    def H(self, rows=None):
        """Rows of H (all rows by default) as CSR."""
        return self._assemble([self.local_entries, self.coupling_entries], rows)

    def H_local(self, rows=None):
        return self._assemble([self.local_entries], rows)

    def S(self, rows=None):
        return self._assemble([self.S_entries], rows)
