"""Three-body kinematics, potentials and angular functions (oracle).

ORACLE -- test infrastructure only (see ``oracle/__init__``).

Particles are labelled 1, 2, 3; arrays here are indexed 0, 1, 2.
"""
from __future__ import annotations

from math import factorial

import numpy as np


# --------------------------------------------------------------------------
# masses and the kinematic rotation (Section 2.1, Eq. JacobiTrans)
# --------------------------------------------------------------------------
def reduced_masses(m):
    """mu_a = m_b m_c/(m_b+m_c) and mu_a(bc) = m_a (m_b+m_c)/M, a = 1, 2, 3."""
    m = np.asarray(m, dtype=np.float64)
    M = m.sum()
    mu_pair = np.empty(3)
    mu_rel = np.empty(3)
    for a in range(3):
        b, c = [i for i in range(3) if i != a]
        mu_pair[a] = m[b] * m[c] / (m[b] + m[c])
        mu_rel[a] = m[a] * (m[b] + m[c]) / M
    return mu_pair, mu_rel


def rotation_cs(m, beta, alpha):
    """(c_beta,alpha, s_beta,alpha) of Eq. JacobiTrans; beta, alpha are 1-based labels."""
    m = np.asarray(m, dtype=np.float64)
    M = m.sum()
    mb, ma = m[beta - 1], m[alpha - 1]
    c = -np.sqrt(mb * ma / ((M - mb) * (M - ma)))
    s = (-1.0) ** (beta - alpha) * np.sign(alpha - beta) * np.sqrt(1.0 - c * c)
    return float(c), float(s)


def rotate_xyz(c, s, x, y, z):
    """X_beta from X_alpha = (x, y, z) (Section 2.2, the x_beta, y_beta, z_beta formulas)."""
    xb = np.sqrt(np.maximum(c * c * x * x + 2 * s * c * x * y * z + s * s * y * y, 0.0))
    yb = np.sqrt(np.maximum(s * s * x * x - 2 * s * c * x * y * z + c * c * y * y, 0.0))
    zb = (s * c * (y * y - x * x) + (c * c - s * s) * x * y * z) / (xb * yb)
    return xb, yb, np.clip(zb, -1.0, 1.0)


def w_angle(beta, alpha, c, s, x, y, z, yb):
    """Angle w_beta,alpha of Eq. euler-ba, with the branch rule of Section 2.2."""
    arg = np.clip((-s * x * z + c * y) / yb, -1.0, 1.0)
    w = np.arccos(arg)
    if (beta, alpha) in ((1, 2), (2, 3), (3, 1)):
        return w
    return 2 * np.pi - w


# --------------------------------------------------------------------------
# potentials (Section 2.1, Eqs. PotSplit, split3b, Mcutoff0)
# --------------------------------------------------------------------------
def coulomb(m, Z, a, x):
    """V^C_a(x) = sqrt(2 mu_a) Z_b Z_c / x in reduced coordinates (a is 1-based)."""
    mu_pair, _ = reduced_masses(m)
    b, c = [i for i in range(3) if i != a - 1]
    return np.sqrt(2 * mu_pair[a - 1]) * Z[b] * Z[c] / x


def cutoff_chi(x, y, nu, x0, y0):
    """Merkuriev cut-off chi = 2 / {1 + exp[(x/x0)^nu / (1 + y/y0)]} (Eq. Mcutoff0)."""
    arg = (x / x0) ** nu
    if np.isfinite(y0):
        arg = arg / (1.0 + y / y0)
    with np.errstate(over="ignore"):
        return 2.0 / (1.0 + np.exp(arg))


def split_potential(m, Z, a, x, y, mode, nu, x0, y0):
    """(V^(s)_a, V^(l)_a) at reduced coordinates (x, y) of pair a.

    mode 0: Merkuriev split (Eq. split3b); mode 1: no splitting, V^(s) = V,
    V^(l) = 0 (standard Faddeev equations, Section 2.1).
    """
    vc = coulomb(m, Z, a, x)
    if mode == 1:
        return vc, np.zeros_like(vc)
    chi = cutoff_chi(x, y, nu, x0, y0)
    return chi * vc, (1.0 - chi) * vc


def vhat(m, Z, a, y, Ry):
    """Preconditioner potential V^_a(y) of Section 4 (reading: sqrt(2 mu_a(bc)) in the numerator).

    Z_a (Z_b + Z_c) sqrt(2 mu_a(bc)) / y * (1 - exp(-(y / (0.05 R_y))^2)).
    It enters only the preconditioner: it cancels in H.
    """
    _, mu_rel = reduced_masses(m)
    b, c = [i for i in range(3) if i != a - 1]
    q = Z[a - 1] * (Z[b] + Z[c]) * np.sqrt(2 * mu_rel[a - 1])
    return q / y * (1.0 - np.exp(-(y / (0.05 * Ry)) ** 2))


# --------------------------------------------------------------------------
# Wigner d-functions and the F basis (Section 2.2, Eqs. D-def, F-def, F-ba)
# --------------------------------------------------------------------------
def _wigner_terms(J, M, Mp):
    """Terms (coef, cos_power, sin_power) of Wigner's explicit sum for d^J_{M M'}.

    Convention of Eq. D-def (Biedenharn / Varshalovich): in the textbook form
    d^j_{m' m}(b) = sum_s (-1)^{m'-m+s} sqrt((j+m')!(j-m')!(j+m)!(j-m)!)
        / ((j+m-s)! s! (m'-m+s)! (j-m'-s)!) cos(b/2)^{2j+m-m'-2s} sin(b/2)^{m'-m+2s}
    with m' = M (first index) and m = Mp (second index).
    """
    mp_, m_ = M, Mp
    pref = np.sqrt(float(factorial(J + mp_) * factorial(J - mp_) * factorial(J + m_) * factorial(J - m_)))
    out = []
    for s in range(0, 2 * J + 1):
        d1, d2, d3, d4 = J + m_ - s, s, mp_ - m_ + s, J - mp_ - s
        if min(d1, d2, d3, d4) < 0:
            continue
        coef = (-1.0) ** (mp_ - m_ + s) * pref / (factorial(d1) * factorial(d2) * factorial(d3) * factorial(d4))
        out.append((coef, 2 * J + m_ - mp_ - 2 * s, mp_ - m_ + 2 * s))
    return out


def wigner_d(J, M, Mp, w):
    """d^J_{M M'}(w) of Eq. D-def by Wigner's explicit sum."""
    if abs(M) > J or abs(Mp) > J:
        return np.zeros_like(np.asarray(w, dtype=np.float64))
    w = np.asarray(w, dtype=np.float64)
    c, s = np.cos(w / 2), np.sin(w / 2)
    tot = np.zeros_like(w)
    for coef, pc, ps in _wigner_terms(J, M, Mp):
        tot = tot + coef * c ** pc * s ** ps
    return tot


def wigner_d_over_sin(J, M, Mp, w, k):
    """d^J_{M M'}(w) / sin(w)^k for k <= min(|M-M'|, |M+M'|), as a regular function.

    Every term of the explicit sum carries cos(w/2)^{>=|M+M'|} sin(w/2)^{>=|M-M'|},
    and sin w = 2 sin(w/2) cos(w/2), so the quotient is a finite sum.
    """
    assert k <= min(abs(M - Mp), abs(M + Mp))
    w = np.asarray(w, dtype=np.float64)
    c, s = np.cos(w / 2), np.sin(w / 2)
    tot = np.zeros_like(w)
    for coef, pc, ps in _wigner_terms(J, M, Mp):
        tot = tot + coef * c ** (pc - k) * s ** (ps - k)
    return tot / 2.0 ** k


def lam(J, Mp):
    """lambda^{J M'} = sqrt(J(J+1) - M'(M'+1)) (Section 2.2)."""
    return np.sqrt(max(J * (J + 1) - Mp * (Mp + 1), 0))


def lam_hat_plus(J, Mp):
    """lambda-hat^{J, +M'} = lambda^{J, M'} sqrt(1 + delta_{M'0}) (Section 3.1)."""
    return lam(J, Mp) * np.sqrt(1.0 + (Mp == 0))


def lam_hat_minus(J, Mp):
    """lambda-hat^{J, -M'} = lambda^{J, -M'} sqrt(1 + delta_{M'1}) (Section 3.1)."""
    return lam(J, -Mp) * np.sqrt(1.0 + (Mp == 1))


def coupling_K(J, tau, Mp, Mpp, w):
    """(-1)^{M''-M'} 2/sqrt(2+2 delta_{M''0}) F^{J tau}_{M'' M'}(0, w, 0) (Eqs. FM, F-def)."""
    F = (wigner_d(J, Mpp, Mp, w) + tau * (-1.0) ** Mp * wigner_d(J, Mpp, -Mp, w)) / np.sqrt(2.0 + 2.0 * (Mp == 0))
    return (-1.0) ** (Mpp - Mp) * 2.0 / np.sqrt(2.0 + 2.0 * (Mpp == 0)) * F


def coupling_K_over_sin(J, tau, Mp, Mpp, w, k):
    """coupling_K(...) / sin(w)^k, regular for k <= M' - M'' (M'' < M')."""
    F = (wigner_d_over_sin(J, Mpp, Mp, w, k) + tau * (-1.0) ** Mp * wigner_d_over_sin(J, Mpp, -Mp, w, k)) \
        / np.sqrt(2.0 + 2.0 * (Mp == 0))
    return (-1.0) ** (Mpp - Mp) * 2.0 / np.sqrt(2.0 + 2.0 * (Mpp == 0)) * F
