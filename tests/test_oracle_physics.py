"""Pins for the oracle's kinematics, potentials and angular functions, checked
against explicit 3D particle geometry and textbook identities."""
import numpy as np
import pytest
from scipy.special import eval_jacobi
from math import factorial

from oracle import physics as ph

MASSES = [(1.0, 1.0, 1e15), (1.0, 1.0, 1.0), (1.0, 3.0, 7.0)]


def jacobi_vectors(r, m):
    """Reduced Jacobi vectors by definition: x_a = sqrt(2 mu_a) (r_c - r_b) for cyclic (a, b, c),
    y_a = sqrt(2 mu_a(bc)) (r_a - centre of mass of (b, c))."""
    mu_pair, mu_rel = ph.reduced_masses(m)
    X, Y = [], []
    for a in range(3):
        b, c = (a + 1) % 3, (a + 2) % 3
        X.append(np.sqrt(2 * mu_pair[a]) * (r[c] - r[b]))
        cm = (m[b] * r[b] + m[c] * r[c]) / (m[b] + m[c])
        Y.append(np.sqrt(2 * mu_rel[a]) * (r[a] - cm))
    return X, Y


def plane_coords(xv, yv):
    x, y = np.linalg.norm(xv), np.linalg.norm(yv)
    return x, y, float(xv @ yv / (x * y))


@pytest.mark.parametrize("m", MASSES)
def test_rotation_matches_geometry(m):
    rng = np.random.default_rng(3)
    m = np.array(m)
    for _ in range(5):
        r = rng.standard_normal((3, 3))
        X, Y = jacobi_vectors(r, m)
        for a in (1, 2, 3):
            for b in (1, 2, 3):
                if a == b:
                    continue
                c, s = ph.rotation_cs(m, b, a)
                assert abs(c * c + s * s - 1) < 1e-14
                # Eq. JacobiTrans
                assert np.allclose(X[b - 1], c * X[a - 1] + s * Y[a - 1], atol=1e-9)
                assert np.allclose(Y[b - 1], -s * X[a - 1] + c * Y[a - 1], atol=1e-9)
                # Section 2.2 formulas for (x_b, y_b, z_b)
                xa, ya, za = plane_coords(X[a - 1], Y[a - 1])
                xb, yb, zb = ph.rotate_xyz(c, s, xa, ya, za)
                assert np.allclose([xb, yb, zb], plane_coords(X[b - 1], Y[b - 1]), atol=1e-9)


@pytest.mark.parametrize("m", MASSES)
def test_w_angle_matches_body_frames(m):
    """w_ba: y_b expressed in alpha's body frame is (sin w, 0, cos w) (Eq. euler-ba)."""
    rng = np.random.default_rng(4)
    m = np.array(m)
    for _ in range(5):
        r = rng.standard_normal((3, 3))
        X, Y = jacobi_vectors(r, m)
        for a in (1, 2, 3):
            xa_v, ya_v = X[a - 1], Y[a - 1]
            ez = ya_v / np.linalg.norm(ya_v)
            ex = xa_v - (xa_v @ ez) * ez
            ex /= np.linalg.norm(ex)
            for b in (1, 2, 3):
                if a == b:
                    continue
                c, s = ph.rotation_cs(m, b, a)
                x, y, z = plane_coords(xa_v, ya_v)
                xb, yb, zb = ph.rotate_xyz(c, s, x, y, z)
                w = ph.w_angle(b, a, c, s, x, y, z, yb)
                yb_v = Y[b - 1] / np.linalg.norm(Y[b - 1])
                assert abs(np.cos(w) - yb_v @ ez) < 1e-9
                assert abs(np.sin(w) - yb_v @ ex) < 1e-9


def test_round_trip_and_invariants():
    m = np.array([1.0, 2.0, 5.0])
    x, y, z = 1.3, 0.7, -0.4
    for a, b in ((1, 2), (2, 3), (3, 1), (2, 1)):
        c, s = ph.rotation_cs(m, b, a)
        xb, yb, zb = ph.rotate_xyz(c, s, x, y, z)
        assert abs(xb ** 2 + yb ** 2 - x ** 2 - y ** 2) < 1e-12  # hyperradius
        assert abs(xb * yb * np.sqrt(1 - zb ** 2) - x * y * np.sqrt(1 - z ** 2)) < 1e-12  # area
        c2, s2 = ph.rotation_cs(m, a, b)
        assert np.allclose(ph.rotate_xyz(c2, s2, xb, yb, zb), (x, y, z), atol=1e-12)


def test_coulomb_in_reduced_coordinates():
    rng = np.random.default_rng(5)
    m = np.array([1.0, 3.0, 7.0])
    Z = np.array([-1.0, 2.0, 1.5])
    r = rng.standard_normal((3, 3))
    X, _ = jacobi_vectors(r, m)
    for a in (1, 2, 3):
        b, c = [i for i in range(3) if i != a - 1]
        dist = np.linalg.norm(r[b] - r[c])
        assert abs(ph.coulomb(m, Z, a, np.linalg.norm(X[a - 1])) - Z[b] * Z[c] / dist) < 1e-12


def test_cutoff():
    assert ph.cutoff_chi(0.0, 1.0, 2.01, 1.0, np.inf) == 1.0
    assert ph.cutoff_chi(40.0, 1.0, 2.01, 1.0, np.inf) == 0.0
    # finite y0: the cut-off widens with y
    assert ph.cutoff_chi(2.0, 10.0, 2.01, 1.0, 1.0) > ph.cutoff_chi(2.0, 0.0, 2.01, 1.0, 1.0)


def jacobi_form(J, M, Mp, w):
    """Eq. D-def with the factorial reading sqrt((J+M')!(J-M')!/((J+M)!(J-M)!)), for M' >= |M|."""
    pref = np.sqrt(factorial(J + Mp) * factorial(J - Mp) / (factorial(J + M) * factorial(J - M)))
    return pref * np.sin(w / 2) ** (Mp - M) * np.cos(w / 2) ** (Mp + M) * eval_jacobi(J - Mp, Mp - M, Mp + M, np.cos(w))


def dmat(J, w):
    return np.array([[ph.wigner_d(J, M, Mp, w) for Mp in range(-J, J + 1)] for M in range(-J, J + 1)])


@pytest.mark.parametrize("J", [0, 1, 2, 3, 5, 10, 11])
def test_wigner_d(J):
    w = np.array([0.0, 0.3, 1.7, 3.0, np.pi, 4.4])
    for M in range(-J, J + 1):
        for Mp in range(abs(M), J + 1):
            assert np.allclose(ph.wigner_d(J, M, Mp, w), jacobi_form(J, M, Mp, w), atol=1e-12)
    assert np.allclose(dmat(J, 0.0), np.eye(2 * J + 1), atol=1e-14)
    for a, b in ((0.4, 1.1), (2.0, 2.5)):
        D = dmat(J, a)
        assert np.allclose(D @ D.T, np.eye(2 * J + 1), atol=1e-12)
        assert np.allclose(dmat(J, a) @ dmat(J, b), dmat(J, a + b), atol=1e-12)


def test_wigner_d_J1_closed_forms():
    w = 0.9
    assert abs(ph.wigner_d(1, 1, 1, w) - (1 + np.cos(w)) / 2) < 1e-14
    assert abs(ph.wigner_d(1, 1, 0, w) + np.sin(w) / np.sqrt(2)) < 1e-14
    assert abs(ph.wigner_d(1, 0, 1, w) - np.sin(w) / np.sqrt(2)) < 1e-14
    assert abs(ph.wigner_d(1, 1, -1, w) - (1 - np.cos(w)) / 2) < 1e-14
    assert abs(ph.wigner_d(1, 0, 0, w) - np.cos(w)) < 1e-14


def test_d_over_sin_is_the_quotient():
    w = np.array([0.2, 1.0, 2.5, 3.5, 5.9])
    for J, M, Mp, k in ((2, 0, 2, 2), (3, 1, 3, 2), (3, 0, -2, 2), (2, 1, 2, 1), (10, 3, 9, 6), (11, 0, 11, 8)):
        assert np.allclose(ph.wigner_d_over_sin(J, M, Mp, w, k), ph.wigner_d(J, M, Mp, w) / np.sin(w) ** k, atol=1e-12)


def test_F_basis_symmetry():
    """F_{M,-M'} = tau (-1)^{M'} F_{M,M'} (Section 2.2), through the d-functions at (0, w, 0)."""
    w = 1.3
    for J in (1, 2, 3, 10):
        for tau in (1, -1):
            for M in range(-J, J + 1):
                for Mp in range(1, J + 1):
                    Fp = (ph.wigner_d(J, M, Mp, w) + tau * (-1) ** Mp * ph.wigner_d(J, M, -Mp, w))
                    Fm = (ph.wigner_d(J, M, -Mp, w) + tau * (-1) ** Mp * ph.wigner_d(J, M, Mp, w))
                    assert abs(Fm - tau * (-1) ** Mp * Fp) < 1e-13


def test_lambda_hat():
    assert abs(ph.lam(2, 0) - np.sqrt(6)) < 1e-15
    assert abs(ph.lam_hat_plus(2, 0) - np.sqrt(12)) < 1e-14
    assert abs(ph.lam_hat_minus(2, 1) - np.sqrt(6) * np.sqrt(2)) < 1e-14
    assert ph.lam(2, 2) == 0.0
