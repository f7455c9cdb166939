"""Pins for the oracle's spline layer: exact polynomial reproduction, node maps,
collocation points, and 1D eigenvalue problems with closed-form limits."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle.splines import Axis, HermiteBasis, nodes_map_pow, nodes_sin, hermite_shapes, MAP_POW, MAP_SIN, MAP_EQUI


def test_map_pow_endpoints_and_monotone():
    t = nodes_map_pow(40.0, 24)
    assert t[0] == 0.0 and t[-1] == 40.0
    assert np.all(np.diff(t) > 0)
    # Eq. map-pow at u = 1/2: 4((1 + R/4)^{1/2} - 1)
    assert abs(t[12] - 4 * (np.sqrt(11.0) - 1)) < 1e-13


def test_sin_nodes_symmetric():
    t = nodes_sin(8)
    assert t[0] == -1.0 and t[-1] == 1.0
    assert np.allclose(t, -t[::-1], atol=1e-15)
    assert abs(t[2] - np.sin(np.pi * (-0.5) / 2)) < 1e-15


def test_shapes_partition_and_endpoint_values():
    s = np.linspace(0, 1, 7)
    h = 0.3
    v = hermite_shapes(s, h, 0)
    assert np.allclose(v[:, 0] + v[:, 2], 1.0)  # value functions sum to one
    assert np.allclose(v[0], [1, 0, 0, 0]) and np.allclose(v[-1], [0, 0, 1, 0])
    d = hermite_shapes(s, h, 1)
    assert np.allclose(d[0], [0, 1, 0, 0]) and np.allclose(d[-1], [0, 0, 0, 1])


def _fd(f, t, k, eps=1e-4):
    if k == 1:
        return (f(t + eps) - f(t - eps)) / (2 * eps)
    return (f(t + eps) - 2 * f(t) + f(t - eps)) / eps ** 2


def test_derivative_shapes_match_finite_differences():
    s = np.array([0.13, 0.5, 0.77])
    h = 0.7
    for k in (1, 2):
        f = lambda tt: hermite_shapes(tt / h, h, 0)
        assert np.allclose(hermite_shapes(s, h, k), _fd(f, s * h, k), atol=1e-6)


@pytest.mark.parametrize("kind,nint,a,b,dirichlet", [
    (MAP_POW, 7, 0.0, 11.0, True), (MAP_EQUI, 5, 0.0, 3.0, True), (MAP_SIN, 6, -1.0, 1.0, False)])
def test_cubic_reproduction(kind, nint, a, b, dirichlet):
    """S c = p, D1 c = p', D2 c = p'' for any cubic p (Dirichlet-compatible in x, y)."""
    ax = Axis(kind, nint, a, b, dirichlet=dirichlet)
    rng = np.random.default_rng(1)
    if dirichlet:
        q0, q1 = rng.standard_normal(2)
        p = lambda t: (t - a) * (b - t) * (q0 + q1 * t)
        dp = lambda t: (b - t) * (q0 + q1 * t) - (t - a) * (q0 + q1 * t) + (t - a) * (b - t) * q1
        ddp = lambda t: -2 * (q0 + q1 * t) + 2 * q1 * (b - t) - 2 * q1 * (t - a)
    else:
        co = rng.standard_normal(4)
        p = lambda t: np.polyval(co, t)
        dp = lambda t: np.polyval(np.polyder(co), t)
        ddp = lambda t: np.polyval(np.polyder(co, 2), t)
    c = ax.basis.coefficients_of(p, dp)
    pts = np.concatenate([ax.pts, rng.uniform(a, b, 50)])
    for k, f in ((0, p), (1, dp), (2, ddp)):
        B = ax.basis.matrix(pts, k)
        assert np.max(np.abs(B @ c - f(pts))) < 1e-10 * max(1.0, np.max(np.abs(f(pts))))


def test_collocation_counts_and_interior():
    for nint in (1, 2, 5, 8):
        az = Axis(MAP_SIN, nint, -1.0, 1.0, dirichlet=False)
        assert len(az.pts) == 2 * nint + 2 == az.n
        assert np.all(np.abs(az.pts) < 1.0) and np.all(np.diff(az.pts) > 0)
    ax = Axis(MAP_POW, 9, 0.0, 40.0, dirichlet=True)
    assert len(ax.pts) == 18 == ax.n and np.all(ax.pts > 0) and np.all(ax.pts < 40.0)


def test_box_eigenvalues_converge_fourth_order():
    """-u'' = eps u, u(0) = u(R) = 0: eps_n = (n pi / R)^2."""
    R = 3.0
    errs = []
    for nint in (8, 16, 32):
        ax = Axis(MAP_EQUI, nint, 0.0, R, dirichlet=True)
        ev = np.sort(sla.eig(-ax.mat(2), ax.mat(0), right=False).real)
        errs.append(abs(ev[0] - (np.pi / R) ** 2))
        assert abs(ev[1] - (2 * np.pi / R) ** 2) < 1e-2
    assert errs[-1] < 1e-6
    assert errs[0] / errs[1] > 12 and errs[1] / errs[2] > 12  # ~2^4


def test_hydrogenic_x_problem():
    """-u'' + sqrt(2 mu) Z1 Z2 / x u = eps u  ->  eps_n = -mu (Z1 Z2)^2 / (2 n^2) (reduced coordinates)."""
    mu, ZZ = 1.0, -2.0
    ax = Axis(MAP_POW, 96, 0.0, 40.0, dirichlet=True)
    x = ax.pts
    A = -ax.mat(2) + (np.sqrt(2 * mu) * ZZ / x)[:, None] * ax.mat(0)
    ev = np.sort(sla.eig(A, ax.mat(0), right=False).real)
    for n in (1, 2, 3):
        assert abs(ev[n - 1] - (-mu * ZZ ** 2 / (2 * n * n))) < 1e-4


def test_out_of_box_points_are_zero():
    b = HermiteBasis(nodes_map_pow(10.0, 4), dirichlet=True)
    cols, vals = b.local(np.array([-0.1, 10.5, 5.0]), 0)
    assert np.all(vals[:2] == 0) and np.any(vals[2] != 0)


# ---------------------------------------------------------------------------------------------------
# quintic Hermite splines S_5^3 (Section 4)
# ---------------------------------------------------------------------------------------------------
def test_quintic_shapes_nodal_conditions_and_derivatives():
    """Each of the six shape functions carries exactly one unit among (value, t-derivative, second
    t-derivative) at the two interval ends; derivatives agree with finite differences."""
    from oracle.splines import QUINTIC
    h = 0.7
    for end, s0 in ((0, 0.0), (1, 1.0)):
        for d in range(3):
            v = hermite_shapes(np.array([s0]), h, d, QUINTIC)[0]
            want = np.zeros(6)
            want[3 * end + d] = 1.0
            assert np.allclose(v, want, atol=1e-12), (end, d, v)
    s = np.array([0.13, 0.5, 0.77])
    for k in (1, 2):
        f = lambda tt: hermite_shapes(tt / h, h, 0, QUINTIC)
        assert np.allclose(hermite_shapes(s, h, k, QUINTIC), _fd(f, s * h, k), atol=1e-5)


@pytest.mark.parametrize("kind,nint,a,b,dirichlet", [
    (MAP_POW, 7, 0.0, 36.0, True), (MAP_EQUI, 5, 0.0, 3.0, True), (MAP_SIN, 6, -1.0, 1.0, False),
    (MAP_SIN, 1, -1.0, 1.0, False), (MAP_SIN, 2, -1.0, 1.0, False)])
def test_quintic_reproduction(kind, nint, a, b, dirichlet):
    """S c = p, D1 c = p', D2 c = p'' for any quintic p (vanishing at both ends in x, y), c its Hermite data."""
    from oracle.splines import QUINTIC
    ax = Axis(kind, nint, a, b, dirichlet=dirichlet, basis=QUINTIC)
    rng = np.random.default_rng(2)
    co = rng.standard_normal(6)
    if dirichlet:
        co = np.polymul(np.polymul([1.0, -a], [-1.0, b]), co[:4])
    p = lambda t: np.polyval(co, t)
    dp = lambda t: np.polyval(np.polyder(co), t)
    ddp = lambda t: np.polyval(np.polyder(co, 2), t)
    c = ax.basis.coefficients_of(p, dp, ddp)
    pts = np.concatenate([ax.pts, rng.uniform(a, b, 50)])
    for k, f in ((0, p), (1, dp), (2, ddp)):
        B = ax.basis.matrix(pts, k)
        assert np.max(np.abs(B @ c - f(pts))) < 1e-10 * max(1.0, np.max(np.abs(f(pts))))


def test_quintic_collocation_counts():
    """Quintic: 3N+1 functions and Gauss points in x, y (the paper's counts, e.g. 22 for N = 7), 3N+3 in z."""
    from oracle.splines import QUINTIC
    for nint in (1, 2, 3, 6):
        az = Axis(MAP_SIN, nint, -1.0, 1.0, dirichlet=False, basis=QUINTIC)
        assert len(az.pts) == 3 * nint + 3 == az.n
        assert np.all(np.abs(az.pts) < 1.0) and np.all(np.diff(az.pts) > 0)
    ax = Axis(MAP_POW, 7, 0.0, 36.0, dirichlet=True, basis=QUINTIC)
    assert len(ax.pts) == 22 == ax.n and np.all(ax.pts > 0) and np.all(ax.pts < 36.0)
    assert np.all(np.diff(ax.pts) > 0)


def test_quintic_box_eigenvalues_converge_faster():
    """-u'' = eps u on [0, R]: the quintic collocation eigenvalue converges at a higher order than the cubic
    (at least sixth: halving h divides the error by more than 50)."""
    from oracle.splines import QUINTIC
    R = 3.0
    errs = []
    for nint in (4, 8, 16):
        ax = Axis(MAP_EQUI, nint, 0.0, R, dirichlet=True, basis=QUINTIC)
        ev = np.sort(sla.eig(-ax.mat(2), ax.mat(0), right=False).real)
        errs.append(abs(ev[0] - (np.pi / R) ** 2))
    assert errs[-1] < 1e-9
    assert errs[0] / errs[1] > 50 and errs[1] / errs[2] > 50


def test_quintic_hydrogenic_x_problem():
    from oracle.splines import QUINTIC
    mu, ZZ = 1.0, -2.0
    ax = Axis(MAP_POW, 40, 0.0, 40.0, dirichlet=True, basis=QUINTIC)
    x = ax.pts
    A = -ax.mat(2) + (np.sqrt(2 * mu) * ZZ / x)[:, None] * ax.mat(0)
    ev = np.sort(sla.eig(A, ax.mat(0), right=False).real)
    for n in (1, 2, 3):
        assert abs(ev[n - 1] - (-mu * ZZ ** 2 / (2 * n * n))) < 1e-6
