"""Host logic of libfm on the CPU (no GPU): the 1D decompositions of the
preconditioner set-up against LAPACK on the collocation matrices the solver uses."""
import numpy as np
import pytest
import scipy.linalg as sla

from fm_inputs import workload
from oracle import physics as ph
from oracle.system import FMSystem


@pytest.fixture(scope="module")
def lib():
    from paper_2005_05398_gb300 import build, _lib
    build.build()
    return _lib


def _check(lib, A1, A2, descending):
    Wb, W, lam = lib.fm_host_decompose(A1, A2, descending)
    n = len(lam)
    scale = np.abs(lam).max()
    assert np.abs(Wb @ A1 @ W - np.diag(lam)).max() < 1e-11 * scale
    assert np.abs(Wb @ A2 @ W - np.eye(n)).max() < 1e-11
    ref = np.sort(sla.eig(A1, A2, right=False).real)
    got = np.sort(lam)
    assert np.abs(got - ref).max() < 1e-10 * scale
    assert np.all(np.diff(lam) <= 0) if descending else np.all(np.diff(lam) >= 0)


@pytest.mark.parametrize("nint", [(7, 9, 5), (24, 24, 8), (64, 64, 16)])
def test_z_and_x_decompositions_match_lapack(lib, nint):
    s = FMSystem(workload("he_l0_24x24x8", nint=nint, R=(40.0, 40.0), J=2))
    g = s.g[1]
    z = g.az.pts
    Sz, D1z, D2z = g.az.mat(0), g.az.mat(1), g.az.mat(2)
    for Mp in (0, 1, 2):
        Dz = (1 - z * z)[:, None] * D2z - (2 * (Mp + 1) * z)[:, None] * D1z - Mp * (Mp + 1) * Sz
        try:
            sla_ev = sla.eig(Dz, Sz, right=False)
        except Exception:
            continue
        if np.abs(sla_ev.imag).max() > 1e-10 * np.abs(sla_ev).max():
            with pytest.raises(lib.FMError):
                lib.fm_host_decompose(Dz, Sz, True)
            continue
        _check(lib, Dz, Sz, True)
    x = g.ax.pts
    Sx, D2x = g.ax.mat(0), g.ax.mat(2)
    for l in (0, 1, 7, 20):
        A1 = -D2x + (l * (l + 1) / x ** 2 + ph.coulomb(s.m, s.Z, 1, x))[:, None] * Sx
        _check(lib, A1, Sx, False)


@pytest.mark.parametrize("zmap", [1, 2])
def test_high_momentum_z_pencils(lib, zmap):
    """The z problems of J = 10 and 11 (M' up to 11; equidistant and sin-mapped z nodes): real pencils
    decompose like LAPACK, complex ones are reported."""
    s = FMSystem(workload("he_l0_24x24x8", nint=(6, 6, 6), R=(40.0, 40.0), J=11, maps=(0, 0, zmap)))
    g = s.g[1]
    z = g.az.pts
    Sz, D1z, D2z = g.az.mat(0), g.az.mat(1), g.az.mat(2)
    checked = 0
    for Mp in range(0, 12):
        Dz = (1 - z * z)[:, None] * D2z - (2 * (Mp + 1) * z)[:, None] * D1z - Mp * (Mp + 1) * Sz
        ev = sla.eig(Dz, Sz, right=False)
        if np.abs(ev.imag).max() > 1e-10 * np.abs(ev).max():
            with pytest.raises(lib.FMError):
                lib.fm_host_decompose(Dz, Sz, True)
            continue
        _check(lib, Dz, Sz, True)
        checked += 1
    assert checked >= 4  # the rest are complex at this z grid and are checked to be reported


def test_y_pencil_and_complex_detection(lib):
    s = FMSystem(workload("he_l0_24x24x8", nint=(24, 24, 8)))
    g = s.g[1]
    y = g.ay.pts
    Sy, D2y = g.ay.mat(0), g.ay.mat(2)
    A1 = -D2y + (ph.vhat(s.m, s.Z, 1, y, g.Ry) + 2.9 - 1.7)[:, None] * Sy
    _check(lib, A1, (1 / y ** 2)[:, None] * Sy, False)
    rot = np.array([[0.0, -1.0], [1.0, 0.0]])
    with pytest.raises(lib.FMError):
        lib.fm_host_decompose(rot, np.eye(2))


@pytest.mark.parametrize("basis", [0, 1])
@pytest.mark.parametrize("kind,nint,a,b,dirichlet", [(0, 7, 0.0, 36.0, True), (0, 1, 0.0, 9.0, True),
                                                    (2, 5, -1.0, 1.0, False), (2, 2, -1.0, 1.0, False),
                                                    (2, 1, -1.0, 1.0, False), (1, 6, -1.0, 1.0, False)])
def test_library_axis_equals_oracle_basis(lib, basis, kind, nint, a, b, dirichlet):
    """The library's spline axis (set-up code, host) against the oracle's basis: the same collocation points,
    function count and, rebuilt from the taps, the same value / first / second derivative matrices
    (cubic and quintic Hermite, Dirichlet x / y axes and closed z axes)."""
    from oracle.splines import Axis
    ax = lib.fm_host_axis(kind, nint, a, b, dirichlet, basis)
    ref = Axis(kind, nint, a, b, dirichlet=dirichlet, basis=basis)
    n, r = ax["n"], ax["r"]
    assert n == ref.n and r == (4 if basis == 0 else 6)
    assert np.abs(ax["pts"] - ref.pts).max() < 1e-14 * max(abs(a), abs(b))
    for d, key in ((0, "S"), (1, "D1"), (2, "D2")):
        M = np.zeros((n, n))
        for e in range(n):
            for t in range(r):
                j = ax["base"][e] + t
                if 0 <= j < n:
                    M[e, j] += ax[key][e, t]
                else:
                    assert ax[key][e, t] == 0.0
        R = ref.mat(d)
        assert np.abs(M - R).max() < 1e-12 * np.abs(R).max(), (key, np.abs(M - R).max())
