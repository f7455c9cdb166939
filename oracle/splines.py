"""Hermite splines (cubic and quintic), node maps and Gauss-point collocation (oracle).

ORACLE -- test infrastructure only (see ``oracle/__init__``).

Section 3.1: each partial component is expanded in products of local basis
functions on [0, R_x] x [0, R_y] x [-1, 1]; the x and y bases satisfy zero
Dirichlet conditions at both ends.  Section 4: spline nodes come from mapping
an equidistant grid (Eq. map-pow for x, y; the sin map for z), and collocation
is at Gaussian points.

Two bases.  Cubic Hermite splines (two functions per node: value and slope,
r = 4) with two Gauss-Legendre points per interval.  The x, y bases drop the
value functions at both end nodes (2N functions on N intervals, 2N collocation
points).  The z basis keeps all 2N+2 functions (no condition at z = -1, +1);
the system is squared by taking three Gauss-Legendre points in the first and
the last z interval and two in every other one (a reading: the paper does not
state how its z system is squared).  All z collocation points are interior, so
no collocation point is a collinear configuration, where the coupling term of
Eq. FM-pre is 0/0.

Quintic Hermite splines S_5^3 (Section 4: degree 5, two continuous
derivatives, three functions per node -- value, first and second derivative --
so r = 6), three Gauss-Legendre points per interval.  The x, y bases drop the
value functions at both ends (3N+1 functions: the counts of the paper's tables,
e.g. 22 = 3*7 + 1); the z basis keeps all 3N+3.  Reading: the paper does not say
how these systems are squared; here the first x / y interval takes four Gauss
points (3N+1), and the first, the last and the middle (index N // 2) z
intervals take one more each (3N+3; a single interval takes six).  Collocating
at an end node instead would put a row of zeros into the value matrix S (every
basis function vanishes where the Dirichlet value function was dropped), which
the 1D decompositions of the preconditioner cannot invert.
"""
from __future__ import annotations

import numpy as np

MAP_POW, MAP_EQUI, MAP_SIN = 0, 1, 2


# --------------------------------------------------------------------------
# node maps (Section 4)
# --------------------------------------------------------------------------
def nodes_map_pow(R, nint):
    """Eq. map-pow: 4((1 + R/4)^u - 1), u = i/N on an equidistant grid."""
    u = np.arange(nint + 1, dtype=np.float64) / nint
    t = 4.0 * ((1.0 + R / 4.0) ** u - 1.0)
    t[0], t[-1] = 0.0, R
    return t


def nodes_equidistant(a, b, nint):
    t = a + (b - a) * np.arange(nint + 1, dtype=np.float64) / nint
    t[0], t[-1] = a, b
    return t


def nodes_sin(nint):
    """sin(pi z(i)/2) for equidistant z(i) on [-1, 1] (Section 4)."""
    zt = -1.0 + 2.0 * np.arange(nint + 1, dtype=np.float64) / nint
    t = np.sin(np.pi * zt / 2.0)
    t[0], t[-1] = -1.0, 1.0
    return t


def make_nodes(kind, nint, a, b):
    if kind == MAP_POW:
        assert a == 0.0
        return nodes_map_pow(b, nint)
    if kind == MAP_EQUI:
        return nodes_equidistant(a, b, nint)
    if kind == MAP_SIN:
        assert (a, b) == (-1.0, 1.0)
        return nodes_sin(nint)
    raise ValueError(kind)


# --------------------------------------------------------------------------
# Hermite shape functions of one interval
# --------------------------------------------------------------------------
CUBIC, QUINTIC = 0, 1


def hermite_shapes(s, h, deriv, basis=CUBIC):
    """Shape functions on an interval of length h at local coordinate s in [0, 1].

    Cubic (4 columns): value at the left node, slope at the left node, value
    at the right node, slope at the right node.  Quintic (6 columns): value,
    first and second derivative at the left node, then the same at the right
    node.  Each is the polynomial whose (value, derivatives) at the two nodes
    are one unit vector of those conditions (first derivatives with respect to
    the global variable t = t_left + h s, hence the factors h, h^2).
    ``deriv`` is the order of the derivative in t.
    """
    s = np.asarray(s, dtype=np.float64)
    h = np.asarray(h, dtype=np.float64)
    if basis == CUBIC:
        if deriv == 0:
            cols = [(1 + 2 * s) * (1 - s) ** 2, s * (1 - s) ** 2 * h, s * s * (3 - 2 * s), s * s * (s - 1) * h]
        elif deriv == 1:
            cols = [6 * s * (s - 1) / h, (1 - s) * (1 - 3 * s), 6 * s * (1 - s) / h, s * (3 * s - 2)]
        elif deriv == 2:
            cols = [(12 * s - 6) / h ** 2, (6 * s - 4) / h, (6 - 12 * s) / h ** 2, (6 * s - 2) / h]
        else:
            raise ValueError(deriv)
        return np.stack(np.broadcast_arrays(*cols), axis=-1)
    if basis != QUINTIC:
        raise ValueError(basis)
    # polynomials in s as coefficient lists (ascending powers), scaled to the global variable
    polys = [
        np.array([1.0, 0.0, 0.0, -10.0, 15.0, -6.0]),           # value, left
        np.array([0.0, 1.0, 0.0, -6.0, 8.0, -3.0]),             # first derivative, left (x h)
        np.array([0.0, 0.0, 0.5, -1.5, 1.5, -0.5]),             # second derivative, left (x h^2)
        np.array([0.0, 0.0, 0.0, 10.0, -15.0, 6.0]),            # value, right
        np.array([0.0, 0.0, 0.0, -4.0, 7.0, -3.0]),             # first derivative, right (x h)
        np.array([0.0, 0.0, 0.0, 0.5, -1.0, 0.5]),              # second derivative, right (x h^2)
    ]
    hpow = [0, 1, 2, 0, 1, 2]
    cols = []
    for c, e in zip(polys, hpow):
        d = np.polynomial.polynomial.polyder(c, deriv) if deriv else c
        cols.append(np.polynomial.polynomial.polyval(s, d) * h ** (e - deriv))
    return np.stack(np.broadcast_arrays(*cols), axis=-1)


class HermiteBasis:
    """Hermite basis on the nodes ``t`` (optionally Dirichlet at both ends).

    Global (full) function numbering with q functions per node (q = 2 cubic,
    3 quintic): q m + d = the function of node m carrying the d-th derivative.
    With Dirichlet conditions the value functions of the first and last nodes
    are dropped; the remaining functions keep their relative order.
    """

    def __init__(self, t, dirichlet, basis=CUBIC):
        self.t = np.asarray(t, dtype=np.float64)
        self.N = len(self.t) - 1
        self.kind = basis
        self.q = 2 if basis == CUBIC else 3
        self.r = 2 * self.q
        self.dirichlet = bool(dirichlet)
        nfull = self.q * (self.N + 1)
        keep = np.ones(nfull, dtype=bool)
        if dirichlet:
            keep[0] = False
            keep[self.q * self.N] = False
        self.full_to_red = np.full(nfull, -1, dtype=np.int64)
        self.full_to_red[keep] = np.arange(int(keep.sum()))
        self.n = int(keep.sum())

    @property
    def a(self):
        return self.t[0]

    @property
    def b(self):
        return self.t[-1]

    def locate(self, p):
        """Interval index m with t_m <= p <= t_{m+1} (the last interval is closed)."""
        m = np.searchsorted(self.t, p, side="right") - 1
        return np.clip(m, 0, self.N - 1)

    def local(self, p, deriv):
        """For points p: (columns (P,r), values (P,r)); column -1 = dropped function.

        Points outside [t_0, t_N] get all-zero values (the expansion is zero
        outside its box).
        """
        p = np.asarray(p, dtype=np.float64)
        m = self.locate(p)
        h = self.t[m + 1] - self.t[m]
        s = (p - self.t[m]) / h
        vals = hermite_shapes(s, h, deriv, self.kind)
        full = self.q * m[:, None] + np.arange(self.r)[None, :]
        cols = self.full_to_red[full]
        outside = (p < self.a) | (p > self.b)
        vals = np.where(outside[:, None], 0.0, vals)
        vals = np.where(cols < 0, 0.0, vals)
        return cols, vals

    def matrix(self, p, deriv):
        """Dense matrix B[q, f] = (d/dt)^deriv S^f(p_q)."""
        cols, vals = self.local(p, deriv)
        B = np.zeros((len(p), self.n))
        for c in range(self.r):
            ok = cols[:, c] >= 0
            np.add.at(B, (np.nonzero(ok)[0], cols[ok, c]), vals[ok, c])
        return B

    def gauss_points(self, counts):
        """counts[m] Gauss-Legendre points in interval m, ascending."""
        out = []
        for m, q in enumerate(counts):
            g, _ = np.polynomial.legendre.leggauss(int(q))
            tl, tr = self.t[m], self.t[m + 1]
            out.append(0.5 * (tl + tr) + 0.5 * (tr - tl) * g)
        return np.concatenate(out)

    def collocation_points(self, closed):
        """Gauss points, as many as functions.  Cubic: two per interval; with ``closed``
        (all 2N+2 functions kept) the first and last intervals take three (one
        interval alone takes four).  Quintic: three per interval; the first interval
        takes four without ``closed`` (3N+1 functions), and with ``closed`` (3N+3) the
        first, the last and the middle interval N // 2 take one more each (one interval
        alone takes six)."""
        if self.kind == CUBIC:
            counts = np.full(self.N, 2)
            if closed:
                if self.N == 1:
                    counts[0] = 4
                else:
                    counts[0] = counts[-1] = 3
            return self.gauss_points(counts)
        counts = np.full(self.N, 3)
        if not closed:
            counts[0] += 1
        elif self.N == 1:
            counts[0] = 6
        else:
            counts[0] += 1
            counts[-1] += 1
            counts[self.N // 2] += 1
        return self.gauss_points(counts)

    def coefficients_of(self, f, df, d2f=None):
        """Hermite interpolation coefficients of f (value and derivatives at every node)."""
        full = np.empty(self.q * (self.N + 1))
        full[0::self.q] = f(self.t)
        full[1::self.q] = df(self.t)
        if self.q == 3:
            full[2::3] = d2f(self.t)
        keep = self.full_to_red >= 0
        return full[keep]


class Axis:
    """One coordinate axis of a component: basis plus collocation points."""

    def __init__(self, kind, nint, a, b, dirichlet, basis=CUBIC):
        self.nodes = make_nodes(kind, nint, a, b)
        self.basis = HermiteBasis(self.nodes, dirichlet, basis)
        self.pts = self.basis.collocation_points(closed=not dirichlet)
        self.n = self.basis.n
        assert len(self.pts) == self.n, (len(self.pts), self.n)

    def mat(self, deriv):
        return self.basis.matrix(self.pts, deriv)
