"""Seeded synthetic inputs shared by the tests, the bench and the oracle.

This module holds data only: the named workloads (particle masses and charges,
total momentum, grid sizes, splitting parameters, shifts) and seeded random
vectors.  It contains none of the method's arithmetic, so both the CUDA path
and the CPU oracle may take their inputs from it without sharing any
computation.

Workloads follow the systems of Section 4 (atomic He with an infinitely heavy
core, ``10^15`` a.u. in practice) and the He-like / Ps- / H- systems of the
benchmark configurations.  Energies are in the units of the reduced-coordinate
equations (Hartree for electron-mass units); box sizes are in reduced
coordinates.
"""
from __future__ import annotations

import copy

import numpy as np

INF_MASS = 1.0e15  # "infinite" core mass, Section 4

SYSTEMS = {
    # masses (m1, m2, m3), charges (Z1, Z2, Z3); particles 1, 2 are identical
    "He": {"mass": (1.0, 1.0, INF_MASS), "charge": (-1.0, -1.0, 2.0)},
    "Hminus": {"mass": (1.0, 1.0, INF_MASS), "charge": (-1.0, -1.0, 1.0)},
    "Psminus": {"mass": (1.0, 1.0, 1.0), "charge": (-1.0, -1.0, 1.0)},
}

# splitting modes
MERKURIEV, NO_SPLIT, SCHRODINGER = 0, 1, 2
# node maps
MAP_POW, MAP_EQUI, MAP_SIN = 0, 1, 2


def make_workload(system="He", J=0, tau=1, p=1, identical_pair=12,
                  nint=(24, 24, 8), R=(40.0, 40.0), maps=(MAP_POW, MAP_POW, MAP_SIN),
                  mode=MERKURIEV, nu=2.01, x0=1.0, y0=float("inf"), vs_cut=1e-20,
                  shift=-2.95, k=1, name=None, basis=0):
    """Return a plain dict describing one Faddeev-Merkuriev problem."""
    sysd = SYSTEMS[system]
    return {
        "name": name or f"{system}_J{J}_{nint[0]}x{nint[1]}x{nint[2]}",
        "system": system,
        "mass": tuple(float(m) for m in sysd["mass"]),
        "charge": tuple(float(z) for z in sysd["charge"]),
        "J": int(J), "tau": int(tau), "p": int(p), "identical_pair": int(identical_pair),
        "nint": tuple(int(n) for n in nint), "R": tuple(float(r) for r in R),
        "maps": tuple(int(m) for m in maps),
        "mode": int(mode), "nu": float(nu), "x0": float(x0), "y0": float(y0),
        "vs_cut": float(vs_cut),
        "shift": float(shift), "k": int(k),
        "basis": int(basis),  # 0 = cubic Hermite, 1 = quintic Hermite (S_5^3, Section 4)
    }


# The named workloads.  Interval counts are the spline intervals per axis;
# cubic Hermite splines give 2*n dofs in x, y (Dirichlet at both ends) and
# 2*n + 2 in z.
WORKLOADS = {
    # He-like, L=0, 24x24 intervals in x, y to 40, 8 in z: small case
    "he_l0_24x24x8": make_workload("He", 0, nint=(24, 24, 8), R=(40.0, 40.0), shift=-2.95, k=1,
                                   name="he_l0_24x24x8"),
    # He-like, L=0, 96x96x24 intervals: the large single-GPU case
    "he_l0_96x96x24": make_workload("He", 0, nint=(96, 96, 24), R=(40.0, 40.0), shift=-2.95, k=1,
                                    name="he_l0_96x96x24"),
}
# He, J = 10 (n_M = 11), the shape of the paper's high-momentum table (Section 4): equidistant z,
# component 1 on a 280 x 280 box with 58 x 58 x 6 intervals, component 3 on a 2 x 2 box with 4 x 4 x 6;
# the level nearest -2.0045 (the paper's lowest is near -2.0041)
WORKLOADS["he_l10_58x58x6"] = make_workload("He", 10, nint=(58, 58, 6), R=(280.0, 280.0),
                                            maps=(MAP_POW, MAP_POW, MAP_EQUI), shift=-2.0045, k=1,
                                            name="he_l10_58x58x6")
WORKLOADS["he_l10_58x58x6"]["grids"] = {1: {"nint": (58, 58, 6), "R": (280.0, 280.0)},
                                        3: {"nint": (4, 4, 6), "R": (2.0, 2.0)}}
# He J = 1 (2^1P, 3^1P), the paper's Table pardiso: quintic Hermite basis, boxes (1: 36, 36; 3: 9, 6) and
# its five basis rows (n_x, n_y, n_z) = (3N+1, 3N+1, 3N_z+3) per component, written here as interval counts
PARDISO_ROWS = [((7, 7, 2), (6, 6, 3)), ((10, 10, 2), (7, 7, 4)), ((13, 13, 3), (8, 8, 5)),
                ((16, 16, 3), (9, 9, 6)), ((19, 19, 3), (9, 9, 6))]
for _r, (_n1, _n3) in enumerate(PARDISO_ROWS, 1):
    WORKLOADS[f"he_j1_pardiso_row{_r}"] = make_workload("He", 1, nint=_n1, R=(36.0, 36.0), shift=-2.10, k=2,
                                                       name=f"he_j1_pardiso_row{_r}", basis=1)
    WORKLOADS[f"he_j1_pardiso_row{_r}"]["grids"] = {1: {"nint": _n1, "R": (36.0, 36.0)},
                                                     3: {"nint": _n3, "R": (9.0, 6.0)}}
# He 3^1D (J = 2, tau = 1, p = 1), the paper's convergence study (Fig. He-conv): quintic Hermite basis on the
# domains (1: 45, 45; 3: 11, 6); its final basis (1: 238, 238, 24; 3: 52, 40, 27), 4 246 848 unknowns, and a
# sequence that refines the radial bases of component 1 toward it (interval counts; n = 3N+1, n_z = 3N_z+3)
CONV3D_FINAL = ((79, 79, 7), (17, 13, 8))


def he_3d_workload(n1=CONV3D_FINAL[0], n3=CONV3D_FINAL[1]):
    w = make_workload("He", 2, nint=n1, R=(45.0, 45.0), shift=-2.0557, k=1,
                      name=f"he_j2_3d_{n1[0]}x{n1[1]}x{n1[2]}", basis=1)
    w["grids"] = {1: {"nint": tuple(n1), "R": (45.0, 45.0)}, 3: {"nint": tuple(n3), "R": (11.0, 6.0)}}
    return w


WORKLOADS["he_j2_3d_final"] = he_3d_workload()
CONV3D_SEQUENCE = [((n, n, 7), CONV3D_FINAL[1]) for n in (31, 43, 55, 67, 79)]
for _J in (1, 2, 3):
    WORKLOADS[f"psm_l{_J}_64x64x16"] = make_workload(
        "Psminus", _J, nint=(64, 64, 16), R=(80.0, 80.0), shift=-0.27, k=4,
        name=f"psm_l{_J}_64x64x16")


def workload(name, **overrides):
    """A copy of a named workload with fields overridden."""
    w = copy.deepcopy(WORKLOADS[name])
    w.update(overrides)
    return w


def rand_vec(n, seed):
    """Seeded N(0,1) vector of length n (float64)."""
    return np.random.default_rng(seed).standard_normal(int(n))


SEED_BASE = 20050539


# Independent-request mixes (batched and served workloads): per request a system drawn from
# H-, He-like and Ps-, total momentum J (tau = +1), interval counts per radial axis and in z,
# an energy, and what to compute (half linear solves with a N(0,1) right-hand side, half
# nearest-eigenvalue solves).  Solves take E uniform in [-3, -0.2]; an eigen-request draws its
# shift from the part of that range next to the system's bound and low box states, so that
# shift-invert converges in a bounded number of Arnoldi steps.
MIX_BOX = {"He": 40.0, "Hminus": 40.0, "Psminus": 80.0}
MIX_EIG_SHIFT = {"He": (-3.0, -2.0), "Hminus": (-0.6, -0.45), "Psminus": (-0.3, -0.22)}
MIX_SCALES = {
    # name: (J range, radial interval range, z interval range)
    "full": ((0, 4), (32, 128), (8, 24)),
    "medium": ((0, 3), (16, 64), (4, 12)),
    "small": ((0, 2), (8, 16), (3, 5)),
}


def request_mix(count, seed, scale="full", systems=("Hminus", "He", "Psminus")):
    """Seeded list of request dicts {'wl', 'kind', 'E', 'k', 'seed'} (kind 'solve' or 'eigs')."""
    rng = np.random.default_rng(seed)
    (j_lo, j_hi), (r_lo, r_hi), (z_lo, z_hi) = MIX_SCALES[scale]
    out = []
    for i in range(int(count)):
        system = systems[int(rng.integers(len(systems)))]
        J = int(rng.integers(j_lo, j_hi + 1))
        nx, ny = (int(v) for v in rng.integers(r_lo, r_hi + 1, size=2))
        nz = int(rng.integers(z_lo, z_hi + 1))
        kind = "solve" if i % 2 == 0 else "eigs"
        if kind == "solve":
            E = float(rng.uniform(-3.0, -0.2))
        else:
            E = float(rng.uniform(*MIX_EIG_SHIFT[system]))
        Rb = MIX_BOX[system]
        wl = make_workload(system, J, nint=(nx, ny, nz), R=(Rb, Rb), shift=E, k=1,
                           name=f"{system}_J{J}_{nx}x{ny}x{nz}")
        out.append({"wl": wl, "kind": kind, "E": E, "k": 1, "seed": int(seed) * 1000 + i})
    return out
