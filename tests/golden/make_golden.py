"""Writes the stored oracle values under tests/golden/ (calls only oracle/).

    python tests/golden/make_golden.py he2p      # He J=1 2^1P / 3^1P sequence
    python tests/golden/make_golden.py cfg1      # He L=0, 24x24x8 intervals: lowest level near -2.95
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from fm_inputs import workload  # noqa: E402
from oracle import solvers  # noqa: E402
from oracle.system import FMSystem  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def he2p():
    runs = []
    for n1, n3 in (((12, 12, 4), (5, 4, 4)), ((16, 16, 4), (6, 5, 5)), ((20, 20, 5), (7, 6, 6))):
        wl = workload("he_l0_24x24x8", J=1, nint=n1, R=(36.0, 36.0))
        wl["grids"] = {3: {"nint": n3, "R": (9.0, 6.0)}}
        t = time.time()
        s = FMSystem(wl)
        E, _ = solvers.eigs_near(s.H(), s.S(), -2.10, 3)
        runs.append({"n1": list(n1), "n3": list(n3), "R1": [36.0, 36.0], "R3": [9.0, 6.0], "N": int(s.N),
                     "E": sorted(float(e) for e in E.real), "seconds": round(time.time() - t, 1)})
        print(runs[-1], flush=True)
    json.dump({"_source": "oracle/ (tests/golden/make_golden.py he2p): He J=1 tau=1 p=1, Merkuriev split, "
               "lowest levels near -2.10", "runs": runs}, open(os.path.join(HERE, "oracle_he_2P.json"), "w"), indent=1)


def cfg1():
    wl = workload("he_l0_24x24x8")
    t = time.time()
    s = FMSystem(wl)
    H, S = s.H(), s.S()
    ta = time.time() - t
    E, v = solvers.eigs_near(H, S, wl["shift"], 4)
    res = [float(solvers.residual(H, S, e.real, v[:, i].real)) for i, e in enumerate(E)]
    out = {"_source": "oracle/ (tests/golden/make_golden.py cfg1): He L=0, 24x24x8 intervals, R=40, Merkuriev split; "
           "eigenvalues of H c = E S c nearest the shift by sparse-LU shift-invert Arnoldi",
           "workload": wl, "N": int(s.N), "E": [float(e) for e in E.real], "residual": res,
           "seconds": round(time.time() - t, 1), "assembly_seconds": round(ta, 1)}
    print(out)
    json.dump(out, open(os.path.join(HERE, "oracle_he_l0_24x24x8.json"), "w"), indent=1)


if __name__ == "__main__":
    for name in sys.argv[1:] or ["he2p", "cfg1"]:
        globals()[name]()
