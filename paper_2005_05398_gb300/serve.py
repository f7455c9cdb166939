"""ctypes binding of libfm's request loop (fm_server_* in include/fm.h).

Argument marshalling only: admission, scheduling, the solves and the timing all run inside
libfm.  A request is a workload dict (fm_inputs) plus what to compute.
"""
from __future__ import annotations

import ctypes
from ctypes import c_int, c_int64, c_void_p

import numpy as np

from ._lib import (FM_REQ_EIGS, FM_REQ_SOLVE, FM_SERVER_DRY_RUN, FMError, _check, fm_request, fm_result, lib,
                   make_structs)

KINDS = {"solve": FM_REQ_SOLVE, "eigs": FM_REQ_EIGS}


def make_request(wl, kind, E, k=1, seed=0, precision=1, sim_ms=0.0, out=None):
    """An fm_request from a workload dict (one grid for every solved component)."""
    s, grids, ng, sp = make_structs(wl)
    r = fm_request()
    r.sys = s
    r.grid = grids[0]
    r.split = sp
    r.kind = KINDS[kind]
    r.E = float(E)
    r.k = int(k)
    r.seed = int(seed)
    r.precision = int(precision)
    r.sim_ms = float(sim_ms)
    r.out_host = c_void_p(out.ctypes.data) if out is not None else None
    return r


class Server:
    """One fm_server: `slots` worker threads admitting requests by device-memory budget."""

    def __init__(self, device=0, hbm_budget=0, slots=4, dry_run=False):
        h = c_void_p()
        _check("fm_server_create", lib().fm_server_create(int(device), int(hbm_budget), int(slots),
                                                          FM_SERVER_DRY_RUN if dry_run else 0, ctypes.byref(h)))
        self.h = h
        self._outs = {}

    def submit(self, wl, kind, E, k=1, seed=0, precision=1, sim_ms=0.0, out=None):
        """Enqueue one request; `out` (float64 numpy array of n or k*n values) receives the
        solution or eigenvectors.  Returns the request id."""
        if out is not None and not (out.dtype == np.float64 and out.flags["C_CONTIGUOUS"]):
            raise ValueError("out must be a contiguous float64 array")
        r = make_request(wl, kind, E, k, seed, precision, sim_ms, out)
        rid = c_int64()
        _check("fm_server_submit", lib().fm_server_submit(self.h, ctypes.byref(r), ctypes.byref(rid)))
        if out is not None:
            self._outs[rid.value] = out  # keep the buffer alive until the request is collected
        return rid.value

    def wait(self, rid, timeout_ms=-1.0):
        """Block until request `rid` finished; its fm_result as a dict (collected once)."""
        res = fm_result()
        _check("fm_server_wait", lib().fm_server_wait(self.h, int(rid), float(timeout_ms), ctypes.byref(res)))
        self._outs.pop(rid, None)
        return res.as_dict()

    def stats(self):
        a, b = c_int64(), c_int64()
        c, d, e = c_int(), c_int(), c_int()
        _check("fm_server_stats", lib().fm_server_stats(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                                        ctypes.byref(d), ctypes.byref(e)))
        return {"in_use": a.value, "peak_in_use": b.value, "busy": c.value, "peak_busy": d.value,
                "queued": e.value}

    def close(self):
        if self.h:
            lib().fm_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


__all__ = ["Server", "make_request", "FMError"]
