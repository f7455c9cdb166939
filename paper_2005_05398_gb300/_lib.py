"""ctypes binding of libfm (include/fm.h): argument marshalling only.

Every computation runs inside libfm's CUDA kernels; PyTorch provides device
memory and streams.  The functions keep the C names (fm_create, fm_apply,
fm_precond_apply, fm_solve, fm_eigs, ...).  Loading fails loudly when the
library has not been built: there is no fallback.
"""
from __future__ import annotations

import ctypes
import math
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfm.so")

c_double, c_int, c_int64, c_void_p = ctypes.c_double, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p


class fm_system(ctypes.Structure):
    _fields_ = [("mass", c_double * 3), ("charge", c_double * 3), ("J", c_int), ("tau", c_int),
                ("exch_p", c_int), ("identical_pair", c_int)]


class fm_grid(ctypes.Structure):
    _fields_ = [("nint_x", c_int), ("nint_y", c_int), ("nint_z", c_int), ("Rx", c_double), ("Ry", c_double),
                ("xmap", c_int), ("ymap", c_int), ("zmap", c_int), ("basis", c_int)]


class fm_splitting(ctypes.Structure):
    _fields_ = [("mode", c_int), ("nu", c_double), ("x0", c_double), ("y0", c_double), ("vs_cut", c_double)]


class fm_opts(ctypes.Structure):
    _fields_ = [("tol", c_double), ("restart_m", c_int), ("max_iters", c_int), ("precision", c_int),
                ("ncv", c_int), ("max_restarts", c_int), ("eig_tol", c_double), ("z_eigs", c_int),
                ("y_solver", c_int), ("tune", c_int), ("mma", c_int), ("start_filter", c_int),
                ("refine", c_int), ("inner_tol32", c_double), ("tc_chain", c_int), ("gram_schmidt", c_int),
                ("mixed_scheme", c_int), ("z_tile", c_int), ("device", c_int), ("stream", c_void_p)]


class fm_info(ctypes.Structure):
    _fields_ = [("iters", c_int), ("restarts", c_int), ("op_applies", c_int), ("converged", c_int),
                ("resid", c_double), ("ms", c_double), ("accept", c_int), ("refine_steps", c_int),
                ("resid_S", c_double), ("norm_H", c_double), ("norm_S", c_double), ("rq_dev", c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class fm_request(ctypes.Structure):
    _fields_ = [("sys", fm_system), ("grid", fm_grid), ("split", fm_splitting), ("kind", c_int), ("E", c_double),
                ("k", c_int), ("seed", ctypes.c_uint64), ("precision", c_int), ("sim_ms", c_double),
                ("out_host", c_void_p)]


class fm_result(ctypes.Structure):
    _fields_ = [("status", c_int), ("iters", c_int), ("n", c_int64), ("bytes", c_int64), ("evals", c_double * 8),
                ("resid", c_double), ("out_norm", c_double), ("t_submit_ms", c_double), ("t_start_ms", c_double),
                ("t_end_ms", c_double)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_}
        d["evals"] = list(self.evals)
        return d


FM_OK, FM_ERR_NOT_CONVERGED, FM_ERR_SCRATCH_LIMIT, FM_ERR_TIMEOUT = 0, -4, -9, -10
FM_REQ_SOLVE, FM_REQ_EIGS, FM_SERVER_DRY_RUN = 0, 1, 1
FM_MMA_AUTO, FM_MMA_SIMT, FM_MMA_TF32 = 0, 1, 2
KERNEL_CLASSES = ["apply_xy", "apply_z", "coupling", "zmix", "xmix", "ysolve", "dot", "axpy", "other"]

_LIB = None

SIGNATURES = {
    "fm_default_opts": (None, [ctypes.POINTER(fm_opts)]),
    "fm_create": (c_int, [ctypes.POINTER(fm_system), ctypes.POINTER(fm_grid), c_int, ctypes.POINTER(fm_splitting),
                          ctypes.POINTER(fm_opts), ctypes.POINTER(c_void_p)]),
    "fm_size": (c_int, [c_void_p, ctypes.POINTER(c_int64), ctypes.POINTER(c_int), ctypes.POINTER(c_int)]),
    "fm_estimate_bytes": (c_int, [ctypes.POINTER(fm_system), ctypes.POINTER(fm_grid), c_int,
                                  ctypes.POINTER(fm_splitting), ctypes.POINTER(fm_opts), ctypes.POINTER(c_int64)]),
    "fm_component": (c_int, [c_void_p, c_int, ctypes.POINTER(c_int), ctypes.POINTER(c_int), ctypes.POINTER(c_int64)]),
    "fm_apply": (c_int, [c_void_p, c_double, c_void_p, c_void_p]),
    "fm_apply_S": (c_int, [c_void_p, c_void_p, c_void_p]),
    "fm_apply_noalloc": (c_int, [c_void_p, c_double, c_void_p, c_void_p]),
    "fm_set_shift": (c_int, [c_void_p, c_double]),
    "fm_precond_apply": (c_int, [c_void_p, c_void_p, c_void_p]),
    "fm_solve": (c_int, [c_void_p, c_double, c_void_p, c_void_p, ctypes.POINTER(fm_info)]),
    "fm_eigs": (c_int, [c_void_p, c_double, c_int, c_void_p, ctypes.POINTER(c_double), c_void_p,
                        ctypes.POINTER(fm_info)]),
    "fm_eigs_host": (c_int, [c_void_p, c_double, c_int, c_void_p, ctypes.POINTER(c_double), c_void_p,
                             ctypes.POINTER(fm_info)]),
    "fm_destroy": (None, [c_void_p]),
    "fm_strerror": (ctypes.c_char_p, [c_int]),
    "fm_stats": (c_int, [c_void_p, ctypes.POINTER(c_int64), ctypes.POINTER(c_int64)]),
    "fm_profile": (c_int, [c_void_p, c_int]),
    "fm_host_decompose": (c_int, [c_int, c_void_p, c_void_p, c_int, c_void_p, c_void_p, c_void_p]),
    "fm_host_axis": (c_int, [c_int, c_int, c_double, c_double, c_int, c_int, ctypes.POINTER(c_int),
                             ctypes.POINTER(c_int), c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "fm_profile_read": (c_int, [c_void_p, ctypes.POINTER(c_double), ctypes.POINTER(c_int64), ctypes.POINTER(c_double),
                                ctypes.POINTER(c_double)]),
    "fm_server_create": (c_int, [c_int, c_int64, c_int, c_int, ctypes.POINTER(c_void_p)]),
    "fm_server_submit": (c_int, [c_void_p, ctypes.POINTER(fm_request), ctypes.POINTER(c_int64)]),
    "fm_server_wait": (c_int, [c_void_p, c_int64, c_double, ctypes.POINTER(fm_result)]),
    "fm_server_stats": (c_int, [c_void_p, ctypes.POINTER(c_int64), ctypes.POINTER(c_int64), ctypes.POINTER(c_int),
                                ctypes.POINTER(c_int), ctypes.POINTER(c_int)]),
    "fm_server_destroy": (None, [c_void_p]),
}


class FMError(RuntimeError):
    def __init__(self, fn, code):
        super().__init__(f"{fn} failed: {lib().fm_strerror(code).decode()} ({code})")
        self.code = code


def lib():
    """The loaded libfm (raises when it has not been built)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libfm.so is not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def _check(fn, rc, allow=()):
    if rc != FM_OK and rc not in allow:
        raise FMError(fn, rc)
    return rc


def _ptr(t):
    """Device pointer of a contiguous float64 CUDA tensor."""
    if t is None:
        return None
    import torch
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError("expected a contiguous float64 CUDA tensor")
    return c_void_p(t.data_ptr())


def make_structs(wl):
    """C structs from a workload dict (fm_inputs)."""
    s = fm_system()
    s.mass[:] = list(wl["mass"])
    s.charge[:] = list(wl["charge"])
    s.J, s.tau, s.exch_p, s.identical_pair = wl["J"], wl["tau"], wl["p"], wl["identical_pair"]
    labels = [1] if wl["mode"] == 2 else ([1, 3] if wl["identical_pair"] == 12 else [1, 2, 3])
    per = wl.get("grids") or {}
    gl = []
    for a in (labels if per else labels[:1]):
        nint = per.get(a, {}).get("nint", wl["nint"])
        R = per.get(a, {}).get("R", wl["R"])
        g = fm_grid()
        g.nint_x, g.nint_y, g.nint_z = nint
        g.Rx, g.Ry = R
        g.xmap, g.ymap, g.zmap = wl["maps"]
        g.basis = int(wl.get("basis", 0))
        gl.append(g)
    grids = (fm_grid * len(gl))(*gl)
    sp = fm_splitting()
    sp.mode, sp.nu, sp.x0 = wl["mode"], wl["nu"], wl["x0"]
    sp.y0 = wl["y0"] if math.isfinite(wl["y0"]) else float("inf")
    sp.vs_cut = wl.get("vs_cut", 0.0)
    return s, grids, len(gl), sp


def make_opts(**opt):
    o = fm_opts()
    lib().fm_default_opts(ctypes.byref(o))
    for k, v in opt.items():
        if k == "stream":
            o.stream = c_void_p(v.cuda_stream if hasattr(v, "cuda_stream") else v)
        else:
            setattr(o, k, v)
    return o


def fm_estimate_bytes(wl, **opt):
    """Device bytes fm_create would hold for this workload and options (no GPU work)."""
    s, grids, ng, sp = make_structs(wl)
    o = make_opts(**opt)
    b = c_int64()
    _check("fm_estimate_bytes", lib().fm_estimate_bytes(ctypes.byref(s), grids, ng, ctypes.byref(sp), ctypes.byref(o),
                                                        ctypes.byref(b)))
    return b.value


def fm_host_decompose(A1, A2, descending=False):
    """(W-bar, W, lam) from libfm's host set-up code (numpy arrays; no GPU)."""
    import numpy as np
    A1 = np.ascontiguousarray(A1, dtype=np.float64)
    A2 = np.ascontiguousarray(A2, dtype=np.float64)
    n = A1.shape[0]
    Wb, W, lam = np.empty((n, n)), np.empty((n, n)), np.empty(n)
    p = lambda a: a.ctypes.data_as(c_void_p)
    _check("fm_host_decompose", lib().fm_host_decompose(n, p(A1), p(A2), int(descending), p(Wb), p(W), p(lam)))
    return Wb, W, lam


def fm_host_axis(kind, nint, a, b, dirichlet, basis=0):
    """One spline axis as libfm's set-up builds it (host only): dict of numpy arrays pts, base, S, D1, D2."""
    import numpy as np
    cap = 3 * (int(nint) + 1)
    pts, base = np.empty(cap), np.empty(cap, dtype=np.int32)
    S, D1, D2 = np.empty((cap, 6)), np.empty((cap, 6)), np.empty((cap, 6))
    n, r = c_int(), c_int()
    p = lambda x: x.ctypes.data_as(c_void_p)
    _check("fm_host_axis", lib().fm_host_axis(int(kind), int(nint), float(a), float(b), int(bool(dirichlet)), int(basis),
                                              ctypes.byref(n), ctypes.byref(r), p(pts), p(base), p(S), p(D1), p(D2)))
    n, r = n.value, r.value
    S, D1, D2 = (np.ascontiguousarray(X.reshape(-1)[: n * r].reshape(n, r)) for X in (S, D1, D2))
    return {"n": n, "r": r, "pts": pts[:n].copy(), "base": base[:n].copy(), "S": S, "D1": D1, "D2": D2}


class Context:
    """One libfm context (fm_create ... fm_destroy)."""

    def __init__(self, wl, **opt):
        L = lib()
        self.wl = dict(wl)
        o = make_opts(**opt)
        self.opts = o
        s, grids, ng, sp = make_structs(wl)
        h = c_void_p()
        _check("fm_create", L.fm_create(ctypes.byref(s), grids, ng, ctypes.byref(sp), ctypes.byref(o), ctypes.byref(h)))
        self.h = h
        n, nc, nM = c_int64(), c_int(), c_int()
        _check("fm_size", L.fm_size(h, ctypes.byref(n), ctypes.byref(nc), ctypes.byref(nM)))
        self.n, self.ncomp, self.nM = n.value, nc.value, nM.value
        self.components = []
        for i in range(self.ncomp):
            lab, dims, off = c_int(), (c_int * 3)(), c_int64()
            _check("fm_component", L.fm_component(h, i, ctypes.byref(lab), dims, ctypes.byref(off)))
            self.components.append({"label": lab.value, "nz": dims[0], "nx": dims[1], "ny": dims[2], "off": off.value})

    def fm_apply(self, E, x, y):
        _check("fm_apply", lib().fm_apply(self.h, float(E), _ptr(x), _ptr(y)))

    def fm_apply_noalloc(self, E, x, y):
        """(H - E S) x with the library's fixed scratch: allocates no device memory (see include/fm.h)."""
        _check("fm_apply_noalloc", lib().fm_apply_noalloc(self.h, float(E), _ptr(x), _ptr(y)))

    def fm_apply_S(self, x, y):
        _check("fm_apply_S", lib().fm_apply_S(self.h, _ptr(x), _ptr(y)))

    def fm_set_shift(self, E):
        _check("fm_set_shift", lib().fm_set_shift(self.h, float(E)))

    def fm_precond_apply(self, x, y):
        _check("fm_precond_apply", lib().fm_precond_apply(self.h, _ptr(x), _ptr(y)))

    def fm_solve(self, E, rhs, x, allow_not_converged=False):
        info = fm_info()
        rc = lib().fm_solve(self.h, float(E), _ptr(rhs), _ptr(x), ctypes.byref(info))
        _check("fm_solve", rc, (FM_ERR_NOT_CONVERGED,) if allow_not_converged else ())
        return info.as_dict()

    def fm_eigs(self, shift, k, v0=None, evecs=None, allow_not_converged=False):
        ev = (c_double * k)()
        info = fm_info()
        rc = lib().fm_eigs(self.h, float(shift), int(k), _ptr(v0), ev, _ptr(evecs), ctypes.byref(info))
        _check("fm_eigs", rc, (FM_ERR_NOT_CONVERGED,) if allow_not_converged else ())
        return list(ev), info.as_dict()

    def fm_eigs_host(self, shift, k, v0_host=None, evecs_host=None, allow_not_converged=False):
        """Host buffers: numpy float64 arrays (v0_host length n, evecs_host k*n) or pinned torch tensors."""
        ev = (c_double * k)()
        info = fm_info()

        def hp(a):
            if a is None:
                return None
            if hasattr(a, "data_ptr"):
                return c_void_p(a.data_ptr())
            return a.ctypes.data_as(c_void_p)
        _check("fm_eigs_host", lib().fm_eigs_host(self.h, float(shift), int(k), hp(v0_host), ev, hp(evecs_host),
                                                  ctypes.byref(info)),
               (FM_ERR_NOT_CONVERGED,) if allow_not_converged else ())
        return list(ev), info.as_dict()

    def fm_stats(self):
        a, b = c_int64(), c_int64()
        _check("fm_stats", lib().fm_stats(self.h, ctypes.byref(a), ctypes.byref(b)))
        return {"launches": a.value, "device_bytes": b.value}

    def fm_profile(self, enable):
        _check("fm_profile", lib().fm_profile(self.h, int(bool(enable))))

    def fm_profile_read(self):
        K = len(KERNEL_CLASSES)
        ms, n, fl, by = (c_double * K)(), (c_int64 * K)(), (c_double * K)(), (c_double * K)()
        _check("fm_profile_read", lib().fm_profile_read(self.h, ms, n, fl, by))
        return {k: {"ms": ms[i], "launches": n[i], "flops": fl[i], "bytes": by[i]} for i, k in enumerate(KERNEL_CLASSES)}

    def fm_destroy(self):
        if getattr(self, "h", None):
            lib().fm_destroy(self.h)
            self.h = None

    close = fm_destroy

    def __del__(self):
        try:
            self.fm_destroy()
        except Exception:
            pass
