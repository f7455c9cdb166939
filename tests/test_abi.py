"""The C-ABI library loads (no GPU needed) and exports every entry point of include/fm.h;
the binding's struct layouts match the header's field lists."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "fm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fm_[A-Za-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2005_05398_gb300 import build
    return build.build()


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (fm_[A-Za-z_0-9]+)", out))
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing
    assert len(declared_functions()) >= 13
    assert set(declared_functions()) == exported, exported ^ set(declared_functions())


def test_library_loads_without_gpu_and_binds(libpath):
    import ctypes
    from paper_2005_05398_gb300 import _lib
    L = _lib.lib()
    for name in declared_functions():
        assert hasattr(L, name)
    assert L.fm_strerror(0).decode() == "ok"
    assert "complex" in L.fm_strerror(-6).decode()
    o = _lib.fm_opts()
    L.fm_default_opts(ctypes.byref(o))
    assert o.tol == 1e-12 and o.restart_m == 64 and o.ncv == 20


def test_struct_fields_match_header():
    from paper_2005_05398_gb300 import _lib
    src = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "fm.h")).read(), flags=re.S)
    for cls, tag in ((_lib.fm_system, "fm_system"), (_lib.fm_grid, "fm_grid"), (_lib.fm_splitting, "fm_splitting"),
                     (_lib.fm_opts, "fm_opts"), (_lib.fm_info, "fm_info"), (_lib.fm_request, "fm_request"),
                     (_lib.fm_result, "fm_result")):
        body = re.search(r"typedef struct \{([^{}]*)\}\s*" + tag + ";", src).group(1)
        body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
        names = re.findall(r"([A-Za-z_][A-Za-z_0-9]*)\s*(?:\[\d+\])?\s*[,;]", body)
        assert [f for f, _ in cls._fields_] == names, (tag, names)


def test_create_rejects_bad_arguments_without_touching_gpu():
    """Argument validation happens before any CUDA call (n_M = 0 for J = 0, tau = -1)."""
    import ctypes
    from paper_2005_05398_gb300 import _lib
    from fm_inputs import workload
    L = _lib.lib()
    wl = workload("he_l0_24x24x8", tau=-1)
    s, grids, ng, sp = _lib.make_structs(wl)
    h = ctypes.c_void_p()
    assert L.fm_create(ctypes.byref(s), grids, ng, ctypes.byref(sp), None, ctypes.byref(h)) == -1
    assert not h.value
