"""GPU: requests served concurrently (several slots, overlapping on the device) give the same
results as each request run alone: eigenvalues to 1e-9 relative, solutions to 1e-8 relative."""
import numpy as np
import pytest

from fm_inputs import request_mix

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def serve():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_05398_gb300 import build
    build.build()
    from paper_2005_05398_gb300 import serve as s
    return s


def _n(wl):
    return (wl["J"] + 1) * 2 * (2 * wl["nint"][0]) * (2 * wl["nint"][1]) * (2 * wl["nint"][2] + 2)


def _run(serve, mix, slots):
    srv = serve.Server(slots=slots)
    outs, ids = [], []
    for r in mix:
        out = np.zeros(_n(r["wl"]) * (1 if r["kind"] == "solve" else r["k"]))
        outs.append(out)
        ids.append(srv.submit(r["wl"], r["kind"], r["E"], k=r["k"], seed=r["seed"], precision=r.get("precision", 1),
                              out=out))
    res = [srv.wait(i) for i in ids]
    st = srv.stats()
    srv.close()
    return res, outs, st


@pytest.mark.parametrize("precision", [1, 2])
def test_results_alone_equal_results_in_mix(serve, precision):
    mix = request_mix(10, 3 + precision, scale="small")
    for r in mix:
        r["precision"] = precision
    res_mix, out_mix, st = _run(serve, mix, slots=5)
    assert st["peak_busy"] >= 2  # requests really overlapped
    for i, r in enumerate(mix):
        ra, oa, _ = _run(serve, [r], slots=1)
        a, m = ra[0], res_mix[i]
        assert a["status"] in (0, -4) and a["status"] == m["status"], (r["wl"]["name"], a["status"], m["status"])
        assert a["n"] == m["n"] == _n(r["wl"])
        if r["kind"] == "eigs":
            assert abs(a["evals"][0] - m["evals"][0]) <= 1e-9 * abs(a["evals"][0])
            va, vm = oa[0], out_mix[i]
            assert np.linalg.norm(va - vm) <= 1e-8 * np.linalg.norm(va)
        else:
            assert a["resid"] <= 1e-12 or a["status"] == -4
            assert np.linalg.norm(oa[0] - out_mix[i]) <= 1e-8 * np.linalg.norm(oa[0])


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_estimate_bounds_the_device_bytes_a_context_holds(serve, precision):
    """Admission trusts fm_estimate_bytes: it must not undercount what fm_create allocates."""
    import paper_2005_05398_gb300 as pkg
    from paper_2005_05398_gb300._lib import fm_estimate_bytes
    for r in request_mix(6, 11, scale="small"):
        wl = r["wl"]
        est = fm_estimate_bytes(wl, restart_m=40, ncv=20, precision=precision)
        ctx = pkg.Context(wl, restart_m=40, ncv=20, precision=precision)
        ctx.fm_set_shift(r["E"])
        held = ctx.fm_stats()["device_bytes"]
        ctx.close()
        assert held <= est <= 1.5 * held + 2**22, (wl["name"], held, est)
