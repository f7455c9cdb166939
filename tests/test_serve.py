"""The request loop's admission and scheduling, exercised on the host (FM_SERVER_DRY_RUN: every
request "runs" for its simulated time and no CUDA call is made)."""
import time

import pytest

from fm_inputs import request_mix, workload


@pytest.fixture(scope="module")
def serve():
    from paper_2005_05398_gb300 import build
    build.build()
    from paper_2005_05398_gb300 import serve as s
    return s


def _bytes(wl, kind="solve", k=1):
    from paper_2005_05398_gb300._lib import fm_estimate_bytes
    n = wl["J"] + 1
    n *= 2 * (2 * wl["nint"][0]) * (2 * wl["nint"][1]) * (2 * wl["nint"][2] + 2)
    return fm_estimate_bytes(wl, restart_m=40, ncv=20, precision=1) + (2 if kind == "solve" else 1) * n * 8


def test_every_request_completes_within_budget_and_slots(serve):
    mix = request_mix(40, 7, scale="medium")
    sizes = [_bytes(r["wl"], r["kind"]) for r in mix]
    budget = int(2.5 * max(sizes))
    srv = serve.Server(hbm_budget=budget, slots=4, dry_run=True)
    ids = [srv.submit(r["wl"], r["kind"], r["E"], seed=r["seed"], sim_ms=5.0 + (i % 7)) for i, r in enumerate(mix)]
    res = [srv.wait(i) for i in ids]
    st = srv.stats()
    srv.close()
    assert all(r["status"] == 0 for r in res)
    assert st["peak_in_use"] <= budget and st["in_use"] == 0 and st["busy"] == 0 and st["queued"] == 0
    assert 1 <= st["peak_busy"] <= 4
    for r, sz in zip(res, sizes):
        assert r["bytes"] == sz  # admitted with the estimate plus the request's vectors
        assert r["t_start_ms"] >= r["t_submit_ms"] and r["t_end_ms"] - r["t_start_ms"] >= 4.9


def test_running_requests_never_exceed_budget(serve):
    """Reconstruct the in-flight set from the start / end times: at every start the admitted bytes
    of the requests running then fit the budget."""
    mix = request_mix(30, 11, scale="medium")
    sizes = [_bytes(r["wl"], r["kind"]) for r in mix]
    budget = int(1.6 * max(sizes))
    srv = serve.Server(hbm_budget=budget, slots=8, dry_run=True)
    ids = [srv.submit(r["wl"], r["kind"], r["E"], sim_ms=8.0) for r in mix]
    res = [srv.wait(i) for i in ids]
    srv.close()
    for r in res:
        t = r["t_start_ms"]
        running = sum(q["bytes"] for q in res if q["t_start_ms"] <= t < q["t_end_ms"])
        assert running <= budget


def test_large_request_is_not_starved(serve):
    """A request that needs the whole budget waits while small ones pass it at most 8 times, then
    runs before any later request."""
    small = workload("he_l0_24x24x8", nint=(8, 8, 3))
    big = workload("he_l0_24x24x8", nint=(40, 40, 8))
    sb, bb = _bytes(small), _bytes(big)
    budget = bb + sb // 2  # the big one never fits next to a small one
    srv = serve.Server(hbm_budget=budget, slots=4, dry_run=True)
    first = [srv.submit(small, "solve", -2.5, sim_ms=30.0) for _ in range(2)]
    time.sleep(0.01)
    big_id = srv.submit(big, "solve", -2.5, sim_ms=5.0)
    later = [srv.submit(small, "solve", -2.5, sim_ms=30.0) for _ in range(20)]
    rb = srv.wait(big_id)
    rl = [srv.wait(i) for i in later]
    for i in first:
        srv.wait(i)
    srv.close()
    passed = [r for r in rl if r["t_start_ms"] < rb["t_start_ms"]]
    assert len(passed) <= 8
    assert all(r["t_start_ms"] >= rb["t_end_ms"] - 1e-6 for r in rl if r not in passed)


def test_rejections(serve):
    from paper_2005_05398_gb300._lib import FMError
    wl = workload("he_l0_24x24x8", nint=(8, 8, 3))
    with pytest.raises(FMError):
        serve.Server(hbm_budget=10**9, slots=0, dry_run=True)
    with pytest.raises(FMError):
        serve.Server(hbm_budget=0, slots=2, dry_run=True)
    srv = serve.Server(hbm_budget=_bytes(wl) - 1, slots=2, dry_run=True)
    with pytest.raises(FMError) as e:  # alone larger than the budget
        srv.submit(wl, "solve", -2.5)
    assert e.value.code == -2
    srv.close()
    srv = serve.Server(hbm_budget=10**12, slots=2, dry_run=True)
    with pytest.raises(FMError):
        srv.submit(wl, "eigs", -2.5, k=9)
    with pytest.raises(FMError):
        srv.submit(workload("he_l0_24x24x8", tau=-1), "solve", -2.5)  # J = 0, tau = -1: no M' block
    rid = srv.submit(wl, "solve", -2.5, sim_ms=200.0)
    with pytest.raises(FMError) as e:
        srv.wait(rid, timeout_ms=1.0)
    assert e.value.code == -10
    assert srv.wait(rid)["status"] == 0
    with pytest.raises(FMError):
        srv.wait(rid)  # collected already
    srv.close()


def test_request_mix_is_seeded_and_in_range():
    from fm_inputs import MIX_EIG_SHIFT, MIX_SCALES
    a, b = request_mix(20, 5), request_mix(20, 5)
    assert [r["wl"]["name"] for r in a] == [r["wl"]["name"] for r in b] and [r["E"] for r in a] == [r["E"] for r in b]
    (j_lo, j_hi), (r_lo, r_hi), (z_lo, z_hi) = MIX_SCALES["full"]
    for i, r in enumerate(a):
        wl = r["wl"]
        assert j_lo <= wl["J"] <= j_hi and wl["tau"] == 1
        assert r_lo <= wl["nint"][0] <= r_hi and r_lo <= wl["nint"][1] <= r_hi and z_lo <= wl["nint"][2] <= z_hi
        assert r["kind"] == ("solve" if i % 2 == 0 else "eigs")
        if r["kind"] == "solve":
            assert -3.0 <= r["E"] <= -0.2
        else:
            lo, hi = MIX_EIG_SHIFT[wl["system"]]
            assert lo <= r["E"] <= hi


def test_memory_estimate_counts_each_precision_mode(serve):
    """fm_estimate_bytes (host only) sizes what fm_create allocates, so admission can trust it: the float32
    Krylov workspace of MIXED precision and the double-float tables and basis of its mixed_scheme 2 each add
    memory, and the vectors alone set a floor (N x 8 bytes x (2 m + ncv) for the float64 bases)."""
    from paper_2005_05398_gb300._lib import fm_estimate_bytes
    wl = workload("he_l0_24x24x8")
    n = 2 * 48 * 48 * 18  # two components, 48 x 48 x 18 functions each
    fp32 = fm_estimate_bytes(wl, restart_m=40, ncv=20, precision=1)
    mixed = fm_estimate_bytes(wl, restart_m=40, ncv=20, precision=2, mixed_scheme=0)
    mixed_dd = fm_estimate_bytes(wl, restart_m=40, ncv=20, precision=2, mixed_scheme=2)
    assert fp32 >= n * 8 * (2 * 40 + 20)
    assert mixed > fp32 + n * 4 * (2 * 40)          # float32 basis and directions
    assert mixed_dd > mixed + n * 8 * (2 * 40 + 1)   # double-float basis and directions on top
