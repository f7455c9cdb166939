"""GPU at the full sizes of the measured workloads (He L=0 on 96x96x24 intervals, 3.69 M unknowns, with the
benchmark's options; Ps- L=3 on 64x64x16 intervals, 4.46 M unknowns; He J=10 with n_M = 11, 2.08 M unknowns),
checked on rows of H and S the oracle assembles one by one: the operator apply, and the residual of the
eigenpairs fm_eigs returns (normwise over the sampled rows)."""
import numpy as np
import pytest

from fm_inputs import workload, rand_vec

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2005_05398_gb300 as p
    from paper_2005_05398_gb300 import build
    build.build()
    p.lib()
    return p


def _rows(s, seed, count=2000):
    rows = np.sort(np.random.default_rng(seed).choice(s.N, count, replace=False))
    return rows, s.H(rows).tocsr(), s.S(rows).tocsr()


@pytest.mark.parametrize("name", ["psm_l3_64x64x16", "he_l10_58x58x6"])
def test_fullsize_apply_on_sampled_rows(pkg, name):
    from oracle.system import FMSystem
    wl = workload(name)
    s = FMSystem(wl)
    ctx = pkg.Context(wl, restart_m=8, ncv=4)
    assert ctx.n == s.N
    rows, Hr, Sr = _rows(s, 12)
    x = rand_vec(s.N, 13)
    E = wl["shift"]
    y = torch.empty(s.N, dtype=torch.float64, device="cuda")
    ctx.fm_apply(E, torch.tensor(x, device="cuda"), y)
    got = y.cpu().numpy()[rows]
    ref = Hr @ x - E * (Sr @ x)
    scale = np.abs(Hr).max(axis=1).toarray().ravel() * np.abs(x).max() + 1e-300
    bound = 1e-13 * np.maximum(1.0, np.sqrt(np.diff(Hr.indptr) / 256.0))  # rounding grows with the row length
    assert np.max(np.abs(got - ref) / scale / bound) < 1.0


@pytest.mark.parametrize("name,precision", [("psm_l3_64x64x16", 1), ("he_l10_58x58x6", 2)])
def test_fullsize_eigenpairs_satisfy_sampled_rows(pkg, name, precision):
    """(H - E S) c = 0 on the oracle's rows for every returned pair, normwise relative to |H||c| + |E||S||c|
    (the Ritz residual 1e-9 and the relaxed inner solves leave about 1e-9 of that scale)."""
    from oracle.system import FMSystem
    wl = workload(name)
    s = FMSystem(wl)
    k = wl["k"]
    ctx = pkg.Context(wl, restart_m=40, precision=precision)
    evecs = torch.empty(k * s.N, dtype=torch.float64, device="cuda")
    ev, info = ctx.fm_eigs(wl["shift"], k, evecs=evecs)
    assert info["converged"] == 1
    rows, Hr, Sr = _rows(s, 14)
    C = evecs.cpu().numpy().reshape(k, s.N)
    aH, aS = abs(Hr), abs(Sr)
    for i in range(k):
        c = C[i]
        r = Hr @ c - ev[i] * (Sr @ c)
        scale = aH @ np.abs(c) + abs(ev[i]) * (aS @ np.abs(c))
        assert np.max(np.abs(r)) < 1e-7 * np.max(scale), (name, i, ev[i])


@pytest.fixture(scope="module")
def he96():
    """The benchmark's workload: oracle rows and the float64 eigenvalue of the same start vector."""
    from oracle.system import FMSystem
    wl = workload("he_l0_96x96x24")
    s = FMSystem(wl)
    rows, Hr, Sr = _rows(s, 14)
    return wl, s, rows, Hr, Sr


@pytest.mark.parametrize("precision", [1, 2])
def test_fullsize_benchmark_eigenpair(pkg, he96, precision):
    """He L=0, 96x96x24 intervals, the benchmark's options (restart 40, 8 start-vector filter passes,
    k = 1, tensor-core float32 preconditioner; and MIXED): the pair is accepted by the Ritz-residual rule,
    its float64 certificate (backward error) is within 1e-9, it satisfies the oracle's sampled rows, and
    its eigenvalue equals the float64-preconditioner mode's to 1e-10."""
    from fm_inputs import SEED_BASE
    wl, s, rows, Hr, Sr = he96
    v0 = torch.tensor(rand_vec(s.N, SEED_BASE), dtype=torch.float64, device="cuda")
    ctx = pkg.Context(wl, restart_m=40, precision=precision, start_filter=8)
    evecs = torch.empty(s.N, dtype=torch.float64, device="cuda")
    ev, info = ctx.fm_eigs(wl["shift"], 1, v0=v0, evecs=evecs)
    ctx.close()
    assert info["converged"] == 1 and info["accept"] == 1 and info["resid"] <= 1e-9, info
    c = evecs.cpu().numpy()
    r = Hr @ c - ev[0] * (Sr @ c)
    scale = abs(Hr) @ np.abs(c) + abs(ev[0]) * (abs(Sr) @ np.abs(c))
    assert np.linalg.norm(r) < 1e-9 * np.linalg.norm(scale), (np.linalg.norm(r), np.linalg.norm(scale))
    ctx64 = pkg.Context(wl, restart_m=40, precision=0, start_filter=8)
    ev64, info64 = ctx64.fm_eigs(wl["shift"], 1, v0=v0)
    ctx64.close()
    assert info64["converged"] == 1
    assert abs(ev[0] - ev64[0]) <= 1e-10 * abs(ev64[0]), (ev, ev64)
