"""fm_apply_noalloc: the operator apply for callers that may not allocate device memory
during the call (memory owned by another allocator, or a time-critical path where
cudaMalloc / cudaFree would synchronise the device).  It must give the same result as
fm_apply, call after call, although its scratch planes are a fixed array shared by every
call instead of the context's own buffers."""
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


@pytest.mark.parametrize("kw", [dict(), dict(J=1, nint=(10, 12, 6), R=(25.0, 30.0))])
def test_noalloc_apply_matches_apply_twice(pkg, kw):
    wl = workload("he_l0_24x24x8", **kw)
    ctx = pkg.Context(wl, restart_m=4, ncv=4)
    n = ctx.n
    assert n <= 1 << 20
    for seed, E in ((11, -2.9), (12, 0.7)):  # two calls in a row, different inputs
        x = torch.tensor(rand_vec(n, seed), dtype=torch.float64, device="cuda")
        ref = torch.empty_like(x)
        got = torch.full_like(x, float("nan"))
        ctx.fm_apply(E, x, ref)
        ctx.fm_apply_noalloc(E, x, got)
        torch.cuda.synchronize()
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        assert np.all(np.isfinite(g))
        assert np.max(np.abs(g - r)) <= 1e-13 * np.max(np.abs(r))
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_scratch(pkg):
    from paper_2005_05398_gb300 import FMError
    wl = workload("he_l0_24x24x8", nint=(64, 64, 16), R=(40.0, 40.0))
    ctx = pkg.Context(wl, restart_m=2, ncv=4)
    assert ctx.n > 1 << 20
    x = torch.zeros(ctx.n, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    with pytest.raises(FMError) as e:
        ctx.fm_apply_noalloc(-2.9, x, y)
    assert e.value.code == -9 and "scratch" in str(e.value)
    ctx.close()
