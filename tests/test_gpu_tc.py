"""GPU: the float32 preconditioner with its x and y stages on the tensor cores (TF32 mode
products, float32 accumulation).  The grids span several 128-row tiles, K blocks with ragged
tails and both y-stage forms (per-l diagonalisation for n_M = 1, banded M'-chain solves)."""
import numpy as np
import pytest

from fm_inputs import workload, rand_vec

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# TF32 keeps 10 mantissa bits (unit roundoff 2^-11); four chained products of length <= 132 with
# the conditioning of the 1D eigenvector bases stay well inside this bound (a layout or index
# error gives O(1)).
TF32_REL = 1e-2
# BF16 keeps 7 (unit roundoff 2^-8, eight times TF32's): the same chain with float32 accumulation
BF16_REL = 8e-2

CASES = {
    "he_l0_rows132": dict(nint=(66, 34, 3), R=(20.0, 17.0)),      # y stage: 2 row tiles (128 + 4)
    "he_l0_rows132y": dict(nint=(34, 66, 3), R=(20.0, 17.0)),     # x stage: 2 row tiles
    "he_l1_banded": dict(J=1, nint=(10, 12, 4), R=(20.0, 17.0)),  # n_M = 2: banded y solves between
    "psm_l2": dict(J=2, nint=(8, 10, 4), R=(30.0, 27.0), mass=(1.0, 1.0, 1.0), charge=(-1.0, -1.0, 1.0),
                   shift=-0.27),
    # n_x = n_y = 256: the float32 slab is too large for the fused per-slab kernel (unfused TF32 chain)
    "he_l0_wide": dict(nint=(128, 128, 2), R=(20.0, 17.0)),
}
# multiples of 8 in n_x and n_y, as the BF16 operands need
BF16_CASES = {
    "he_l0_rows136": dict(nint=(68, 36, 3), R=(20.0, 17.0)),      # fused chain, 2 row tiles in x
    "he_l0_rows136y": dict(nint=(36, 68, 3), R=(20.0, 17.0)),     # fused chain, 2 row tiles in y
    "he_l0_wide": dict(nint=(128, 128, 2), R=(20.0, 17.0)),       # n = 256: fused in BF16
    "he_l1_banded": dict(J=1, nint=(12, 8, 4), R=(20.0, 17.0)),   # n_M = 2: banded y, TF32 x stages
    # n_x = 24, n_y = 16: the fused BF16 chain on a grid whose sparse LU (the oracle's eigen-solve)
    # takes seconds; the two-row-tile grids above have 1.6e5 unknowns and 2e7 nonzeros
    "he_l0_small": dict(nint=(12, 8, 3), R=(20.0, 17.0)),
}


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2005_05398_gb300 as p
    from paper_2005_05398_gb300 import build
    build.build()
    p.lib()
    return p


def _dev(a):
    return torch.tensor(np.asarray(a), dtype=torch.float64, device="cuda")


def _wl(name):
    return workload("he_l0_24x24x8", **CASES[name])


def test_tc_eligibility(pkg):
    from paper_2005_05398_gb300._lib import FMError
    ctx = pkg.Context(_wl("he_l1_banded"), precision=1, mma=2)
    ctx.close()
    with pytest.raises(FMError) as e:  # n_x = 14, n_y = 18: not multiples of 4
        pkg.Context(workload("he_l0_24x24x8", nint=(7, 9, 5)), precision=1, mma=2)
    assert e.value.code == -1


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("y_solver", [0, 1])
@pytest.mark.parametrize("tc_chain", [0, 1])
def test_tc_precond_close_to_fp64(pkg, name, y_solver, tc_chain):
    """TF32 tensor-core chain (z stages, fused or unfused x / y stages, banded y solves) against the float64
    chain, which is itself equal to the paper's literal form (test_gpu_parity); tc_chain 0 is the chain with
    tensor-core z stages and the fused per-slab x / y stages, 1 the chain with SIMT z stages."""
    wl = _wl(name)
    E = wl["shift"] + 0.011
    ref_ctx = pkg.Context(wl, precision=0, y_solver=y_solver)
    tc = pkg.Context(wl, precision=1, mma=2, y_solver=y_solver, tc_chain=tc_chain)
    simt = pkg.Context(wl, precision=1, mma=1, y_solver=y_solver)
    v = _dev(rand_vec(ref_ctx.n, 21))
    out = {}
    for key, c in (("ref", ref_ctx), ("tc", tc), ("simt", simt)):
        c.fm_set_shift(E)
        y = torch.empty_like(v)
        c.fm_precond_apply(v, y)
        out[key] = y
        c.close()
    nref = torch.linalg.norm(out["ref"]).item()
    e_simt = torch.linalg.norm(out["simt"] - out["ref"]).item() / nref
    e_tc = torch.linalg.norm(out["tc"] - out["ref"]).item() / nref
    print(name, y_solver, "float32 SIMT", e_simt, "TF32 tensor cores", e_tc)
    assert e_simt < 1e-4
    assert e_tc < TF32_REL, name


@pytest.mark.parametrize("name,mma", [("he_l0_rows132", 2), ("he_l1_banded", 2), ("psm_l2", 2), ("he_l0_rows136", 3)])
def test_z_tile_widths_agree_bitwise(pkg, name, mma):
    """The z-stage tile width (points per tensor-core tile: 128, 64, 32, or the autotuner's choice) changes
    only which points share an MMA, not the K accumulation of any output element: every width gives the
    same preconditioner output bit for bit (an index or layout error in a narrow tile does not)."""
    wl = workload("he_l0_24x24x8", **(BF16_CASES[name] if mma == 3 else CASES[name]))
    E = wl["shift"] + 0.011
    out = {}
    for zt in (128, 64, 32, 256 + 128, 256 + 64, 256 + 32, 0):
        c = pkg.Context(wl, precision=1, mma=mma, z_tile=zt)
        c.fm_set_shift(E)
        v = _dev(rand_vec(c.n, 31))
        y = torch.empty_like(v)
        c.fm_precond_apply(v, y)
        torch.cuda.synchronize()
        out[zt] = y
        c.close()
    assert torch.isfinite(out[128]).all()
    for zt in (64, 32, 256 + 128, 256 + 64, 256 + 32, 0):
        assert torch.equal(out[zt], out[128]), (name, zt, (out[zt] - out[128]).abs().max().item())


def test_tc_computed_z_inverts_fmfin(pkg):
    """n_M = 1, computed z eigenvalues: the preconditioner is the exact inverse of Eq. FM-fin's left
    operator, so P^{-1} L v returns v to TF32 accuracy through the tensor-core chain."""
    from oracle.system import FMSystem
    from oracle.precond import Preconditioner
    wl = workload("he_l0_24x24x8", nint=(10, 8, 3), R=(10.0, 12.0))
    s = FMSystem(wl)
    E = -2.7
    P = Preconditioner(s, E, z_eigs="computed")
    ctx = pkg.Context(wl, z_eigs=1, precision=1, mma=2)
    ctx.fm_set_shift(E)
    v = rand_vec(s.N, 22)
    Lv = np.zeros(s.N)
    for a in s.comps:
        g = s.g[a]
        Lv[s.off[a]:s.off[a] + g.csize] = P.dense_L_fmfin(a) @ v[s.off[a]:s.off[a] + g.csize]
    y = torch.empty(s.N, dtype=torch.float64, device="cuda")
    ctx.fm_precond_apply(_dev(Lv), y)
    # L v is dominated by its high-frequency part, which the inverse cancels: the TF32 truncation
    # of the stages (2^-10 relative) is amplified by ||L^{-1}|| ||L v|| / ||v|| and by the condition of
    # the 1D eigenvector bases, to about 1.4e-2 on this grid; an index or layout error gives O(1)
    err = np.linalg.norm(y.cpu().numpy() - v) / np.linalg.norm(v)
    print("computed-z TF32 identity error", err)
    assert err < 5e-2


@pytest.mark.parametrize("precision,tc_chain,gram_schmidt", [(1, 0, 0), (2, 0, 0), (1, 1, 0), (1, 0, 1), (2, 1, 1)])
def test_tc_solve_matches_sparse_lu(pkg, precision, tc_chain, gram_schmidt):
    """FGMRES with the TF32 preconditioner (either tensor-core chain; CGS2 or single-pass DGKS
    orthogonalisation) reaches the sparse-LU solution of Eq. FM-lin."""
    from oracle.system import FMSystem
    from oracle import solvers
    wl = workload("he_l0_24x24x8", nint=(10, 12, 4), R=(20.0, 17.0))
    s = FMSystem(wl)
    H, S = s.H(), s.S()
    E = -2.5
    b = rand_vec(s.N, 23)
    ref = solvers.solve(H, S, E, b)
    ctx = pkg.Context(wl, precision=precision, mma=2, restart_m=40, tc_chain=tc_chain, gram_schmidt=gram_schmidt)
    x = torch.zeros(s.N, dtype=torch.float64, device="cuda")
    info = ctx.fm_solve(E, _dev(b), x)
    got = x.cpu().numpy()
    assert info["converged"] == 1 and info["resid"] <= 1e-12
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-8


@pytest.mark.parametrize("mixed_scheme", [0, 1, 2])
def test_mixed_schemes_match_sparse_lu(pkg, mixed_scheme):
    """FM_PREC_MIXED, flexible inner-outer scheme (float64 FGMRES over float32 FGMRES preconditioner steps),
    iterative refinement, and the flexible scheme with double-float inner solves: each reaches the float64
    tolerance and the sparse-LU solution of Eq. FM-lin."""
    from oracle.system import FMSystem
    from oracle import solvers
    wl = workload("he_l0_24x24x8", nint=(10, 12, 4), R=(20.0, 17.0))
    s = FMSystem(wl)
    E = -2.5
    b = rand_vec(s.N, 29)
    ref = solvers.solve(s.H(), s.S(), E, b)
    ctx = pkg.Context(wl, precision=2, mma=2, restart_m=40, mixed_scheme=mixed_scheme)
    x = torch.zeros(s.N, dtype=torch.float64, device="cuda")
    info = ctx.fm_solve(E, _dev(b), x)
    print("mixed scheme", mixed_scheme, info)
    assert info["converged"] == 1 and info["resid"] <= 1e-12
    assert np.linalg.norm(x.cpu().numpy() - ref) / np.linalg.norm(ref) < 1e-8


@pytest.mark.parametrize("name", ["he_l1_banded", "psm_l2", "he_l0_small"])
def test_dd_inner_eigs_match_oracle(pkg, name):
    """Double-float inner solves (mixed_scheme 2) inside the flexible float64 iteration: the certified
    eigenvalues equal the oracle's to 1e-9 (n_M = 2 and 3 with banded y solves; n_M = 1 with the fused chain)."""
    from oracle.system import FMSystem
    from oracle import solvers
    wl = workload("he_l0_24x24x8", **BF16_CASES[name]) if name == "he_l0_small" else _wl(name)
    s = FMSystem(wl)
    shift = wl["shift"] if name != "he_l1_banded" else -2.12
    Eo, _ = solvers.eigs_near(s.H(), s.S(), shift, 6)
    Eo = Eo[np.abs(Eo.imag) <= 1e-10 * np.abs(Eo)][:2].real
    ctx = pkg.Context(wl, restart_m=40, precision=2, mixed_scheme=2)
    ev, info = ctx.fm_eigs(shift, 2)
    print(name, "double-float inner", info)
    assert info["converged"] == 1 and info["resid"] <= 1e-9, info
    for i in range(2):
        assert abs(ev[i] - Eo[i]) <= 1e-9 * abs(Eo[i]), (ev, Eo)


@pytest.mark.parametrize("name,k,precision", [("he_l1_banded", 2, 1), ("psm_l2", 2, 2), ("he_l1_banded", 2, 2)])
def test_tc_eigs_match_oracle(pkg, name, k, precision):
    from oracle.system import FMSystem
    from oracle import solvers
    wl = _wl(name)
    s = FMSystem(wl)
    H, S = s.H(), s.S()
    shift = wl["shift"] if name != "he_l1_banded" else -2.12
    Eo, _ = solvers.eigs_near(H, S, shift, k + 4)
    real = np.abs(Eo.imag) <= 1e-10 * np.abs(Eo)
    Eo = Eo[real][:k].real
    ctx = pkg.Context(wl, restart_m=40, precision=precision, mma=2)
    ev, info = ctx.fm_eigs(shift, k)
    assert info["converged"] == 1
    for i in range(k):
        assert abs(ev[i] - Eo[i]) <= 1e-9 * abs(Eo[i]), (ev, Eo)


@pytest.mark.parametrize("name", list(BF16_CASES))
@pytest.mark.parametrize("y_solver", [0, 1])
def test_bf16_precond_close_to_fp64(pkg, name, y_solver):
    """BF16 operands (float32 accumulation) in the z stages and the fused chain, against the float64 chain,
    and within a few times the TF32 chain's error."""
    wl = workload("he_l0_24x24x8", **BF16_CASES[name])
    E = wl["shift"] + 0.011
    out = {}
    for key, kw in (("ref", dict(precision=0)), ("tf32", dict(precision=1, mma=2)), ("bf16", dict(precision=1, mma=3))):
        c = pkg.Context(wl, y_solver=y_solver, **kw)
        c.fm_set_shift(E)
        v = _dev(rand_vec(c.n, 24))
        y = torch.empty_like(v)
        c.fm_precond_apply(v, y)
        out[key] = y
        c.close()
    nref = torch.linalg.norm(out["ref"]).item()
    e32 = torch.linalg.norm(out["tf32"] - out["ref"]).item() / nref
    e16 = torch.linalg.norm(out["bf16"] - out["ref"]).item() / nref
    print(name, y_solver, "TF32", e32, "BF16", e16)
    assert e32 < TF32_REL and e16 < BF16_REL, (name, e32, e16)


def test_bf16_eligibility(pkg):
    from paper_2005_05398_gb300._lib import FMError
    with pytest.raises(FMError) as e:  # n_x = 20: a multiple of 4, not of 8
        pkg.Context(workload("he_l0_24x24x8", nint=(10, 12, 3)), precision=1, mma=3)
    assert e.value.code == -1


@pytest.mark.parametrize("precision", [1, 2])
def test_bf16_solve_matches_sparse_lu(pkg, precision):
    """A looser preconditioner, the same float64 solution."""
    from oracle.system import FMSystem
    from oracle import solvers
    wl = workload("he_l0_24x24x8", nint=(12, 8, 4), R=(20.0, 17.0))
    s = FMSystem(wl)
    H, S = s.H(), s.S()
    E = -2.5
    b = rand_vec(s.N, 25)
    ref = solvers.solve(H, S, E, b)
    ctx = pkg.Context(wl, precision=precision, mma=3, restart_m=40)
    x = torch.zeros(s.N, dtype=torch.float64, device="cuda")
    info = ctx.fm_solve(E, _dev(b), x)
    got = x.cpu().numpy()
    assert info["converged"] == 1 and info["resid"] <= 1e-12
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-8


@pytest.mark.parametrize("name,k,precision", [("he_l0_small", 2, 1), ("he_l0_small", 2, 2), ("he_l1_banded", 2, 2)])
def test_bf16_eigs_match_oracle(pkg, name, k, precision):
    from oracle.system import FMSystem
    from oracle import solvers
    wl = workload("he_l0_24x24x8", **BF16_CASES[name])
    s = FMSystem(wl)
    H, S = s.H(), s.S()
    shift = wl["shift"] if name != "he_l1_banded" else -2.12
    Eo, _ = solvers.eigs_near(H, S, shift, k + 4)
    real = np.abs(Eo.imag) <= 1e-10 * np.abs(Eo)
    Eo = Eo[real][:k].real
    ctx = pkg.Context(wl, restart_m=40, precision=precision, mma=3)
    ev, info = ctx.fm_eigs(shift, k)
    assert info["converged"] == 1 and info["resid"] <= 1e-9
    for i in range(k):
        assert abs(ev[i] - Eo[i]) <= 1e-9 * abs(Eo[i]), (ev, Eo)
