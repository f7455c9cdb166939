/*
 * libfm -- GB300 (sm_103a) solver for the spline-collocation discretisation of the
 * three-body Faddeev-Merkuriev equations in total orbital momentum representation
 * (Gradusov, Roudnev, Yarevsky, Yakovlev, arXiv:2005.05398).
 *
 * The problem (Section 3.1, Eq. FM-lin): find E and c with H c = E S c, or solve
 * (H - E S) x = b, where H is the collocation matrix of Eq. FM-fin (equivalently
 * Eq. FM-pre with its right-hand side moved to the left) and S has entries
 * S^k(z) S^i(x) S^j(y) at the collocation points.  The iterative solves are
 * preconditioned by the tensor-trick inverse of Eq. prec-2 (Section 3.2).
 *
 * Conventions
 *  - Every function returns an fm_status (0 on success).  fm_strerror() names a code.
 *  - Vectors are float64 and live in device memory of the context's GPU unless the
 *    entry point says "host".  Their length is n_unknowns (fm_size()).  The caller
 *    owns every buffer it passes; the library never frees caller memory and keeps
 *    no pointer to it after the call returns.
 *  - Vector layout (Section 3.2 ordering): [solved component a][M' = M0..J][k_z][i_x][j_y],
 *    j_y fastest.  Solved components: particles {1, 3} when particles 1 and 2 are
 *    identical (Eq. 2-sym-part), {1, 2, 3} otherwise, {1} in the Schrodinger limit.
 *  - All work is ordered on the context's stream (fm_opts.stream, or the legacy
 *    default stream when NULL).  fm_apply / fm_apply_S return without synchronising;
 *    fm_precond_apply synchronises when its tensor-core stages ran (it reads their wait
 *    flag); fm_solve / fm_eigs synchronise before they return.
 *  - A context is used by one host thread at a time.
 *  - Energies are in the units of the reduced-coordinate equations (Hartree for
 *    electron-mass units); box sizes R_x, R_y are in reduced Jacobi coordinates.
 */
#ifndef FM_H
#define FM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FM_OK = 0,
  FM_ERR_ARG = -1,              /* invalid argument (sizes, n_M = 0, null pointers, ...) */
  FM_ERR_OOM = -2,              /* device or host allocation failed */
  FM_ERR_CUDA = -3,             /* a CUDA runtime call failed */
  FM_ERR_NOT_CONVERGED = -4,    /* iteration limit reached; outputs hold the best iterate */
  FM_ERR_BREAKDOWN = -5,        /* Krylov breakdown (zero or non-finite norm) */
  FM_ERR_COMPLEX_SPECTRUM = -6, /* a 1D generalized eigenproblem has complex eigenvalues */
  FM_ERR_NO_SHIFT = -7,         /* preconditioner used before fm_set_shift */
  FM_ERR_NUMERIC = -8,          /* singular 1D or banded factor, non-finite setup value */
  FM_ERR_SCRATCH_LIMIT = -9,    /* problem larger than the fixed scratch of fm_apply_noalloc */
  FM_ERR_TIMEOUT = -10          /* a bounded wait inside a device kernel expired (results invalid) */
} fm_status;

/* Three particles (Section 2.1).  Masses in electron masses ("infinite" core: 1e15,
 * Section 4), charges in units of e.  J = total orbital momentum, tau = +1/-1 the
 * parity label of the F basis (Eq. F-def), exch_p = +1/-1 exchange symmetry of the
 * identical pair (Eq. 2-sym), identical_pair = 12 when particles 1 and 2 are
 * identical (solve components 1 and 3), 0 otherwise (solve 1, 2, 3). */
typedef struct {
  double mass[3];
  double charge[3];
  int J;
  int tau;
  int exch_p;
  int identical_pair;
} fm_system;

enum { FM_MAP_POW = 0, FM_MAP_EQUI = 1, FM_MAP_SIN = 2 };

/* Spline grid of one solved component, notation (n_x, n_y, n_z; R_x, R_y) of Section 4.
 * nint intervals per axis.  Cubic Hermite splines: 2*nint functions in x and y (Dirichlet at 0
 * and R), 2*nint + 2 in z on [-1, 1].  Quintic Hermite (value, first and second derivative per node):
 * 3*nint + 1 in x and y, 3*nint + 3 in z (the counts of the paper's tables).  Collocation at Gauss
 * points, as many as functions.  Node maps: Eq. map-pow (FM_MAP_POW, x and y), equidistant, and
 * sin(pi u / 2) (FM_MAP_SIN, z only). */
typedef struct {
  int nint_x, nint_y, nint_z;
  double Rx, Ry;
  int xmap, ymap, zmap;
  int basis; /* 0 = cubic Hermite (r = 4), 1 = quintic Hermite S_5^3 (r = 6, Section 4); one basis for all */
} fm_grid;

enum { FM_SPLIT_MERKURIEV = 0, FM_SPLIT_NONE = 1, FM_SPLIT_SCHRODINGER = 2 };

/* Potential splitting (Eqs. PotSplit, split3b, Mcutoff0): mode 0 = Merkuriev cut-off
 * chi = 2/(1+exp[(x/x0)^nu/(1+y/y0)]) (y0 = +inf allowed), mode 1 = no splitting
 * (V^(s) = V: standard Faddeev equations), mode 2 = Schrodinger limit (one component,
 * all pair potentials on the left, Section 2.1).  In mode 0 a collocation point
 * carries the V^(s) coupling only where chi > vs_cut (0 keeps every nonzero chi). */
typedef struct {
  int mode;
  double nu, x0, y0;
  double vs_cut;
} fm_splitting;

/* Precision modes.  FP64: float64 everywhere.  FP32: float32 preconditioner, float64 operator,
 * FGMRES and Gram-Schmidt.  MIXED: float32 FGMRES solves (float32 operator, preconditioner and
 * Gram-Schmidt) inside a float64 iteration on the true float64 residual, chosen by
 * fm_opts.mixed_scheme: a flexible float64 FGMRES whose preconditioner is the float32 solve
 * (default), or iterative refinement; the result meets the same float64 tolerance. */
enum { FM_PREC_FP64 = 0, FM_PREC_FP32 = 1, FM_PREC_MIXED = 2 };

/* Mode products of the float32 preconditioner (FP32 and MIXED precision).  AUTO: TF32 tensor-core
 * GEMMs (float32 accumulation) on every component whose n_x and n_y are multiples of 4 in [16, 256],
 * float32 CUDA cores otherwise.  SIMT: float32 CUDA cores always.  TF32: tensor cores, FM_ERR_ARG
 * from fm_create when a component is not eligible.  BF16: BF16 operands with float32 accumulation
 * (8 significand bits per operand: a looser preconditioner, the same float64 results) for the z stages
 * and, with n_M = 1, the fused x / y chain; the x stages around the banded y solves (n_M > 1) stay
 * TF32; needs n_x, n_y multiples of 8 in [16, 256] and n_z <= 128 (else FM_ERR_ARG).
 * On the tensor cores the z stages run as tcgen05 GEMMs when n_z <= 128, and for n_M = 1 the x and y
 * stages of one slab (z mode) run in one kernel that keeps the slab on chip. */
enum { FM_MMA_AUTO = 0, FM_MMA_SIMT = 1, FM_MMA_TF32 = 2, FM_MMA_BF16 = 3 };

typedef struct {
  double tol;        /* relative residual of fm_solve (FGMRES true residual), e.g. 1e-12 */
  int restart_m;     /* FGMRES restart length (1..128) */
  int max_iters;     /* total FGMRES iteration limit per fm_solve */
  int precision;     /* FM_PREC_FP64, FM_PREC_FP32 or FM_PREC_MIXED */
  int ncv;           /* Arnoldi basis size of fm_eigs (>= 2k + 1) */
  int max_restarts;  /* Arnoldi restarts of fm_eigs */
  double eig_tol;    /* fm_eigs: relative Ritz residual |h_{m+1,m} y_m| / |theta| at which a Ritz pair is
                        accepted (default 1e-9); a pair whose energy changed by less than 1e-3 * eig_tol
                        (relative) over three Arnoldi steps while its residual is below sqrt(eig_tol) is
                        accepted too (its accuracy is then set by the inner solves) */
  int z_eigs;        /* 0 = replace z eigenvalues by -l(l+1) (Eq. prop-eq); 1 = keep them (n_M = 1 only) */
  int y_solver;      /* y stage of the preconditioner: 0 = automatic (per-l diagonalisation for n_M = 1 with the
                        float32 preconditioner, banded LU otherwise), 1 = banded LU, 2 = per-l
                        diagonalisation of (A_l, S_y) when n_M = 1 (both invert the same matrix) */
  int tune;          /* fm_eigs: 1 = tune the preconditioner to the current Ritz vectors U (rank-k update
                        P + (A U - P U) U^T, Freitag & Spence), dropped once an inner solve stalls;
                        0 = plain preconditioner (default: with the relaxed inner tolerance the tuning no
                        longer saves time, and near clusters of levels it misleads inexact solves) */
  int mma;           /* FM_MMA_AUTO, FM_MMA_SIMT, FM_MMA_TF32 or FM_MMA_BF16 */
  int start_filter;  /* fm_eigs: passes v <- P^{-1} S v / |.| applied to the start vector before the Arnoldi
                        process (the tensor preconditioner approximates (H - E* S)^{-1}, so each pass
                        enriches the directions of the levels nearest the shift); 0..16, or -1 (default):
                        16 when one level is wanted, 6 when several are (more passes then filter the other
                        wanted levels out) */
  int refine;        /* fm_eigs: most inverse-iteration steps c <- (H - shift S)^{-1} S c / |.| (float64 solves
                        to tol) given to a returned pair whose backward error is above eig_tol; 0..8, default 2 */
  double inner_tol32; /* FM_PREC_MIXED: relative residual of each float32 inner solve, in [1e-7, 0.5], or 0 for
                        the scheme's default (1e-3 flexible, 3e-5 refinement, half the outer tolerance but at least 3e-9 for
                        double-float); smaller means fewer float64
                        steps and more float32 iterations in each */
  int tc_chain;      /* tensor-core preconditioner chain: 0 = z stages on the tensor cores and, for n_M = 1, the
                        x / y stages of a slab in one fused kernel; 1 = z stages on CUDA cores and one
                        tensor-core launch per x / y stage (TF32) */
  int gram_schmidt;  /* float64 FGMRES orthogonalisation: 0 = two classical Gram-Schmidt passes, the first on
                        the FP32 pipe from the leading bits, the closing update on the FP32 pipe too while the
                        second projection is below 1e-5 of the vector (float64 otherwise); 1 = one float64
                        pass, repeated only when it cancelled more than half of the vector's norm (DGKS test) */
  int mixed_scheme;  /* FM_PREC_MIXED: 0 = flexible inner-outer iteration (float64 FGMRES on the float64 operator,
                        each of its preconditioner steps a float32 FGMRES solve of the normalised basis
                        vector, so the float64 Krylov space is kept across the float32 solves; default);
                        1 = iterative refinement x += float32 solve of the normalised float64 residual,
                        each refinement step starting a new float32 Krylov space; 2 = the flexible iteration
                        with double-float inner solves (operator, basis and Gram-Schmidt as pairs of floats,
                        about 48 significand bits, on the FP32 pipe; the float32 tensor preconditioner) */
  int z_tile;        /* tensor-core tile of the z stages: 0 = chosen per shape by fm_create's autotuner (widths 128,
                        64 and 32 points in two shapes each, timed on the context's buffers, results cached per
                        shape for the process); or fixed: 128, 64, 32 (runs along the output's contiguous
                        index), + 256 for the shape with runs of 8 on the input side too */
  int device;        /* CUDA device ordinal */
  void* stream;      /* cudaStream_t, NULL = legacy default stream */
} fm_opts;

/* How fm_eigs' Arnoldi iteration stopped (fm_info.accept). */
enum {
  FM_ACCEPT_NONE = 0,    /* restart limit or breakdown before either rule held */
  FM_ACCEPT_RITZ = 1,    /* every wanted Ritz pair met |h_{m+1,m} y_m| / |theta| <= eig_tol */
  FM_ACCEPT_STABLE = 2   /* some pair only met the stable-energy rule (see fm_opts.eig_tol) */
};

typedef struct {
  int iters;          /* FGMRES iterations (fm_solve; float32 iterations in FM_PREC_MIXED) or total inner
                         iterations (fm_eigs, refinement included) */
  int restarts;       /* FGMRES restarts (FM_PREC_MIXED: float64 outer iterations of the flexible scheme or
                         refinement steps) or Arnoldi restarts */
  int op_applies;     /* shift-invert operator applications (fm_eigs, refinement included) */
  int converged;      /* 1 when every requested quantity met its tolerance */
  double resid;       /* fm_solve: final relative residual |b - (H - E S) x| / |b|;
                         fm_eigs: largest backward error eta of the returned pairs (see fm_eigs) */
  double ms;          /* wall time of the call */
  int accept;         /* fm_eigs: FM_ACCEPT_* rule that stopped the Arnoldi iteration */
  int refine_steps;   /* fm_eigs: inverse-iteration steps taken by the final float64 refinement (all pairs) */
  double resid_S;     /* fm_eigs: largest |H c - E S c| / |S c| of the returned pairs */
  double norm_H;      /* fm_eigs: the estimates of |H|_2 and |S|_2 in the backward error (power-iteration */
  double norm_S;      /*          lower bounds, so that eta is never underestimated through them) */
  double rq_dev;      /* fm_eigs: largest |E_R - E| / |E|, E_R = (S c)^T (H c) / |S c|^2 the Rayleigh estimate */
} fm_info;

/* A context holds one problem's tables, factors and Krylov workspace on one device.  Different
 * contexts may be used concurrently from different host threads (each on its own stream), which is
 * how the request loop below runs several problems side by side. */
typedef struct fm_ctx fm_ctx;

/* Default options: tol 1e-12, restart 64, max_iters 2000, FP64, ncv 20, 50 restarts,
 * eig_tol 1e-9, replaced z eigenvalues, plain preconditioner, start-vector filter passes by k, 2 refinement
 * steps, device 0, default stream. */
void fm_default_opts(fm_opts* opts);

/* Build a context: 1D bases and collocation points (Section 3.1), pointwise potential
 * tables, the V^(s) coupling geometry (Eqs. r-form, s-rot), the E-independent z and x
 * decompositions of the preconditioner (Eq. z-dec and the x problems of Section 3.2)
 * and the Krylov workspace.  grids: n_grids = 1 (same grid for every solved component)
 * or one per solved component.  On error *out is NULL. */
int fm_create(const fm_system* sys, const fm_grid* grids, int n_grids, const fm_splitting* split,
              const fm_opts* opts, fm_ctx** out);

/* Device memory (bytes) that fm_create with these arguments would hold, from the same size
 * plan (no allocation, no GPU work, no eigen-decompositions; within a few percent).  For
 * admission control of concurrent solves.  fm_eigs_host adds k vectors on first use. */
int fm_estimate_bytes(const fm_system* sys, const fm_grid* grids, int n_grids, const fm_splitting* split,
                      const fm_opts* opts, int64_t* bytes);

/* Sizes: total unknowns, solved components, n_M = J - M0 + 1 (Section 2.2). */
int fm_size(const fm_ctx* ctx, int64_t* n_unknowns, int* n_components, int* n_M);

/* Per solved component: particle label (1..3), dims = {n_z, n_x, n_y}, offset of its block. */
int fm_component(const fm_ctx* ctx, int comp, int* label, int dims[3], int64_t* offset);

/* y = (H - E S) x (Eq. FM-lin).  x and y: device, length n_unknowns, must not overlap. */
int fm_apply(fm_ctx* ctx, double E, const double* x, double* y);

/* y = S x.  Device buffers, no overlap. */
int fm_apply_S(fm_ctx* ctx, const double* x, double* y);

/* Build the E*-dependent part of the preconditioner (the banded y systems of
 * Eq. ops / the tridiagonal M' chains, Section 3.2) for shift Estar. */
int fm_set_shift(fm_ctx* ctx, double Estar);

/* y = L^{-1}(E*) x, the tensor-trick preconditioner of Eq. prec-2.  Device buffers,
 * no overlap.  FM_ERR_NO_SHIFT before the first fm_set_shift. */
int fm_precond_apply(fm_ctx* ctx, const double* x, double* y);

/* Solve (H - E S) x = rhs by right-preconditioned FGMRES (restarted) with the
 * preconditioner built for E (fm_set_shift is called when E differs from the current
 * shift).  x (device) is the initial guess on entry (pass zeros for none) and the
 * solution on return.  Converged when ||rhs - (H - E S) x|| <= tol ||rhs|| in float64.
 * A restart cycle that fails to halve the true residual ends the solve (the float64
 * residual has reached its rounding floor); FM_ERR_NOT_CONVERGED then, or at max_iters,
 * with the best iterate in x and info->resid the reached relative residual.  info may be NULL. */
int fm_solve(fm_ctx* ctx, double E, const double* rhs, double* x, fm_info* info);

/* k eigenpairs of H c = E S c nearest 'shift' by restarted Arnoldi on the
 * shift-invert operator (H - shift S)^{-1} S (Eq. FM-lin; E = shift + 1/theta), each
 * operator application an FGMRES solve to max(tol, eig_tol / 10).  v0 (device, may be NULL = seeded normal start)
 * starts the iteration.  Only real eigenvalues are returned: complex-conjugate pairs of the
 * non-symmetric collocation pencil (non-physical in the bound-state problem) are passed over,
 * so the result is the k real eigenvalues nearest the shift.
 * Final float64 certificate: for each returned pair, E = shift + 1/theta (the Ritz value) and its Ritz
 * vector c (|c| = 1), the library forms H c and S c with the float64 operator and the backward error
 * eta = |H c - E S c| / (|H| + |E| |S|): (E, c) is an exact eigenpair of a pencil within relative distance
 * eta of (H, S).  A pair with eta > eig_tol gets up to opts.refine inverse-iteration steps
 * c <- (H - shift S)^{-1} S c / |.|, E = shift + 1 / (c^T (H - shift S)^{-1} S c), a step kept only when it
 * lowers eta.  The call returns FM_OK only when every pair ends with eta <= eig_tol, whichever rule stopped
 * the Arnoldi iteration (info->accept); otherwise FM_ERR_NOT_CONVERGED with the pairs as computed.  The
 * Rayleigh estimate E_R = (S c)^T (H c) / |S c|^2 is reported as a check (info->rq_dev): it weighs the
 * high-frequency error of c with |H| and is less accurate than the Ritz value of the shift-invert operator.
 * evals (host, k doubles) receive the certified E sorted by |E - shift|;
 * evecs (device, k * n_unknowns, may be NULL) the eigenvectors normalised to unit
 * 2-norm with their largest-magnitude entry positive.  info may be NULL. */
int fm_eigs(fm_ctx* ctx, double shift, int k, const double* v0, double* evals, double* evecs, fm_info* info);

/* fm_eigs with HOST buffers: v0_host (may be NULL) is copied to the device, evecs_host
 * (may be NULL) receives the eigenvectors.  The copies run on the context's stream. */
int fm_eigs_host(fm_ctx* ctx, double shift, int k, const double* v0_host, double* evals,
                 double* evecs_host, fm_info* info);

/* Release every resource of the context.  NULL is allowed. */
void fm_destroy(fm_ctx* ctx);

/* Static description of a status code. */
const char* fm_strerror(int status);

/* Diagnostics: counts of the library's own kernel launches since the context was
 * created (launches) and bytes of device memory the context holds. */
int fm_stats(const fm_ctx* ctx, int64_t* launches, int64_t* device_bytes);

/* Largest n_unknowns accepted by fm_apply_noalloc. */
#define FM_NOALLOC_MAX_UNKNOWNS (1 << 20)

/* y = (H - E S) x like fm_apply, for callers that must not allocate device memory during
 * the call: code whose device memory is owned by another allocator (a framework's caching
 * allocator or a pool sized at start-up, where a cudaMalloc can fail or fragment the pool)
 * and code on a time-critical path, where cudaMalloc / cudaFree can synchronise the device.
 * The paper has no counterpart: it is an interface for such callers.  The context is built
 * by fm_create beforehand (which does allocate); this call allocates nothing.  Its scratch
 * (three planes of n_unknowns doubles) is a fixed array inside the library, 24 MiB that every
 * GPU loading the library holds until the process exits; n_unknowns above
 * FM_NOALLOC_MAX_UNKNOWNS gives FM_ERR_SCRATCH_LIMIT.  The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress, with that device current); make that first
 * call before any stream capture begins.  The address is kept per device and CUDA context: after a
 * cudaDeviceReset (or a new primary context) the next call looks it up again, so that call, too,
 * must come before any stream capture.  All calls
 * share the array: two calls whose kernels overlap on the GPU (different streams or
 * contexts running concurrently) race on it and produce wrong results.  Nothing in the
 * array needs clearing between calls.  Device buffers x and y must not overlap. */
int fm_apply_noalloc(fm_ctx* ctx, double E, const double* x, double* y);

/* Host-side diagnostic (no GPU involved): the 1D decomposition D(A1, A2) of
 * Eq. WW-scale exactly as fm_create computes it for the preconditioner: W-bar A1 W =
 * diag(lam), W-bar A2 W = I, eigenvalues ascending (descending if 'descending').
 * Row-major n x n arrays owned by the caller.  FM_ERR_COMPLEX_SPECTRUM when the
 * pencil has complex eigenvalues, FM_ERR_NUMERIC when A2 or W is singular. */
int fm_host_decompose(int n, const double* A1, const double* A2, int descending, double* Wbar, double* W,
                      double* lam);

/* Host-side diagnostic (no GPU involved): one spline axis exactly as fm_create builds it (Section 3.1,
 * Section 4): node map 'map' (FM_MAP_*) of 'nint' intervals on [a, b], Dirichlet at both ends or not,
 * basis 0 (cubic Hermite, r = 4) or 1 (quintic Hermite, r = 6).  Outputs: *n functions (= collocation
 * points), *r taps per point; pts[n] the collocation points, base[n] the first tap's function index, and
 * S, D1, D2 [n][r] the values, first and second derivatives of functions base + t at each point.  The
 * caller provides arrays for n <= 3 (nint + 1) points and r = 6 taps.  FM_ERR_ARG for invalid input. */
int fm_host_axis(int map, int nint, double a, double b, int dirichlet, int basis, int* n, int* r, double* pts,
                 int* base, double* S, double* D1, double* D2);

/* Kernel classes of the per-kernel timing below. */
enum {
  FM_KERNEL_APPLY_XY = 0,  /* operator apply, y and x passes */
  FM_KERNEL_APPLY_Z,       /* operator apply, z pass + pointwise terms + M' couplings */
  FM_KERNEL_COUPLING,      /* V^(s) coupling gather */
  FM_KERNEL_ZMIX,          /* preconditioner z mode products */
  FM_KERNEL_XMIX,          /* preconditioner x mode products (with the y stage where they run fused) */
  FM_KERNEL_YSOLVE,        /* preconditioner banded y solves */
  FM_KERNEL_DOT,           /* Krylov multi-dot products */
  FM_KERNEL_AXPY,          /* Krylov multi-axpy updates */
  FM_KERNEL_OTHER,         /* copies, scalings, start vectors, combinations */
  FM_NUM_KERNEL_CLASSES
};

/* Per-kernel timing with CUDA events recorded on the context's stream around every
 * launch.  enable = 1 clears the accumulators and starts recording, 0 stops. */
int fm_profile(fm_ctx* ctx, int enable);

/* Accumulated device time (ms), launch counts and algorithmic work (FLOPs and DRAM-level
 * bytes by the per-kernel formulas of the library's documentation; flops and bytes may be
 * NULL) per kernel class since fm_profile(ctx, 1).  Arrays have FM_NUM_KERNEL_CLASSES
 * entries.  Synchronises the stream. */
int fm_profile_read(fm_ctx* ctx, double* ms, int64_t* launches, double* flops, double* bytes);

/* ---------------------------------------------------------------------------------------
 * Request loop for independent problems (serving).  The paper solves one problem at a time;
 * this part has no counterpart there.  A server owns `slots` worker threads, each with its
 * own CUDA stream.  A submitted request waits in arrival order until a slot is free and its
 * device working set (fm_estimate_bytes plus the request's two vectors) fits the HBM budget
 * next to the requests already running; a request that has been passed over 8 times by
 * later, smaller ones blocks further passing until it is admitted.  Each admitted request
 * gets its own context (1D factor sets, Krylov state) on the device for its lifetime, so
 * the requests in flight overlap on the GPU and their results do not depend on the mix
 * (every kernel reduces in a fixed order).
 * ------------------------------------------------------------------------------------- */
typedef struct fm_server fm_server;

enum { FM_REQ_SOLVE = 0, FM_REQ_EIGS = 1 };
enum { FM_SERVER_DRY_RUN = 1 }; /* host only: requests "run" for sim_ms, no CUDA call is made */

/* One request: a problem (one grid for every solved component) and what to compute.
 * kind FM_REQ_SOLVE: (H - E S) x = b with b ~ N(0,1) drawn from `seed` on the device;
 * FM_REQ_EIGS: the k (1..8) eigenvalues nearest E, Arnoldi start ~ N(0,1) from `seed`.
 * out_host (optional, host memory the caller keeps alive until fm_server_wait returns)
 * receives x (n values) or the k eigenvectors (k n values). */
typedef struct {
  fm_system sys;
  fm_grid grid;
  fm_splitting split;
  int kind;
  double E;
  int k;
  uint64_t seed;
  int precision;     /* FM_PREC_* */
  double sim_ms;     /* FM_SERVER_DRY_RUN: simulated run time of the request */
  double* out_host;
} fm_request;

/* Outcome of one request.  Times in ms on the server's steady clock (0 = creation). */
typedef struct {
  int status;         /* fm_status of the solve or eigen-solve */
  int iters;          /* FGMRES iterations */
  int64_t n;          /* unknowns */
  int64_t bytes;      /* device bytes the request was admitted with */
  double evals[8];    /* FM_REQ_EIGS: eigenvalues, nearest first */
  double resid;       /* relative residual (solve) or largest eigen-residual (eigs) */
  double out_norm;    /* ||x|| (solve); 1 per eigenvector (eigs) */
  double t_submit_ms, t_start_ms, t_end_ms;
} fm_result;

/* hbm_budget <= 0: the device memory free at creation (cudaMemGetInfo) less 5 % of the device, so that
 * memory already held by other allocators in the process (a framework's caching allocator, other
 * contexts) is not promised to requests; FM_ERR_OOM when nothing is left.  With FM_SERVER_DRY_RUN the
 * budget must be given (> 0).  slots in 1..64. */
int fm_server_create(int device, int64_t hbm_budget, int slots, int flags, fm_server** out);

/* Enqueue a request (copied); *id identifies it.  FM_ERR_OOM when the request alone exceeds the
 * budget, FM_ERR_ARG for invalid requests (checked as fm_create and fm_eigs would). */
int fm_server_submit(fm_server* s, const fm_request* r, int64_t* id);

/* Block until request id has finished (timeout_ms < 0: no limit) and return its result once;
 * FM_ERR_TIMEOUT when the limit passed first, FM_ERR_ARG for an unknown or collected id. */
int fm_server_wait(fm_server* s, int64_t id, double timeout_ms, fm_result* out);

/* Device bytes admitted now and at most so far, requests running now and at most so far,
 * requests waiting for admission (any pointer may be NULL). */
int fm_server_stats(fm_server* s, int64_t* in_use, int64_t* peak_in_use, int* busy, int* peak_busy, int* queued);

/* Finish the queued and running requests, stop the workers, free the server. */
void fm_server_destroy(fm_server* s);

#ifdef __cplusplus
}
#endif
#endif /* FM_H */
