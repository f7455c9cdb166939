// Internal structures of libfm (not part of the C ABI).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/fm.h"
#include "fm_dd.h"

namespace fmi {

// One spline axis (Section 3.1): nodes, collocation points and, per collocation
// point, the r nonzero basis functions as taps base+t, t = 0..r-1 (a tap outside
// [0, n) carries the value 0).  Cubic Hermite: q = 2 functions per node, r = 4;
// quintic Hermite S_5^3: q = 3, r = 6.
constexpr int kMaxTaps = 6;
struct Axis {
  int kind = 0, nint = 0, n = 0;
  int q = 2, r = 4;                    // functions per node, taps per point
  int kl = 0, ku = 0;                  // band half-widths of the 1D collocation matrices (row - col, col - row)
  double a = 0, b = 0;
  bool dirichlet = false;
  std::vector<double> nodes, pts;
  std::vector<int> base;               // per point
  std::vector<double> S, D1, D2;       // per point, r values each
  void build(int kind, int nint, double a, double b, bool dirichlet, int basis = 0);
  int locate(double p) const;          // interval m with nodes[m] <= p <= nodes[m+1]
  // taps of an arbitrary point (values, first derivatives or second derivatives); v holds r values
  void eval(double p, int deriv, int* base_out, double v[kMaxTaps]) const;
  // rows of c[x][y] a tile of tx consecutive collocation points reads (from the base of its first point)
  int tile_rows(int tx) const;
};

// Half-width of the banded y systems of one l (Section 3.2, the M' chain of n_c components interleaved
// with y): the 1D band of the y collocation matrices times n_c, plus the M' coupling to the neighbours.
inline int band_kl(const Axis& ay, int nc) {
  const int k = ay.kl > ay.ku ? ay.kl : ay.ku;
  return nc == 1 ? k : k * nc + 1;
}
constexpr int kMaxBandKL = 25;  // widest banded y system the y-solve kernel takes

// Device-side 1D tap tables of one axis.
struct AxisDev {
  int* base = nullptr;
  double* S = nullptr;   // [n][4]
  double* D1 = nullptr;
  double* D2 = nullptr;
  double* pts = nullptr;
};

struct Source {          // one V^(s) coupling source of a component (Eq. FM-pre right side)
  int beta = 0;          // particle label of the source pair
  int src = 0;           // index of the solved component whose expansion is evaluated
  double zsign = 1.0;    // -1: psi_2(x, y, z) = p (-1)^{M'} psi_1(x, y, -z) (Eq. 2-sym-part)
  bool sym = false;
};

// float32 copies of the operator tables (mixed-precision inner solves)
struct Tabs32 {
  float *Sx = nullptr, *D2x = nullptr, *Sy = nullptr, *D2y = nullptr, *Sz = nullptr, *D1z = nullptr, *D2z = nullptr;
  float *zp = nullptr, *W = nullptr, *A = nullptr, *B = nullptr, *iy2 = nullptr, *cval = nullptr, *cw = nullptr;
};

// double-float copies of the operator tables (mixed_scheme 2: double-float inner solves)
struct TabsDD {
  dd *Sx = nullptr, *D2x = nullptr, *Sy = nullptr, *D2y = nullptr, *Sz = nullptr, *D1z = nullptr, *D2z = nullptr;
  dd *zp = nullptr, *W = nullptr, *A = nullptr, *B = nullptr, *iy2 = nullptr, *cval = nullptr, *cw = nullptr;
};

struct Comp {
  int label = 0;                 // particle label alpha
  int r = 4;                     // taps per point of the component's basis (4 cubic, 6 quintic)
  int64_t ystage_off = 0;        // offset of the component in fm_ctx::ystage32 ([nM][nz][nx][nint_y][r])
  Tabs32 f32;
  TabsDD tdd;
  Axis ax, ay, az;
  int nx = 0, ny = 0, nz = 0;
  int64_t npts = 0, off = 0;     // points per M' block, offset in the vector
  double Rx = 0, Ry = 0;
  std::vector<Source> sources;
  // device tables
  AxisDev dx, dy, dz;
  double* W = nullptr;           // [nM][nz][nx][ny] V_a + sum V^(l)_b + q M'(M'+1) + (J(J+1)-2M'^2)/y^2, q = 1/x^2+1/y^2
  double* A = nullptr;           // [nz][nx][ny] q (1 - z^2)
  double* B = nullptr;           // [nM][nz][nx][ny] 2 (M'+1) z q
  double* iy2 = nullptr;         // [ny] 1/y^2
  // coupling tables: n_act active points, per (source s): taps and weights
  int n_act = 0;
  int* act_pt = nullptr;         // [n_act] point index (k*nx + i)*ny + j
  int* cpl_base = nullptr;       // [ns][3][n_act]  (z, x, y tap bases)
  double* cpl_val = nullptr;     // [ns][3 r][n_act] (Sz[r], Sx[r], Sy[r])
  double* cpl_w = nullptr;       // [ns][nM*nM][n_act] weight of (M', M'')
  // preconditioner, E-independent
  double* Wz = nullptr;          // [nM][nz][nz]
  double* Wzb = nullptr;         // [nM][nz][nz]
  double* Wx = nullptr;          // [nl][nx][nx], l = M0 .. J + nz - 1
  double* Wxb = nullptr;
  float* Wz32 = nullptr; float* Wzb32 = nullptr; float* Wx32 = nullptr; float* Wxb32 = nullptr;
  std::vector<double> Lz;        // [nM][nz] computed z eigenvalues
  std::vector<double> Lx;        // [nl][nx]
  int nl = 0;
  // preconditioner, E-dependent banded y systems: per l a group of nx lines
  std::vector<int> chain_lo, chain_n;   // per l: first iM and length of the M' chain
  int* d_chain_lo = nullptr; int* d_chain_n = nullptr;
  int64_t* d_band_off = nullptr; int64_t* d_lmul_off = nullptr; int64_t* d_piv_off = nullptr;
  std::vector<int64_t> band_off;        // per l: offset (in elements) of its group in yU / yL
  std::vector<int64_t> piv_off;
  int64_t band_total = 0, lmul_total = 0, piv_total = 0;
  double* yU = nullptr;          // per l: [n][kl+ku+1][nx], reciprocal pivot first
  double* yL = nullptr;          // per l: [n][kl+1][nx], slot 0 the pivot offset, then the multipliers
  float* yU32 = nullptr; float* yL32 = nullptr;
  std::vector<int64_t> lmul_off;
  // n_M = 1: per-l diagonalisation of (A_l, S_y), A_l = -D_y + (c_l Y_r2 + V^ - E*) S_y, used by the
  // float32 preconditioner (same inverse as the banded y solves)
  bool ydiag_ok = false;
  float* Wy32 = nullptr; float* Wyb32 = nullptr;   // [nl][ny][ny]
  float* dLy32 = nullptr;                          // [nl][ny]
  float* dLx32 = nullptr;                          // [nl][nx]
  double* Wy64 = nullptr; double* Wyb64 = nullptr; double* dLy64 = nullptr; double* dLx64 = nullptr;
  float2* dLx2 = nullptr;                          // [nl][nx] lambda_x as (hi, lo) float pairs
  float2* dLy2 = nullptr;                          // [nl][ny] lambda_y as (hi, lo) float pairs
  // tensor-core chain: TMA maps of the stage buffers and of the float32 W matrices
  // 0 t[slab][j][i], 1 u[slab][j][i], 2 W-bar_x, 3 W_x, 4 u[slab][i][j], 5 t[slab][i][j], 6 W-bar_y, 7 W_y
  CUtensorMap tm[8];
  // tensor-core z stages and the fused n_M = 1 x / y chain (BF16 or TF32 operands)
  void* Wz_tc = nullptr;         // [nM][nz][ldz] W_z, rows zero-padded to ldz (16-byte TMA strides)
  void* Wzb_tc = nullptr;        // [nM][nz][ldz] W-bar_z
  int ldz = 0;
  uint16_t *Wx16 = nullptr, *Wxb16 = nullptr, *Wy16 = nullptr, *Wyb16 = nullptr;  // BF16 copies
  CUtensorMap tmz[2];            // W-bar_z, W_z for the z-stage kernel
  CUtensorMap tmf[5];            // fused chain: slab t[slab][j][i], W-bar_x, W-bar_y, W_y, W_x
  bool tcz = false;              // z stages on the tensor cores
  int tcz_np[2] = {128, 128};    // their tile widths (points per tile), forward / inverse
  int x_pair_ls = 0;             // x pencils (values of l) with complex-conjugate pairs, kept in a real basis
  bool fused = false;            // n_M = 1: x / y stages in one kernel per slab (with the y diagonalisation)
};

}  // namespace fmi

struct fm_ctx {
  fm_system sys{};
  fm_splitting split{};
  fm_opts opts{};
  int device = 0;
  cudaStream_t stream = nullptr;
  bool pool_alloc = false;  // allocations stream-ordered on `stream` (cudaMallocAsync / cudaFreeAsync)
  int M0 = 0, nM = 0;
  std::vector<int> Mps;
  std::vector<fmi::Comp> comps;
  int64_t N = 0;
  double mu_pair[3]{}, mu_rel[3]{};
  // preconditioner state
  bool have_shift = false;
  double Estar = 0.0;
  // workspace
  double* P = nullptr;           // [N] y/x-pass planes for the apply (S_x S_y c)
  double* Q = nullptr;           // [N] (D_x S_y c)
  double* R = nullptr;           // [N] (S_x D_y c)
  float* P32 = nullptr; float* Q32 = nullptr; float* R32 = nullptr;  // float32 apply scratch
  double* t64 = nullptr;         // [N] preconditioner stage buffer
  double* u64 = nullptr;
  float* t32 = nullptr;
  float* u32 = nullptr;
  int m_alloc = 0;
  float* V32 = nullptr;          // float32 FGMRES basis [(m+1)][N] (mixed precision)
  float* Z32 = nullptr;          // [m][N]
  float* w32 = nullptr;          // [N]
  float* r32 = nullptr;          // [N]
  float* d32 = nullptr;          // [N]
  float* e32 = nullptr;          // [N]
  float* ystage32 = nullptr;     // float32 sources of the coupling regrouped by y interval (MIXED precision)
  bool use_dd = false;           // MIXED precision, mixed_scheme 2: double-float inner solves
  fmi::dd* Vdd = nullptr;             // their FGMRES basis [(m+1)][N]
  fmi::dd* Zdd = nullptr;             // [m][N]
  fmi::dd* wdd = nullptr;             // [N]
  fmi::dd* rdd = nullptr;             // [N]
  fmi::dd* bdd = nullptr;             // [N] right-hand side
  fmi::dd* xdd = nullptr;             // [N] solution
  double* V = nullptr;           // FGMRES basis [(m+1)][N]
  double* Z = nullptr;           // FGMRES preconditioned directions [m][N]
  double* w = nullptr;           // [N]
  double* r = nullptr;           // [N]
  double* red = nullptr;         // reduction scratch (per-block partial sums)
  double* gsd = nullptr;         // Gram-Schmidt coefficients and norms kept on the device
  unsigned* gs_cnt = nullptr;    // arrival counter of the last-block reductions
  double* tuneG_dev = nullptr;   // (U^T W)^{-1} of the tuned preconditioner, on the device
  double* red_host = nullptr;    // pinned
  int red_blocks = 0;
  // eigen workspace
  int ncv_alloc = 0;
  double* AV = nullptr;          // Arnoldi basis [(ncv+1)][N]
  double* tmpN = nullptr;        // [N]
  double* tmpN2 = nullptr;
  double* tmpN3 = nullptr;
  double* evec_stage = nullptr;  // fm_eigs_host staging (k vectors)
  int evec_stage_k = 0;
  // tuned preconditioner used by the eigen-solver: P_t = P + (A U - P U) U^T with orthonormal U
  // (n_tune columns), applied through P_t^{-1} = P^{-1} - (W - U) (U^T W)^{-1} U^T P^{-1}, W = P^{-1} A U
  int n_tune = 0;
  double* tuneU = nullptr;       // [8][N]
  double* tuneWU = nullptr;      // [8][N]  W - U
  std::vector<double> tuneGinv;  // (U^T W)^{-1}, n_tune x n_tune, row-major
  double normH = 0.0, normS = 0.0;  // power-iteration lower bounds of |H|_2 and |S|_2 (0 = not yet estimated)
  bool tc_active = false;        // float32 preconditioner x / y stages on the tensor cores
  bool bf16 = false;             // ... with BF16 operands (z stages and the fused chain), else TF32
  int* tc_err = nullptr;         // device flag: a bounded wait of a tensor-core kernel expired
  int64_t launches = 0;
  int64_t device_bytes = 0;
  // per-kernel timing (fm_profile)
  bool prof = false;
  std::vector<cudaEvent_t> ev_free;
  struct ProfRec { int cls; cudaEvent_t a, b; };
  std::vector<ProfRec> recs;
  double prof_ms[FM_NUM_KERNEL_CLASSES]{};
  int64_t prof_n[FM_NUM_KERNEL_CLASSES]{};
  double prof_flops[FM_NUM_KERNEL_CLASSES]{};   // algorithmic work of the recorded launches
  double prof_bytes[FM_NUM_KERNEL_CLASSES]{};
  std::vector<void*> allocs;
};

// helpers shared by the translation units
namespace fmi {
int dev_alloc(fm_ctx* c, void** p, size_t bytes);
int upload(fm_ctx* c, void** p, const void* host, size_t bytes);
int setup_host(fm_ctx* c, const fm_grid* grids, int n_grids);       // grids, tables, coupling, z/x decompositions
int setup_shift(fm_ctx* c, double Estar);                            // banded y systems
int estimate_bytes(const fm_system* S, const fm_grid* grids, int n_grids, const fm_splitting* split, const fm_opts* o,
                   int64_t* out);
// kernels (fm_kernels.cu)
int launch_apply(fm_ctx* c, double E, const double* x, double* y, bool only_S);
int launch_apply32(fm_ctx* c, double E, const float* x, float* y, bool only_S);
int launch_precond(fm_ctx* c, const double* x, double* y);
int launch_precond32(fm_ctx* c, const float* x, float* y);
int dot_many32(fm_ctx* c, const float* V, int64_t ldv, int nv, const float* w, double* h_host);
int axpy_many_norm32(fm_ctx* c, const float* V, int64_t ldv, int nv, const double* h_host, float sign, float* w,
                     double* nrm2_out);
int to32(fm_ctx* c, const double* x, double a, float* y);
int add32(fm_ctx* c, const float* y, double a, double* x);
int axpby32(fm_ctx* c, float a, const float* x, float b, float* y);
int dot_many(fm_ctx* c, const double* V, int64_t ldv, int nv, const double* w, double* h_host);
int dot_many_x(fm_ctx* c, const double* V, int64_t ldv, int nv, const double* w, const double* extra, double* h_host);
int axpy_many(fm_ctx* c, const double* V, int64_t ldv, int nv, const double* h_host, double* w, double sign);
int dot_many_dev(fm_ctx* c, const double* V, int64_t ldv, int nv, const double* w, const double* extra, double* h_dev,
                 bool lowp = false);
int gs_cgs2(fm_ctx* c, const double* V, int nv, double* w, double* vout, double* h, double* hn);
int gs_cgs1(fm_ctx* c, const double* V, int nv, double* w, double* vout, double* h, double* hn);
int gs_cgs2_32(fm_ctx* c, const float* V, int nv, float* w, float* vout, double* h, double* hn);
// double-float inner solves (mixed_scheme 2)
int launch_apply_dd(fm_ctx* c, double E, const dd* x, dd* y, bool only_S);
int launch_precond_dd(fm_ctx* c, const dd* x, dd* y);  // the float32 tensor preconditioner on the leading parts
int to_dd(fm_ctx* c, const double* x, double a, dd* y);    // y = a x
int add_dd(fm_ctx* c, const dd* y, double a, double* x);   // x += a y
int axpby_dd(fm_ctx* c, double a, const dd* x, double b, dd* y);  // y = a x + b y
int dot_many_dd(fm_ctx* c, const dd* V, int64_t ldv, int nv, const dd* w, double* h_host);
int axpy_many_dd(fm_ctx* c, const dd* V, int64_t ldv, int nv, const double* h_host, dd* w);  // w += sum h_j V_j
int gs_cgs2_dd(fm_ctx* c, const dd* V, int nv, dd* w, dd* vout, double* h, double* hn);
int tuning_correct(fm_ctx* c, const double* U, const double* WmU, const double* Gdev, int k, double* z);
int scale_copy(fm_ctx* c, const double* x, double a, double* y);   // y = a x
int axpby(fm_ctx* c, double a, const double* x, double b, double* y);  // y = a x + b y
int fill_normal(fm_ctx* c, double* x, uint64_t seed);
int combine(fm_ctx* c, const double* V, int64_t ldv, int nv, const double* Q_host, int nc, double* out, int64_t ldo);
int absmax(fm_ctx* c, const double* x, double* val);
int kernels_init(fm_ctx* c);
int launch_apply_scratch(fm_ctx* c, double E, const double* x, double* y, double* P, double* Q, double* R);
// timing helpers: begin() returns a token for end(); no-ops unless profiling
int prof_begin(fm_ctx* c, int cls);
void prof_end(fm_ctx* c, int token, double flops, double bytes);
int prof_harvest(fm_ctx* c);   // after a stream synchronisation: fold finished records
// tensor-core preconditioner stages (fm_tc.cu)
bool tc_component_ok(const Comp& cp);
int tc_setup(fm_ctx* c);       // after the stage buffers exist: encode the TMA maps
int tc_kernels_init();
int tc_check(fm_ctx* c);       // FM_ERR_TIMEOUT when a tensor-core kernel gave up a wait
int* tc_flag_slot(fm_ctx* c);  // the wait flag's place in the Gram-Schmidt result buffer (read every step)
// tensor-core chain over all components: z and x forward (+ y for the diagonalised n_M = 1 form, fused
// per slab where eligible); the components left for the banded y solves are returned in 'banded'
template <typename TIO>
int precond_tc_front(fm_ctx* c, const TIO* x, std::vector<Comp*>* banded);
template <typename TIO>
int precond_tc_back(fm_ctx* c, TIO* y);                                 // x, z inverse
bool tc_uses_ydiag(const fm_ctx* c, const Comp& cp);                    // the n_M = 1 y diagonalisation runs
uint16_t f2bf(float v);                                                 // float -> bfloat16 bits (nearest even)
}  // namespace fmi

#define FM_CUDA(call)                                   \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return FM_ERR_CUDA;          \
  } while (0)
