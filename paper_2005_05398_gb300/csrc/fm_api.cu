// The C ABI of libfm (include/fm.h): context life cycle, operator and preconditioner
// applications, the FGMRES linear solver and the shift-invert Arnoldi eigensolver
// (Eq. FM-lin; the paper runs IRAM (ARPACK) around a preconditioned GMRES, Section 4).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "fm_dense.h"
#include "fm_internal.h"

namespace fmi {

// Context memory is stream-ordered on the context's stream where the device has memory pools: its release
// (cudaFreeAsync) then waits for that stream only, so a context destroyed beside others running on their own
// streams (the request loop) does not stall them as a device-wide cudaFree would.
int dev_alloc(fm_ctx* c, void** p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  cudaError_t e = c->pool_alloc ? cudaMallocAsync(p, bytes, c->stream) : cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return FM_ERR_OOM;
  }
  c->allocs.push_back(*p);
  c->device_bytes += (int64_t)bytes;
  return FM_OK;
}

int upload(fm_ctx* c, void** p, const void* host, size_t bytes) {
  int rc = dev_alloc(c, p, bytes);
  if (rc) return rc;
  if (bytes) {
    FM_CUDA(cudaMemcpyAsync(*p, host, bytes, cudaMemcpyHostToDevice, c->stream));
    FM_CUDA(cudaStreamSynchronize(c->stream));
  }
  return FM_OK;
}

static double wall_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

static int nrm2(fm_ctx* c, const double* v, double* out) {
  double h = 0.0;
  int rc = dot_many(c, v, c->N, 1, v, &h);
  *out = std::sqrt(std::max(h, 0.0));
  return rc;
}

// z <- P_t^{-1}-correction of z = P^{-1} v:  z -= (W - U) (U^T W)^{-1} (U^T z)
static int apply_tuning(fm_ctx* c, double* z) {
  return tuning_correct(c, c->tuneU, c->tuneWU, c->tuneG_dev, c->n_tune, z);
}

// Tune the preconditioner to the columns of U (device, orthonormal, k <= 8): W = P^{-1} (H - E S) U.
static int set_tuning(fm_ctx* c, double E, const double* U, int k) {
  int rc;
  c->n_tune = 0;
  if (k <= 0) return FM_OK;
  const int64_t N = c->N;
  FM_CUDA(cudaMemcpyAsync(c->tuneU, U, (size_t)k * N * 8, cudaMemcpyDeviceToDevice, c->stream));
  std::vector<double> G((size_t)k * k);
  for (int j = 0; j < k; ++j) {
    double* wj = c->tuneWU + (int64_t)j * N;
    if ((rc = launch_apply(c, E, c->tuneU + (int64_t)j * N, c->tmpN2, false))) return rc;
    if ((rc = launch_precond(c, c->tmpN2, wj))) return rc;
    std::vector<double> col(k);
    if ((rc = dot_many(c, c->tuneU, N, k, wj, col.data()))) return rc;  // U^T w_j
    for (int i = 0; i < k; ++i) G[(size_t)i * k + j] = col[i];
    if ((rc = axpby(c, -1.0, c->tuneU + (int64_t)j * N, 1.0, wj))) return rc;  // w_j - u_j
  }
  c->tuneGinv.assign((size_t)k * k, 0.0);
  if (!fmh::invert(k, G.data(), c->tuneGinv.data())) return FM_OK;  // singular: leave untuned
  FM_CUDA(cudaMemcpy(c->tuneG_dev, c->tuneGinv.data(), (size_t)k * k * sizeof(double), cudaMemcpyHostToDevice));
  c->n_tune = k;
  return FM_OK;
}

// Right-preconditioned restarted FGMRES for (H - E S) x = b (x: initial guess in, solution out).
static int fgmres32(fm_ctx* c, double E, const float* b, float* d, double tol, int max_iters, int* iters_out);

// Relative residual of each float32 inner solve in FM_PREC_MIXED (0 selects the scheme's default).
static double inner_tol32(const fm_ctx* c) {
  if (c->opts.inner_tol32 > 0.0) return c->opts.inner_tol32;
  return c->opts.mixed_scheme == 0 ? 1e-3 : (c->opts.mixed_scheme == 2 ? 1e-6 : 3e-5);
}

// Preconditioner step of the flexible scheme: z <- float32 FGMRES solution of (H - E S) z = v for a unit
// float64 vector v (float32 operator, preconditioner and basis), widened to float64.
static int precond_flex32(fm_ctx* c, double E, const double* v, double* z, int max_iters, int* iters) {
  int rc;
  if ((rc = to32(c, v, 1.0, c->d32))) return rc;
  if ((rc = fgmres32(c, E, c->d32, c->e32, inner_tol32(c), max_iters, iters))) return rc;
  FM_CUDA(cudaMemsetAsync(z, 0, c->N * sizeof(double), c->stream));
  return add32(c, c->e32, 1.0, z);
}

// double-float right-preconditioned FGMRES for (H - E S) d = b (double-float operator and basis, the
// float32 tensor preconditioner on the leading parts; Givens and the small least-squares problem in float64).
// d starts at zero.  Mirrors fgmres32.
static int fgmres_dd(fm_ctx* c, double E, const fmi::dd* b, fmi::dd* d, double tol, int max_iters, int* iters_out) {
  using fmi::dd;
  int rc;
  const int m = c->opts.restart_m;
  const int64_t N = c->N;
  double b2;
  if ((rc = dot_many_dd(c, b, N, 1, b, &b2))) return rc;
  const double bnorm = std::sqrt(std::max(b2, 0.0));
  *iters_out = 0;
  FM_CUDA(cudaMemsetAsync(d, 0, N * sizeof(dd), c->stream));
  if (!(bnorm > 0.0)) return FM_OK;
  dd* r = c->rdd;
  FM_CUDA(cudaMemcpyAsync(r, b, N * sizeof(dd), cudaMemcpyDeviceToDevice, c->stream));
  double beta = bnorm, beta_prev = HUGE_VAL;
  std::vector<double> R((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), h(m + 1), y(m);
  int total = 0;
  while (beta > tol * bnorm && total < max_iters && beta <= 0.5 * beta_prev) {
    beta_prev = beta;
    if ((rc = axpby_dd(c, 1.0 / beta, r, 0.0, c->Vdd))) return rc;
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int jdone = 0;
    for (int j = 0; j < m && total < max_iters; ++j) {
      dd* Vj = c->Vdd + (int64_t)j * N;
      dd* Zj = c->Zdd + (int64_t)j * N;
      if ((rc = launch_precond_dd(c, Vj, Zj))) return rc;
      if ((rc = launch_apply_dd(c, E, Zj, c->wdd, false))) return rc;
      double hn;  // CGS2 writes the next basis vector Vdd[j+1] = (w - V h) / hn
      if ((rc = gs_cgs2_dd(c, c->Vdd, j + 1, c->wdd, c->Vdd + (int64_t)(j + 1) * N, h.data(), &hn))) return rc;
      if (!std::isfinite(hn)) return FM_ERR_BREAKDOWN;
      for (int i = 0; i < j; ++i) {
        const double t = cs[i] * h[i] + sn[i] * h[i + 1];
        h[i + 1] = -sn[i] * h[i] + cs[i] * h[i + 1];
        h[i] = t;
      }
      const double rr = std::hypot(h[j], hn);
      cs[j] = (rr == 0.0) ? 1.0 : h[j] / rr;
      sn[j] = (rr == 0.0) ? 0.0 : hn / rr;
      h[j] = rr;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      for (int i = 0; i <= j; ++i) R[(size_t)i * m + j] = h[i];
      ++total;
      jdone = j + 1;
      if (std::fabs(g[j + 1]) <= tol * bnorm || hn == 0.0) break;
    }
    for (int i = jdone - 1; i >= 0; --i) {
      double sacc = g[i];
      for (int k = i + 1; k < jdone; ++k) sacc -= R[(size_t)i * m + k] * y[k];
      if (R[(size_t)i * m + i] == 0.0) return FM_ERR_BREAKDOWN;
      y[i] = sacc / R[(size_t)i * m + i];
    }
    if ((rc = axpy_many_dd(c, c->Zdd, N, jdone, y.data(), d))) return rc;
    if ((rc = launch_apply_dd(c, E, d, c->wdd, false))) return rc;  // double-float residual r = b - A d
    if ((rc = axpby_dd(c, 1.0, b, 0.0, r))) return rc;
    if ((rc = axpby_dd(c, -1.0, c->wdd, 1.0, r))) return rc;
    double r2;
    if ((rc = dot_many_dd(c, r, N, 1, r, &r2))) return rc;
    beta = std::sqrt(std::max(r2, 0.0));
    if (!std::isfinite(beta)) return FM_ERR_BREAKDOWN;
  }
  *iters_out = total;
  return FM_OK;
}

// Preconditioner step of the flexible scheme with double-float inner solves (mixed_scheme 2).
// Its inner tolerance: fm_opts.inner_tol32 when set; by default half the outer tolerance, so that one
// double-float Krylov space does the work (the float64 outer iteration then checks the true residual and
// corrects what the double-float rounding left), but not below 3e-9, above the double-float rounding floor
// of the operator (about 1e-14 relative per operation times its conditioning), where an inner solve
// would only stagnate.
static int precond_flexdd(fm_ctx* c, double E, const double* v, double* z, int max_iters, int* iters,
                          double tol_outer) {
  int rc;
  const double tin = c->opts.inner_tol32 > 0.0 ? c->opts.inner_tol32 : std::max(0.5 * tol_outer, 3e-9);
  if ((rc = to_dd(c, v, 1.0, c->bdd))) return rc;
  if ((rc = fgmres_dd(c, E, c->bdd, c->xdd, tin, max_iters, iters))) return rc;
  FM_CUDA(cudaMemsetAsync(z, 0, c->N * sizeof(double), c->stream));
  return add_dd(c, c->xdd, 1.0, z);
}

// Right-preconditioned flexible GMRES (restart m) for (H - E S) x = b on the float64 operator.  The
// preconditioner step is the tensor preconditioner (FP64 / FP32 modes, optionally tuned) or, with flex32, a
// float32 FGMRES solve (FM_PREC_MIXED, flexible scheme); iters_out then counts the float32 iterations and
// restarts_out the float64 outer iterations.
static int fgmres(fm_ctx* c, double E, const double* b, double* x, double tol, int max_iters, int* iters_out,
                  int* restarts_out, double* resid_out, bool flex32 = false) {
  int rc;
  const int m = c->opts.restart_m;
  const int64_t N = c->N;
  double bnorm;
  if ((rc = nrm2(c, b, &bnorm))) return rc;
  *iters_out = 0;
  *restarts_out = 0;
  if (!(bnorm > 0.0)) {
    FM_CUDA(cudaMemsetAsync(x, 0, N * sizeof(double), c->stream));
    *resid_out = 0.0;
    return std::isfinite(bnorm) ? FM_OK : FM_ERR_BREAKDOWN;
  }
  double* r = c->r;
  if ((rc = launch_apply(c, E, x, r, false))) return rc;
  if ((rc = axpby(c, 1.0, b, -1.0, r))) return rc;
  double beta;
  if ((rc = nrm2(c, r, &beta))) return rc;
  std::vector<double> R((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), h(m + 1), y(m);
  int total = 0, inner32 = 0, outer = 0;
  bool converged = false;
  double beta_prev = HUGE_VAL;
  while (true) {
    if (!std::isfinite(beta)) return FM_ERR_BREAKDOWN;
    if (beta <= tol * bnorm) {
      converged = true;
      break;
    }
    if (total >= max_iters) break;
    // a whole restart cycle that did not halve the true residual: the float64 residual has
    // reached its rounding floor (about eps ||A|| ||x||), further cycles only chase noise
    if (beta > 0.5 * beta_prev) break;
    beta_prev = beta;
    if ((rc = scale_copy(c, r, 1.0 / beta, c->V))) return rc;
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int jdone = 0;
    for (int j = 0; j < m && total < max_iters; ++j) {
      double* Vj = c->V + (int64_t)j * N;
      double* Zj = c->Z + (int64_t)j * N;
      if (flex32) {
        int it = 0;
        if (c->use_dd) rc = precond_flexdd(c, E, Vj, Zj, std::max(1, max_iters - total), &it, tol);
        else rc = precond_flex32(c, E, Vj, Zj, std::max(1, max_iters - total), &it);
        if (rc) return rc;
        inner32 += it;
        total += std::max(it, 1) - 1;  // the float32 iterations count against max_iters (+1 below)
        ++outer;
      } else {
        if ((rc = launch_precond(c, Vj, Zj))) return rc;
        if ((rc = apply_tuning(c, Zj))) return rc;
      }
      if ((rc = launch_apply(c, E, Zj, c->w, false))) return rc;
      double hn;  // Gram-Schmidt writes the next basis vector V[j+1] = (w - V h) / hn
      if (c->opts.gram_schmidt == 1) rc = gs_cgs1(c, c->V, j + 1, c->w, c->V + (int64_t)(j + 1) * N, h.data(), &hn);
      else rc = gs_cgs2(c, c->V, j + 1, c->w, c->V + (int64_t)(j + 1) * N, h.data(), &hn);
      if (rc) return rc;
      if (!std::isfinite(hn)) return FM_ERR_BREAKDOWN;
      for (int i = 0; i < j; ++i) {  // previous Givens rotations
        const double t = cs[i] * h[i] + sn[i] * h[i + 1];
        h[i + 1] = -sn[i] * h[i] + cs[i] * h[i + 1];
        h[i] = t;
      }
      const double rr = std::hypot(h[j], hn);
      cs[j] = (rr == 0.0) ? 1.0 : h[j] / rr;
      sn[j] = (rr == 0.0) ? 0.0 : hn / rr;
      h[j] = rr;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      for (int i = 0; i <= j; ++i) R[(size_t)i * m + j] = h[i];
      ++total;
      jdone = j + 1;
      if (std::fabs(g[j + 1]) <= tol * bnorm || hn == 0.0) break;
    }
    for (int i = jdone - 1; i >= 0; --i) {  // R y = g
      double s = g[i];
      for (int k = i + 1; k < jdone; ++k) s -= R[(size_t)i * m + k] * y[k];
      if (R[(size_t)i * m + i] == 0.0) return FM_ERR_BREAKDOWN;
      y[i] = s / R[(size_t)i * m + i];
    }
    if ((rc = axpy_many(c, c->Z, N, jdone, y.data(), x, 1.0))) return rc;
    ++*restarts_out;
    if ((rc = launch_apply(c, E, x, r, false))) return rc;
    if ((rc = axpby(c, 1.0, b, -1.0, r))) return rc;
    if ((rc = nrm2(c, r, &beta))) return rc;
  }
  *iters_out = flex32 ? inner32 : total;
  if (flex32) *restarts_out = outer;
  *resid_out = beta / bnorm;
  return converged ? FM_OK : FM_ERR_NOT_CONVERGED;
}

// float32 right-preconditioned FGMRES for (H - E S) d = b (float32 operator, preconditioner and basis;
// Givens and the small least-squares problem in float64).  d starts at zero.
static int fgmres32(fm_ctx* c, double E, const float* b, float* d, double tol, int max_iters, int* iters_out) {
  int rc;
  const int m = c->opts.restart_m;
  const int64_t N = c->N;
  double b2;
  if ((rc = dot_many32(c, b, N, 1, b, &b2))) return rc;
  const double bnorm = std::sqrt(std::max(b2, 0.0));
  *iters_out = 0;
  FM_CUDA(cudaMemsetAsync(d, 0, N * sizeof(float), c->stream));
  if (!(bnorm > 0.0)) return FM_OK;
  float* r = c->r32;
  FM_CUDA(cudaMemcpyAsync(r, b, N * sizeof(float), cudaMemcpyDeviceToDevice, c->stream));
  double beta = bnorm, beta_prev = HUGE_VAL;
  std::vector<double> R((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), h(m + 1), y(m);
  int total = 0;
  while (beta > tol * bnorm && total < max_iters && beta <= 0.5 * beta_prev) {
    beta_prev = beta;
    if ((rc = axpby32(c, (float)(1.0 / beta), r, 0.0f, c->V32))) return rc;
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int jdone = 0;
    for (int j = 0; j < m && total < max_iters; ++j) {
      float* Vj = c->V32 + (int64_t)j * N;
      float* Zj = c->Z32 + (int64_t)j * N;
      if ((rc = launch_precond32(c, Vj, Zj))) return rc;
      if ((rc = launch_apply32(c, E, Zj, c->w32, false))) return rc;
      double hn;  // CGS2 writes the next basis vector V32[j+1] = (w - V h) / hn
      if ((rc = gs_cgs2_32(c, c->V32, j + 1, c->w32, c->V32 + (int64_t)(j + 1) * N, h.data(), &hn))) return rc;
      if (!std::isfinite(hn)) return FM_ERR_BREAKDOWN;
      for (int i = 0; i < j; ++i) {
        const double t = cs[i] * h[i] + sn[i] * h[i + 1];
        h[i + 1] = -sn[i] * h[i] + cs[i] * h[i + 1];
        h[i] = t;
      }
      const double rr = std::hypot(h[j], hn);
      cs[j] = (rr == 0.0) ? 1.0 : h[j] / rr;
      sn[j] = (rr == 0.0) ? 0.0 : hn / rr;
      h[j] = rr;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      for (int i = 0; i <= j; ++i) R[(size_t)i * m + j] = h[i];
      ++total;
      jdone = j + 1;
      if (std::fabs(g[j + 1]) <= tol * bnorm || hn == 0.0) break;
    }
    for (int i = jdone - 1; i >= 0; --i) {
      double sacc = g[i];
      for (int k = i + 1; k < jdone; ++k) sacc -= R[(size_t)i * m + k] * y[k];
      if (R[(size_t)i * m + i] == 0.0) return FM_ERR_BREAKDOWN;
      y[i] = sacc / R[(size_t)i * m + i];
    }
    if ((rc = axpy_many_norm32(c, c->Z32, N, jdone, y.data(), 1.0f, d, nullptr))) return rc;
    if ((rc = launch_apply32(c, E, d, c->w32, false))) return rc;  // float32 residual r = b - A d
    if ((rc = axpby32(c, 1.0f, b, 0.0f, r))) return rc;
    if ((rc = axpby32(c, -1.0f, c->w32, 1.0f, r))) return rc;
    double r2;
    if ((rc = dot_many32(c, r, N, 1, r, &r2))) return rc;
    beta = std::sqrt(std::max(r2, 0.0));
    if (!std::isfinite(beta)) return FM_ERR_BREAKDOWN;
  }
  *iters_out = total;
  return FM_OK;
}

// Mixed precision: float64 iterative refinement (true residual r = b - (H - E S) x in float64)
// around float32 FGMRES corrections, each solved to the relative residual opts.inner_tol32.
static int ir_solve(fm_ctx* c, double E, const double* b, double* x, double tol, int max_iters, int* iters_out,
                    int* outer_out, double* resid_out) {
  int rc;
  double bnorm;
  if ((rc = nrm2(c, b, &bnorm))) return rc;
  *iters_out = 0;
  *outer_out = 0;
  if (!(bnorm > 0.0)) {
    FM_CUDA(cudaMemsetAsync(x, 0, c->N * sizeof(double), c->stream));
    *resid_out = 0.0;
    return std::isfinite(bnorm) ? FM_OK : FM_ERR_BREAKDOWN;
  }
  double* r = c->r;
  if ((rc = launch_apply(c, E, x, r, false))) return rc;
  if ((rc = axpby(c, 1.0, b, -1.0, r))) return rc;
  double beta;
  if ((rc = nrm2(c, r, &beta))) return rc;
  double beta_prev = HUGE_VAL;
  int total = 0;
  bool converged = false;
  while (true) {
    if (!std::isfinite(beta)) return FM_ERR_BREAKDOWN;
    if (beta <= tol * bnorm) {
      converged = true;
      break;
    }
    if (total >= max_iters || beta > 0.5 * beta_prev) break;
    beta_prev = beta;
    if ((rc = to32(c, r, 1.0 / beta, c->d32))) return rc;  // normalised residual as the float32 right-hand side
    int it = 0;
    if ((rc = fgmres32(c, E, c->d32, c->e32, inner_tol32(c), max_iters - total, &it))) return rc;
    total += it;
    ++*outer_out;
    if ((rc = add32(c, c->e32, beta, x))) return rc;  // x += beta * correction
    if ((rc = launch_apply(c, E, x, r, false))) return rc;
    if ((rc = axpby(c, 1.0, b, -1.0, r))) return rc;
    if ((rc = nrm2(c, r, &beta))) return rc;
  }
  *iters_out = total;
  *resid_out = beta / bnorm;
  return converged ? FM_OK : FM_ERR_NOT_CONVERGED;
}

// (H - E S) x = b with the context's precision mode: float64 FGMRES (modes 0, 1) or float64
// iterative refinement around float32 FGMRES (mode 2).
static int solve_any(fm_ctx* c, double E, const double* b, double* x, double tol, int max_iters, int* iters_out,
                     int* restarts_out, double* resid_out) {
  if (c->opts.precision == FM_PREC_MIXED) {
    if (c->opts.mixed_scheme == 1) return ir_solve(c, E, b, x, tol, max_iters, iters_out, restarts_out, resid_out);
    return fgmres(c, E, b, x, tol, max_iters, iters_out, restarts_out, resid_out, true);
  }
  return fgmres(c, E, b, x, tol, max_iters, iters_out, restarts_out, resid_out);
}

// Householder-free modified Gram-Schmidt QR of an m x k matrix (row-major), twice.
static bool small_qr(int m, int k, std::vector<double>& Y) {
  for (int pass = 0; pass < 2; ++pass)
    for (int j = 0; j < k; ++j) {
      for (int i = 0; i < j; ++i) {
        double d = 0.0;
        for (int r = 0; r < m; ++r) d += Y[(size_t)r * k + i] * Y[(size_t)r * k + j];
        for (int r = 0; r < m; ++r) Y[(size_t)r * k + j] -= d * Y[(size_t)r * k + i];
      }
      double nr = 0.0;
      for (int r = 0; r < m; ++r) nr += Y[(size_t)r * k + j] * Y[(size_t)r * k + j];
      nr = std::sqrt(nr);
      if (!(nr > 1e-14)) return false;
      for (int r = 0; r < m; ++r) Y[(size_t)r * k + j] /= nr;
    }
  return true;
}

struct Ritz {
  double theta;
  int col;
  bool real;
};

// Lower bounds of |H|_2 and |S|_2: the largest |A v| over four normalised power steps from a seeded
// start (|A v| <= |A|_2 for every unit v).  The backward error of fm_eigs divides by them, so an
// underestimate can only make the reported error larger.  Computed once per context.
static int operator_norms(fm_ctx* c, double* nH, double* nS) {
  int rc;
  if (!(c->normH > 0.0 && c->normS > 0.0)) {
    double est[2] = {0.0, 0.0};
    for (int which = 0; which < 2; ++which) {
      double* v = c->tmpN;
      double* w = c->tmpN2;
      if ((rc = fill_normal(c, v, 0x5eedf00dull + (uint64_t)which))) return rc;
      double nv;
      if ((rc = nrm2(c, v, &nv))) return rc;
      if ((rc = scale_copy(c, v, 1.0 / nv, v))) return rc;
      for (int it = 0; it < 4; ++it) {
        if ((rc = launch_apply(c, 0.0, v, w, which == 1))) return rc;
        double nw;
        if ((rc = nrm2(c, w, &nw))) return rc;
        if (!(nw > 0.0) || !std::isfinite(nw)) return FM_ERR_NUMERIC;
        est[which] = std::max(est[which], nw);
        if ((rc = scale_copy(c, w, 1.0 / nw, v))) return rc;
      }
    }
    c->normH = est[0];
    c->normS = est[1];
  }
  *nH = c->normH;
  *nS = c->normS;
  return FM_OK;
}

// Float64 certificate of the pair (E, c) with |c| = 1: the backward error eta = |H c - E S c| / (|H| + |E| |S|),
// |H c - E S c| / |S c|, and the Rayleigh estimate E_R = (S c)^T (H c) / |S c|^2 (the E that minimises the
// residual, reported as a consistency check).  Uses tmpN and tmpN2.
static int certify(fm_ctx* c, const double* cv, double E, double nH, double nS, double* eta, double* resS,
                   double* E_R) {
  int rc;
  double* Hc = c->tmpN;
  double* Sc = c->tmpN2;
  if ((rc = launch_apply(c, 0.0, cv, Hc, false))) return rc;
  if ((rc = launch_apply(c, 0.0, cv, Sc, true))) return rc;
  double sh = 0.0, ss = 0.0;
  if ((rc = dot_many(c, Sc, c->N, 1, Hc, &sh)) || (rc = dot_many(c, Sc, c->N, 1, Sc, &ss))) return rc;
  if (!(ss > 0.0) || !std::isfinite(ss) || !std::isfinite(sh)) return FM_ERR_BREAKDOWN;
  *E_R = sh / ss;
  if ((rc = axpby(c, -E, Sc, 1.0, Hc))) return rc;  // Hc <- H c - E S c
  double rn;
  if ((rc = nrm2(c, Hc, &rn))) return rc;
  *eta = rn / (nH + std::fabs(E) * nS);
  *resS = rn / std::sqrt(ss);
  return FM_OK;
}

}  // namespace fmi

using namespace fmi;

extern "C" {

void fm_default_opts(fm_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->tol = 1e-12;
  o->restart_m = 64;
  o->max_iters = 2000;
  o->precision = FM_PREC_FP64;
  o->ncv = 20;
  o->max_restarts = 50;
  o->eig_tol = 1e-9;
  o->z_eigs = 0;
  o->tune = 0;
  o->y_solver = 0;
  o->mma = FM_MMA_AUTO;
  o->start_filter = -1;
  o->refine = 2;
  o->inner_tol32 = 0.0;
  o->tc_chain = 0;
  o->gram_schmidt = 0;
  o->mixed_scheme = 0;
  o->z_tile = 0;
  o->device = 0;
  o->stream = nullptr;
}

const char* fm_strerror(int s) {
  switch (s) {
    case FM_OK: return "ok";
    case FM_ERR_ARG: return "invalid argument";
    case FM_ERR_OOM: return "out of memory";
    case FM_ERR_CUDA: return "CUDA runtime error";
    case FM_ERR_NOT_CONVERGED: return "iteration limit reached without convergence";
    case FM_ERR_BREAKDOWN: return "Krylov breakdown (zero or non-finite norm)";
    case FM_ERR_COMPLEX_SPECTRUM: return "a 1D generalized eigenproblem has complex eigenvalues";
    case FM_ERR_NO_SHIFT: return "preconditioner used before fm_set_shift";
    case FM_ERR_NUMERIC: return "singular or non-finite set-up quantity";
    case FM_ERR_SCRATCH_LIMIT: return "problem larger than the fixed scratch of fm_apply_noalloc (FM_NOALLOC_MAX_UNKNOWNS)";
    case FM_ERR_TIMEOUT: return "a bounded wait inside a device kernel expired";
    default: return "unknown status";
  }
}

void fm_destroy(fm_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  for (auto& r : c->recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : c->ev_free) cudaEventDestroy(e);
  if (c->pool_alloc) {
    for (void* p : c->allocs) cudaFreeAsync(p, c->stream);
    cudaStreamSynchronize(c->stream);  // the memory is back in the pool when fm_destroy returns
  } else {
    for (void* p : c->allocs) cudaFree(p);
  }
  if (c->red_host) cudaFreeHost(c->red_host);
  delete c;
}

int fm_create(const fm_system* sys, const fm_grid* grids, int n_grids, const fm_splitting* split, const fm_opts* opts,
              fm_ctx** out) {
  if (!out) return FM_ERR_ARG;
  *out = nullptr;
  if (!sys || !grids || !split || n_grids < 1) return FM_ERR_ARG;
  fm_opts o;
  if (opts) o = *opts;
  else fm_default_opts(&o);
  if (sys->J < 0 || (sys->tau != 1 && sys->tau != -1) || (sys->exch_p != 1 && sys->exch_p != -1)) return FM_ERR_ARG;
  if (sys->identical_pair != 0 && sys->identical_pair != 12) return FM_ERR_ARG;
  for (int i = 0; i < 3; ++i)
    if (!(sys->mass[i] > 0.0) || !std::isfinite(sys->charge[i])) return FM_ERR_ARG;
  if (sys->identical_pair == 12 && (sys->mass[0] != sys->mass[1] || sys->charge[0] != sys->charge[1])) return FM_ERR_ARG;
  if (split->mode < 0 || split->mode > 2 || !(split->nu > 0) || !(split->x0 > 0) || !(split->y0 > 0) || split->vs_cut < 0)
    return FM_ERR_ARG;
  const int M0 = (1 - sys->tau) / 2, nM = sys->J - M0 + 1;
  if (nM <= 0 || nM > 12) return FM_ERR_ARG;
  if (o.z_eigs == 1 && nM != 1) return FM_ERR_ARG;
  if (o.restart_m < 1 || o.restart_m > 256 || o.max_iters < 1 || !(o.tol > 0) || o.ncv < 3 || o.ncv > 64 ||
      o.max_restarts < 0 || !(o.eig_tol > 0) || o.precision < 0 || o.precision > 2 || o.y_solver < 0 ||
      o.y_solver > 2 || o.mma < 0 || o.mma > 3 || o.start_filter < -1 || o.start_filter > 16 || o.refine < 0 || o.refine > 8 ||
      !(o.inner_tol32 == 0.0 || (o.inner_tol32 >= 1e-7 && o.inner_tol32 <= 0.5)) || o.gram_schmidt < 0 ||
      o.gram_schmidt > 1 || o.mixed_scheme < 0 || o.mixed_scheme > 2 ||
      !(o.z_tile == 0 || (((o.z_tile & ~256) == 32 || (o.z_tile & ~256) == 64 || (o.z_tile & ~256) == 128) &&
        (o.z_tile & ~(256 | 255)) == 0)) ||
      o.tc_chain < 0 || o.tc_chain > 1 || (o.tc_chain == 1 && o.mma == FM_MMA_BF16))
    return FM_ERR_ARG;
  fm_ctx* c = new fm_ctx();
  c->sys = *sys;
  c->split = *split;
  c->opts = o;
  c->device = o.device;
  c->stream = (cudaStream_t)o.stream;
  c->M0 = M0;
  c->nM = nM;
  for (int i = 0; i < nM; ++i) c->Mps.push_back(M0 + i);
  int rc = FM_OK;
  auto fail = [&](int e) {
    fm_destroy(c);
    return e;
  };
  const bool verbose = getenv("FM_VERBOSE") != nullptr;
  double tph = wall_ms();
  auto phase = [&](const char* what) {
    if (!verbose) return;
    const double now = wall_ms();
    fprintf(stderr, "[fm_create] %-26s %8.1f ms\n", what, now - tph);
    tph = now;
  };
  if (cudaSetDevice(c->device) != cudaSuccess) return fail(FM_ERR_CUDA);
  {
    int pools = 0;
    if (cudaDeviceGetAttribute(&pools, cudaDevAttrMemoryPoolsSupported, c->device) != cudaSuccess) return fail(FM_ERR_CUDA);
    c->pool_alloc = pools != 0;
  }
  if ((rc = kernels_init(c))) return fail(rc);
  phase("kernel attributes");
  c->use_dd = o.precision == FM_PREC_MIXED && o.mixed_scheme == 2;
  if ((rc = setup_host(c, grids, n_grids))) return fail(rc);
  phase("tables and decompositions");
  const int64_t N = c->N;
  const int m = o.restart_m;
  c->red_blocks = 4 * 152;  // reduction blocks: four per SM
  if ((rc = dev_alloc(c, (void**)&c->P, N * 8)) || (rc = dev_alloc(c, (void**)&c->Q, N * 8)) ||
      (rc = dev_alloc(c, (void**)&c->R, N * 8)) || (rc = dev_alloc(c, (void**)&c->t64, N * 8)) ||
      (rc = dev_alloc(c, (void**)&c->u64, N * 8)) || (rc = dev_alloc(c, (void**)&c->t32, N * 4)) ||
      (rc = dev_alloc(c, (void**)&c->u32, N * 4)) || (rc = dev_alloc(c, (void**)&c->V, (size_t)(m + 1) * N * 8)) ||
      (rc = dev_alloc(c, (void**)&c->Z, (size_t)std::max(m, o.ncv) * N * 8)) || (rc = dev_alloc(c, (void**)&c->w, N * 8)) ||
      (rc = dev_alloc(c, (void**)&c->r, N * 8)) ||
      (rc = dev_alloc(c, (void**)&c->red, ((size_t)c->red_blocks * 256 + 8192) * 8)) ||
      (rc = dev_alloc(c, (void**)&c->AV, (size_t)(o.ncv + 1) * N * 8)) ||
      (rc = dev_alloc(c, (void**)&c->tmpN, N * 8)) || (rc = dev_alloc(c, (void**)&c->tmpN2, N * 8)) ||
      (rc = dev_alloc(c, (void**)&c->tmpN3, N * 8)) || (rc = dev_alloc(c, (void**)&c->tuneU, (size_t)8 * N * 8)) ||
      (rc = dev_alloc(c, (void**)&c->tuneWU, (size_t)8 * N * 8)) || (rc = dev_alloc(c, (void**)&c->gsd, 4096 * 8)) ||
      (rc = dev_alloc(c, (void**)&c->gs_cnt, 256)) || (rc = dev_alloc(c, (void**)&c->tuneG_dev, 64 * 8)))
    return fail(rc);
  if (cudaMemset(c->gs_cnt, 0, 256) != cudaSuccess) return fail(FM_ERR_CUDA);
  if (cudaMallocHost((void**)&c->red_host, 8192 * 8) != cudaSuccess) return fail(FM_ERR_OOM);
  if (c->use_dd) {  // double-float Krylov workspace; float32 buffers of the preconditioner's input and output
    if ((rc = dev_alloc(c, (void**)&c->Vdd, (size_t)(m + 1) * N * 8)) || (rc = dev_alloc(c, (void**)&c->Zdd, (size_t)m * N * 8)) ||
        (rc = dev_alloc(c, (void**)&c->wdd, N * 8)) || (rc = dev_alloc(c, (void**)&c->rdd, N * 8)) ||
        (rc = dev_alloc(c, (void**)&c->bdd, N * 8)) || (rc = dev_alloc(c, (void**)&c->xdd, N * 8)) ||
        (rc = dev_alloc(c, (void**)&c->d32, N * 4)) || (rc = dev_alloc(c, (void**)&c->e32, N * 4)))
      return fail(rc);
  } else if (o.precision == FM_PREC_MIXED) {  // float32 Krylov workspace of the mixed-precision solves
    if ((rc = dev_alloc(c, (void**)&c->V32, (size_t)(m + 1) * N * 4)) || (rc = dev_alloc(c, (void**)&c->Z32, (size_t)m * N * 4)) ||
        (rc = dev_alloc(c, (void**)&c->w32, N * 4)) || (rc = dev_alloc(c, (void**)&c->r32, N * 4)) ||
        (rc = dev_alloc(c, (void**)&c->d32, N * 4)) || (rc = dev_alloc(c, (void**)&c->e32, N * 4)) ||
        (rc = dev_alloc(c, (void**)&c->P32, N * 4)) || (rc = dev_alloc(c, (void**)&c->Q32, N * 4)) ||
        (rc = dev_alloc(c, (void**)&c->R32, N * 4)))
      return fail(rc);
    int64_t st = 0;  // coupling sources regrouped by y interval for the float32 gather
    for (auto& cp : c->comps) {
      cp.ystage_off = st;
      st += (int64_t)c->nM * cp.nz * cp.nx * cp.ay.nint * cp.r;
    }
    if ((rc = dev_alloc(c, (void**)&c->ystage32, (size_t)st * 4))) return fail(rc);
  }
  phase("workspace allocation");
  if ((rc = tc_setup(c))) return fail(rc);
  phase("tensor maps");
  c->m_alloc = m;
  c->ncv_alloc = o.ncv;
  *out = c;
  return FM_OK;
}

int fm_estimate_bytes(const fm_system* sys, const fm_grid* grids, int n_grids, const fm_splitting* split,
                      const fm_opts* opts, int64_t* bytes) {
  if (!sys || !grids || !split || !bytes || n_grids < 1) return FM_ERR_ARG;
  fm_opts o;
  if (opts) o = *opts;
  else fm_default_opts(&o);
  return estimate_bytes(sys, grids, n_grids, split, &o, bytes);
}

int fm_size(const fm_ctx* c, int64_t* n, int* ncomp, int* nM) {
  if (!c) return FM_ERR_ARG;
  if (n) *n = c->N;
  if (ncomp) *ncomp = (int)c->comps.size();
  if (nM) *nM = c->nM;
  return FM_OK;
}

int fm_component(const fm_ctx* c, int comp, int* label, int dims[3], int64_t* offset) {
  if (!c || comp < 0 || comp >= (int)c->comps.size()) return FM_ERR_ARG;
  const auto& cp = c->comps[comp];
  if (label) *label = cp.label;
  if (dims) {
    dims[0] = cp.nz;
    dims[1] = cp.nx;
    dims[2] = cp.ny;
  }
  if (offset) *offset = cp.off;
  return FM_OK;
}

int fm_stats(const fm_ctx* c, int64_t* launches, int64_t* bytes) {
  if (!c) return FM_ERR_ARG;
  if (launches) *launches = c->launches;
  if (bytes) *bytes = c->device_bytes;
  return FM_OK;
}

int fm_host_decompose(int n, const double* A1, const double* A2, int descending, double* Wbar, double* W,
                      double* lam) {
  if (n < 1 || !A1 || !A2 || !Wbar || !W || !lam) return FM_ERR_ARG;
  const int e = fmh::decompose(n, A1, A2, descending != 0, Wbar, W, lam);
  if (e == -1) return FM_ERR_COMPLEX_SPECTRUM;
  if (e != 0) return FM_ERR_NUMERIC;
  return FM_OK;
}

int fm_profile(fm_ctx* c, int enable) {
  if (!c) return FM_ERR_ARG;
  FM_CUDA(cudaSetDevice(c->device));
  FM_CUDA(cudaStreamSynchronize(c->stream));
  prof_harvest(c);
  if (enable) {
    for (int i = 0; i < FM_NUM_KERNEL_CLASSES; ++i) {
      c->prof_ms[i] = 0.0;
      c->prof_n[i] = 0;
      c->prof_flops[i] = 0.0;
      c->prof_bytes[i] = 0.0;
    }
  }
  c->prof = enable != 0;
  return FM_OK;
}

int fm_profile_read(fm_ctx* c, double* ms, int64_t* n, double* flops, double* bytes) {
  if (!c || !ms || !n) return FM_ERR_ARG;
  FM_CUDA(cudaSetDevice(c->device));
  FM_CUDA(cudaStreamSynchronize(c->stream));
  prof_harvest(c);
  for (int i = 0; i < FM_NUM_KERNEL_CLASSES; ++i) {
    ms[i] = c->prof_ms[i];
    n[i] = c->prof_n[i];
    if (flops) flops[i] = c->prof_flops[i];
    if (bytes) bytes[i] = c->prof_bytes[i];
  }
  return FM_OK;
}

int fm_apply(fm_ctx* c, double E, const double* x, double* y) {
  if (!c || !x || !y || x == y || !std::isfinite(E)) return FM_ERR_ARG;
  FM_CUDA(cudaSetDevice(c->device));
  return launch_apply(c, E, x, y, false);
}

int fm_apply_S(fm_ctx* c, const double* x, double* y) {
  if (!c || !x || !y || x == y) return FM_ERR_ARG;
  FM_CUDA(cudaSetDevice(c->device));
  return launch_apply(c, 0.0, x, y, true);
}

int fm_set_shift(fm_ctx* c, double Estar) {
  if (!c || !std::isfinite(Estar)) return FM_ERR_ARG;
  FM_CUDA(cudaSetDevice(c->device));
  return setup_shift(c, Estar);
}

int fm_precond_apply(fm_ctx* c, const double* x, double* y) {
  if (!c || !x || !y || x == y) return FM_ERR_ARG;
  if (!c->have_shift) return FM_ERR_NO_SHIFT;
  FM_CUDA(cudaSetDevice(c->device));
  int rc = launch_precond(c, x, y);
  return rc ? rc : tc_check(c);
}

int fm_solve(fm_ctx* c, double E, const double* rhs, double* x, fm_info* info) {
  if (!c || !rhs || !x || rhs == x || !std::isfinite(E)) return FM_ERR_ARG;
  FM_CUDA(cudaSetDevice(c->device));
  const double t0 = wall_ms();
  int rc;
  if (!c->have_shift || c->Estar != E)
    if ((rc = setup_shift(c, E))) return rc;
  int it = 0, rs = 0;
  double res = 0.0;
  rc = solve_any(c, E, rhs, x, c->opts.tol, c->opts.max_iters, &it, &rs, &res);
  FM_CUDA(cudaStreamSynchronize(c->stream));
  if (rc == FM_OK || rc == FM_ERR_NOT_CONVERGED) {
    const int tc = tc_check(c);
    if (tc) rc = tc;
  }
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->iters = it;
    info->restarts = rs;
    info->resid = res;
    info->converged = (rc == FM_OK);
    info->ms = wall_ms() - t0;
  }
  return rc;
}

static int eigs_impl(fm_ctx* c, double shift, int k, const double* v0, double* evals, double* evecs, fm_info* info);

int fm_eigs(fm_ctx* c, double shift, int k, const double* v0, double* evals, double* evecs, fm_info* info) {
  int rc = eigs_impl(c, shift, k, v0, evals, evecs, info);
  if (c) {
    c->n_tune = 0;
    if (rc == FM_OK || rc == FM_ERR_NOT_CONVERGED) {
      const int tc = tc_check(c);
      if (tc) rc = tc;
    }
  }
  return rc;
}

static int eigs_impl(fm_ctx* c, double shift, int k, const double* v0, double* evals, double* evecs, fm_info* info) {
  if (!c || !evals || k < 1 || !std::isfinite(shift)) return FM_ERR_ARG;
  const int m = c->ncv_alloc;
  if (m < k + 2) return FM_ERR_ARG;
  FM_CUDA(cudaSetDevice(c->device));
  const double t0 = wall_ms();
  const int64_t N = c->N;
  int rc;
  if (!c->have_shift || c->Estar != shift)
    if ((rc = setup_shift(c, shift))) return rc;
  double* V = c->AV;
  if (v0) FM_CUDA(cudaMemcpyAsync(V, v0, N * 8, cudaMemcpyDeviceToDevice, c->stream));
  else if ((rc = fill_normal(c, V, 20050539ull))) return rc;
  double nv;
  if ((rc = nrm2(c, V, &nv))) return rc;
  if (!(nv > 0.0) || !std::isfinite(nv)) return FM_ERR_ARG;
  if ((rc = scale_copy(c, V, 1.0 / nv, V))) return rc;
  // -1 (default): 16 passes for one wanted level, 6 for several (more passes filter the other wanted levels
  // out of the start vector: measured on He L=0 with k = 1 and Ps- L=3 with k = 4)
  const int n_filter = c->opts.start_filter >= 0 ? c->opts.start_filter : (k == 1 ? 16 : 6);
  for (int pass = 0; pass < n_filter; ++pass) {  // v <- P^{-1} S v / ||P^{-1} S v||
    if ((rc = launch_apply(c, 0.0, V, c->tmpN, true))) return rc;
    if ((rc = launch_precond(c, c->tmpN, c->tmpN2))) return rc;
    if ((rc = nrm2(c, c->tmpN2, &nv))) return rc;
    if (!(nv > 0.0) || !std::isfinite(nv)) return FM_ERR_BREAKDOWN;
    if ((rc = scale_copy(c, c->tmpN2, 1.0 / nv, V))) return rc;
  }
  std::vector<double> G((size_t)(m + 1) * m, 0.0);  // projected matrix, row-major (m+1) x m
  int kcur = 0, restarts = 0, inner = 0, ops = 0, nsz = 0;
  bool converged = false, accepted_stable = false;
  std::vector<Ritz> best;
  std::vector<double> Y;  // eigenvectors of the projected matrix (nsz x nsz)
  std::vector<std::vector<double>> hist;  // eigenvalue history of each wanted Ritz value
  const bool verbose = getenv("FM_VERBOSE") != nullptr;
  // The tuned preconditioner speeds up inner solves that converge; once an inner solve stalls far above
  // its tolerance (the shift sits in a cluster of levels and the solves reach their float64 floor), the
  // tuning is dropped for the rest of the eigen-solve: its rank-k correction then steers the inexact
  // solves away from the wanted direction.
  bool tune_ok = true;
  double max_res = 0.0;
  // Inner solves to base_tol while the wanted Ritz pairs are far from converged; once their largest
  // relative Ritz residual r is small, the next operator application may be inexact by about
  // 0.1 base_tol / r (relaxation of inexact Arnoldi, Simoncini and Szyld, with a factor 10 of margin),
  // at most 1e-7.
  const double base_tol = std::max(c->opts.tol, 0.1 * c->opts.eig_tol);
  double prev_res = 1.0;
  while (true) {
    bool done = false;
    for (int j = kcur; j < m; ++j) {
      double* Vj = V + (int64_t)j * N;
      double* w = V + (int64_t)(j + 1) * N;
      if (c->opts.tune && tune_ok && c->opts.precision != FM_PREC_MIXED && nsz >= 1 && !best.empty()) {
        // tuned preconditioner (Freitag-Spence): U = orthonormalised Ritz vectors of the wanted values
        std::vector<int> cols;
        for (const auto& rz : best)
          if (rz.real && (int)cols.size() < std::min(k, 8)) cols.push_back(rz.col);
        const int nt = (int)cols.size();
        std::vector<double> Yt((size_t)nsz * nt);
        for (int r = 0; r < nsz; ++r)
          for (int q = 0; q < nt; ++q) Yt[(size_t)r * nt + q] = Y[(size_t)r * nsz + cols[q]];
        if (nt > 0 && small_qr(nsz, nt, Yt)) {
          if ((rc = combine(c, V, N, nsz, Yt.data(), nt, c->tuneU, N))) return rc;
          if ((rc = set_tuning(c, shift, c->tuneU, nt))) return rc;
        }
      }
      if ((rc = launch_apply(c, 0.0, Vj, c->tmpN, true))) return rc;  // S v_j
      FM_CUDA(cudaMemsetAsync(w, 0, N * 8, c->stream));
      int it = 0, rs = 0;
      double res = 0.0;
      const double inner_tol = std::max(base_tol, std::min(1e-7, 0.1 * base_tol / std::max(prev_res, 1e-300)));
      rc = solve_any(c, shift, c->tmpN, w, inner_tol, c->opts.max_iters, &it, &rs, &res);
      inner += it;
      ++ops;
      if (rc != FM_OK && rc != FM_ERR_NOT_CONVERGED) return rc;
      if (res > 100.0 * inner_tol && c->n_tune > 0) {
        tune_ok = false;
        c->n_tune = 0;
      }
      std::vector<double> h(j + 1);
      double hn;
      if ((rc = gs_cgs2(c, V, j + 1, w, w, h.data(), &hn))) return rc;  // w <- (w - V h) / hn
      if (!std::isfinite(hn)) return FM_ERR_BREAKDOWN;
      for (int i = 0; i <= j; ++i) G[(size_t)i * m + j] = h[i];
      G[(size_t)(j + 1) * m + j] = hn;
      nsz = j + 1;
      if (nsz < k) continue;
      // Ritz pairs of the nsz x nsz projected matrix
      std::vector<double> A((size_t)nsz * nsz), re(nsz), im(nsz);
      Y.assign((size_t)nsz * nsz, 0.0);
      for (int r = 0; r < nsz; ++r)
        for (int q = 0; q < nsz; ++q) A[(size_t)r * nsz + q] = G[(size_t)r * m + q];
      if (fmh::eig_general(nsz, A.data(), re.data(), im.data(), Y.data()) < 0) return FM_ERR_NUMERIC;
      std::vector<int> order(nsz);
      for (int i = 0; i < nsz; ++i) order[i] = i;
      std::sort(order.begin(), order.end(),
                [&](int a, int b) { return std::hypot(re[a], im[a]) > std::hypot(re[b], im[b]); });
      best.clear();
      bool ok = true, stagnant = true, wanted_real = true;
      max_res = 0.0;
      for (int t = 0; t < nsz; ++t) {
        const int e = order[t];
        Ritz rz{re[e], e, im[e] == 0.0};
        best.push_back(rz);
        if ((int)best.size() <= k) {
          const int i = (int)best.size() - 1;
          if (!rz.real) {
            ok = stagnant = wanted_real = false;
            continue;
          }
          const double resid = std::fabs(hn * Y[(size_t)(nsz - 1) * nsz + e]) / std::max(std::fabs(rz.theta), 1e-300);
          max_res = std::max(max_res, resid);
          if (resid > c->opts.eig_tol) ok = false;
          // eigenvalue E = shift + 1/theta stable over the last steps while the Ritz residual is small:
          // its accuracy is then limited by the inner solves, far below the requested level
          const double Ei = shift + 1.0 / rz.theta;
          if ((int)hist.size() <= i) hist.resize(i + 1);
          hist[i].push_back(Ei);
          const auto& hv = hist[i];
          bool st = hv.size() >= 3 && resid < std::sqrt(c->opts.eig_tol);
          for (size_t q = hv.size() >= 3 ? hv.size() - 3 : 0; st && q + 1 < hv.size(); ++q)
            if (std::fabs(hv[q + 1] - hv[q]) > 1e-3 * c->opts.eig_tol * std::fabs(Ei)) st = false;
          if (!st) stagnant = false;
        }
      }
      prev_res = wanted_real ? std::min(1.0, std::max(max_res, 1e-300)) : 1.0;
      if (verbose)
        fprintf(stderr, "[fm_eigs] step %d restart %d inner %d ritz_res %.3e E0 %.15f%s\n", nsz, restarts, inner,
                max_res, best.empty() ? 0.0 : shift + 1.0 / best[0].theta, ok ? " (residual)" : (stagnant ? " (stable)" : ""));
      if (ok || stagnant || hn == 0.0) {
        converged = ok || stagnant;
        accepted_stable = stagnant && !ok;
        done = true;
        break;
      }
    }
    if (done || restarts >= c->opts.max_restarts) break;
    // thick restart: keep the real Ritz vectors of the kk largest |theta|
    const int kk = std::min(m - 1, std::max(k, (m + k) / 2));
    std::vector<int> keep;
    for (const auto& rz : best)
      if (rz.real && (int)keep.size() < kk) keep.push_back(rz.col);
    const int nk = (int)keep.size();
    if (nk < 1) break;
    std::vector<double> Qy((size_t)m * nk);
    for (int r = 0; r < m; ++r)
      for (int q = 0; q < nk; ++q) Qy[(size_t)r * nk + q] = Y[(size_t)r * m + keep[q]];
    if (!small_qr(m, nk, Qy)) break;
    // T = Qy^T G Qy, b = g_{m+1,m} Qy[m-1, :]
    std::vector<double> GQ((size_t)m * nk, 0.0), T((size_t)nk * nk, 0.0);
    for (int r = 0; r < m; ++r)
      for (int q = 0; q < nk; ++q) {
        double s = 0.0;
        for (int t = 0; t < m; ++t) s += G[(size_t)r * m + t] * Qy[(size_t)t * nk + q];
        GQ[(size_t)r * nk + q] = s;
      }
    for (int a = 0; a < nk; ++a)
      for (int q = 0; q < nk; ++q) {
        double s = 0.0;
        for (int r = 0; r < m; ++r) s += Qy[(size_t)r * nk + a] * GQ[(size_t)r * nk + q];
        T[(size_t)a * nk + q] = s;
      }
    const double gl = G[(size_t)m * m + (m - 1)];
    if ((rc = combine(c, V, N, m, Qy.data(), nk, c->Z, N))) return rc;  // new basis into Z (scratch)
    FM_CUDA(cudaMemcpyAsync(V, c->Z, (size_t)nk * N * 8, cudaMemcpyDeviceToDevice, c->stream));
    FM_CUDA(cudaMemcpyAsync(V + (int64_t)nk * N, V + (int64_t)m * N, N * 8, cudaMemcpyDeviceToDevice, c->stream));
    std::fill(G.begin(), G.end(), 0.0);
    for (int a = 0; a < nk; ++a)
      for (int q = 0; q < nk; ++q) G[(size_t)a * m + q] = T[(size_t)a * nk + q];
    for (int q = 0; q < nk; ++q) G[(size_t)nk * m + q] = gl * Qy[(size_t)(m - 1) * nk + q];
    kcur = nk;
    ++restarts;
  }
  c->n_tune = 0;
  const int accept = converged ? (accepted_stable ? FM_ACCEPT_STABLE : FM_ACCEPT_RITZ) : FM_ACCEPT_NONE;
  if (nsz < k || (int)best.size() < k) return FM_ERR_NOT_CONVERGED;
  std::vector<double> Ek(k);
  for (int i = 0; i < k; ++i) {
    if (!best[i].real) return FM_ERR_NOT_CONVERGED;
    Ek[i] = shift + 1.0 / best[i].theta;
  }
  std::vector<int> ord(k);
  for (int i = 0; i < k; ++i) ord[i] = i;
  std::sort(ord.begin(), ord.end(), [&](int a, int b) { return std::fabs(Ek[a] - shift) < std::fabs(Ek[b] - shift); });
  // Float64 certificate of every returned pair, whichever rule stopped the iteration above: the Ritz value
  // E = shift + 1/theta with its Ritz vector c, and the backward error eta of (E, c) formed with the float64
  // operator.  A pair above eig_tol gets inverse-iteration steps z = (H - shift S)^{-1} S c with the
  // shift-invert operator's Rayleigh quotient theta = c^T z (|c| = 1), E = shift + 1/theta, a step kept only
  // when it lowers eta.  The call converges when every pair ends at eta <= eig_tol.  (The energy stays the
  // operator's Ritz value: the one-sided Rayleigh estimate through H weighs the high-frequency error of c
  // with |H| and is the less accurate of the two; it is reported as a check.)
  double nH, nS;
  if ((rc = operator_norms(c, &nH, &nS))) return rc;
  std::vector<double> eta_k(k, 0.0), resS_k(k, 0.0);
  double rq_dev = 0.0;
  int refine_steps = 0;
  bool certified = true;
  double* cvec = c->tmpN3;
  double* z = c->tuneU;           // free once the eigen-iteration has ended (n_tune = 0)
  double* keep = c->tuneU + N;
  for (int ii = 0; ii < k; ++ii) {
    const int i = ord[ii];
    std::vector<double> yv(nsz);
    for (int r = 0; r < nsz; ++r) yv[r] = Y[(size_t)r * nsz + best[i].col];
    if ((rc = combine(c, V, N, nsz, yv.data(), 1, cvec, N))) return rc;
    double nr;
    if ((rc = nrm2(c, cvec, &nr))) return rc;
    if (!(nr > 0.0) || !std::isfinite(nr)) return FM_ERR_BREAKDOWN;
    if ((rc = scale_copy(c, cvec, 1.0 / nr, cvec))) return rc;
    double E = Ek[i], eta, resS, ER;
    if ((rc = certify(c, cvec, E, nH, nS, &eta, &resS, &ER))) return rc;
    for (int step = 0; step < c->opts.refine && eta > c->opts.eig_tol; ++step) {
      if ((rc = launch_apply(c, 0.0, cvec, c->tmpN2, true))) return rc;  // S c
      FM_CUDA(cudaMemsetAsync(z, 0, N * 8, c->stream));
      int it = 0, rs = 0;
      double res = 0.0;
      rc = solve_any(c, shift, c->tmpN2, z, c->opts.tol, c->opts.max_iters, &it, &rs, &res);
      inner += it;
      ++ops;
      ++refine_steps;
      if (rc != FM_OK && rc != FM_ERR_NOT_CONVERGED) return rc;
      double th = 0.0, nz;
      if ((rc = dot_many(c, cvec, N, 1, z, &th)) || (rc = nrm2(c, z, &nz))) return rc;
      if (!(nz > 0.0) || !std::isfinite(nz) || th == 0.0 || !std::isfinite(th)) break;
      FM_CUDA(cudaMemcpyAsync(keep, cvec, N * 8, cudaMemcpyDeviceToDevice, c->stream));
      if ((rc = scale_copy(c, z, 1.0 / nz, cvec))) return rc;
      const double E2 = shift + 1.0 / th;
      double eta2, resS2, ER2;
      if ((rc = certify(c, cvec, E2, nH, nS, &eta2, &resS2, &ER2))) return rc;
      if (!(eta2 < eta)) {  // no gain: keep the previous pair and stop
        FM_CUDA(cudaMemcpyAsync(cvec, keep, N * 8, cudaMemcpyDeviceToDevice, c->stream));
        break;
      }
      E = E2;
      eta = eta2;
      resS = resS2;
      ER = ER2;
    }
    double mx;
    if ((rc = absmax(c, cvec, &mx))) return rc;
    if (mx < 0) {
      if ((rc = scale_copy(c, cvec, -1.0, cvec))) return rc;
    }
    eta_k[ii] = eta;
    resS_k[ii] = resS;
    rq_dev = std::max(rq_dev, std::fabs(ER - E) / std::max(std::fabs(E), 1e-300));
    evals[ii] = E;
    if (!(eta <= c->opts.eig_tol)) certified = false;
    if (evecs) FM_CUDA(cudaMemcpyAsync(evecs + (int64_t)ii * N, cvec, N * 8, cudaMemcpyDeviceToDevice, c->stream));
  }
  FM_CUDA(cudaStreamSynchronize(c->stream));
  if (verbose)
    for (int ii = 0; ii < k; ++ii)
      fprintf(stderr, "[fm_eigs] pair %d: E %.15f eta %.3e |r|/|Sc| %.3e (|H| %.3e |S| %.3e)\n", ii, evals[ii],
              eta_k[ii], resS_k[ii], nH, nS);
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->iters = inner;
    info->restarts = restarts;
    info->op_applies = ops;
    info->converged = certified ? 1 : 0;
    info->resid = *std::max_element(eta_k.begin(), eta_k.end());
    info->resid_S = *std::max_element(resS_k.begin(), resS_k.end());
    info->norm_H = nH;
    info->norm_S = nS;
    info->rq_dev = rq_dev;
    info->accept = accept;
    info->refine_steps = refine_steps;
    info->ms = wall_ms() - t0;
  }
  return certified ? FM_OK : FM_ERR_NOT_CONVERGED;
}

int fm_eigs_host(fm_ctx* c, double shift, int k, const double* v0_host, double* evals, double* evecs_host, fm_info* info) {
  if (!c || !evals || k < 1) return FM_ERR_ARG;
  FM_CUDA(cudaSetDevice(c->device));
  const int64_t N = c->N;
  int rc;
  if (evecs_host && c->evec_stage_k < k) {
    if ((rc = dev_alloc(c, (void**)&c->evec_stage, (size_t)k * N * 8))) return rc;
    c->evec_stage_k = k;
  }
  const double* v0d = nullptr;
  if (v0_host) {
    FM_CUDA(cudaMemcpyAsync(c->tmpN3, v0_host, N * 8, cudaMemcpyHostToDevice, c->stream));
    v0d = c->tmpN3;
  }
  rc = fm_eigs(c, shift, k, v0d, evals, evecs_host ? c->evec_stage : nullptr, info);
  if (rc != FM_OK && rc != FM_ERR_NOT_CONVERGED) return rc;
  if (evecs_host)
    FM_CUDA(cudaMemcpyAsync(evecs_host, c->evec_stage, (size_t)k * N * 8, cudaMemcpyDeviceToHost, c->stream));
  FM_CUDA(cudaStreamSynchronize(c->stream));
  return rc;
}

}  // extern "C"
