// Host set-up of libfm: spline axes and collocation (Section 3.1, Section 4), the
// kinematics and potentials of Section 2, the V^(s) coupling geometry (Eqs. r-form,
// s-rot), the z and x decompositions of the preconditioner (Eq. z-dec and the x
// problems of Section 3.2) and the E*-dependent banded y systems.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <thread>
#include <vector>

#include "fm_dense.h"
#include "fm_internal.h"

namespace fmi {

// ---------------------------------------------------------------------------
// Hermite shape functions on [t_m, t_m + h], local coordinate s in [0, 1].
// Cubic (q = 2): value left, slope left, value right, slope right.
// Quintic (q = 3, S_5^3 of Section 4): value, first and second derivative at the left node, then at the
// right node -- the degree-5 polynomials with one unit condition among those six; derivative dofs are
// with respect to t, hence the powers of h.  deriv = order of the t-derivative returned.
// ---------------------------------------------------------------------------
static void shapes(double s, double h, int deriv, int q, double* v) {
  const double u = 1.0 - s;
  if (q == 2) {
    if (deriv == 0) {
      v[0] = (1.0 + 2.0 * s) * u * u;
      v[1] = s * u * u * h;
      v[2] = s * s * (3.0 - 2.0 * s);
      v[3] = s * s * (s - 1.0) * h;
    } else if (deriv == 1) {
      v[0] = 6.0 * s * (s - 1.0) / h;
      v[1] = u * (1.0 - 3.0 * s);
      v[2] = 6.0 * s * u / h;
      v[3] = s * (3.0 * s - 2.0);
    } else {
      v[0] = (12.0 * s - 6.0) / (h * h);
      v[1] = (6.0 * s - 4.0) / h;
      v[2] = (6.0 - 12.0 * s) / (h * h);
      v[3] = (6.0 * s - 2.0) / h;
    }
    return;
  }
  const double s2 = s * s, s3 = s2 * s, s4 = s3 * s, s5 = s4 * s;
  if (deriv == 0) {
    v[0] = 1.0 - 10.0 * s3 + 15.0 * s4 - 6.0 * s5;
    v[1] = (s - 6.0 * s3 + 8.0 * s4 - 3.0 * s5) * h;
    v[2] = 0.5 * s2 * u * u * u * h * h;
    v[3] = 10.0 * s3 - 15.0 * s4 + 6.0 * s5;
    v[4] = (-4.0 * s3 + 7.0 * s4 - 3.0 * s5) * h;
    v[5] = 0.5 * s3 * u * u * h * h;
  } else if (deriv == 1) {
    v[0] = (-30.0 * s2 + 60.0 * s3 - 30.0 * s4) / h;
    v[1] = 1.0 - 18.0 * s2 + 32.0 * s3 - 15.0 * s4;
    v[2] = 0.5 * (2.0 * s - 9.0 * s2 + 12.0 * s3 - 5.0 * s4) * h;
    v[3] = (30.0 * s2 - 60.0 * s3 + 30.0 * s4) / h;
    v[4] = -12.0 * s2 + 28.0 * s3 - 15.0 * s4;
    v[5] = 0.5 * (3.0 * s2 - 8.0 * s3 + 5.0 * s4) * h;
  } else {
    v[0] = (-60.0 * s + 180.0 * s2 - 120.0 * s3) / (h * h);
    v[1] = (-36.0 * s + 96.0 * s2 - 60.0 * s3) / h;
    v[2] = 0.5 * (2.0 - 18.0 * s + 36.0 * s2 - 20.0 * s3);
    v[3] = (60.0 * s - 180.0 * s2 + 120.0 * s3) / (h * h);
    v[4] = (-24.0 * s + 84.0 * s2 - 60.0 * s3) / h;
    v[5] = 0.5 * (6.0 * s - 24.0 * s2 + 20.0 * s3);
  }
}

// q Gauss-Legendre nodes on [-1, 1], ascending: closed forms for q <= 4, Newton on P_q otherwise
static void gauss(int q, double* g) {
  if (q == 2) {
    const double a = 1.0 / std::sqrt(3.0);
    g[0] = -a; g[1] = a;
  } else if (q == 3) {
    const double a = std::sqrt(0.6);
    g[0] = -a; g[1] = 0.0; g[2] = a;
  } else if (q == 4) {
    const double a = std::sqrt(3.0 / 7.0 - 2.0 / 7.0 * std::sqrt(1.2));
    const double b = std::sqrt(3.0 / 7.0 + 2.0 / 7.0 * std::sqrt(1.2));
    g[0] = -b; g[1] = -a; g[2] = a; g[3] = b;
  } else {
    for (int i = 0; i < q; ++i) {
      double x = std::cos(M_PI * (i + 0.75) / (q + 0.5));  // the i-th largest root, approximately
      for (int it = 0; it < 100; ++it) {
        double p0 = 1.0, p1 = x;  // Legendre recurrence (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}
        for (int k = 1; k < q; ++k) {
          const double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
          p0 = p1;
          p1 = p2;
        }
        const double dp = q * (x * p1 - p0) / (x * x - 1.0);
        const double dx = p1 / dp;
        x -= dx;
        if (std::fabs(dx) < 1e-16) break;
      }
      g[q - 1 - i] = x;
    }
  }
}

// taps for interval m: base q m (- 1 with the Dirichlet basis, which drops the value functions of the
// end nodes: the first interval's tap 0 is then outside the basis, and in the last interval the taps
// after the dropped value function move down one place so that the r taps stay contiguous).
static void place(const Axis& A, int m, const double* sh, int* base, double* v) {
  const int q = A.q, r = A.r;
  if (!A.dirichlet) {
    *base = q * m;
    for (int t = 0; t < r; ++t) v[t] = sh[t];
    return;
  }
  *base = q * m - 1;
  for (int t = 0; t < r; ++t) v[t] = sh[t];
  if (m == 0) v[0] = 0.0;
  if (m == A.nint - 1) {
    for (int t = q; t < r - 1; ++t) v[t] = sh[t + 1];
    v[r - 1] = 0.0;
  }
}

void Axis::build(int kind_, int nint_, double a_, double b_, bool dirichlet_, int basis) {
  kind = kind_; nint = nint_; a = a_; b = b_; dirichlet = dirichlet_;
  q = (basis == 1) ? 3 : 2;
  r = 2 * q;
  nodes.resize(nint + 1);
  for (int i = 0; i <= nint; ++i) {
    const double u = (double)i / nint;
    if (kind == FM_MAP_POW) nodes[i] = 4.0 * (std::pow(1.0 + b / 4.0, u) - 1.0);
    else if (kind == FM_MAP_SIN) nodes[i] = std::sin(M_PI * (-1.0 + 2.0 * u) / 2.0);
    else nodes[i] = a + (b - a) * u;
  }
  nodes[0] = a;
  nodes[nint] = b;
  n = q * (nint + 1) - (dirichlet ? 2 : 0);
  pts.clear(); base.clear(); S.clear(); D1.clear(); D2.clear();
  // Gauss points per interval, as many in all as functions: cubic 2 (closed z: 3 in the first and last
  // intervals); quintic 3 (x, y: 4 in the first interval; closed z: one more in the first, the last and
  // the middle interval nint / 2; a single interval takes all)
  std::vector<int> cnt(nint, q);
  if (q == 2) {
    if (!dirichlet) {
      if (nint == 1) cnt[0] = 4;
      else cnt[0] = cnt[nint - 1] = 3;
    }
  } else if (dirichlet) {
    cnt[0] += 1;
  } else if (nint == 1) {
    cnt[0] = 6;
  } else {
    cnt[0] += 1;
    cnt[nint - 1] += 1;
    cnt[nint / 2] += 1;
  }
  for (int m = 0; m < nint; ++m) {
    double g[8];
    gauss(cnt[m], g);
    const double h = nodes[m + 1] - nodes[m];
    for (int e = 0; e < cnt[m]; ++e) {
      const double s = 0.5 * (1.0 + g[e]);
      const double p = nodes[m] + h * s;
      pts.push_back(p);
      double sh[kMaxTaps], v[kMaxTaps];
      int bb;
      for (int d = 0; d < 3; ++d) {
        shapes(s, h, d, q, sh);
        place(*this, m, sh, &bb, v);
        std::vector<double>& dst = d == 0 ? S : (d == 1 ? D1 : D2);
        for (int t = 0; t < r; ++t) dst.push_back(v[t]);
      }
      base.push_back(bb);
    }
  }
  kl = ku = 0;
  for (int e = 0; e < (int)pts.size(); ++e) {
    const int lo = std::max(base[e], 0), hi = std::min(base[e] + r - 1, n - 1);
    kl = std::max(kl, e - lo);
    ku = std::max(ku, hi - e);
  }
}

int Axis::tile_rows(int tx) const {
  int rows = 1;
  for (int e0 = 0; e0 < (int)pts.size(); e0 += tx) {
    const int e1 = std::min((int)pts.size(), e0 + tx) - 1;
    rows = std::max(rows, base[e1] + r - base[e0]);
  }
  return rows;
}

int Axis::locate(double p) const {
  int m = (int)(std::upper_bound(nodes.begin(), nodes.end(), p) - nodes.begin()) - 1;
  return std::min(std::max(m, 0), nint - 1);
}

void Axis::eval(double p, int deriv, int* base_out, double v[kMaxTaps]) const {
  if (!(p >= a && p <= b)) {
    *base_out = 0;
    for (int t = 0; t < kMaxTaps; ++t) v[t] = 0.0;
    return;
  }
  const int m = locate(p);
  const double h = nodes[m + 1] - nodes[m];
  double sh[kMaxTaps];
  shapes((p - nodes[m]) / h, h, deriv, q, sh);
  place(*this, m, sh, base_out, v);
}

// ---------------------------------------------------------------------------
// kinematics and potentials (Section 2)
// ---------------------------------------------------------------------------
static void rotation(const double* m, int beta, int alpha, double* c, double* s) {
  const double M = m[0] + m[1] + m[2];
  const double mb = m[beta - 1], ma = m[alpha - 1];
  *c = -std::sqrt(mb * ma / ((M - mb) * (M - ma)));
  const double sg = ((beta - alpha) % 2 == 0 ? 1.0 : -1.0) * (alpha > beta ? 1.0 : -1.0);
  *s = sg * std::sqrt(1.0 - (*c) * (*c));
}

static void rotate(double c, double s, double x, double y, double z, double* xb, double* yb, double* zb) {
  *xb = std::sqrt(std::max(c * c * x * x + 2.0 * s * c * x * y * z + s * s * y * y, 0.0));
  *yb = std::sqrt(std::max(s * s * x * x - 2.0 * s * c * x * y * z + c * c * y * y, 0.0));
  double t = (s * c * (y * y - x * x) + (c * c - s * s) * x * y * z) / ((*xb) * (*yb));
  *zb = std::min(1.0, std::max(-1.0, t));
}

static bool first_branch(int beta, int alpha) {
  return (beta == 1 && alpha == 2) || (beta == 2 && alpha == 3) || (beta == 3 && alpha == 1);
}

static double w_angle(int beta, int alpha, double c, double s, double x, double y, double z, double yb) {
  const double arg = std::min(1.0, std::max(-1.0, (-s * x * z + c * y) / yb));
  const double w = std::acos(arg);
  return first_branch(beta, alpha) ? w : 2.0 * M_PI - w;
}

static double coulomb(const fm_ctx* c, int a, double x) {
  int b = -1, g = -1;
  for (int i = 0; i < 3; ++i)
    if (i != a - 1) (b < 0 ? b : g) = i;
  return std::sqrt(2.0 * c->mu_pair[a - 1]) * c->sys.charge[b] * c->sys.charge[g] / x;
}

static double chi(const fm_splitting& sp, double x, double y) {
  double arg = std::pow(x / sp.x0, sp.nu);
  if (std::isfinite(sp.y0)) arg /= (1.0 + y / sp.y0);
  return 2.0 / (1.0 + std::exp(arg));
}

static double vhat(const fm_ctx* c, int a, double y, double Ry) {
  double zz = 0.0;
  for (int i = 0; i < 3; ++i)
    if (i != a - 1) zz += c->sys.charge[i];
  const double qv = c->sys.charge[a - 1] * zz * std::sqrt(2.0 * c->mu_rel[a - 1]);
  const double u = y / (0.05 * Ry);
  return qv / y * (1.0 - std::exp(-u * u));
}

// ---------------------------------------------------------------------------
// Wigner d (Eq. D-def) through the Jacobi-polynomial form, valid for M' >= |M|, and
// the symmetries d_{M M'} = (-1)^{M-M'} d_{M' M} = d_{-M', -M} for the other indices.
// d_over_sin returns d / sin(w)^k (k <= min(|M-M'|, |M+M'|)).
// ---------------------------------------------------------------------------
// a float64 value as an unevaluated sum of two floats (hi, lo)
static float2 split2(double v) {
  const float hi = (float)v;
  return make_float2(hi, (float)(v - (double)hi));
}

// log n! and binomial coefficients from tables (the arguments here are small integers: J <= 11)
constexpr int kFactTab = 64;
struct FactTables {
  double lf[kFactTab];
  double bin[kFactTab][kFactTab];
  FactTables() {
    for (int n = 0; n < kFactTab; ++n) lf[n] = std::lgamma(n + 1.0);
    for (int n = 0; n < kFactTab; ++n)
      for (int k = 0; k < kFactTab; ++k) bin[n][k] = (k == 0 || k == n) ? 1.0 : (k > n ? 0.0 : bin[n - 1][k - 1] + bin[n - 1][k]);
  }
};
static const FactTables& fact_tables() {
  static const FactTables t;
  return t;
}

static double lfact(int n) { return (n >= 0 && n < kFactTab) ? fact_tables().lf[n] : std::lgamma(n + 1.0); }

static double binom(int n, int k) {
  if (k < 0 || k > n) return 0.0;
  if (n < kFactTab) return fact_tables().bin[n][k];
  return std::exp(lfact(n) - lfact(k) - lfact(n - k));
}

// x^e for a non-negative integer e by repeated squaring
static double ipow(double x, int e) {
  double r = 1.0;
  while (e > 0) {
    if (e & 1) r *= x;
    x *= x;
    e >>= 1;
  }
  return r;
}

static double jacobi_poly(int n, int al, int be, double x) {
  const double xm = (x - 1.0) / 2.0, xp = (x + 1.0) / 2.0;
  double s = 0.0;
  for (int k = 0; k <= n; ++k) s += binom(n + al, n - k) * binom(n + be, k) * ipow(xm, k) * ipow(xp, n - k);
  return s;
}

static double wigner_d_sin(int J, int M, int Mp, double w, int k) {
  if (std::abs(M) > J || std::abs(Mp) > J) return 0.0;
  double sign = 1.0;
  int m = M, mp = Mp;
  if (mp >= std::abs(m)) {
  } else if (m >= std::abs(mp)) {  // d_{M M'} = (-1)^{M-M'} d_{M' M}
    sign = ((m - mp) % 2 == 0) ? 1.0 : -1.0;
    std::swap(m, mp);
  } else if (-mp >= std::abs(m)) {  // d_{M M'} = (-1)^{M-M'} d_{-M, -M'}
    sign = ((m - mp) % 2 == 0) ? 1.0 : -1.0;
    m = -m;
    mp = -mp;
  } else {  // -M >= |M'|: d_{M M'} = d_{-M', -M}
    const int t = m;
    m = -mp;
    mp = -t;
  }
  const double pref = std::exp(0.5 * (lfact(J + mp) + lfact(J - mp) - lfact(J + m) - lfact(J - m)));
  const double sh = std::sin(0.5 * w), ch = std::cos(0.5 * w);
  const double val = pref * ipow(sh, mp - m - k) * ipow(ch, mp + m - k) * jacobi_poly(J - mp, mp - m, mp + m, std::cos(w));
  return sign * std::ldexp(val, -k);
}

// (-1)^{M''-M'} 2/sqrt(2+2 d_{M''0}) F^{J tau}_{M'' M'}(0, w, 0), divided by sin(w)^k
static double coupling_K(int J, int tau, int Mp, int Mpp, double w, int k) {
  const double F = (wigner_d_sin(J, Mpp, Mp, w, k) + tau * ((Mp % 2 == 0) ? 1.0 : -1.0) * wigner_d_sin(J, Mpp, -Mp, w, k)) /
                   std::sqrt(2.0 + (Mp == 0 ? 2.0 : 0.0));
  return (((Mpp - Mp) % 2 == 0) ? 1.0 : -1.0) * 2.0 / std::sqrt(2.0 + (Mpp == 0 ? 2.0 : 0.0)) * F;
}

static double lam(int J, int Mp) {
  const double v = (double)(J * (J + 1) - Mp * (Mp + 1));
  return v > 0 ? std::sqrt(v) : 0.0;
}
static double lam_hat_plus(int J, int Mp) { return lam(J, Mp) * std::sqrt(Mp == 0 ? 2.0 : 1.0); }
static double lam_hat_minus(int J, int Mp) { return lam(J, -Mp) * std::sqrt(Mp == 1 ? 2.0 : 1.0); }

// g_l^{M'}(1) (Appendix, Eq. g-def, Condon-Shortley phase)
static double g_at_one(int l, int Mp) {
  const double nrm = std::sqrt((2 * l + 1) / 2.0 * std::exp(lfact(l - Mp) - lfact(l + Mp)));
  return nrm * ((Mp % 2 == 0) ? 1.0 : -1.0) * std::exp(lfact(l + Mp) - lfact(Mp) - lfact(l - Mp)) / std::pow(2.0, Mp);
}

// ---------------------------------------------------------------------------
template <typename F>
static void parallel_for(int n, F f) {
  unsigned nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
  if (n < 2 || nt == 1) {
    for (int i = 0; i < n; ++i) f(i);
    return;
  }
  std::vector<std::thread> th;
  std::atomic<int> next{0};
  for (unsigned t = 0; t < nt; ++t)
    th.emplace_back([&]() {
      for (int i = next++; i < n; i = next++) f(i);
    });
  for (auto& t : th) t.join();
}

// Wall-clock phases of the set-up, printed to stderr when FM_VERBOSE is set.
struct PhaseTimer {
  bool on = getenv("FM_VERBOSE") != nullptr;
  std::chrono::steady_clock::time_point t = std::chrono::steady_clock::now();
  void mark(const char* what) {
    if (!on) return;
    const auto now = std::chrono::steady_clock::now();
    fprintf(stderr, "[fm_setup] %-28s %8.1f ms\n", what, std::chrono::duration<double, std::milli>(now - t).count());
    t = now;
  }
};

static int upload_axis(fm_ctx* c, const Axis& A, AxisDev& D) {
  int rc;
  if ((rc = upload(c, (void**)&D.base, A.base.data(), A.base.size() * sizeof(int)))) return rc;
  if ((rc = upload(c, (void**)&D.S, A.S.data(), A.S.size() * sizeof(double)))) return rc;
  if ((rc = upload(c, (void**)&D.D1, A.D1.data(), A.D1.size() * sizeof(double)))) return rc;
  if ((rc = upload(c, (void**)&D.D2, A.D2.data(), A.D2.size() * sizeof(double)))) return rc;
  if ((rc = upload(c, (void**)&D.pts, A.pts.data(), A.pts.size() * sizeof(double)))) return rc;
  return FM_OK;
}

static std::vector<double> dense_of(const Axis& A, const std::vector<double>& vals) {
  std::vector<double> M((size_t)A.n * A.n, 0.0);
  for (int q = 0; q < A.n; ++q)
    for (int t = 0; t < A.r; ++t) {
      const int j = A.base[q] + t;
      if (j >= 0 && j < A.n) M[(size_t)q * A.n + j] += vals[q * A.r + t];
    }
  return M;
}

static std::vector<float> to_f32(const std::vector<double>& v) { return std::vector<float>(v.begin(), v.end()); }

// bfloat16 bits of v: the high half of the float32 pattern, rounded to nearest even
uint16_t f2bf(float v) {
  uint32_t u;
  std::memcpy(&u, &v, 4);
  if ((u & 0x7fffffffu) > 0x7f800000u) return (uint16_t)((u >> 16) | 0x40u);  // NaN stays NaN
  u += 0x7fffu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}

static std::vector<uint16_t> to_bf16(const std::vector<double>& v) {
  std::vector<uint16_t> o(v.size());
  for (size_t i = 0; i < v.size(); ++i) o[i] = f2bf((float)v[i]);
  return o;
}

static bool tc_requested(const fm_ctx* c) {
  return c->opts.precision != FM_PREC_FP64 && c->opts.mma != FM_MMA_SIMT;
}

int setup_host(fm_ctx* c, const fm_grid* grids, int n_grids) {
  const fm_system& S = c->sys;
  const double* m = S.mass;
  const double M = m[0] + m[1] + m[2];
  for (int a = 0; a < 3; ++a) {
    int b = -1, g = -1;
    for (int i = 0; i < 3; ++i)
      if (i != a) (b < 0 ? b : g) = i;
    c->mu_pair[a] = m[b] * m[g] / (m[b] + m[g]);
    c->mu_rel[a] = m[a] * (m[b] + m[g]) / M;
  }
  std::vector<int> labels;
  if (c->split.mode == FM_SPLIT_SCHRODINGER) labels = {1};
  else if (S.identical_pair == 12) labels = {1, 3};
  else labels = {1, 2, 3};
  if (n_grids != 1 && n_grids != (int)labels.size()) return FM_ERR_ARG;
  c->comps.resize(labels.size());
  int64_t off = 0;
  for (size_t ic = 0; ic < labels.size(); ++ic) {
    Comp& cp = c->comps[ic];
    const fm_grid& g = grids[n_grids == 1 ? 0 : ic];
    if (g.nint_x < 1 || g.nint_y < 1 || g.nint_z < 1 || !(g.Rx > 0) || !(g.Ry > 0) || g.basis < 0 || g.basis > 1)
      return FM_ERR_ARG;
    if (g.zmap == FM_MAP_POW || g.xmap == FM_MAP_SIN || g.ymap == FM_MAP_SIN) return FM_ERR_ARG;
    cp.label = labels[ic];
    cp.ax.build(g.xmap, g.nint_x, 0.0, g.Rx, true, g.basis);
    cp.ay.build(g.ymap, g.nint_y, 0.0, g.Ry, true, g.basis);
    cp.az.build(g.zmap, g.nint_z, -1.0, 1.0, false, g.basis);
    cp.r = cp.ax.r;
    if (ic > 0 && cp.r != c->comps[0].r) return FM_ERR_ARG;  // one basis for every solved component
    cp.nx = cp.ax.n; cp.ny = cp.ay.n; cp.nz = cp.az.n;
    cp.Rx = g.Rx; cp.Ry = g.Ry;
    cp.npts = (int64_t)cp.nz * cp.nx * cp.ny;
    cp.off = off;
    off += cp.npts * c->nM;
  }
  c->N = off;
  // sources (Eq. FM-pre right-hand side with Eq. 2-sym-part)
  for (auto& cp : c->comps) {
    cp.sources.clear();
    if (c->split.mode == FM_SPLIT_SCHRODINGER) continue;
    for (int beta = 1; beta <= 3; ++beta) {
      if (beta == cp.label) continue;
      Source s;
      s.beta = beta;
      int idx = -1;
      for (size_t i = 0; i < labels.size(); ++i)
        if (labels[i] == beta) idx = (int)i;
      if (idx >= 0) {
        s.src = idx;
        s.zsign = 1.0;
        s.sym = false;
      } else {  // beta = 2 of the identical pair: component 1 at (x, y, -z) times p (-1)^{M''}
        s.src = 0;
        s.zsign = -1.0;
        s.sym = true;
      }
      cp.sources.push_back(s);
    }
  }
  const int J = S.J, nM = c->nM;
  int rc;
  PhaseTimer tm;
  // x decompositions of every component in one thread pool (they need only the x axis, unless the computed
  // z eigenvalues replace l(l+1): then they follow the z decompositions below)
  struct XD {
    std::vector<double> Wx, Wxb;
    std::vector<int> err, pairs;
  };
  std::vector<XD> xd(c->comps.size());
  auto x_task = [&](const Comp& cp, int il, XD& d) {
    const int nx = cp.nx, l = c->M0 + il;
    const double ll1 = (c->opts.z_eigs == 1) ? -cp.Lz[il] : (double)l * (l + 1);
    static thread_local std::vector<double> Sxd, D2xd;
    Sxd = dense_of(cp.ax, cp.ax.S);
    D2xd = dense_of(cp.ax, cp.ax.D2);
    std::vector<double> A1((size_t)nx * nx);
    for (int q = 0; q < nx; ++q) {
      const double x = cp.ax.pts[q];
      const double f = ll1 / (x * x) + coulomb(c, cp.label, x);
      for (int j = 0; j < nx; ++j) A1[(size_t)q * nx + j] = -D2xd[(size_t)q * nx + j] + f * Sxd[(size_t)q * nx + j];
    }
    Comp& cw = const_cast<Comp&>(cp);
    d.err[il] = fmh::decompose(nx, A1.data(), Sxd.data(), false, &d.Wxb[(size_t)il * nx * nx],
                               &d.Wx[(size_t)il * nx * nx], &cw.Lx[(size_t)il * nx]);
    if (d.err[il] == -1) {
      // complex-conjugate pairs (quintic collocation pencils, Section 4): each pair in a real basis (real and
      // imaginary parts of its eigenvector), its real part as the diagonal value of both columns.  The
      // preconditioner then leaves out the pair's 2 x 2 rotation (relative size |Im| / |Re + lambda_y +
      // lambda_z - E|), an approximation of the tensor-trick inverse that FGMRES absorbs; the operator, and
      // so every result, is unchanged.
      std::vector<int> kind(nx);
      d.err[il] = fmh::decompose_pairs(nx, A1.data(), Sxd.data(), -1, &d.Wxb[(size_t)il * nx * nx],
                                       &d.Wx[(size_t)il * nx * nx], &cw.Lx[(size_t)il * nx], kind.data());
      if (d.err[il] == 0) d.pairs[il] = 1;
    }
  };
  const bool x_first = c->opts.z_eigs != 1;
  if (x_first) {
    std::vector<std::pair<int, int>> tasks;
    for (size_t q = 0; q < c->comps.size(); ++q) {
      Comp& cp = c->comps[q];
      cp.nl = nM + cp.nz - 1;
      xd[q].Wx.resize((size_t)cp.nl * cp.nx * cp.nx);
      xd[q].Wxb.resize((size_t)cp.nl * cp.nx * cp.nx);
      xd[q].err.assign(cp.nl, 0);
      xd[q].pairs.assign(cp.nl, 0);
      cp.Lx.assign((size_t)cp.nl * cp.nx, 0.0);
      for (int il = 0; il < cp.nl; ++il) tasks.push_back({(int)q, il});
    }
    parallel_for((int)tasks.size(), [&](int t) { x_task(c->comps[tasks[t].first], tasks[t].second, xd[tasks[t].first]); });
    tm.mark("x decompositions");
  }
  for (auto& cp : c->comps) {
    tm.mark("(previous component)");
    if ((rc = upload_axis(c, cp.ax, cp.dx))) return rc;
    if ((rc = upload_axis(c, cp.ay, cp.dy))) return rc;
    if ((rc = upload_axis(c, cp.az, cp.dz))) return rc;
    // pointwise coefficients of Eq. FM-pre: the left-hand potential V_a(x) + sum_{b != a} V^(l)_b(x_b, y_b)
    // folded with the M'-dependent diagonal terms, and the coefficients of the z derivatives
    std::vector<double> W((size_t)nM * cp.npts), Atab((size_t)cp.npts), Btab((size_t)nM * cp.npts), iy2(cp.ny);
    for (int j = 0; j < cp.ny; ++j) iy2[j] = 1.0 / (cp.ay.pts[j] * cp.ay.pts[j]);
    std::vector<int> bad_plane(cp.nz, 0);
    const Comp* cq = &cp;
    parallel_for(cp.nz, [&](int k) {  // one z plane per task
      for (int i = 0; i < cq->nx; ++i)
        for (int j = 0; j < cq->ny; ++j) {
          const double z = cq->az.pts[k], x = cq->ax.pts[i], y = cq->ay.pts[j];
          double tot = coulomb(c, cq->label, x);
          for (int beta = 1; beta <= 3; ++beta) {
            if (beta == cq->label) continue;
            double cc, ss, xb, yb, zb;
            rotation(m, beta, cq->label, &cc, &ss);
            rotate(cc, ss, x, y, z, &xb, &yb, &zb);
            const double vc = coulomb(c, beta, xb);
            if (c->split.mode == FM_SPLIT_SCHRODINGER) tot += vc;
            else if (c->split.mode == FM_SPLIT_MERKURIEV) tot += (1.0 - chi(c->split, xb, yb)) * vc;
          }
          if (!std::isfinite(tot)) bad_plane[k] = 1;
          const size_t pt = ((size_t)k * cq->nx + i) * cq->ny + j;
          const double q = 1.0 / (x * x) + iy2[j];
          Atab[pt] = q * (1.0 - z * z);
          for (int iM = 0; iM < nM; ++iM) {
            const int Mp = c->Mps[iM];
            W[(size_t)iM * cq->npts + pt] = tot + q * Mp * (Mp + 1.0) + (J * (J + 1.0) - 2.0 * Mp * Mp) * iy2[j];
            Btab[(size_t)iM * cq->npts + pt] = 2.0 * (Mp + 1) * z * q;
          }
        }
    });
    for (int b : bad_plane)
      if (b) return FM_ERR_NUMERIC;
    tm.mark("potential tables");
    if ((rc = upload(c, (void**)&cp.W, W.data(), W.size() * sizeof(double)))) return rc;
    if ((rc = upload(c, (void**)&cp.A, Atab.data(), Atab.size() * sizeof(double)))) return rc;
    if ((rc = upload(c, (void**)&cp.B, Btab.data(), Btab.size() * sizeof(double)))) return rc;
    if ((rc = upload(c, (void**)&cp.iy2, iy2.data(), iy2.size() * sizeof(double)))) return rc;
    {  // float32 copies for the mixed-precision inner solves
      auto up32 = [&](float** dst, const std::vector<double>& v) {
        std::vector<float> f(v.begin(), v.end());
        return upload(c, (void**)dst, f.data(), f.size() * sizeof(float));
      };
      if ((rc = up32(&cp.f32.Sx, cp.ax.S)) || (rc = up32(&cp.f32.D2x, cp.ax.D2)) || (rc = up32(&cp.f32.Sy, cp.ay.S)) ||
          (rc = up32(&cp.f32.D2y, cp.ay.D2)) || (rc = up32(&cp.f32.Sz, cp.az.S)) || (rc = up32(&cp.f32.D1z, cp.az.D1)) ||
          (rc = up32(&cp.f32.D2z, cp.az.D2)) || (rc = up32(&cp.f32.zp, cp.az.pts)) || (rc = up32(&cp.f32.W, W)) ||
          (rc = up32(&cp.f32.A, Atab)) || (rc = up32(&cp.f32.B, Btab)) || (rc = up32(&cp.f32.iy2, iy2)))
        return rc;
    }
    if (c->use_dd) {  // double-float copies for the double-float inner solves
      auto updd = [&](dd** dst, const std::vector<double>& v) {
        std::vector<dd> f(v.begin(), v.end());
        return upload(c, (void**)dst, f.data(), f.size() * sizeof(dd));
      };
      if ((rc = updd(&cp.tdd.Sx, cp.ax.S)) || (rc = updd(&cp.tdd.D2x, cp.ax.D2)) || (rc = updd(&cp.tdd.Sy, cp.ay.S)) ||
          (rc = updd(&cp.tdd.D2y, cp.ay.D2)) || (rc = updd(&cp.tdd.Sz, cp.az.S)) || (rc = updd(&cp.tdd.D1z, cp.az.D1)) ||
          (rc = updd(&cp.tdd.D2z, cp.az.D2)) || (rc = updd(&cp.tdd.zp, cp.az.pts)) || (rc = updd(&cp.tdd.W, W)) ||
          (rc = updd(&cp.tdd.A, Atab)) || (rc = updd(&cp.tdd.B, Btab)) || (rc = updd(&cp.tdd.iy2, iy2)))
        return rc;
    }

    // coupling geometry (Eqs. r-form, s-rot): active points and, per source, taps and weights
    if (!cp.sources.empty()) {
      std::vector<int> act;
      std::vector<char> on_xy((size_t)cp.nx * cp.ny, 1);  // chi depends on (x, y) only
      if (c->split.mode == FM_SPLIT_MERKURIEV)
        for (int i = 0; i < cp.nx; ++i)
          for (int j = 0; j < cp.ny; ++j) on_xy[(size_t)i * cp.ny + j] = chi(c->split, cp.ax.pts[i], cp.ay.pts[j]) > c->split.vs_cut;
      for (int k = 0; k < cp.nz; ++k)
        for (int i = 0; i < cp.nx; ++i)
          for (int j = 0; j < cp.ny; ++j)
            if (on_xy[(size_t)i * cp.ny + j]) act.push_back((int)(((int64_t)k * cp.nx + i) * cp.ny + j));
      cp.n_act = (int)act.size();
      const int ns = (int)cp.sources.size(), na = cp.n_act;
      std::vector<int> base((size_t)ns * 3 * na);
      const int R = cp.r, R3 = 3 * cp.r;
      std::vector<double> val((size_t)ns * R3 * na), wt((size_t)ns * nM * nM * na);
      std::atomic<int> bad_w{0};
      const int chunk = 4096, nchunks = (na + chunk - 1) / chunk;
      for (int s = 0; s < ns; ++s) {
        const Source& src = cp.sources[s];
        const Comp& sc = c->comps[src.src];
        double cc, ss;
        rotation(m, src.beta, cp.label, &cc, &ss);
        parallel_for(nchunks, [&](int ch) {
        for (int p = ch * chunk; p < std::min(na, (ch + 1) * chunk); ++p) {
          const int pt = act[p];
          const int k = pt / (cp.nx * cp.ny), rem = pt % (cp.nx * cp.ny), i = rem / cp.ny, j = rem % cp.ny;
          const double z = cp.az.pts[k], x = cp.ax.pts[i], y = cp.ay.pts[j];
          double xb, yb, zb;
          rotate(cc, ss, x, y, z, &xb, &yb, &zb);
          const double w = w_angle(src.beta, cp.label, cc, ss, x, y, z, yb);
          int b3[3];
          double v[3 * kMaxTaps];
          sc.az.eval(src.zsign * zb, 0, &b3[0], v);
          sc.ax.eval(xb, 0, &b3[1], v + R);
          sc.ay.eval(yb, 0, &b3[2], v + 2 * R);
          for (int d = 0; d < 3; ++d) base[((size_t)s * 3 + d) * na + p] = b3[d];
          for (int t = 0; t < R3; ++t) val[((size_t)s * R3 + t) * na + p] = v[t];
          // weight V^(s)_a * rho * rho^{M''} * angular(M', M'') * [p (-1)^{M''}]
          const double vc = coulomb(c, cp.label, x);
          const double vs = (c->split.mode == FM_SPLIT_MERKURIEV) ? chi(c->split, x, y) * vc : vc;
          const double rho = x * y / (xb * yb);
          const double sin_t = std::sqrt(std::max(0.0, 1.0 - z * z));
          const double sgnw = first_branch(src.beta, cp.label) ? 1.0 : -1.0;
          for (int iM = 0; iM < nM; ++iM)
            for (int jM = 0; jM < nM; ++jM) {
              const int Mp = c->Mps[iM], Mpp = c->Mps[jM];
              double ang;
              if (Mpp >= Mp) {
                ang = ipow(sin_t, Mpp - Mp) * coupling_K(J, S.tau, Mp, Mpp, w, 0);
              } else {
                const int kk = Mp - Mpp;
                ang = ipow(std::fabs(ss) * x / yb, kk) * ipow(sgnw, kk) * coupling_K(J, S.tau, Mp, Mpp, w, kk);
              }
              double wv = vs * rho * ipow(rho, Mpp) * ang;
              if (src.sym) wv *= S.exch_p * ((Mpp % 2 == 0) ? 1.0 : -1.0);
              if (!std::isfinite(wv)) bad_w = 1;
              wt[(((size_t)s * nM * nM) + (size_t)iM * nM + jM) * na + p] = wv;
            }
        }
        });
      }
      if (bad_w) return FM_ERR_NUMERIC;
      tm.mark("coupling geometry");
      if ((rc = upload(c, (void**)&cp.act_pt, act.data(), act.size() * sizeof(int)))) return rc;
      if ((rc = upload(c, (void**)&cp.cpl_base, base.data(), base.size() * sizeof(int)))) return rc;
      if ((rc = upload(c, (void**)&cp.cpl_val, val.data(), val.size() * sizeof(double)))) return rc;
      if ((rc = upload(c, (void**)&cp.cpl_w, wt.data(), wt.size() * sizeof(double)))) return rc;
      std::vector<float> val32(val.begin(), val.end()), wt32(wt.begin(), wt.end());
      if ((rc = upload(c, (void**)&cp.f32.cval, val32.data(), val32.size() * sizeof(float)))) return rc;
      if ((rc = upload(c, (void**)&cp.f32.cw, wt32.data(), wt32.size() * sizeof(float)))) return rc;
      if (c->use_dd) {
        std::vector<dd> vdd(val.begin(), val.end()), wdd(wt.begin(), wt.end());
        if ((rc = upload(c, (void**)&cp.tdd.cval, vdd.data(), vdd.size() * sizeof(dd)))) return rc;
        if ((rc = upload(c, (void**)&cp.tdd.cw, wdd.data(), wdd.size() * sizeof(dd)))) return rc;
      }
    }

    tm.mark("coupling upload");
    // z decompositions per M' (Eq. z-dec), columns normalised to g_l^{M'}(1)
    const int nz = cp.nz, nx = cp.nx;
    std::vector<double> Wz((size_t)nM * nz * nz), Wzb((size_t)nM * nz * nz);
    cp.Lz.assign((size_t)nM * nz, 0.0);
    const std::vector<double> Szd = dense_of(cp.az, cp.az.S);
    for (int iM = 0; iM < nM; ++iM) {
      const int Mp = c->Mps[iM];
      std::vector<double> A1((size_t)nz * nz, 0.0);
      for (int q = 0; q < nz; ++q) {
        const double z = cp.az.pts[q];
        const int R = cp.az.r;
        for (int t = 0; t < R; ++t) {
          const int j = cp.az.base[q] + t;
          if (j < 0 || j >= nz) continue;
          A1[(size_t)q * nz + j] += (1.0 - z * z) * cp.az.D2[q * R + t] - 2.0 * (Mp + 1) * z * cp.az.D1[q * R + t] -
                                    Mp * (Mp + 1.0) * cp.az.S[q * R + t];
        }
      }
      double* Wb = &Wzb[(size_t)iM * nz * nz];
      double* Wr = &Wz[(size_t)iM * nz * nz];
      const int top = cp.az.q * cp.az.nint;  // value function of the node z = 1
      std::vector<int> kind(nz, 0);
      const int e = fmh::decompose_pairs(nz, A1.data(), Szd.data(), top, Wb, Wr, &cp.Lz[(size_t)iM * nz], kind.data());
      if (e == -1) return FM_ERR_COMPLEX_SPECTRUM;
      if (e != 0) return FM_ERR_NUMERIC;
      bool has_pairs = false;
      for (int kd : kind) has_pairs = has_pairs || kd != 0;
      if (has_pairs && c->opts.z_eigs == 1) return FM_ERR_COMPLEX_SPECTRUM;
      // columns scaled so their spline equals g_l^{M'}(1); the imaginary-part column of a
      // complex pair takes the scale of its real-part column
      double sc = 1.0;
      for (int l = 0; l < nz; ++l) {
        if (kind[l] != 2) {
          const double f1 = Wr[(size_t)top * nz + l];
          if (f1 == 0.0) return FM_ERR_NUMERIC;
          sc = g_at_one(Mp + l, Mp) / f1;
        }
        for (int q = 0; q < nz; ++q) Wr[(size_t)q * nz + l] *= sc;
        for (int q = 0; q < nz; ++q) Wb[(size_t)l * nz + q] /= sc;
      }
    }
    if ((rc = upload(c, (void**)&cp.Wz, Wz.data(), Wz.size() * 8))) return rc;
    if ((rc = upload(c, (void**)&cp.Wzb, Wzb.data(), Wzb.size() * 8))) return rc;
    {
      auto f = to_f32(Wz), fb = to_f32(Wzb);
      if ((rc = upload(c, (void**)&cp.Wz32, f.data(), f.size() * 4))) return rc;
      if ((rc = upload(c, (void**)&cp.Wzb32, fb.data(), fb.size() * 4))) return rc;
    }
    if (tc_requested(c) && nz <= 128) {  // tensor-core z stages: rows padded to 16-byte TMA strides
      const bool bf = c->opts.mma == FM_MMA_BF16;
      const int ld = bf ? (nz + 7) / 8 * 8 : (nz + 3) / 4 * 4;
      cp.ldz = ld;
      for (int which = 0; which < 2; ++which) {
        const std::vector<double>& src = which ? Wz : Wzb;
        std::vector<double> pad((size_t)nM * nz * ld, 0.0);
        for (int iM = 0; iM < nM; ++iM)
          for (int r = 0; r < nz; ++r)
            for (int q = 0; q < nz; ++q) pad[((size_t)iM * nz + r) * ld + q] = src[((size_t)iM * nz + r) * nz + q];
        void** dst = which ? &cp.Wz_tc : &cp.Wzb_tc;
        if (bf) {
          auto h = to_bf16(pad);
          if ((rc = upload(c, dst, h.data(), h.size() * 2))) return rc;
        } else {
          auto h = to_f32(pad);
          if ((rc = upload(c, dst, h.data(), h.size() * 4))) return rc;
        }
      }
    }
    // x decompositions per l = M0 .. J + nz - 1 (already done above unless computed z eigenvalues are kept)
    XD& d = xd[&cp - c->comps.data()];
    cp.nl = nM + nz - 1;
    const int nl = cp.nl;
    if (!x_first) {
      d.Wx.resize((size_t)nl * nx * nx);
      d.Wxb.resize((size_t)nl * nx * nx);
      d.err.assign(nl, 0);
      d.pairs.assign(nl, 0);
      cp.Lx.assign((size_t)nl * nx, 0.0);
      parallel_for(nl, [&](int il) { x_task(cp, il, d); });
    }
    for (int e : d.err) {
      if (e == -1) return FM_ERR_COMPLEX_SPECTRUM;
      if (e != 0) return FM_ERR_NUMERIC;
    }
    cp.x_pair_ls = 0;
    for (int p : d.pairs) cp.x_pair_ls += p;
    if (cp.x_pair_ls && getenv("FM_VERBOSE"))
      fprintf(stderr, "[fm_setup] component %d: %d x pencils with complex-conjugate pairs (real basis)\n", cp.label,
              cp.x_pair_ls);
    const std::vector<double>& Wx = d.Wx;
    const std::vector<double>& Wxb = d.Wxb;
    tm.mark("z decompositions");
    if ((rc = upload(c, (void**)&cp.Wx, Wx.data(), Wx.size() * 8))) return rc;
    if ((rc = upload(c, (void**)&cp.Wxb, Wxb.data(), Wxb.size() * 8))) return rc;
    {
      auto f = to_f32(Wx), fb = to_f32(Wxb);
      if ((rc = upload(c, (void**)&cp.Wx32, f.data(), f.size() * 4))) return rc;
      if ((rc = upload(c, (void**)&cp.Wxb32, fb.data(), fb.size() * 4))) return rc;
    }
    if (tc_requested(c) && c->opts.mma == FM_MMA_BF16) {
      auto h = to_bf16(Wx), hb = to_bf16(Wxb);
      if ((rc = upload(c, (void**)&cp.Wx16, h.data(), h.size() * 2))) return rc;
      if ((rc = upload(c, (void**)&cp.Wxb16, hb.data(), hb.size() * 2))) return rc;
    }
    // M' chains per l and the storage plan of the banded y factors
    cp.chain_lo.assign(nl, 0);
    cp.chain_n.assign(nl, 0);
    cp.band_off.assign(nl, 0);
    cp.lmul_off.assign(nl, 0);
    cp.piv_off.assign(nl, 0);
    int64_t bo = 0, lo = 0, po = 0;
    for (int il = 0; il < nl; ++il) {
      const int l = c->M0 + il;
      int first = -1, cnt = 0;
      for (int iM = 0; iM < nM; ++iM) {
        const int Mp = c->Mps[iM];
        if (Mp <= l && l <= Mp + nz - 1) {
          if (first < 0) first = iM;
          ++cnt;
        }
      }
      cp.chain_lo[il] = first;
      cp.chain_n[il] = cnt;
      const int n = cnt * cp.ny, kl = band_kl(cp.ay, cnt);
      if (kl > kMaxBandKL) return FM_ERR_ARG;  // M' chain too long for the banded y solve of this basis
      cp.band_off[il] = bo;
      cp.lmul_off[il] = lo;
      cp.piv_off[il] = po;
      bo += (int64_t)n * (2 * kl + 1) * nx;
      lo += (int64_t)n * (kl + 1) * nx;
      po += (int64_t)n * nx;
    }
    cp.band_total = bo;
    cp.lmul_total = lo;
    cp.piv_total = po;
    if ((rc = upload(c, (void**)&cp.d_chain_lo, cp.chain_lo.data(), nl * sizeof(int)))) return rc;
    if ((rc = upload(c, (void**)&cp.d_chain_n, cp.chain_n.data(), nl * sizeof(int)))) return rc;
    if ((rc = upload(c, (void**)&cp.d_band_off, cp.band_off.data(), nl * sizeof(int64_t)))) return rc;
    if ((rc = upload(c, (void**)&cp.d_lmul_off, cp.lmul_off.data(), nl * sizeof(int64_t)))) return rc;
    if ((rc = upload(c, (void**)&cp.d_piv_off, cp.piv_off.data(), nl * sizeof(int64_t)))) return rc;
    if ((rc = dev_alloc(c, (void**)&cp.yU, bo * 8))) return rc;
    if ((rc = dev_alloc(c, (void**)&cp.yL, lo * 8))) return rc;
    if ((rc = dev_alloc(c, (void**)&cp.yU32, bo * 4))) return rc;
    if ((rc = dev_alloc(c, (void**)&cp.yL32, lo * 4))) return rc;
    if (nM == 1) {
      const int ny = cp.ny;
      if ((rc = dev_alloc(c, (void**)&cp.Wy32, (size_t)nl * ny * ny * 4))) return rc;
      if ((rc = dev_alloc(c, (void**)&cp.Wyb32, (size_t)nl * ny * ny * 4))) return rc;
      if ((rc = dev_alloc(c, (void**)&cp.dLy32, (size_t)nl * ny * 4))) return rc;
      std::vector<float> lx32(cp.Lx.begin(), cp.Lx.end());
      if ((rc = upload(c, (void**)&cp.dLx32, lx32.data(), lx32.size() * 4))) return rc;
      if ((rc = dev_alloc(c, (void**)&cp.Wy64, (size_t)nl * ny * ny * 8))) return rc;
      if ((rc = dev_alloc(c, (void**)&cp.Wyb64, (size_t)nl * ny * ny * 8))) return rc;
      if ((rc = dev_alloc(c, (void**)&cp.dLy64, (size_t)nl * ny * 8))) return rc;
      if ((rc = upload(c, (void**)&cp.dLx64, cp.Lx.data(), cp.Lx.size() * 8))) return rc;
      std::vector<float2> lx2(cp.Lx.size());
      for (size_t q = 0; q < lx2.size(); ++q) lx2[q] = split2(cp.Lx[q]);
      if ((rc = upload(c, (void**)&cp.dLx2, lx2.data(), lx2.size() * sizeof(float2)))) return rc;
      if ((rc = dev_alloc(c, (void**)&cp.dLy2, (size_t)nl * ny * sizeof(float2)))) return rc;
      if (tc_requested(c) && c->opts.mma == FM_MMA_BF16) {
        if ((rc = dev_alloc(c, (void**)&cp.Wy16, (size_t)nl * ny * ny * 2))) return rc;
        if ((rc = dev_alloc(c, (void**)&cp.Wyb16, (size_t)nl * ny * ny * 2))) return rc;
      }
    }
    tm.mark("factor uploads");
  }
  return FM_OK;
}

// Device bytes a context with these parameters holds (the allocations of setup_host and fm_create,
// computed from the same size plan without allocating or decomposing anything).
int estimate_bytes(const fm_system* S, const fm_grid* grids, int n_grids, const fm_splitting* split, const fm_opts* o,
                   int64_t* out) {
  const int M0 = (1 - S->tau) / 2, nM = S->J - M0 + 1;
  if (nM <= 0 || nM > 12) return FM_ERR_ARG;
  std::vector<int> labels;
  if (split->mode == FM_SPLIT_SCHRODINGER) labels = {1};
  else if (S->identical_pair == 12) labels = {1, 3};
  else labels = {1, 2, 3};
  if (n_grids != 1 && n_grids != (int)labels.size()) return FM_ERR_ARG;
  double bytes = 0.0, dd_tables = 0.0;
  int64_t N = 0;
  for (size_t ic = 0; ic < labels.size(); ++ic) {
    const fm_grid& g = grids[n_grids == 1 ? 0 : ic];
    if (g.nint_x < 1 || g.nint_y < 1 || g.nint_z < 1 || !(g.Rx > 0) || !(g.Ry > 0)) return FM_ERR_ARG;
    if (g.basis < 0 || g.basis > 1) return FM_ERR_ARG;
    Axis ax, ay, az;
    ax.build(g.xmap, g.nint_x, 0.0, g.Rx, true, g.basis);
    ay.build(g.ymap, g.nint_y, 0.0, g.Ry, true, g.basis);
    az.build(g.zmap, g.nint_z, -1.0, 1.0, false, g.basis);
    const double R = ax.r;
    const double nx = ax.n, ny = ay.n, nz = az.n, npts = nx * ny * nz;
    N += (int64_t)(npts * nM);
    bytes += (nx + ny + nz) * (4 + 3 * R * 12 + 8) * 1.5;              // tap tables (float64 + float32)
    bytes += (2.0 * nM + 1.0) * npts * 12.0 + ny * 12.0;                 // W, B per M'; A; iy2 (+ float32)
    dd_tables += (nx + ny + nz) * 3 * R * 8 + (2.0 * nM + 1.0) * npts * 8.0;
    if (split->mode != FM_SPLIT_SCHRODINGER) {                           // coupling geometry
      double act = 0.0;
      for (int i = 0; i < ax.n; ++i)
        for (int j = 0; j < ay.n; ++j)
          if (split->mode != FM_SPLIT_MERKURIEV || chi(*split, ax.pts[i], ay.pts[j]) > split->vs_cut) act += 1.0;
      act *= nz;
      const double ns = 2.0;
      bytes += act * (4.0 + ns * (12.0 + 3.0 * R * 12.0 + nM * nM * 12.0));
      dd_tables += act * ns * (3.0 * R + nM * nM) * 8.0;
    }
    const double nl = nM + nz - 1;
    bytes += 2.0 * nM * nz * nz * 12.0 + 2.0 * nl * nx * nx * 12.0;     // z and x decompositions
    double bo = 0.0, lo = 0.0;                                           // banded y factors
    for (int il = 0; il < (int)nl; ++il) {
      const int l = M0 + il;
      int cnt = 0;
      for (int iM = 0; iM < nM; ++iM) {
        const int Mp = M0 + iM;
        if (Mp <= l && l <= Mp + (int)nz - 1) ++cnt;
      }
      const double n = cnt * ny, kl = band_kl(ay, cnt);
      bo += n * (2 * kl + 1) * nx;
      lo += n * (kl + 1) * nx;
    }
    bytes += bo * 12.0 + lo * 12.0;
    if (nM == 1) bytes += 2.0 * nl * ny * ny * 12.0 + nl * (nx + ny) * 20.0;  // per-l y diagonalisation
    if (o->precision != FM_PREC_FP64 && o->mma != FM_MMA_SIMT) {
      bytes += 2.0 * nM * nz * (nz + 8) * 4.0;                           // padded z factors of the tensor cores
      if (o->mma == FM_MMA_BF16) bytes += 2.0 * nl * (nx * nx + (nM == 1 ? ny * ny : 0.0)) * 2.0;
    }
  }
  const double m = o->restart_m, ncv = o->ncv, n = (double)N;
  if (o->precision == FM_PREC_MIXED && o->mixed_scheme == 2)
    bytes += dd_tables + n * 8.0 * ((m + 1) + m + 4);                  // double-float tables and Krylov vectors
  bytes += n * 8.0 * (5 + 2 + 3 + 16) + n * 4.0 * 2;                    // apply scratch, stage buffers, tuning
  bytes += n * 8.0 * ((m + 1) + std::max(m, ncv) + (ncv + 1));          // FGMRES and Arnoldi bases
  if (o->precision == FM_PREC_MIXED) bytes += n * 4.0 * ((m + 1) + m + 7 + 2.5);  // + y-interval sources
  bytes += (4.0 * 152 * 256 + 8192 + 4096) * 8.0;
  *out = (int64_t)bytes;
  return FM_OK;
}

// The E*-dependent banded y systems: for each (l, i_x) the block-tridiagonal (in M')
// system with banded blocks N^{M'}_{l i} = A1 + (J(J+1) - 2M'^2 + l(l+1)) A2 and
// N^{M'+-} = (off-diagonal coefficient) A2, where A1 = -D_y + V^ S_y - E* S_y +
// (Lambda_x^l)_{ii} S_y and A2 = Y_r2 S_y (Section 3.2, Eq. ops and the matrix L0).
// Factorised by banded LU with the unknowns ordered r = j * n_c + c.
int setup_shift(fm_ctx* c, double Estar) {
  const int J = c->sys.J;
  int rc;
  PhaseTimer tm;
  for (auto& cp : c->comps) {
    const int nx = cp.nx, ny = cp.ny;
    std::vector<double> U((size_t)cp.band_total), L((size_t)cp.lmul_total);
    std::vector<double> vh(ny);
    for (int j = 0; j < ny; ++j) vh[j] = vhat(c, cp.label, cp.ay.pts[j], cp.Ry);
    std::vector<int> bad(cp.nl, 0);
    const Comp* cpp = &cp;
    parallel_for(cp.nl, [&](int il) {
      const int l = c->M0 + il;
      const double ll1 = (c->opts.z_eigs == 1) ? -cpp->Lz[il] : (double)l * (l + 1);
      const int nc = cpp->chain_n[il], lo = cpp->chain_lo[il];
      const int n = nc * ny, kl = band_kl(cpp->ay, nc), ku = kl, wb = 2 * kl + ku + 1, wu = kl + ku + 1;
      const int R = cpp->ay.r;
      std::vector<double> B((size_t)n * wb), Lm((size_t)n * kl);
      std::vector<int> piv(n);
      for (int ix = 0; ix < nx; ++ix) {
        const double lx = cpp->Lx[(size_t)il * nx + ix];
        std::fill(B.begin(), B.end(), 0.0);
        for (int eta = 0; eta < ny; ++eta) {
          const double y = cpp->ay.pts[eta];
          for (int t = 0; t < R; ++t) {
            const int j = cpp->ay.base[eta] + t;
            if (j < 0 || j >= ny) continue;
            const double s = cpp->ay.S[eta * R + t], d2 = cpp->ay.D2[eta * R + t];
            const double a1 = -d2 + (vh[eta] - Estar + lx) * s;
            const double a2 = s / (y * y);
            for (int cc = 0; cc < nc; ++cc) {
              const int Mp = c->Mps[lo + cc];
              const int row = eta * nc + cc;
              auto put = [&](int col, double v) { B[(size_t)row * wb + (col - row + kl)] += v; };
              put(j * nc + cc, a1 + (J * (J + 1.0) - 2.0 * Mp * Mp + ll1) * a2);
              if (cc + 1 < nc) put(j * nc + cc + 1, lam_hat_plus(J, Mp) * (-lam(l, Mp)) * a2);
              if (cc >= 1) put(j * nc + cc - 1, -lam_hat_minus(J, Mp) * lam(l, -Mp) * a2);
            }
          }
        }
        if (!fmh::band_lu(n, kl, ku, B.data(), Lm.data(), piv.data())) {
          bad[il] = 1;
          return;
        }
        // per row r: U[r][0] = 1 / pivot, U[r][1..wu) the upper band; L[r][0] = pivot offset,
        // L[r][1..kl] = multipliers
        double* Ug = &U[cpp->band_off[il]];
        double* Lg = &L[cpp->lmul_off[il]];
        for (int r = 0; r < n; ++r) {
          Ug[((size_t)r * wu) * nx + ix] = 1.0 / B[(size_t)r * wb + kl];  // reciprocal of the pivot
          for (int d = 1; d < wu; ++d) Ug[((size_t)r * wu + d) * nx + ix] = B[(size_t)r * wb + kl + d];
          Lg[((size_t)r * (kl + 1)) * nx + ix] = (double)(piv[r] - r);
          for (int d = 0; d < kl; ++d) Lg[((size_t)r * (kl + 1) + d + 1) * nx + ix] = Lm[(size_t)r * kl + d];
        }
      }
    });
    for (int b : bad)
      if (b) return FM_ERR_NUMERIC;
    tm.mark("banded y factors");
    FM_CUDA(cudaMemcpyAsync(cp.yU, U.data(), U.size() * 8, cudaMemcpyHostToDevice, c->stream));
    FM_CUDA(cudaMemcpyAsync(cp.yL, L.data(), L.size() * 8, cudaMemcpyHostToDevice, c->stream));
    std::vector<float> U32(U.begin(), U.end()), L32(L.begin(), L.end());
    FM_CUDA(cudaMemcpyAsync(cp.yU32, U32.data(), U32.size() * 4, cudaMemcpyHostToDevice, c->stream));
    FM_CUDA(cudaMemcpyAsync(cp.yL32, L32.data(), L32.size() * 4, cudaMemcpyHostToDevice, c->stream));
    FM_CUDA(cudaStreamSynchronize(c->stream));
    tm.mark("banded y upload");
    cp.ydiag_ok = false;
  }
  // n_M = 1: (W-bar_y^l, W_y^l, Lambda_y^l) = D(A_l, S_y) with A_l = -D_y + (c_l / y^2 + V^ - E*) S_y; the block of
  // l is I (x) A_l + Lambda_x^l (x) S_y, inverted line by line as W_y (Lambda_y + lambda_x)^{-1} W-bar_y.  The
  // decompositions of every component run in one thread pool.
  if (c->nM == 1) {
    struct YD {
      Comp* cp;
      std::vector<double> Syd, D2yd, vh, Wy, Wyb, Ly;
      std::vector<int> err;
    };
    std::vector<YD> yd;
    for (auto& cp : c->comps) {
      if (!cp.Wy32) continue;
      YD d;
      d.cp = &cp;
      const int ny = cp.ny;
      d.Syd = dense_of(cp.ay, cp.ay.S);
      d.D2yd = dense_of(cp.ay, cp.ay.D2);
      d.vh.resize(ny);
      for (int j = 0; j < ny; ++j) d.vh[j] = vhat(c, cp.label, cp.ay.pts[j], cp.Ry);
      d.Wy.resize((size_t)cp.nl * ny * ny);
      d.Wyb.resize((size_t)cp.nl * ny * ny);
      d.Ly.resize((size_t)cp.nl * ny);
      d.err.assign(cp.nl, 0);
      yd.push_back(std::move(d));
    }
    std::vector<std::pair<int, int>> tasks;
    for (int q = 0; q < (int)yd.size(); ++q)
      for (int il = 0; il < yd[q].cp->nl; ++il) tasks.push_back({q, il});
    const int Mp = c->Mps[0];
    parallel_for((int)tasks.size(), [&](int ti) {
      YD& d = yd[tasks[ti].first];
      const Comp* cpp = d.cp;
      const int il = tasks[ti].second, ny = cpp->ny, l = c->M0 + il;
      const double ll1 = (c->opts.z_eigs == 1) ? -cpp->Lz[il] : (double)l * (l + 1);
      const double cl = J * (J + 1.0) - 2.0 * Mp * Mp + ll1;
      std::vector<double> A((size_t)ny * ny);
      for (int q = 0; q < ny; ++q) {
        const double y = cpp->ay.pts[q];
        const double f = cl / (y * y) + d.vh[q] - Estar;
        for (int j = 0; j < ny; ++j) A[(size_t)q * ny + j] = -d.D2yd[(size_t)q * ny + j] + f * d.Syd[(size_t)q * ny + j];
      }
      d.err[il] = fmh::decompose(ny, A.data(), d.Syd.data(), false, &d.Wyb[(size_t)il * ny * ny],
                                 &d.Wy[(size_t)il * ny * ny], &d.Ly[(size_t)il * ny]);
    });
    tm.mark("y diagonalisations");
    for (YD& d : yd) {
      Comp& cp = *d.cp;
      bool ok = true;
      for (int e : d.err) ok = ok && (e == 0);
      if (!ok) continue;  // complex or singular: the banded y solves serve this component
      std::vector<float> a32(d.Wy.begin(), d.Wy.end()), b32(d.Wyb.begin(), d.Wyb.end()), l32(d.Ly.begin(), d.Ly.end());
      FM_CUDA(cudaMemcpyAsync(cp.Wy32, a32.data(), a32.size() * 4, cudaMemcpyHostToDevice, c->stream));
      FM_CUDA(cudaMemcpyAsync(cp.Wyb32, b32.data(), b32.size() * 4, cudaMemcpyHostToDevice, c->stream));
      FM_CUDA(cudaMemcpyAsync(cp.dLy32, l32.data(), l32.size() * 4, cudaMemcpyHostToDevice, c->stream));
      FM_CUDA(cudaMemcpyAsync(cp.Wy64, d.Wy.data(), d.Wy.size() * 8, cudaMemcpyHostToDevice, c->stream));
      FM_CUDA(cudaMemcpyAsync(cp.Wyb64, d.Wyb.data(), d.Wyb.size() * 8, cudaMemcpyHostToDevice, c->stream));
      FM_CUDA(cudaMemcpyAsync(cp.dLy64, d.Ly.data(), d.Ly.size() * 8, cudaMemcpyHostToDevice, c->stream));
      std::vector<float2> ly2(d.Ly.size());
      for (size_t q = 0; q < ly2.size(); ++q) ly2[q] = split2(d.Ly[q]);
      FM_CUDA(cudaMemcpyAsync(cp.dLy2, ly2.data(), ly2.size() * sizeof(float2), cudaMemcpyHostToDevice, c->stream));
      std::vector<uint16_t> a16, b16;
      if (cp.Wy16) {
        a16 = to_bf16(d.Wy);
        b16 = to_bf16(d.Wyb);
        FM_CUDA(cudaMemcpyAsync(cp.Wy16, a16.data(), a16.size() * 2, cudaMemcpyHostToDevice, c->stream));
        FM_CUDA(cudaMemcpyAsync(cp.Wyb16, b16.data(), b16.size() * 2, cudaMemcpyHostToDevice, c->stream));
      }
      FM_CUDA(cudaStreamSynchronize(c->stream));
      cp.ydiag_ok = true;
    }
    tm.mark("y diagonalisation upload");
  }
  c->Estar = Estar;
  c->have_shift = true;
  (void)rc;
  return FM_OK;
}

}  // namespace fmi

extern "C" int fm_host_axis(int map, int nint, double a, double b, int dirichlet, int basis, int* n, int* r,
                            double* pts, int* base, double* S, double* D1, double* D2) {
  if (nint < 1 || !(b > a) || basis < 0 || basis > 1 || map < 0 || map > 2 || !n || !r || !pts || !base || !S || !D1 ||
      !D2)
    return FM_ERR_ARG;
  fmi::Axis A;
  A.build(map, nint, a, b, dirichlet != 0, basis);
  *n = A.n;
  *r = A.r;
  for (int e = 0; e < A.n; ++e) {
    pts[e] = A.pts[e];
    base[e] = A.base[e];
    for (int t = 0; t < A.r; ++t) {
      S[e * A.r + t] = A.S[e * A.r + t];
      D1[e * A.r + t] = A.D1[e * A.r + t];
      D2[e * A.r + t] = A.D2[e * A.r + t];
    }
  }
  return FM_OK;
}
