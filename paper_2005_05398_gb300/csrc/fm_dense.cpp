// Small dense and banded linear algebra on the host (row-major, float64).
// See fm_dense.h.  Algorithms: Gaussian elimination with partial pivoting;
// balancing by powers of two (Parlett-Reinsch); Householder reduction to
// Hessenberg form; the Francis implicit double-shift QR iteration for the
// eigenvalues of a Hessenberg matrix; inverse iteration for eigenvectors;
// banded Gaussian elimination with row interchanges.
#include "fm_dense.h"

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <numeric>

namespace fmh {

static inline double& at(double* A, int n, int i, int j) { return A[(size_t)i * n + j]; }

// sum_j a[j] b[j] in four independent partial sums (instruction-level parallelism; vectorisable)
static inline double dot4(const double* a, const double* b, int m) {
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  int j = 0;
  for (; j + 4 <= m; j += 4) {
    s0 += a[j] * b[j];
    s1 += a[j + 1] * b[j + 1];
    s2 += a[j + 2] * b[j + 2];
    s3 += a[j + 3] * b[j + 3];
  }
  for (; j < m; ++j) s0 += a[j] * b[j];
  return (s0 + s1) + (s2 + s3);
}

bool lu_factor(int n, double* A, int* piv) {
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = std::fabs(at(A, n, k, k));
    for (int i = k + 1; i < n; ++i) {
      double v = std::fabs(at(A, n, i, k));
      if (v > best) { best = v; p = i; }
    }
    piv[k] = p;
    if (best == 0.0 || !std::isfinite(best)) return false;
    if (p != k)  // swap the active part only: multipliers stay where step k made them
      for (int j = k; j < n; ++j) std::swap(at(A, n, k, j), at(A, n, p, j));
    const double inv = 1.0 / at(A, n, k, k);
    for (int i = k + 1; i < n; ++i) {
      double l = at(A, n, i, k) * inv;
      at(A, n, i, k) = l;
      if (l != 0.0)
        for (int j = k + 1; j < n; ++j) at(A, n, i, j) -= l * at(A, n, k, j);
    }
  }
  return true;
}

void lu_solve(int n, const double* LU, const int* piv, double* b) {
  for (int k = 0; k < n; ++k) {
    if (piv[k] != k) std::swap(b[k], b[piv[k]]);
    for (int i = k + 1; i < n; ++i) b[i] -= LU[(size_t)i * n + k] * b[k];
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = b[i];
    for (int j = i + 1; j < n; ++j) s -= LU[(size_t)i * n + j] * b[j];
    b[i] = s / LU[(size_t)i * n + i];
  }
}

// X = A^{-1} B for n x n row-major B (m columns = n) from the LU factors, by whole-row operations (the
// rows are contiguous: forward and back substitution as row AXPYs instead of strided column walks)
static void lu_solve_rows(int n, const double* LU, const int* piv, double* B) {
  // forward: the swaps interleaved with the elimination steps, as lu_factor made them (its multipliers
  // of step k are not permuted by the later swaps)
  for (int k = 0; k < n; ++k) {
    double* bk = B + (size_t)k * n;
    if (piv[k] != k)
      for (int j = 0; j < n; ++j) std::swap(bk[j], B[(size_t)piv[k] * n + j]);
    for (int i = k + 1; i < n; ++i) {
      const double l = LU[(size_t)i * n + k];
      if (l == 0.0) continue;
      double* bi = B + (size_t)i * n;
      for (int j = 0; j < n; ++j) bi[j] -= l * bk[j];
    }
  }
  for (int i = n - 1; i >= 0; --i) {
    double* bi = B + (size_t)i * n;
    for (int k = i + 1; k < n; ++k) {
      const double u = LU[(size_t)i * n + k];
      if (u == 0.0) continue;
      const double* bk = B + (size_t)k * n;
      for (int j = 0; j < n; ++j) bi[j] -= u * bk[j];
    }
    const double inv = 1.0 / LU[(size_t)i * n + i];
    for (int j = 0; j < n; ++j) bi[j] *= inv;
  }
}

bool invert(int n, const double* A, double* Ainv) {
  std::vector<double> LU(A, A + (size_t)n * n);
  std::vector<int> piv(n);
  if (!lu_factor(n, LU.data(), piv.data())) return false;
  std::fill(Ainv, Ainv + (size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) Ainv[(size_t)i * n + i] = 1.0;
  lu_solve_rows(n, LU.data(), piv.data(), Ainv);
  return true;
}

// Scale rows/columns by powers of two so that row and column norms are comparable:
// B = D^{-1} A D, returns D.
static void balance(int n, double* A, double* D) {
  for (int i = 0; i < n; ++i) D[i] = 1.0;
  bool changed = true;
  for (int sweep = 0; changed && sweep < 100; ++sweep) {
    changed = false;
    for (int i = 0; i < n; ++i) {
      double c = 0.0, r = 0.0;
      for (int j = 0; j < n; ++j) {
        if (j == i) continue;
        c += std::fabs(at(A, n, j, i));
        r += std::fabs(at(A, n, i, j));
      }
      if (c == 0.0 || r == 0.0 || !std::isfinite(c) || !std::isfinite(r)) continue;
      const double total = c + r;
      double f = 1.0;
      while (c * f < r / f * 0.5) f *= 2.0;
      while (c * f > r / f * 2.0) f *= 0.5;
      if ((c * f + r / f) < 0.95 * total) {
        D[i] *= f;
        for (int j = 0; j < n; ++j) at(A, n, i, j) /= f;  // row i of D^{-1} A
        for (int j = 0; j < n; ++j) at(A, n, j, i) *= f;  // column i of A D
        changed = true;
      }
    }
  }
}

// Householder reduction: A := Q^T A Q upper Hessenberg, Q accumulated (Q may be null).
static void hessenberg(int n, double* A, double* Q) {
  if (Q) {
    std::fill(Q, Q + (size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) at(Q, n, i, i) = 1.0;
  }
  std::vector<double> v(n), srow(n);
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1;  // length of the reflector, rows k+1..n-1
    double nrm = 0.0;
    for (int i = 0; i < m; ++i) nrm += at(A, n, k + 1 + i, k) * at(A, n, k + 1 + i, k);
    nrm = std::sqrt(nrm);
    if (nrm == 0.0) continue;
    const double x0 = at(A, n, k + 1, k);
    const double alpha = (x0 >= 0.0) ? -nrm : nrm;
    for (int i = 0; i < m; ++i) v[i] = at(A, n, k + 1 + i, k);
    v[0] -= alpha;
    double vn = 0.0;
    for (int i = 0; i < m; ++i) vn += v[i] * v[i];
    if (vn == 0.0) continue;
    const double beta = 2.0 / vn;
    {  // left: rows k+1..n-1, s = beta v^T A[k+1.., k..] accumulated row by row (contiguous)
      std::fill(srow.begin() + k, srow.end(), 0.0);
      for (int i = 0; i < m; ++i) {
        const double vi = v[i];
        const double* ar = A + (size_t)(k + 1 + i) * n;
        for (int j = k; j < n; ++j) srow[j] += vi * ar[j];
      }
      for (int j = k; j < n; ++j) srow[j] *= beta;
      for (int i = 0; i < m; ++i) {
        const double vi = v[i];
        double* ar = A + (size_t)(k + 1 + i) * n;
        for (int j = k; j < n; ++j) ar[j] -= srow[j] * vi;
      }
    }
    for (int i = 0; i < n; ++i) {  // right: columns k+1..n-1
      double* ar = A + (size_t)i * n + k + 1;
      const double s = beta * dot4(ar, v.data(), m);
      for (int j = 0; j < m; ++j) ar[j] -= s * v[j];
    }
    if (Q)
      for (int i = 0; i < n; ++i) {
        double* qr = Q + (size_t)i * n + k + 1;
        const double s = beta * dot4(qr, v.data(), m);
        for (int j = 0; j < m; ++j) qr[j] -= s * v[j];
      }
    at(A, n, k + 1, k) = alpha;
    for (int i = k + 2; i < n; ++i) at(A, n, i, k) = 0.0;
  }
}

// Reflector P = I - beta u u^T with P [a b c]^T = (r, 0, 0)^T; u[0] = 1 convention not used.
static void make_reflector(int len, const double* x, double* u, double& beta) {
  double nrm = 0.0;
  for (int i = 0; i < len; ++i) nrm += x[i] * x[i];
  nrm = std::sqrt(nrm);
  for (int i = 0; i < len; ++i) u[i] = x[i];
  if (nrm == 0.0) { beta = 0.0; return; }
  u[0] += (x[0] >= 0.0 ? nrm : -nrm);
  double un = 0.0;
  for (int i = 0; i < len; ++i) un += u[i] * u[i];
  beta = (un == 0.0) ? 0.0 : 2.0 / un;
}

int hess_eigvals(int n, const double* Hin, double* re, double* im) {
  std::vector<double> H(Hin, Hin + (size_t)n * n);
  double* A = H.data();
  double anorm = 0.0;
  for (int i = 0; i < n; ++i)
    for (int j = std::max(0, i - 1); j < n; ++j) anorm += std::fabs(at(A, n, i, j));
  if (anorm == 0.0) {
    for (int i = 0; i < n; ++i) re[i] = im[i] = 0.0;
    return 0;
  }
  const double eps = 2.220446049250313e-16;
  int hi = n - 1;
  int its = 0;
  while (hi >= 0) {
    // find the start of the unreduced block ending at hi
    int lo = hi;
    while (lo > 0) {
      double s = std::fabs(at(A, n, lo - 1, lo - 1)) + std::fabs(at(A, n, lo, lo));
      if (s == 0.0) s = anorm;
      if (std::fabs(at(A, n, lo, lo - 1)) <= eps * s) {
        at(A, n, lo, lo - 1) = 0.0;
        break;
      }
      --lo;
    }
    if (lo == hi) {  // 1x1 block
      re[hi] = at(A, n, hi, hi);
      im[hi] = 0.0;
      --hi;
      its = 0;
      continue;
    }
    if (lo == hi - 1) {  // 2x2 block: eigenvalues of [[a b][c d]]
      const double a = at(A, n, hi - 1, hi - 1), b = at(A, n, hi - 1, hi);
      const double c = at(A, n, hi, hi - 1), d = at(A, n, hi, hi);
      const double p = 0.5 * (a - d), disc = p * p + b * c;
      const double mid = 0.5 * (a + d);
      if (disc >= 0.0) {
        const double sq = std::sqrt(disc);
        // root of larger magnitude first (no cancellation), the other from the determinant
        const double r1 = mid + (mid >= 0.0 ? sq : -sq);
        const double det = a * d - b * c;
        const double r2 = (r1 != 0.0) ? det / r1 : 0.0;
        re[hi - 1] = r1; re[hi] = r2;
        im[hi - 1] = im[hi] = 0.0;
      } else {
        const double sq = std::sqrt(-disc);
        re[hi - 1] = re[hi] = mid;
        im[hi - 1] = sq; im[hi] = -sq;
      }
      hi -= 2;
      its = 0;
      continue;
    }
    if (++its > 60) return -1;
    // double-shift polynomial from the trailing 2x2 (exceptional shifts now and then)
    double s, t;
    if (its % 11 == 10) {
      const double w = std::fabs(at(A, n, hi, hi - 1)) + std::fabs(at(A, n, hi - 1, hi - 2));
      s = 1.5 * w + at(A, n, hi, hi);
      t = w * w;
    } else {
      s = at(A, n, hi - 1, hi - 1) + at(A, n, hi, hi);
      t = at(A, n, hi - 1, hi - 1) * at(A, n, hi, hi) - at(A, n, hi - 1, hi) * at(A, n, hi, hi - 1);
    }
    double x[3];
    x[0] = at(A, n, lo, lo) * at(A, n, lo, lo) + at(A, n, lo, lo + 1) * at(A, n, lo + 1, lo) - s * at(A, n, lo, lo) + t;
    x[1] = at(A, n, lo + 1, lo) * (at(A, n, lo, lo) + at(A, n, lo + 1, lo + 1) - s);
    x[2] = at(A, n, lo + 1, lo) * at(A, n, lo + 2, lo + 1);
    for (int k = lo; k <= hi - 2; ++k) {
      double u[3], beta;
      make_reflector(3, x, u, beta);
      if (beta != 0.0) {
        const int c0 = std::max(lo, k - 1);
        for (int j = c0; j <= hi; ++j) {
          double d = u[0] * at(A, n, k, j) + u[1] * at(A, n, k + 1, j) + u[2] * at(A, n, k + 2, j);
          d *= beta;
          at(A, n, k, j) -= d * u[0];
          at(A, n, k + 1, j) -= d * u[1];
          at(A, n, k + 2, j) -= d * u[2];
        }
        const int r1 = std::min(k + 3, hi);
        for (int i = lo; i <= r1; ++i) {
          double d = u[0] * at(A, n, i, k) + u[1] * at(A, n, i, k + 1) + u[2] * at(A, n, i, k + 2);
          d *= beta;
          at(A, n, i, k) -= d * u[0];
          at(A, n, i, k + 1) -= d * u[1];
          at(A, n, i, k + 2) -= d * u[2];
        }
      }
      x[0] = at(A, n, k + 1, k);
      x[1] = at(A, n, k + 2, k);
      x[2] = (k + 3 <= hi) ? at(A, n, k + 3, k) : 0.0;
    }
    {  // final 2-element reflector on rows/cols hi-1, hi
      double u[2], beta;
      make_reflector(2, x, u, beta);
      const int k = hi - 1;
      if (beta != 0.0) {
        for (int j = std::max(lo, k - 1); j <= hi; ++j) {
          double d = beta * (u[0] * at(A, n, k, j) + u[1] * at(A, n, k + 1, j));
          at(A, n, k, j) -= d * u[0];
          at(A, n, k + 1, j) -= d * u[1];
        }
        for (int i = lo; i <= hi; ++i) {
          double d = beta * (u[0] * at(A, n, i, k) + u[1] * at(A, n, i, k + 1));
          at(A, n, i, k) -= d * u[0];
          at(A, n, i, k + 1) -= d * u[1];
        }
      }
    }
    // clean the entries below the subdiagonal the bulge chase leaves by rounding (the 3-element reflectors
    // touch only (i, i-2) and (i, i-3))
    for (int i = lo + 2; i <= hi; ++i) {
      at(A, n, i, i - 2) = 0.0;
      if (i - 3 >= lo) at(A, n, i, i - 3) = 0.0;
    }
  }
  return 0;
}

// LU factors of (H - mu I) for upper-Hessenberg H by elimination with adjacent-row pivoting: M holds U
// (rows from their diagonal on), l[k] the multiplier of step k and sw[k] whether rows k, k+1 were swapped.
static void hess_shifted_factor(int n, const double* H, double mu, double tiny, double* M, double* l, char* sw) {
  for (int i = 0; i < n; ++i) {
    const int j0 = std::max(0, i - 1);
    for (int j = j0; j < n; ++j) M[(size_t)i * n + j] = H[(size_t)i * n + j] - (i == j ? mu : 0.0);
  }
  for (int k = 0; k + 1 < n; ++k) {
    double* rk = M + (size_t)k * n;
    double* r1 = M + (size_t)(k + 1) * n;
    sw[k] = std::fabs(r1[k]) > std::fabs(rk[k]);
    if (sw[k])
      for (int j = k; j < n; ++j) std::swap(rk[j], r1[j]);
    if (rk[k] == 0.0) rk[k] = tiny;
    l[k] = r1[k] / rk[k];
    if (l[k] != 0.0)
      for (int j = k + 1; j < n; ++j) r1[j] -= l[k] * rk[j];
  }
  if (M[(size_t)(n - 1) * n + n - 1] == 0.0) M[(size_t)(n - 1) * n + n - 1] = tiny;
}

// y <- (H - mu I)^{-1} y with the factors of hess_shifted_factor
static void hess_shifted_lu_solve(int n, const double* M, const double* l, const char* sw, double* b) {
  for (int k = 0; k + 1 < n; ++k) {
    if (sw[k]) std::swap(b[k], b[k + 1]);
    b[k + 1] -= l[k] * b[k];
  }
  for (int i = n - 1; i >= 0; --i) {
    const double* ri = M + (size_t)i * n;
    b[i] = (b[i] - dot4(ri + i + 1, b + i + 1, n - i - 1)) / ri[i];
  }
}

using cplx = std::complex<double>;

// Solve (H - mu I) y = b for upper-Hessenberg H and complex mu (adjacent-row pivoting).
static void hess_shifted_solve_c(int n, const double* H, cplx mu, double tiny, cplx* b, cplx* M) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      M[(size_t)i * n + j] = (j >= i - 1) ? cplx(H[(size_t)i * n + j]) - (i == j ? mu : cplx(0.0)) : cplx(0.0);
  for (int k = 0; k + 1 < n; ++k) {
    cplx* rk = M + (size_t)k * n;
    cplx* r1 = M + (size_t)(k + 1) * n;
    if (std::abs(r1[k]) > std::abs(rk[k])) {
      for (int j = k; j < n; ++j) std::swap(rk[j], r1[j]);
      std::swap(b[k], b[k + 1]);
    }
    if (rk[k] == cplx(0.0)) rk[k] = tiny;
    const cplx l = r1[k] / rk[k];
    if (l != cplx(0.0)) {
      for (int j = k; j < n; ++j) r1[j] -= l * rk[j];
      b[k + 1] -= l * b[k];
    }
  }
  for (int i = n - 1; i >= 0; --i) {
    cplx* ri = M + (size_t)i * n;
    if (ri[i] == cplx(0.0)) ri[i] = tiny;
    cplx sacc = b[i];
    for (int j = i + 1; j < n; ++j) sacc -= ri[j] * b[j];
    b[i] = sacc / ri[i];
  }
}

// All eigenvalues (re, im) of A and unit eigenvectors (real part Vr, imaginary part Vi; Vi = 0 for
// real eigenvalues).  Returns -1 on no convergence, 1 if a complex eigenvalue occurred, 0 otherwise.
int eig_general2(int n, const double* Ain, double* re, double* im, double* Vr, double* Vi) {
  std::vector<double> A(Ain, Ain + (size_t)n * n), D(n), Q((size_t)n * n);
  balance(n, A.data(), D.data());
  hessenberg(n, A.data(), Q.data());
  if (hess_eigvals(n, A.data(), re, im) != 0) return -1;
  double maxabs = 0.0, hn = 0.0;
  for (int i = 0; i < n; ++i) maxabs = std::max(maxabs, std::hypot(re[i], im[i]));
  for (size_t i = 0; i < A.size(); ++i) hn = std::max(hn, std::fabs(A[i]));
  int status = 0;
  std::vector<double> work((size_t)n * n), y(n), lmul(n);
  std::vector<char> swp(n);
  std::vector<cplx> cwork((size_t)n * n), cy(n);
  std::vector<double> Yh((size_t)n * n, 0.0);  // Hessenberg-basis eigenvectors of the real eigenvalues
  std::vector<int> real_cols;
  const double tiny = 1e-15 * (hn > 0 ? hn : 1.0);
  for (int e = 0; e < n; ++e) {
    const bool cx = std::fabs(im[e]) > 1e-10 * maxabs;
    if (!cx) {
      im[e] = 0.0;
      for (int i = 0; i < n; ++i) y[i] = 1.0 + 0.1 * std::sin(1.0 + 3.7 * i + 0.3 * e);
      hess_shifted_factor(n, A.data(), re[e], tiny, work.data(), lmul.data(), swp.data());
      for (int it = 0; it < 3; ++it) {
        hess_shifted_lu_solve(n, work.data(), lmul.data(), swp.data(), y.data());
        double nr = 0.0;
        for (int i = 0; i < n; ++i) nr += y[i] * y[i];
        nr = std::sqrt(nr);
        if (!(nr > 0.0) || !std::isfinite(nr)) return -1;
        for (int i = 0; i < n; ++i) y[i] /= nr;
      }
      // Hessenberg-basis eigenvector, column e of Y; all real ones are back-transformed together below
      for (int i = 0; i < n; ++i) Yh[(size_t)i * n + e] = y[i];
      real_cols.push_back(e);
      for (int i = 0; i < n; ++i) Vi[(size_t)i * n + e] = 0.0;
      continue;
    }
    status = 1;
    const cplx mu(re[e], im[e]);
    for (int i = 0; i < n; ++i) cy[i] = cplx(1.0 + 0.1 * std::sin(1.0 + 3.7 * i + 0.3 * e), 0.05 * std::cos(0.7 * i));
    for (int it = 0; it < 3; ++it) {
      hess_shifted_solve_c(n, A.data(), mu, tiny, cy.data(), cwork.data());
      double nr = 0.0;
      for (int i = 0; i < n; ++i) nr += std::norm(cy[i]);
      nr = std::sqrt(nr);
      if (!(nr > 0.0) || !std::isfinite(nr)) return -1;
      for (int i = 0; i < n; ++i) cy[i] /= nr;
    }
    double nr = 0.0;
    std::vector<cplx> v(n);
    for (int i = 0; i < n; ++i) {
      cplx sacc = 0.0;
      for (int j = 0; j < n; ++j) sacc += Q[(size_t)i * n + j] * cy[j];
      v[i] = D[i] * sacc;
      nr += std::norm(v[i]);
    }
    nr = std::sqrt(nr);
    for (int i = 0; i < n; ++i) {
      Vr[(size_t)i * n + e] = v[i].real() / nr;
      Vi[(size_t)i * n + e] = v[i].imag() / nr;
    }
  }
  if (!real_cols.empty()) {
    // V = D Q Y for the real eigenvectors at once, by rows (row i of Q times the rows of Y: contiguous AXPYs)
    std::vector<double> Vt((size_t)n * n, 0.0), nrm2(n, 0.0);
    for (int i = 0; i < n; ++i) {
      double* vt = Vt.data() + (size_t)i * n;
      const double* qi = Q.data() + (size_t)i * n;
      for (int j = 0; j < n; ++j) {
        const double q = qi[j];
        if (q == 0.0) continue;
        const double* yj = Yh.data() + (size_t)j * n;
        for (int e = 0; e < n; ++e) vt[e] += q * yj[e];
      }
      for (int e = 0; e < n; ++e) {
        vt[e] *= D[i];
        nrm2[e] += vt[e] * vt[e];
      }
    }
    for (int e : real_cols) {
      const double inv = 1.0 / std::sqrt(nrm2[e]);
      for (int i = 0; i < n; ++i) Vr[(size_t)i * n + e] = Vt[(size_t)i * n + e] * inv;
    }
  }
  return status;
}

int eig_general(int n, const double* Ain, double* re, double* im, double* V) {
  std::vector<double> Vi((size_t)n * n);
  const int st = eig_general2(n, Ain, re, im, V, Vi.data());
  if (st < 0) return st;
  for (int e = 0; e < n; ++e)
    if (im[e] != 0.0)
      for (int i = 0; i < n; ++i) V[(size_t)i * n + e] = 0.0;
  return st;
}

int eig_real(int n, const double* Ain, double* lam, double* V) {
  std::vector<double> im(n);
  const int st = eig_general(n, Ain, lam, im.data(), V);
  return st == 0 ? 0 : -1;
}

int decompose(int n, const double* A1, const double* A2, bool descending, double* Wbar, double* W, double* lam) {
  // C = A2^{-1} A1
  std::vector<double> LU(A2, A2 + (size_t)n * n), C(A1, A1 + (size_t)n * n);
  std::vector<int> piv(n);
  if (!lu_factor(n, LU.data(), piv.data())) return -2;
  lu_solve_rows(n, LU.data(), piv.data(), C.data());
  std::vector<double> l(n), V((size_t)n * n);
  if (eig_real(n, C.data(), l.data(), V.data()) != 0) return -1;
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::sort(order.begin(), order.end(), [&](int a, int b) { return descending ? l[a] > l[b] : l[a] < l[b]; });
  for (int e = 0; e < n; ++e) {
    lam[e] = l[order[e]];
    for (int i = 0; i < n; ++i) W[(size_t)i * n + e] = V[(size_t)i * n + order[e]];
  }
  // W-bar = (A2 W)^{-1}
  std::vector<double> A2W((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k) {
      const double a = A2[(size_t)i * n + k];
      if (a == 0.0) continue;
      for (int j = 0; j < n; ++j) A2W[(size_t)i * n + j] += a * W[(size_t)k * n + j];
    }
  if (!invert(n, A2W.data(), Wbar)) return -2;
  return 0;
}

int decompose_pairs(int n, const double* A1, const double* A2, int top, double* Wbar, double* W, double* lam,
                    int* kind) {
  std::vector<double> LU(A2, A2 + (size_t)n * n), C(A1, A1 + (size_t)n * n);
  std::vector<int> piv(n);
  if (!lu_factor(n, LU.data(), piv.data())) return -2;
  lu_solve_rows(n, LU.data(), piv.data(), C.data());
  std::vector<double> re(n), im(n), Vr((size_t)n * n), Vi((size_t)n * n);
  if (eig_general2(n, C.data(), re.data(), im.data(), Vr.data(), Vi.data()) < 0) return -1;
  std::vector<int> order;
  for (int e = 0; e < n; ++e)
    if (im[e] >= 0.0) order.push_back(e);  // one member of every conjugate pair
  std::sort(order.begin(), order.end(), [&](int a, int b) { return re[a] > re[b] || (re[a] == re[b] && a < b); });
  int c = 0;
  for (int e : order) {
    if (im[e] == 0.0) {
      for (int i = 0; i < n; ++i) W[(size_t)i * n + c] = Vr[(size_t)i * n + e];
      lam[c] = re[e];
      kind[c] = 0;
      ++c;
    } else {
      if (c + 1 >= n) return -1;
      // phase so that coefficient 'top' (the value at z = 1 for the z axis; the largest coefficient when
      // top < 0) is real and positive
      int tp = top;
      if (tp < 0) {
        tp = 0;
        for (int i = 1; i < n; ++i)
          if (std::hypot(Vr[(size_t)i * n + e], Vi[(size_t)i * n + e]) >
              std::hypot(Vr[(size_t)tp * n + e], Vi[(size_t)tp * n + e]))
            tp = i;
      }
      const cplx f(Vr[(size_t)tp * n + e], Vi[(size_t)tp * n + e]);
      if (std::abs(f) == 0.0) return -1;
      const cplx ph = std::conj(f) / std::abs(f);
      for (int i = 0; i < n; ++i) {
        const cplx w = cplx(Vr[(size_t)i * n + e], Vi[(size_t)i * n + e]) * ph;
        W[(size_t)i * n + c] = w.real();
        W[(size_t)i * n + c + 1] = w.imag();
      }
      lam[c] = lam[c + 1] = re[e];
      kind[c] = 1;
      kind[c + 1] = 2;
      c += 2;
    }
  }
  if (c != n) return -1;
  std::vector<double> A2W((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k) {
      const double a = A2[(size_t)i * n + k];
      if (a == 0.0) continue;
      for (int j = 0; j < n; ++j) A2W[(size_t)i * n + j] += a * W[(size_t)k * n + j];
    }
  if (!invert(n, A2W.data(), Wbar)) return -2;
  return 0;
}

bool band_lu(int n, int kl, int ku, double* B, double* Lmul, int* piv) {
  const int w = 2 * kl + ku + 1;
  auto el = [&](int i, int j) -> double& { return B[(size_t)i * w + (j - i + kl)]; };
  for (int j = 0; j < n; ++j) {
    const int last = std::min(n - 1, j + kl);
    int p = j;
    double best = std::fabs(el(j, j));
    for (int i = j + 1; i <= last; ++i) {
      double v = std::fabs(el(i, j));
      if (v > best) { best = v; p = i; }
    }
    piv[j] = p;
    if (best == 0.0 || !std::isfinite(best)) return false;
    const int cmax = std::min(n - 1, j + kl + ku);
    if (p != j)
      for (int c = j; c <= cmax; ++c) std::swap(el(j, c), el(p, c));
    const double inv = 1.0 / el(j, j);
    for (int r = 1; r <= kl; ++r) {
      const int i = j + r;
      double l = 0.0;
      if (i <= last) {
        l = el(i, j) * inv;
        el(i, j) = 0.0;
        if (l != 0.0)
          for (int c = j + 1; c <= cmax; ++c) el(i, c) -= l * el(j, c);
      }
      Lmul[(size_t)j * kl + (r - 1)] = l;
    }
  }
  return true;
}

void band_solve(int n, int kl, int ku, const double* B, const double* Lmul, const int* piv, double* x) {
  const int w = 2 * kl + ku + 1;
  for (int j = 0; j < n; ++j) {
    if (piv[j] != j) std::swap(x[j], x[piv[j]]);
    for (int r = 1; r <= kl && j + r < n; ++r) x[j + r] -= Lmul[(size_t)j * kl + (r - 1)] * x[j];
  }
  for (int j = n - 1; j >= 0; --j) {
    double s = x[j];
    for (int d = 1; d <= kl + ku && j + d < n; ++d) s -= B[(size_t)j * w + kl + d] * x[j + d];
    x[j] = s / B[(size_t)j * w + kl];
  }
}

}  // namespace fmh
