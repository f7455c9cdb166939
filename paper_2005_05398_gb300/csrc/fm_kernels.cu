// CUDA kernels of libfm (sm_103a).
//
//  * operator apply y = (H - E S) x (Eq. FM-lin; H from Eq. FM-pre, storage idea of
//    Eq. l-form): sum-factorised banded contractions, y/x pass then z pass with the
//    pointwise coefficients and the M' +- 1 couplings fused;
//  * the V^(s) coupling term (Eqs. r-form, s-rot): a gather of the source
//    component's spline coefficients at the rotated collocation points;
//  * the tensor-trick preconditioner (Eq. prec-2): z and x mode products and the
//    banded y solves that replace the y eigen-transforms and the tridiagonal M'
//    chains (the same operator, factorised by banded LU);
//  * deterministic Krylov reductions (fixed grid, fixed reduction order).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>
#include <type_traits>
#include <vector>

#include "fm_internal.h"

namespace {

constexpr int kMaxM = 12;  // largest n_M (J <= 11 for tau = +1)

// ---------------------------------------------------------------------------
// apply, pass 1: for one (component, M', z-dof k) plane c[i][j] (n_x x n_y) and a tile
// of TX x-collocation points: P = (S_x (x) S_y) c, Q = (D2_x (x) S_y) c, R = (S_x (x) D2_y) c.
// R taps per point (4 cubic, 6 quintic); the tile reads 'rows' rows of c from the base of its
// first point (the host sizes 'rows' from the axis' tap structure).
// ---------------------------------------------------------------------------
template <int TX, int R, typename T>
__global__ void __launch_bounds__(256) k_apply_xy(const T* __restrict__ c, T* __restrict__ P,
                                                  T* __restrict__ Q, T* __restrict__ Rr, int nx, int ny, int rows,
                                                  const int* __restrict__ bx, const T* __restrict__ Sx,
                                                  const T* __restrict__ D2x, const int* __restrict__ by,
                                                  const T* __restrict__ Sy, const T* __restrict__ D2y,
                                                  bool only_S) {
  extern __shared__ unsigned char smraw_xy[];
  T* sm = reinterpret_cast<T*>(smraw_xy);
  T* cs = sm;                 // [rows][ny]
  T* As = sm + rows * ny;     // [rows][ny]  S_y pass
  T* Bs = As + rows * ny;     // [rows][ny]  D2_y pass
  const int64_t plane = (int64_t)blockIdx.y * nx * ny;
  const int xi0 = blockIdx.x * TX;
  const int r0 = bx[xi0];
  for (int idx = threadIdx.x; idx < rows * ny; idx += blockDim.x) {
    const int r = r0 + idx / ny;
    cs[idx] = (r >= 0 && r < nx) ? c[plane + (int64_t)r * ny + (idx % ny)] : (T)0;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < rows * ny; idx += blockDim.x) {
    const int r = idx / ny, eta = idx % ny;
    const int b = by[eta];
    T a = 0, d = 0;
#pragma unroll
    for (int t = 0; t < R; ++t) {
      const int j = b + t;
      if (j >= 0 && j < ny) {
        const T v = cs[r * ny + j];
        a = fma(Sy[eta * R + t], v, a);
        d = fma(D2y[eta * R + t], v, d);
      }
    }
    As[idx] = a;
    Bs[idx] = d;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < TX * ny; idx += blockDim.x) {
    const int xi = xi0 + idx / ny, eta = idx % ny;
    if (xi >= nx) continue;
    const int b = bx[xi] - r0;
    T p = 0, q = 0, rr = 0;
#pragma unroll
    for (int t = 0; t < R; ++t) {
      const int lr = b + t;
      if (lr >= 0 && lr < rows) {
        const T a = As[lr * ny + eta];
        p = fma(Sx[xi * R + t], a, p);
        q = fma(D2x[xi * R + t], a, q);
        rr = fma(Sx[xi * R + t], Bs[lr * ny + eta], rr);
      }
    }
    const int64_t o = plane + (int64_t)xi * ny + eta;
    P[o] = p;
    if (!only_S) {
      Q[o] = q;
      Rr[o] = rr;
    }
  }
}

template <typename T>
struct ZPassArgs {
  const T* P;
  const T* Q;
  const T* R;
  T* y;
  const T* W;       // [nM][nz][nx][ny] folded diagonal coefficient (without -E)
  const T* A;       // [nz][nx][ny] (1/x^2 + 1/y^2)(1 - z^2)
  const T* B;       // [nM][nz][nx][ny] 2 (M'+1) z (1/x^2 + 1/y^2)
  const T* iy2;     // [ny] 1/y^2
  const int* bz;
  const T* Sz;
  const T* D1z;
  const T* D2z;
  const T* zp;
  int nx, ny, nz, nM, M0, J;
  T E;
  T lamp[kMaxM];    // lambda-hat^{J, M'} for M'+1 coupling
  T lamm[kMaxM];    // lambda-hat^{J, -M'} for M'-1 coupling
};

// apply, pass 2: one thread per output point (M', zeta, xi, eta) of a component (R taps in z).
template <int R, typename T>
__global__ void __launch_bounds__(256) k_apply_z(ZPassArgs<T> a, bool only_S) {
  const int64_t npts = (int64_t)a.nz * a.nx * a.ny;
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= npts * a.nM) return;
  const int iM = (int)(gid / npts);
  const int64_t pt = gid - (int64_t)iM * npts;
  const int zeta = (int)(pt / ((int64_t)a.nx * a.ny));
  const int64_t xy = pt - (int64_t)zeta * a.nx * a.ny;
  const int b = a.bz[zeta];
  const int64_t blk = (int64_t)iM * npts;
  T U = 0, Uz = 0, Uzz = 0, Uxx = 0, Uyy = 0;
#pragma unroll
  for (int t = 0; t < R; ++t) {
    const int k = b + t;
    if (k >= 0 && k < a.nz) {
      const int64_t o = blk + (int64_t)k * a.nx * a.ny + xy;
      const T p = a.P[o];
      U = fma(a.Sz[zeta * R + t], p, U);
      if (!only_S) {
        Uz = fma(a.D1z[zeta * R + t], p, Uz);
        Uzz = fma(a.D2z[zeta * R + t], p, Uzz);
        Uxx = fma(a.Sz[zeta * R + t], a.Q[o], Uxx);
        Uyy = fma(a.Sz[zeta * R + t], a.R[o], Uyy);
      }
    }
  }
  if (only_S) {
    a.y[gid] = U;
    return;
  }
  // pointwise coefficients folded at set-up: W = V_a + sum V^(l) + q M'(M'+1) + (J(J+1) - 2M'^2)/y^2
  const T C = a.W[blk + pt] - a.E;
  T out = fma(C, U, fma(a.B[blk + pt], Uz, fma(-a.A[pt], Uzz, -Uyy - Uxx)));
  if (a.nM == 1) {
    a.y[gid] = out;
    return;
  }
  const int eta = (int)(xy % a.ny);
  const T z = a.zp[zeta];
  const T iy2 = a.iy2[eta];
  const int Mp = a.M0 + iM;
  if (iM + 1 < a.nM) {  // lambda-hat^{J,M'}/y^2 [-(1-z^2) d/dz + 2(M'+1) z] psi_{M'+1}
    T Up = 0, Uzp = 0;
#pragma unroll
    for (int t = 0; t < R; ++t) {
      const int k = b + t;
      if (k >= 0 && k < a.nz) {
        const T p = a.P[blk + npts + (int64_t)k * a.nx * a.ny + xy];
        Up = fma(a.Sz[zeta * R + t], p, Up);
        Uzp = fma(a.D1z[zeta * R + t], p, Uzp);
      }
    }
    out += a.lamp[iM] * iy2 * (-((T)1 - z * z) * Uzp + (T)(2 * (Mp + 1)) * z * Up);
  }
  if (iM >= 1) {  // lambda-hat^{J,-M'}/y^2 d/dz psi_{M'-1}
    T Uzm = 0;
#pragma unroll
    for (int t = 0; t < R; ++t) {
      const int k = b + t;
      if (k >= 0 && k < a.nz) Uzm = fma(a.D1z[zeta * R + t], a.P[blk - npts + (int64_t)k * a.nx * a.ny + xy], Uzm);
    }
    out += a.lamm[iM] * iy2 * Uzm;
  }
  a.y[gid] = out;
}

template <typename T>
struct CouplingArgs {
  const T* x;           // full input vector
  T* y;                 // full output vector (accumulated)
  int64_t row_off;      // offset of the target component
  int64_t npts;         // points per M' block of the target component
  int n_act;
  const int* act_pt;
  int ns;
  const int* base[3];   // per source: [3][n_act]
  const T* val[3];      // per source: [12][n_act]
  const T* w[3];        // per source: [nM*nM][n_act]
  int64_t src_off[3];
  int64_t src_npts[3];
  int snx[3], sny[3], snz[3];
  int nM;
  // staged source (float32 path): per source, the y coefficients regrouped by y interval
  const T* stage[3];    // [nM][nz][nx][nint_y][R] of the source component
  int snint[3];         // y intervals of the source
  int sdir;             // 1: Dirichlet y basis (base = q m - 1), so interval m = (base + 1) / q
  int sq;               // functions per node
};

// V^(s) coupling: one thread per active collocation point of a component; R x R x R taps of the source
// expansion at the rotated point.
template <int R, typename T>
__global__ void __launch_bounds__(128) k_apply_coupling(CouplingArgs<T> a) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= a.n_act) return;
  T acc[kMaxM];
#pragma unroll
  for (int m = 0; m < kMaxM; ++m) acc[m] = (T)0;
  for (int s = 0; s < a.ns; ++s) {
    const int bz = a.base[s][p], bx = a.base[s][a.n_act + p], by = a.base[s][2 * a.n_act + p];
    T vz[R], vx[R], vy[R];
    int iz[R], ix[R], iy[R];
#pragma unroll
    for (int t = 0; t < R; ++t) {
      vz[t] = a.val[s][(0 * R + t) * (int64_t)a.n_act + p];
      vx[t] = a.val[s][(1 * R + t) * (int64_t)a.n_act + p];
      vy[t] = a.val[s][(2 * R + t) * (int64_t)a.n_act + p];
      iz[t] = min(max(bz + t, 0), a.snz[s] - 1);
      ix[t] = min(max(bx + t, 0), a.snx[s] - 1);
      iy[t] = min(max(by + t, 0), a.sny[s] - 1);
    }
    for (int jM = 0; jM < a.nM; ++jM) {
      const T* cb = a.x + a.src_off[s] + (int64_t)jM * a.src_npts[s];
      T sz = 0;
#pragma unroll
      for (int tz = 0; tz < R; ++tz) {
        T sx = 0;
#pragma unroll
        for (int tx = 0; tx < R; ++tx) {
          const T* row = cb + ((int64_t)iz[tz] * a.snx[s] + ix[tx]) * a.sny[s];
          T sy = vy[0] * row[iy[0]];
#pragma unroll
          for (int ty = 1; ty < R; ++ty) sy = fma(vy[ty], row[iy[ty]], sy);
          sx = fma(vx[tx], sy, sx);
        }
        sz = fma(vz[tz], sx, sz);
      }
      for (int iM = 0; iM < a.nM; ++iM)
        acc[iM] = fma(a.w[s][(int64_t)(iM * a.nM + jM) * a.n_act + p], sz, acc[iM]);
    }
  }
  const int pt = a.act_pt[p];
  for (int iM = 0; iM < a.nM; ++iM) a.y[a.row_off + (int64_t)iM * a.npts + pt] += acc[iM];
}

// The y coefficients of a component regrouped by y interval: T[row][m][t] = c[row][q m - d + t] for every
// (M', k, i) row, interval m and tap t (0 outside the basis), so that the R taps a point of interval m
// reads are contiguous and aligned.  One thread per (row, interval).
template <int R>
__global__ void __launch_bounds__(256) k_stage_ytaps(const float* __restrict__ c, float* __restrict__ T, int64_t rows,
                                                     int ny, int nint, int q, int d) {
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= rows * nint) return;
  const int64_t row = gid / nint;
  const int m = (int)(gid - row * nint);
  const float* cr = c + row * ny;
  float v[R];
#pragma unroll
  for (int t = 0; t < R; ++t) {
    const int j = q * m - d + t;
    v[t] = (j >= 0 && j < ny) ? cr[j] : 0.f;
  }
  float* o = T + gid * R;
  if constexpr (R == 4) {
    *reinterpret_cast<float4*>(o) = make_float4(v[0], v[1], v[2], v[3]);
  } else {
#pragma unroll
    for (int t = 0; t < R; t += 2) *reinterpret_cast<float2*>(o + t) = make_float2(v[t], v[t + 1]);
  }
}

// The float32 V^(s) coupling on staged sources: the R y taps of a source row are one aligned vector load
// (float4 for R = 4, three float2 for R = 6) instead of R scattered 4-byte loads.
template <int R>
__global__ void __launch_bounds__(128) k_apply_coupling_staged(CouplingArgs<float> a) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= a.n_act) return;
  float acc[kMaxM];
#pragma unroll
  for (int m = 0; m < kMaxM; ++m) acc[m] = 0.f;
  for (int s = 0; s < a.ns; ++s) {
    const int bz = a.base[s][p], bx = a.base[s][a.n_act + p], by = a.base[s][2 * a.n_act + p];
    float vz[R], vx[R], vy[R];
    int iz[R], ix[R];
#pragma unroll
    for (int t = 0; t < R; ++t) {
      vz[t] = a.val[s][(0 * R + t) * (int64_t)a.n_act + p];
      vx[t] = a.val[s][(1 * R + t) * (int64_t)a.n_act + p];
      vy[t] = a.val[s][(2 * R + t) * (int64_t)a.n_act + p];
      iz[t] = min(max(bz + t, 0), a.snz[s] - 1);
      ix[t] = min(max(bx + t, 0), a.snx[s] - 1);
    }
    // y interval of the point (a point outside the source box has base 0 and zero values)
    const int my = min(max((by + a.sdir) / a.sq, 0), a.snint[s] - 1);
    for (int jM = 0; jM < a.nM; ++jM) {
      const float* tb = a.stage[s] + (int64_t)jM * a.snz[s] * a.snx[s] * a.snint[s] * R;
      float sz = 0.f;
#pragma unroll
      for (int tz = 0; tz < R; ++tz) {
        float sx = 0.f;
#pragma unroll
        for (int tx = 0; tx < R; ++tx) {
          const float* row = tb + (((int64_t)iz[tz] * a.snx[s] + ix[tx]) * a.snint[s] + my) * R;
          float sy;
          if constexpr (R == 4) {
            const float4 c4 = __ldg(reinterpret_cast<const float4*>(row));
            sy = vy[0] * c4.x;
            sy = fmaf(vy[1], c4.y, sy);
            sy = fmaf(vy[2], c4.z, sy);
            sy = fmaf(vy[3], c4.w, sy);
          } else {
            sy = 0.f;
#pragma unroll
            for (int t = 0; t < R; t += 2) {
              const float2 c2 = __ldg(reinterpret_cast<const float2*>(row + t));
              sy = fmaf(vy[t], c2.x, sy);
              sy = fmaf(vy[t + 1], c2.y, sy);
            }
          }
          sx = fmaf(vx[tx], sy, sx);
        }
        sz = fmaf(vz[tz], sx, sz);
      }
      for (int iM = 0; iM < a.nM; ++iM)
        acc[iM] = fmaf(a.w[s][(int64_t)(iM * a.nM + jM) * a.n_act + p], sz, acc[iM]);
    }
  }
  const int pt = a.act_pt[p];
  for (int iM = 0; iM < a.nM; ++iM) a.y[a.row_off + (int64_t)iM * a.npts + pt] += acc[iM];
}

// ---------------------------------------------------------------------------
// preconditioner: z mode product  out[l][p] = sum_k W[l][k] in[k][p] for one (component, M').
// A CTA stages W (n_z x n_z) and an n_z x 128 column tile of the input in shared memory;
// each thread produces the n_z outputs of its column.
// ---------------------------------------------------------------------------
template <typename TI, typename TO, typename TW>
__global__ void __launch_bounds__(128) k_zmix(const TW* __restrict__ Wall, const TI* __restrict__ in,
                                              TO* __restrict__ out, int nz, int64_t nxy, int64_t comp_off) {
  extern __shared__ unsigned char smraw[];
  TW* Ws = reinterpret_cast<TW*>(smraw);  // [nz][nz]
  TW* Vs = Ws + nz * nz;                  // [nz][128]
  const int iM = blockIdx.y;
  const TW* W = Wall + (int64_t)iM * nz * nz;
  for (int i = threadIdx.x; i < nz * nz; i += blockDim.x) Ws[i] = W[i];
  const int64_t p0 = (int64_t)blockIdx.x * 128;
  const int64_t base = comp_off + (int64_t)iM * nz * nxy + p0;
  const int cols = (int)min((int64_t)128, nxy - p0);
  for (int k = 0; k < nz; ++k)
    Vs[k * 128 + threadIdx.x] = (threadIdx.x < cols) ? (TW)in[base + (int64_t)k * nxy + threadIdx.x] : (TW)0;
  __syncthreads();
  if ((int)threadIdx.x >= cols) return;
  constexpr int CH = 10;
  for (int l0 = 0; l0 < nz; l0 += CH) {
    TW acc[CH];
#pragma unroll
    for (int u = 0; u < CH; ++u) acc[u] = 0;
    for (int k = 0; k < nz; ++k) {
      const TW v = Vs[k * 128 + threadIdx.x];
#pragma unroll
      for (int u = 0; u < CH; ++u)
        if (l0 + u < nz) acc[u] = fma(Ws[(l0 + u) * nz + k], v, acc[u]);
    }
#pragma unroll
    for (int u = 0; u < CH; ++u)
      if (l0 + u < nz) out[base + (int64_t)(l0 + u) * nxy + threadIdx.x] = (TO)acc[u];
  }
}

// Mode product on every (M', z-mode) slab of a component, slab l = M' + k:
//   out[r][c] = sum_r' W^{l}[r][r'] in[r'][c]   (R x R matrix per l, slabs of R x C)
// x stage: R = n_x, C = n_y; y stage on transposed slabs: R = n_y, C = n_x.  TIN / TOUT read /
// write the slab transposed ([c][r]); SCALE divides the result by lamR[l][r] + lamC[l][c]
// (the diagonal of the tensor-trick inverse).  64x64 output tiles, 256 threads, 4x4 outputs per
// thread, K in steps of 16.
template <typename T, bool TIN, bool TOUT, bool SCALE>
__global__ void __launch_bounds__(256) k_mix(const T* __restrict__ Wall, const T* __restrict__ in, T* __restrict__ out,
                                             int R, int C, int nz, int64_t comp_off, int M0,
                                             const T* __restrict__ lamR, const T* __restrict__ lamC) {
  constexpr int BT = 64, BK = 16;
  __shared__ T smem[BT * (BT + 1) > 2 * BK * (BT + 1) ? BT * (BT + 1) : 2 * BK * (BT + 1)];
  T (*As)[BT + 1] = reinterpret_cast<T (*)[BT + 1]>(smem);
  T (*Bs)[BT + 1] = reinterpret_cast<T (*)[BT + 1]>(smem + BK * (BT + 1));
  const int slab = blockIdx.z;  // iM * nz + k
  const int iM = slab / nz, k = slab % nz;
  const int il = iM + k;        // l - M0
  const T* W = Wall + (int64_t)il * R * R;
  const int64_t so = comp_off + (int64_t)slab * R * C;
  const int row0 = blockIdx.y * BT, col0 = blockIdx.x * BT;
  const int tr = threadIdx.x / 16, tc = threadIdx.x % 16;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0;
  for (int k0 = 0; k0 < R; k0 += BK) {
    for (int e = threadIdx.x; e < BK * BT; e += 256) {
      const int kk = e % BK, rr = e / BK;  // A tile: W[row0+rr][k0+kk]
      const int gr = row0 + rr, gk = k0 + kk;
      As[kk][rr] = (gr < R && gk < R) ? W[(int64_t)gr * R + gk] : (T)0;
      if (TIN) {  // in stored [c][r']: consecutive threads walk r'
        const int kb = e % BK, cc = e / BK;
        const int gk2 = k0 + kb, gc = col0 + cc;
        Bs[kb][cc] = (gk2 < R && gc < C) ? in[so + (int64_t)gc * R + gk2] : (T)0;
      } else {
        const int cc = e % BT, kb = e / BT;
        const int gk2 = k0 + kb, gc = col0 + cc;
        Bs[kb][cc] = (gk2 < R && gc < C) ? in[so + (int64_t)gk2 * C + gc] : (T)0;
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][tr + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tc + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  if (SCALE) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int gr = row0 + tr + 16 * i, gc = col0 + tc + 16 * j;
        if (gr < R && gc < C) acc[i][j] = acc[i][j] / (lamR[(int64_t)il * R + gr] + lamC[(int64_t)il * C + gc]);
      }
  }
  if (!TOUT) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int gr = row0 + tr + 16 * i, gc = col0 + tc + 16 * j;
        if (gr < R && gc < C) out[so + (int64_t)gr * C + gc] = acc[i][j];
      }
  } else {  // stage the tile, then store [c][r] with consecutive threads along r
    T (*Cs)[BT + 1] = reinterpret_cast<T (*)[BT + 1]>(smem);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) Cs[tc + 16 * j][tr + 16 * i] = acc[i][j];
    __syncthreads();
    for (int e = threadIdx.x; e < BT * BT; e += 256) {
      const int rr = e % BT, cc = e / BT;
      const int gr = row0 + rr, gc = col0 + cc;
      if (gr < R && gc < C) out[so + (int64_t)gc * R + gr] = Cs[cc][rr];
    }
  }
}

// banded y solves: one thread per (l, i_x) line of a component; the right-hand side is
// the M'-chain of y-vectors t[iM][l - M'][i_x][:] interleaved as r = j * nc + c.
struct YArgs {
  int nx, ny, nz, M0, nl, maxn;
  int kq;                   // band half-width of the 1D y matrices (2 cubic, 4 quintic)
  int pb;                   // cp.async piece bytes: 16, 8 or 4, dividing n_x and the component offset in bytes
  int64_t comp_off;
  const int* chain_lo;   // [nl]
  const int* chain_n;    // [nl]
  const int64_t* band_off;  // [nl] offset into U
  const int64_t* lmul_off;  // [nl] offset into L
};

// Transposed slabs [j][i_x]: element (iM, k, j, i_x) of a component lives at
// comp_off + ((iM * nz + k) * ny + j) * nx + i_x.  One thread per line (l, i_x), LPB consecutive
// lines of one l per CTA, the unknowns of a line ordered r = j * n_c + c.  A factor "segment" is
// one (row, slot) entry for the CTA's LPB lines: contiguous in memory, and contiguous in the
// shared-memory ring.  The CTA copies segments with cooperative cp.async pieces of PB bytes (a
// thread copies pieces of other threads' lines), so every wait is followed by a CTA barrier:
//   [copy chunk ch+1] [wait chunk ch] [barrier] [eliminate the R rows of chunk ch] [barrier]
// The line itself is staged in shared memory the same way.
__device__ __forceinline__ void cp_async_pb(void* dst, const void* src, int pb) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  if (pb == 16) asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
  else if (pb == 8) asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
  else asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all_but_one() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Copy nseg segments: segment s goes from src(s) (LPB elements, contiguous) to dst(s); only the
// first 'valid' lines are copied (valid is a multiple of the piece length).  Thread t copies piece
// t % pps of segments t / pps, t / pps + LPB / pps, ...
template <typename T, int LPB, typename SrcF, typename DstF>
__device__ __forceinline__ void copy_segments(int nseg, int valid, int pb, SrcF src, DstF dst) {
  const int ep = pb / (int)sizeof(T);  // elements per piece
  const int pps = (valid + ep - 1) / ep;
  const int spr = LPB / pps;           // segments per pass of the CTA
  const int t = threadIdx.x;
  if (t >= spr * pps) return;
  const int k = t % pps;
  for (int sg = t / pps; sg < nseg; sg += spr) cp_async_pb(dst(sg) + k * ep, src(sg) + k * ep, pb);
}

// w[p] for 0 <= p < N through a binary tree of selects (depth log2 N instead of a chain of N)
template <typename T, int N>
__device__ __forceinline__ T pick_window(const T* w, int p) {
  T s[N];
#pragma unroll
  for (int i = 0; i < N; ++i) s[i] = w[i];
  int n = N;
#pragma unroll
  for (int b = 0; (1 << b) < N; ++b) {
    const bool hi = (p >> b) & 1;
#pragma unroll
    for (int i = 0; i < (N + 1) / 2; ++i)
      if (i < (n + 1) / 2) s[i] = (hi && 2 * i + 1 < n) ? s[2 * i + 1] : s[2 * i];
    n = (n + 1) / 2;
  }
  return s[0];
}

// Row walker of a line: row r = j * n_c + c lives at P0 + c * DC + j * nx (DC the distance between the
// chain's neighbouring M' components), stepped without divisions.
template <typename T>
struct RowPtr {
  T* p;
  int c, nc;
  int64_t dc, nx;
  __device__ __forceinline__ void next() {
    p += dc;
    if (++c == nc) {
      c = 0;
      p += nx - (int64_t)nc * dc;
    }
  }
  __device__ __forceinline__ void prev() {
    p -= dc;
    if (--c < 0) {
      c = nc - 1;
      p -= nx - (int64_t)nc * dc;
    }
  }
};

// One line through the banded LU factors, in place on the line's entries in global memory: seg(r) is the
// entry of row r of the CTA's first line, and this thread's line is tid entries further.  Every row of both
// sweeps streams through a shared-memory ring filled a chunk ahead by cooperative cp.async: a ring row holds
// the row's factor slots and, in its last slot, one line value -- the right-hand side entry x[r + KL + 1]
// that enters the forward window at row r, or the forward result z[r] the backward sweep starts from.  The
// forward sweep keeps x[r .. r+KL] in a register window (the pivot row is picked from it by a select tree,
// its index read one row ahead) and writes z[r] back; the backward sweep keeps the KL+KU solved values
// x[r+1 ..] in registers (four independent FMA chains), adds the newest one last and writes x[r].  The
// rows' addresses are walked (RowPtr) rather than recomputed.
template <typename T, int LPB, int KL, typename SegF>
__device__ __forceinline__ void ysolve_line(const T* __restrict__ Lb, const T* __restrict__ Ub, int64_t nx, int n,
                                            int R, SegF seg, RowPtr<T> rp0, T* ring, int Wring, int tid, bool live,
                                            int valid, int pb) {
  constexpr int W = 2 * KL + 1;
  const int nch = (n + R - 1) / R;
  const int RS = Wring + 1;  // slots per ring row (factor slots + the line value)
  const size_t half = (size_t)R * RS * LPB;
  // forward: L z = P b, row r uses L[r][0] (pivot offset) and L[r][1..KL]
  auto issue_f = [&](int ch) {
    T* buf = ring + (ch & 1) * half;
    const int r0 = ch * R, rows = min(R, n - r0);
    copy_segments<T, LPB>(
        rows * (KL + 1), valid, pb,
        [&](int sg) { return Lb + ((int64_t)(r0 + sg / (KL + 1)) * (KL + 1) + sg % (KL + 1)) * nx; },
        [&](int sg) { return buf + ((size_t)(sg / (KL + 1)) * RS + sg % (KL + 1)) * LPB; });
    const int lo = r0 + KL + 1, cnt = max(0, min(rows, n - lo));  // window refills of rows r0 .. r0 + cnt - 1
    copy_segments<T, LPB>(cnt, valid, pb, [&](int sg) { return (const T*)seg(lo + sg); },
                          [&](int sg) { return buf + ((size_t)sg * RS + Wring) * LPB; });
    cp_commit();
  };
  T w[KL + 1];
#pragma unroll
  for (int i = 0; i <= KL; ++i) w[i] = (live && i < n) ? seg(i)[tid] : (T)0;
  RowPtr<T> rp = rp0;  // row 0
  issue_f(0);
  for (int ch = 0; ch < nch; ++ch) {
    if (ch + 1 < nch) {
      issue_f(ch + 1);
      cp_wait_all_but_one();
    } else {
      cp_wait_all();
    }
    __syncthreads();
    if (live) {
      const T* buf = ring + (ch & 1) * half;
      const int r0 = ch * R, rows = min(R, n - r0);
      int p = (int)buf[tid];
      for (int q = 0; q < rows; ++q) {
        const int r = r0 + q;
        const T* f = buf + (size_t)q * RS * LPB + tid;
        const int pn = (q + 1 < rows) ? (int)f[RS * LPB] : 0;  // next row's pivot offset, ahead of use
        const T xr = pick_window<T, KL + 1>(w, p);
        const T w0 = w[0];
        // swap (the pivot row's entry takes w[0]), elimination and window shift in one pass:
        // new w[i] = (old w[i+1], or w[0] where it was the pivot row) - L[r][i+1] x_r
#pragma unroll
        for (int i = 0; i < KL; ++i) {
          const T src = (p == i + 1) ? w0 : w[i + 1];
          w[i] = src - f[(i + 1) * LPB] * xr;
        }
        rp.p[tid] = xr;
        rp.next();
        w[KL] = (r + KL + 1 < n) ? f[Wring * LPB] : (T)0;
        p = pn;
      }
    }
    __syncthreads();
  }
  // the forward results must be in memory before the backward sweep reads them back through the ring
  __threadfence();
  __syncthreads();
  // backward: U x = z, rows descending, U[r][0] the reciprocal of the pivot, U[r][d] the coefficient
  // of x[r + d]; v[i] = x[r + 1 + i] (0 beyond the line, where the band entries are 0)
  auto issue_b = [&](int ch) {
    T* buf = ring + (ch & 1) * half;
    const int rtop = n - 1 - ch * R, rows = min(R, rtop + 1);
    copy_segments<T, LPB>(
        rows * W, valid, pb, [&](int sg) { return Ub + ((int64_t)(rtop - sg / W) * W + sg % W) * nx; },
        [&](int sg) { return buf + ((size_t)(sg / W) * RS + sg % W) * LPB; });
    copy_segments<T, LPB>(rows, valid, pb, [&](int sg) { return (const T*)seg(rtop - sg); },
                          [&](int sg) { return buf + ((size_t)sg * RS + Wring) * LPB; });
    cp_commit();
  };
  T v[W - 1];
#pragma unroll
  for (int i = 0; i < W - 1; ++i) v[i] = (T)0;
  rp.prev();  // row n - 1
  issue_b(0);
  for (int ch = 0; ch < nch; ++ch) {
    if (ch + 1 < nch) {
      issue_b(ch + 1);
      cp_wait_all_but_one();
    } else {
      cp_wait_all();
    }
    __syncthreads();
    if (live) {
      const T* buf = ring + (ch & 1) * half;
      const int rows = min(R, n - ch * R);
      for (int q = 0; q < rows; ++q) {
        const T* f = buf + (size_t)q * RS * LPB + tid;
        T s0 = f[Wring * LPB], s1 = 0, s2 = 0, s3 = 0;
#pragma unroll
        for (int d = 2; d < W; d += 4) s0 -= f[d * LPB] * v[d - 1];
#pragma unroll
        for (int d = 3; d < W; d += 4) s1 -= f[d * LPB] * v[d - 1];
#pragma unroll
        for (int d = 4; d < W; d += 4) s2 -= f[d * LPB] * v[d - 1];
#pragma unroll
        for (int d = 5; d < W; d += 4) s3 -= f[d * LPB] * v[d - 1];
        const T x = (((s0 + s1) + (s2 + s3)) - f[LPB] * v[0]) * f[0];
        rp.p[tid] = x;
        rp.prev();
#pragma unroll
        for (int i = W - 2; i > 0; --i) v[i] = v[i - 1];
        v[0] = x;
      }
    }
    __syncthreads();
  }
}

// the components of one launch (blockIdx.z selects one)
template <typename T>
struct YBatch {
  YArgs a[3];
  const T* U[3];
  const T* L[3];
};

template <typename T, int LPB>
__global__ void __launch_bounds__(LPB) k_ysolve(const YBatch<T> yb, int R, int Wring, int maxn, T* __restrict__ t) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const YArgs& a = yb.a[blockIdx.z];
  const T* __restrict__ U = yb.U[blockIdx.z];
  const T* __restrict__ L = yb.L[blockIdx.z];
  const int il = blockIdx.y;
  const int ix0 = blockIdx.x * LPB;
  if (il >= a.nl || ix0 >= a.nx) return;  // grid sized for the largest component (uniform per CTA)
  const int nc = a.chain_n[il], lo = a.chain_lo[il];
  const int n = nc * a.ny;
  T* ring = reinterpret_cast<T*>(smraw);  // [2][R][Wring + 1][LPB]
  const int tid = threadIdx.x;
  const int valid = min(LPB, a.nx - ix0);
  const bool live = tid < valid;
  // piece size chosen on the host so that every segment start (line rows and factor rows) is aligned to it
  // and every CTA's valid line count is a whole number of pieces
  const int pb = a.pb;
  const int l = a.M0 + il;
  // entry of row r of the CTA's first line (the line of thread tid is tid elements further)
  auto seg = [&](int r) -> T* {
    const int j = r / nc, c = r - j * nc;
    const int iM = lo + c, k = l - a.M0 - iM;
    return t + a.comp_off + (((int64_t)iM * a.nz + k) * a.ny + j) * a.nx + ix0;
  };
  (void)maxn;
  const T* Lb = L + a.lmul_off[il] + ix0;
  const T* Ub = U + a.band_off[il] + ix0;
  RowPtr<T> rp0;
  rp0.p = seg(0);
  rp0.c = 0;
  rp0.nc = nc;
  rp0.dc = (int64_t)(a.nz - 1) * a.ny * a.nx;  // (iM + 1, k - 1) from (iM, k): row r + 1 within one j
  rp0.nx = a.nx;
  // band half-width of this chain (band_kl on the host; at most kMaxBandKL there)
  const int KLc = (nc == 1) ? a.kq : a.kq * nc + 1;
#define FM_YS(KLV) ysolve_line<T, LPB, KLV>(Lb, Ub, a.nx, n, R, seg, rp0, ring, Wring, tid, live, valid, pb)
  switch (KLc) {
    case 2: FM_YS(2); break;
    case 4: FM_YS(4); break;
    case 5: FM_YS(5); break;
    case 7: FM_YS(7); break;
    case 9: FM_YS(9); break;
    case 11: FM_YS(11); break;
    case 13: FM_YS(13); break;
    case 15: FM_YS(15); break;
    case 17: FM_YS(17); break;
    case 19: FM_YS(19); break;
    case 21: FM_YS(21); break;
    case 23: FM_YS(23); break;
    default: FM_YS(25); break;
  }
#undef FM_YS
}

// ---------------------------------------------------------------------------
// Krylov helpers
// ---------------------------------------------------------------------------
constexpr int kRedThreads = 256;
constexpr int kGsMaxVec = 264;  // basis vectors one Gram-Schmidt pass takes (restart length <= 256)
// gsd layout: [0, kGsMaxVec) first-pass coefficients, [kGsMaxVec, 2 kGsMaxVec) second pass, [3 kGsMaxVec, +4)
// scalars, [kGsFlag] the tensor-core kernels' wait flag (an int), read back with every Gram-Schmidt result
constexpr int kGsFlag = 3 * kGsMaxVec + 8;
constexpr int kGsRead = kGsFlag + 1;

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += sh[i];
  __syncthreads();
  return r;
}

// Called by every thread of every block at the end of a reduction kernel, after each block has
// written partial[j * nb + b] (j < nv, nb = gridDim.x): the block that arrives last sums the
// partials in a fixed order (lane-strided, then a shuffle tree) into out[j] and resets the
// counter, so the reduction needs neither a second kernel nor a host round trip.
__device__ void last_block_reduce(const double* partial, int nv, unsigned* counter, double* out) {
  __shared__ unsigned ticket;
  const int nb = (int)gridDim.x;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) ticket = atomicAdd(counter, 1u);
  __syncthreads();
  if (ticket != (unsigned)(nb - 1)) return;
  __threadfence();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
  for (int j = wid; j < nv; j += nw) {
    double s = 0.0;
    for (int b = lane; b < nb; b += 32) s += __ldcg(&partial[(int64_t)j * nb + b]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) out[j] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) *counter = 0u;
}

// The float with the sign, the exponent and the 20 leading mantissa bits of a double (truncated;
// 0 below the float range), built with integer operations so that no FP64 instruction is issued.
__device__ __forceinline__ float f64_lead_f32(double d) {
  const unsigned hi = (unsigned)((unsigned long long)__double_as_longlong(d) >> 32);
  const unsigned fe = ((hi >> 20) & 0x7FFu) - 896u;  // float exponent (wraps below the float range)
  const unsigned sign = hi & 0x80000000u;
  return __uint_as_float((fe - 1u < 254u) ? (sign | (fe << 23) | ((hi & 0xFFFFFu) << 3)) : sign);
}

// a float64 value truncated to float32 by integer operations (1 + 23 significand bits; relative error < 2^-23),
// without the FP64 pipe; values outside float32's normal range become signed zero
__device__ __forceinline__ float f64_trunc_f32(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned fe = ((hi >> 20) & 0x7FFu) - 896u;  // float exponent (wraps below the float range)
  const unsigned sign = hi & 0x80000000u;
  const unsigned mant = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
  return __uint_as_float((fe - 1u < 254u) ? (sign | (fe << 23) | mant) : sign);
}

// partial[j][block] = sum over this block's slice of V[j] . w  (j < nv), and for j = nv, when
// 'extra' is given, extra . w; the last block reduces the partials into out[j].  The vectors are read
// as 16-byte element pairs (n even, 16-byte aligned vectors), eight vectors and two pairs per thread
// and iteration with every load issued before the FMAs, so that a thread keeps 18 loads of 16 bytes
// in flight: the kernel is bound by memory latency otherwise.
// LOWP: products and per-thread sums in float32 from the leading bits of the operands (relative
// accuracy about 1e-6 of sum |V_j| |w|), for the first Gram-Schmidt pass only.
__device__ __forceinline__ double dot2(double2 a, double2 b, double acc) { return fma(a.y, b.y, fma(a.x, b.x, acc)); }
__device__ __forceinline__ float dot2f(double2 a, double2 b, float acc) {
  return fmaf(f64_lead_f32(a.y), f64_lead_f32(b.y), fmaf(f64_lead_f32(a.x), f64_lead_f32(b.x), acc));
}

template <bool LOWP>
__global__ void __launch_bounds__(kRedThreads) k_dot_many(const double* __restrict__ V, int64_t ldv, int nv,
                                                         const double* __restrict__ w, int64_t n,
                                                         double* __restrict__ partial, const double* __restrict__ extra,
                                                         unsigned* counter, double* __restrict__ out) {
  constexpr int JT = 8;
  __shared__ double sh[JT][kRedThreads / 32];
  const int64_t npair = n / 2;
  const int64_t chunk = (npair + gridDim.x - 1) / gridDim.x;
  const int64_t lo = (int64_t)blockIdx.x * chunk;
  const int64_t hi = min(npair, lo + chunk);
  const int nt = nv + (extra ? 1 : 0);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const double2* w2 = reinterpret_cast<const double2*>(w);
  const int64_t bs = blockDim.x;
  for (int j0 = 0; j0 < nt; j0 += JT) {
    const int nj = min(JT, nt - j0);
    const double2* vp[JT];
#pragma unroll
    for (int u = 0; u < JT; ++u) {
      const int j = j0 + min(u, nj - 1);
      vp[u] = reinterpret_cast<const double2*>((j < nv) ? V + (int64_t)j * ldv : extra);
    }
    double acc[JT];
    float accf[JT];
#pragma unroll
    for (int u = 0; u < JT; ++u) {
      acc[u] = 0.0;
      accf[u] = 0.f;
    }
    int64_t p = lo + threadIdx.x;
    for (; p + bs < hi; p += 2 * bs) {
      const double2 wa = w2[p], wb = w2[p + bs];
      double2 va[JT], vb[JT];
#pragma unroll
      for (int u = 0; u < JT; ++u)
        if (u < nj) {
          va[u] = vp[u][p];
          vb[u] = vp[u][p + bs];
        }
#pragma unroll
      for (int u = 0; u < JT; ++u)
        if (u < nj) {
          if (LOWP) accf[u] = dot2f(vb[u], wb, dot2f(va[u], wa, accf[u]));
          else acc[u] = dot2(vb[u], wb, dot2(va[u], wa, acc[u]));
        }
    }
    for (; p < hi; p += bs) {
      const double2 wa = w2[p];
#pragma unroll
      for (int u = 0; u < JT; ++u)
        if (u < nj) {
          if (LOWP) accf[u] = dot2f(vp[u][p], wa, accf[u]);
          else acc[u] = dot2(vp[u][p], wa, acc[u]);
        }
    }
    if ((n & 1) && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {  // odd length: the last element
      const int64_t e = n - 1;
#pragma unroll
      for (int u = 0; u < JT; ++u)
        if (u < nj) {
          const double* vv = reinterpret_cast<const double*>(vp[u]);
          if (LOWP) accf[u] = fmaf(f64_lead_f32(vv[e]), f64_lead_f32(w[e]), accf[u]);
          else acc[u] = fma(vv[e], w[e], acc[u]);
        }
    }
#pragma unroll
    for (int u = 0; u < JT; ++u) {
      double v = LOWP ? (double)accf[u] : acc[u];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0) sh[u][wid] = v;
    }
    __syncthreads();
    if ((int)threadIdx.x < nj) {
      double r = 0.0;
      for (int q = 0; q < kRedThreads / 32; ++q) r += sh[threadIdx.x][q];
      partial[(int64_t)(j0 + threadIdx.x) * gridDim.x + blockIdx.x] = r;
    }
    __syncthreads();
  }
  last_block_reduce(partial, nt, counter, out);
}

// k_dot_many with scalar loads: for vectors that do not all start on 16-byte boundaries (odd strides)
template <bool LOWP>
__global__ void __launch_bounds__(kRedThreads) k_dot_many_s(const double* __restrict__ V, int64_t ldv, int nv,
                                                           const double* __restrict__ w, int64_t n,
                                                           double* __restrict__ partial, const double* __restrict__ extra,
                                                           unsigned* counter, double* __restrict__ out) {
  constexpr int JT = 8;
  __shared__ double sh[JT][kRedThreads / 32];
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t lo = (int64_t)blockIdx.x * chunk;
  const int64_t hi = min(n, lo + chunk);
  const int nt = nv + (extra ? 1 : 0);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int j0 = 0; j0 < nt; j0 += JT) {
    const int nj = min(JT, nt - j0);
    const double* vp[JT];
#pragma unroll
    for (int u = 0; u < JT; ++u) {
      const int j = j0 + min(u, nj - 1);
      vp[u] = (j < nv) ? V + (int64_t)j * ldv : extra;
    }
    double acc[JT];
    float accf[JT];
#pragma unroll
    for (int u = 0; u < JT; ++u) {
      acc[u] = 0.0;
      accf[u] = 0.f;
    }
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
      const double wi = w[i];
#pragma unroll
      for (int u = 0; u < JT; ++u)
        if (u < nj) {
          if (LOWP) accf[u] = fmaf(f64_lead_f32(vp[u][i]), f64_lead_f32(wi), accf[u]);
          else acc[u] = fma(vp[u][i], wi, acc[u]);
        }
    }
#pragma unroll
    for (int u = 0; u < JT; ++u) {
      double v = LOWP ? (double)accf[u] : acc[u];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0) sh[u][wid] = v;
    }
    __syncthreads();
    if ((int)threadIdx.x < nj) {
      double r = 0.0;
      for (int q = 0; q < kRedThreads / 32; ++q) r += sh[threadIdx.x][q];
      partial[(int64_t)(j0 + threadIdx.x) * gridDim.x + blockIdx.x] = r;
    }
    __syncthreads();
  }
  last_block_reduce(partial, nt, counter, out);
}

// float32 vectors: partial[j][block] (float64) = V[j] . w over the block's slice (eight vectors per pass)
__global__ void __launch_bounds__(kRedThreads) k_dot_many32(const float* __restrict__ V, int64_t ldv, int nv,
                                                           const float* __restrict__ w, int64_t n,
                                                           double* __restrict__ partial, unsigned* counter,
                                                           double* __restrict__ out) {
  constexpr int JT = 8;
  __shared__ double sh[JT][kRedThreads / 32];
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t lo = (int64_t)blockIdx.x * chunk;
  const int64_t hi = min(n, lo + chunk);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int j0 = 0; j0 < nv; j0 += JT) {
    const int nj = min(JT, nv - j0);
    float acc[JT];
#pragma unroll
    for (int u = 0; u < JT; ++u) acc[u] = 0.0f;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
      const float wi = w[i];
#pragma unroll
      for (int u = 0; u < JT; ++u)
        if (u < nj) acc[u] = fmaf(V[(int64_t)(j0 + u) * ldv + i], wi, acc[u]);
    }
#pragma unroll
    for (int u = 0; u < JT; ++u) {
      double v = (double)acc[u];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0) sh[u][wid] = v;
    }
    __syncthreads();
    if ((int)threadIdx.x < nj) {
      double r = 0.0;
      for (int q = 0; q < kRedThreads / 32; ++q) r += sh[threadIdx.x][q];
      partial[(int64_t)(j0 + threadIdx.x) * gridDim.x + blockIdx.x] = r;
    }
    __syncthreads();
  }
  last_block_reduce(partial, nv, counter, out);
}

// float32: w += sign * sum_j h[j] V[j], partial[block] = sum of the new w^2 (float64)
__global__ void __launch_bounds__(kRedThreads) k_axpy_many_norm32(const float* __restrict__ V, int64_t ldv, int nv,
                                                                 const float* __restrict__ h, float sign,
                                                                 float* __restrict__ w, int64_t n,
                                                                 double* __restrict__ partial, unsigned* counter,
                                                                 double* __restrict__ out) {
  __shared__ double sh[32];
  float acc = 0.0f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
    int j = 0;
    for (; j + 3 < nv; j += 4) {
      s0 = fmaf(h[j], V[(int64_t)j * ldv + i], s0);
      s1 = fmaf(h[j + 1], V[(int64_t)(j + 1) * ldv + i], s1);
      s2 = fmaf(h[j + 2], V[(int64_t)(j + 2) * ldv + i], s2);
      s3 = fmaf(h[j + 3], V[(int64_t)(j + 3) * ldv + i], s3);
    }
    for (; j < nv; ++j) s0 = fmaf(h[j], V[(int64_t)j * ldv + i], s0);
    const float v = fmaf(sign, (s0 + s1) + (s2 + s3), w[i]);
    w[i] = v;
    acc = fmaf(v, v, acc);
  }
  const double a = block_sum((double)acc, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = a;
  last_block_reduce(partial, 1, counter, out);
}

// y32 = (float)(a * x64)
__global__ void k_to32(const double* __restrict__ x, double a, float* __restrict__ y, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (float)(a * x[i]);
}

// x64 += a * (double)y32
__global__ void k_add32(const float* __restrict__ y, double a, double* __restrict__ x, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = fma(a, (double)y[i], x[i]);
}

// float32 y = a x + b y
__global__ void k_axpby32(float a, const float* __restrict__ x, float b, float* __restrict__ y, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a * x[i] + (b == 0.0f ? 0.0f : b * y[i]);
}

// One pass of classical Gram-Schmidt with the coefficients on the device:
//   w' = w - sum_j c_j V_j,  c = h, or c = G a (G k x k row-major, a of length k) when G is given.
// MODE 0: w <- w', out[0] = ||w'||^2.
// MODE 1 (closing pass): nu^2 = nrm2_prev - |c|^2 (the norm of w' by Pythagoras, V orthonormal and
// c = V^T w), vout <- w' / nu (0 when nu^2 <= 0), out[0] = ||vout||^2 (1 up to rounding), out[1] = nu.
// MODE 2 (single pass with the DGKS test): as MODE 1 when nu^2 >= nrm2_prev / 2 (little cancellation: one
// float64 projection is enough), out[2] = 0; otherwise as MODE 0 (w <- w', out[0] = ||w'||^2) with
// out[2] = 1, and the caller re-orthogonalises.  Every block takes the same decision from the same values.
template <int MODE>
__global__ void __launch_bounds__(kRedThreads) k_gs_axpy(const double* __restrict__ V, int64_t ldv, int nv,
                                                        const double* __restrict__ h, const double* __restrict__ G,
                                                        const double* __restrict__ a, double* w, double* vout,
                                                        int64_t n, double* __restrict__ partial, unsigned* counter,
                                                        double* __restrict__ out, const double* __restrict__ nrm2_prev) {
  __shared__ double cs[kGsMaxVec];
  __shared__ double sh[32];
  __shared__ double inv_nu;
  __shared__ int reorth;
  __shared__ int corr32;
  for (int j = threadIdx.x; j < nv; j += blockDim.x) {
    double cj;
    if (G) {
      cj = 0.0;
      for (int q = 0; q < nv; ++q) cj = fma(G[(int64_t)j * nv + q], a[q], cj);
    } else {
      cj = h[j];
    }
    cs[j] = cj;
  }
  __syncthreads();
  if (MODE >= 1 && threadIdx.x == 0) {
    double c2 = 0.0;
    for (int j = 0; j < nv; ++j) c2 = fma(cs[j], cs[j], c2);
    const double nu2 = *nrm2_prev - c2;
    const double nu = nu2 > 0.0 ? sqrt(nu2) : 0.0;
    inv_nu = nu > 0.0 ? 1.0 / nu : 0.0;
    reorth = (MODE == 2 && !(nu2 >= 0.5 * *nrm2_prev)) ? 1 : 0;
    // closing update on the FP32 pipe only while |h| <= 1e-5 |w'| (its float32 error, ~1e-7 |V h|, then stays
    // below 1e-12 |w'|); with heavier cancellation the float64 path below
    corr32 = (MODE == 1 && c2 <= 1e-10 * *nrm2_prev) ? 1 : 0;
    if (blockIdx.x == 0) {
      out[1] = nu;
      if (MODE == 2) out[2] = (double)reorth;
    }
  }
  __syncthreads();
  const bool write_w = MODE == 0 || (MODE == 2 && reorth);
  double acc = 0.0;
  if (MODE == 1 && corr32) {
    // the closing update of CGS2: its coefficients are the second projection, of relative size ~1e-6 (the
    // error of the first, FP32-pipe projection), so V h is summed on the FP32 pipe from 24-bit truncations
    // (error ~1e-7 of a term <= 1e-5 |w'|) and only w - corr, the scaling and the norm run in float64
    __shared__ float csf[kGsMaxVec];
    for (int j = threadIdx.x; j < nv; j += blockDim.x) csf[j] = (float)cs[j];
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
      float c0 = 0.f, c1 = 0.f;
      int j = 0;
      for (; j + 7 < nv; j += 8) {
        double t[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) t[u] = V[(int64_t)(j + u) * ldv + i];
#pragma unroll
        for (int u = 0; u < 8; u += 2) {
          c0 = fmaf(csf[j + u], f64_trunc_f32(t[u]), c0);
          c1 = fmaf(csf[j + u + 1], f64_trunc_f32(t[u + 1]), c1);
        }
      }
      for (; j < nv; ++j) c0 = fmaf(csf[j], f64_trunc_f32(V[(int64_t)j * ldv + i]), c0);
      const double o = (w[i] - (double)(c0 + c1)) * inv_nu;
      vout[i] = o;
      acc = fma(o, o, acc);
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = acc;
    last_block_reduce(partial, 1, counter, out);
    return;
  }
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    // one FMA per basis vector on a single chain (no partial sums to add: FP64 issue is the bound);
    // eight loads issued ahead of their FMAs
    double v = w[i];
    int j = 0;
    for (; j + 7 < nv; j += 8) {
      double t[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) t[u] = V[(int64_t)(j + u) * ldv + i];
#pragma unroll
      for (int u = 0; u < 8; ++u) v = fma(-cs[j + u], t[u], v);
    }
    for (; j < nv; ++j) v = fma(-cs[j], V[(int64_t)j * ldv + i], v);
    if (write_w) {
      w[i] = v;
      acc = fma(v, v, acc);
    } else {
      const double o = v * inv_nu;
      vout[i] = o;
      acc = fma(o, o, acc);
    }
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = acc;
  last_block_reduce(partial, 1, counter, out);
}

// float32 counterparts of the Gram-Schmidt kernels (MIXED precision inner solves): vectors of
// float32, coefficients, norms and reductions in float64.
// Multi-dot: partial[j][block] of V[j] . w over 16-byte quads (n a multiple of 4, 16-byte aligned
// vectors), eight vectors and two quads per thread and iteration, loads issued before the FMAs.
__device__ __forceinline__ float dot4f(float4 a, float4 b, float acc) {
  return fmaf(a.w, b.w, fmaf(a.z, b.z, fmaf(a.y, b.y, fmaf(a.x, b.x, acc))));
}

__global__ void __launch_bounds__(kRedThreads) k_dot_many32v(const float* __restrict__ V, int64_t ldv, int nv,
                                                            const float* __restrict__ w, int64_t n,
                                                            double* __restrict__ partial, unsigned* counter,
                                                            double* __restrict__ out) {
  constexpr int JT = 8;
  __shared__ double sh[JT][kRedThreads / 32];
  const int64_t nq = n / 4;
  const int64_t chunk = (nq + gridDim.x - 1) / gridDim.x;
  const int64_t lo = (int64_t)blockIdx.x * chunk;
  const int64_t hi = min(nq, lo + chunk);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const float4* w4 = reinterpret_cast<const float4*>(w);
  const int64_t bs = blockDim.x;
  for (int j0 = 0; j0 < nv; j0 += JT) {
    const int nj = min(JT, nv - j0);
    const float4* vp[JT];
#pragma unroll
    for (int u = 0; u < JT; ++u) vp[u] = reinterpret_cast<const float4*>(V + (int64_t)(j0 + min(u, nj - 1)) * ldv);
    float acc[JT];
#pragma unroll
    for (int u = 0; u < JT; ++u) acc[u] = 0.f;
    int64_t p = lo + threadIdx.x;
    for (; p + bs < hi; p += 2 * bs) {
      const float4 wa = w4[p], wb = w4[p + bs];
      float4 va[JT], vb[JT];
#pragma unroll
      for (int u = 0; u < JT; ++u)
        if (u < nj) {
          va[u] = vp[u][p];
          vb[u] = vp[u][p + bs];
        }
#pragma unroll
      for (int u = 0; u < JT; ++u)
        if (u < nj) acc[u] = dot4f(vb[u], wb, dot4f(va[u], wa, acc[u]));
    }
    for (; p < hi; p += bs) {
      const float4 wa = w4[p];
#pragma unroll
      for (int u = 0; u < JT; ++u)
        if (u < nj) acc[u] = dot4f(vp[u][p], wa, acc[u]);
    }
#pragma unroll
    for (int u = 0; u < JT; ++u) {
      double v = (double)acc[u];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0) sh[u][wid] = v;
    }
    __syncthreads();
    if ((int)threadIdx.x < nj) {
      double r = 0.0;
      for (int q = 0; q < kRedThreads / 32; ++q) r += sh[threadIdx.x][q];
      partial[(int64_t)(j0 + threadIdx.x) * gridDim.x + blockIdx.x] = r;
    }
    __syncthreads();
  }
  last_block_reduce(partial, nv, counter, out);
}

// w' = w - sum_j h_j V_j (float32, h from the device); MODE 0: w <- w', out[0] = ||w'||^2;
// MODE 1: vout = w' / nu with nu^2 = nrm2_prev - |h|^2, out[0] = ||vout||^2, out[1] = nu.
template <int MODE>
__global__ void __launch_bounds__(kRedThreads) k_gs_axpy32(const float* __restrict__ V, int64_t ldv, int nv,
                                                          const double* __restrict__ h, float* w, float* vout,
                                                          int64_t n, double* __restrict__ partial, unsigned* counter,
                                                          double* __restrict__ out,
                                                          const double* __restrict__ nrm2_prev) {
  __shared__ float cs[kGsMaxVec];
  __shared__ double sh[32];
  __shared__ float inv_nu;
  for (int j = threadIdx.x; j < nv; j += blockDim.x) cs[j] = (float)h[j];
  __syncthreads();
  if (MODE == 1 && threadIdx.x == 0) {
    double c2 = 0.0;
    for (int j = 0; j < nv; ++j) c2 = fma(h[j], h[j], c2);
    const double nu2 = *nrm2_prev - c2;
    const double nu = nu2 > 0.0 ? sqrt(nu2) : 0.0;
    inv_nu = nu > 0.0 ? (float)(1.0 / nu) : 0.f;
    if (blockIdx.x == 0) out[1] = nu;
  }
  __syncthreads();
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float v = w[i];
    int j = 0;
    for (; j + 7 < nv; j += 8) {
      float t[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) t[u] = V[(int64_t)(j + u) * ldv + i];
#pragma unroll
      for (int u = 0; u < 8; ++u) v = fmaf(-cs[j + u], t[u], v);
    }
    for (; j < nv; ++j) v = fmaf(-cs[j], V[(int64_t)j * ldv + i], v);
    if (MODE == 0) {
      w[i] = v;
      acc += (double)v * (double)v;
    } else {
      const float o = v * inv_nu;
      vout[i] = o;
      acc += (double)o * (double)o;
    }
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = acc;
  last_block_reduce(partial, 1, counter, out);
}

// w += sign * sum_j h[j] V[j]
__global__ void __launch_bounds__(256) k_axpy_many(const double* __restrict__ V, int64_t ldv, int nv,
                                                   const double* __restrict__ h, double sign, double* __restrict__ w,
                                                   int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int j = 0;
    for (; j + 3 < nv; j += 4) {
      s0 = fma(h[j], V[(int64_t)j * ldv + i], s0);
      s1 = fma(h[j + 1], V[(int64_t)(j + 1) * ldv + i], s1);
      s2 = fma(h[j + 2], V[(int64_t)(j + 2) * ldv + i], s2);
      s3 = fma(h[j + 3], V[(int64_t)(j + 3) * ldv + i], s3);
    }
    for (; j < nv; ++j) s0 = fma(h[j], V[(int64_t)j * ldv + i], s0);
    w[i] = fma(sign, (s0 + s1) + (s2 + s3), w[i]);
  }
}

__global__ void k_axpby(double a, const double* __restrict__ x, double b, double* __restrict__ y, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a * x[i] + (b == 0.0 ? 0.0 : b * y[i]);
}

// counter-based normal deviates: splitmix64 -> two uniforms -> Box-Muller
__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__global__ void k_fill_normal(double* x, int64_t n, uint64_t seed) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t a = splitmix64(seed ^ (2 * (uint64_t)i)), b = splitmix64(seed ^ (2 * (uint64_t)i + 1));
    const double u1 = ((a >> 11) + 1.0) * (1.0 / 9007199254740993.0);
    const double u2 = (b >> 11) * (1.0 / 9007199254740992.0);
    x[i] = sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
  }
}

// out[c][i] = sum_j V[j][i] Q[j][c]  (Q row-major nv x nc on the device)
__global__ void __launch_bounds__(256) k_combine(const double* __restrict__ V, int64_t ldv, int nv,
                                                 const double* __restrict__ Qm, int nc, double* __restrict__ out,
                                                 int64_t ldo, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    for (int cc = 0; cc < nc; ++cc) {
      double s = 0.0;
      for (int j = 0; j < nv; ++j) s = fma(V[(int64_t)j * ldv + i], Qm[j * nc + cc], s);
      out[(int64_t)cc * ldo + i] = s;
    }
  }
}

// per block: the entry of largest magnitude (value), first index on ties
__global__ void __launch_bounds__(256) k_absmax(const double* __restrict__ x, int64_t n, double* __restrict__ pval,
                                                long long* __restrict__ pidx) {
  __shared__ double sv[256];
  __shared__ long long si[256];
  double best = 0.0;
  long long bi = -1;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = x[i];
    if (bi < 0 || fabs(v) > fabs(best)) { best = v; bi = i; }
  }
  sv[threadIdx.x] = best;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      const double a = sv[threadIdx.x], b = sv[threadIdx.x + o];
      const long long ia = si[threadIdx.x], ib = si[threadIdx.x + o];
      if (ia < 0 || (ib >= 0 && (fabs(b) > fabs(a) || (fabs(b) == fabs(a) && ib < ia)))) {
        sv[threadIdx.x] = b;
        si[threadIdx.x] = ib;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    pval[blockIdx.x] = sv[0];
    pidx[blockIdx.x] = si[0];
  }
}

// ---------------------------------------------------------------------------
// Double-float Krylov kernels (mixed_scheme 2 inner solves): vectors of dd, reductions summed in dd per
// thread and in float64 across threads (fixed order, deterministic).
// ---------------------------------------------------------------------------
using fmi::dd;

__device__ __forceinline__ double dd_d(dd v) { return (double)v.hi + (double)v.lo; }

// y = dd(a x)
__global__ void k_to_dd(const double* __restrict__ x, double a, dd* __restrict__ y, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = dd(a * x[i]);
}
// x += a y
__global__ void k_add_dd(const dd* __restrict__ y, double a, double* __restrict__ x, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = fma(a, dd_d(y[i]), x[i]);
}
// leading parts as float32 (the tensor preconditioner's input), and back (its output, lo = 0)
__global__ void k_dd_hi(const dd* __restrict__ x, float* __restrict__ y, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = x[i].hi;
}
__global__ void k_f_to_dd(const float* __restrict__ x, dd* __restrict__ y, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = dd(x[i], 0.f);
}
// y = a x + b y (y is not read when b = 0)
__global__ void k_axpby_dd(dd a, const dd* x, dd b, bool b_zero, dd* y, int64_t n) {  // x may be y
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = b_zero ? a * x[i] : fma(a, x[i], b * y[i]);
}

// out[j] = V_j . w for j < nv (eight vectors per pass)
__global__ void __launch_bounds__(kRedThreads) k_dot_many_dd(const dd* __restrict__ V, int64_t ldv, int nv,
                                                            const dd* __restrict__ w, int64_t n,
                                                            double* __restrict__ partial, unsigned* counter,
                                                            double* __restrict__ out) {
  constexpr int JT = 8;
  __shared__ double sh[JT][kRedThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int j0 = 0; j0 < nv; j0 += JT) {
    const int nj = min(JT, nv - j0);
    dd acc[JT];
#pragma unroll
    for (int u = 0; u < JT; ++u) acc[u] = dd(0.f, 0.f);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
      const dd wi = w[i];
#pragma unroll
      for (int u = 0; u < JT; ++u)
        if (u < nj) acc[u] = fma(V[(int64_t)(j0 + u) * ldv + i], wi, acc[u]);
    }
#pragma unroll
    for (int u = 0; u < JT; ++u) {
      double v = dd_d(acc[u]);
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0) sh[u][wid] = v;
    }
    __syncthreads();
    if ((int)threadIdx.x < nj) {
      double r = 0.0;
      for (int q = 0; q < kRedThreads / 32; ++q) r += sh[threadIdx.x][q];
      partial[(int64_t)(j0 + threadIdx.x) * gridDim.x + blockIdx.x] = r;
    }
    __syncthreads();
  }
  last_block_reduce(partial, nv, counter, out);
}

// w' = w - sum_j h_j V_j in dd (h from the device); MODE 0: w <- w', out[0] = ||w'||^2; MODE 1:
// vout = w' / nu with nu^2 = nrm2_prev - |h|^2, out[0] = ||vout||^2, out[1] = nu.  MODE 2: w <- w + sum_j
// h_j V_j (sign +, no norm).
template <int MODE>
__global__ void __launch_bounds__(kRedThreads) k_gs_axpy_dd(const dd* __restrict__ V, int64_t ldv, int nv,
                                                           const double* __restrict__ h, dd* w, dd* vout, int64_t n,
                                                           double* __restrict__ partial, unsigned* counter,
                                                           double* __restrict__ out,
                                                           const double* __restrict__ nrm2_prev) {
  __shared__ dd cs[kGsMaxVec];
  __shared__ double sh[32];
  __shared__ dd inv_nu;
  for (int j = threadIdx.x; j < nv; j += blockDim.x) cs[j] = MODE == 2 ? dd(h[j]) : dd(-h[j]);
  if (MODE == 1 && threadIdx.x == 0) {
    double c2 = 0.0;
    for (int j = 0; j < nv; ++j) c2 = fma(h[j], h[j], c2);
    const double nu2 = *nrm2_prev - c2;
    const double nu = nu2 > 0.0 ? sqrt(nu2) : 0.0;
    inv_nu = nu > 0.0 ? dd(1.0 / nu) : dd(0.f, 0.f);
    if (blockIdx.x == 0) out[1] = nu;
  }
  __syncthreads();
  dd acc(0.f, 0.f);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    dd v = w[i];
    for (int j = 0; j < nv; ++j) v = fma(cs[j], V[(int64_t)j * ldv + i], v);
    if (MODE == 1) {
      v = v * inv_nu;
      vout[i] = v;
    } else {
      w[i] = v;
    }
    if (MODE != 2) acc = fma(v, v, acc);
  }
  if (MODE == 2) return;
  const double a = block_sum(dd_d(acc), sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = a;
  last_block_reduce(partial, 1, counter, out);
}

inline int grid_for(int64_t n, int threads, int cap = 152 * 16) {
  int64_t g = (n + threads - 1) / threads;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

namespace fmi {

template <typename T>
struct ApplyTabs {
  const T *Sx, *D2x, *Sy, *D2y, *Sz, *D1z, *D2z, *zp, *W, *A, *B, *iy2, *cval, *cw;
};

template <typename T>
static ApplyTabs<T> tabs_of(const Comp& cp);

template <>
ApplyTabs<double> tabs_of<double>(const Comp& cp) {
  return {cp.dx.S, cp.dx.D2, cp.dy.S, cp.dy.D2, cp.dz.S, cp.dz.D1, cp.dz.D2, cp.dz.pts, cp.W, cp.A, cp.B, cp.iy2,
          cp.cpl_val, cp.cpl_w};
}

template <>
ApplyTabs<float> tabs_of<float>(const Comp& cp) {
  return {cp.f32.Sx, cp.f32.D2x, cp.f32.Sy, cp.f32.D2y, cp.f32.Sz, cp.f32.D1z, cp.f32.D2z, cp.f32.zp, cp.f32.W,
          cp.f32.A, cp.f32.B, cp.f32.iy2, cp.f32.cval, cp.f32.cw};
}

template <>
ApplyTabs<dd> tabs_of<dd>(const Comp& cp) {
  return {cp.tdd.Sx, cp.tdd.D2x, cp.tdd.Sy, cp.tdd.D2y, cp.tdd.Sz, cp.tdd.D1z, cp.tdd.D2z, cp.tdd.zp, cp.tdd.W,
          cp.tdd.A, cp.tdd.B, cp.tdd.iy2, cp.tdd.cval, cp.tdd.cw};
}

// y = (H - E S) x (only_S: y = S x) with scratch planes P, Q, R, in the element type T.
template <typename T>
static int apply_t(fm_ctx* c, double E, const T* x, T* y, bool only_S, T* P, T* Q, T* R, bool timed) {
  const double fscale = std::is_same<T, float>::value ? 1.0 : 1.0;
  for (auto& cp : c->comps) {
    const ApplyTabs<T> tb = tabs_of<T>(cp);
    const int64_t off = cp.off;
    constexpr int TX = 8;
    const int rows = cp.ax.tile_rows(TX), RT = cp.r;
    const size_t smem = (size_t)3 * rows * cp.ny * sizeof(T);
    dim3 g1((cp.nx + TX - 1) / TX, cp.nz * c->nM);
    {
      const int tk_ = timed ? prof_begin(c, FM_KERNEL_APPLY_XY) : -1;
      if (RT == 6)
        k_apply_xy<TX, 6, T><<<g1, 256, smem, c->stream>>>(x + off, P + off, Q + off, R + off, cp.nx, cp.ny, rows,
                                                           cp.dx.base, tb.Sx, tb.D2x, cp.dy.base, tb.Sy, tb.D2y, only_S);
      else
        k_apply_xy<TX, 4, T><<<g1, 256, smem, c->stream>>>(x + off, P + off, Q + off, R + off, cp.nx, cp.ny, rows,
                                                           cp.dx.base, tb.Sx, tb.D2x, cp.dy.base, tb.Sy, tb.D2y, only_S);
      prof_end(c, tk_, fscale * cp.npts * c->nM * RT * (only_S ? 4.0 : 10.0),
               (double)cp.npts * c->nM * (only_S ? 2.0 : 4.0) * sizeof(T));
    }
    c->launches++;
    ZPassArgs<T> a;
    a.P = P + off; a.Q = Q + off; a.R = R + off; a.y = y + off; a.W = tb.W; a.A = tb.A; a.B = tb.B; a.iy2 = tb.iy2;
    a.bz = cp.dz.base; a.Sz = tb.Sz; a.D1z = tb.D1z; a.D2z = tb.D2z; a.zp = tb.zp;
    a.nx = cp.nx; a.ny = cp.ny; a.nz = cp.nz; a.nM = c->nM; a.M0 = c->M0; a.J = c->sys.J; a.E = (T)E;
    for (int i = 0; i < kMaxM; ++i) a.lamp[i] = a.lamm[i] = (T)0;
    for (int iM = 0; iM < c->nM; ++iM) {
      const int Mp = c->Mps[iM], J = c->sys.J;
      const double vp = (double)(J * (J + 1) - Mp * (Mp + 1)), vm = (double)(J * (J + 1) - Mp * (Mp - 1));
      a.lamp[iM] = (T)((vp > 0 ? sqrt(vp) : 0.0) * sqrt(Mp == 0 ? 2.0 : 1.0));
      a.lamm[iM] = (T)((vm > 0 ? sqrt(vm) : 0.0) * sqrt(Mp == 1 ? 2.0 : 1.0));
    }
    const int64_t tot = cp.npts * c->nM;
    {
      const int tk_ = timed ? prof_begin(c, FM_KERNEL_APPLY_Z) : -1;
      if (RT == 6) k_apply_z<6, T><<<(unsigned)((tot + 255) / 256), 256, 0, c->stream>>>(a, only_S);
      else k_apply_z<4, T><<<(unsigned)((tot + 255) / 256), 256, 0, c->stream>>>(a, only_S);
      prof_end(c, tk_, (double)tot * (only_S ? 2.0 * RT : (10.0 + (c->nM > 1 ? 8.0 * RT : 0.0) + 10.0 * RT)),
               (double)tot * (only_S ? 2.0 : 7.0) * sizeof(T));
    }
    c->launches++;
  }
  const bool staged = std::is_same<T, float>::value && c->ystage32 != nullptr;
  if (!only_S && staged) {  // float32: regroup every source component's y coefficients by y interval
    for (auto& cp : c->comps) {
      const int64_t rows = (int64_t)c->nM * cp.nz * cp.nx, items = rows * cp.ay.nint;
      const int tk_ = timed ? prof_begin(c, FM_KERNEL_COUPLING) : -1;
      const float* xs = reinterpret_cast<const float*>(x) + cp.off;
      float* ts = c->ystage32 + cp.ystage_off;
      if (cp.r == 6) k_stage_ytaps<6><<<(unsigned)((items + 255) / 256), 256, 0, c->stream>>>(xs, ts, rows, cp.ny, cp.ay.nint, cp.ay.q, 1);
      else k_stage_ytaps<4><<<(unsigned)((items + 255) / 256), 256, 0, c->stream>>>(xs, ts, rows, cp.ny, cp.ay.nint, cp.ay.q, 1);
      prof_end(c, tk_, 0.0, (double)rows * cp.ny * 4.0 + (double)items * cp.r * 4.0);
      c->launches++;
    }
  }
  if (!only_S) {
    for (auto& cp : c->comps) {
      if (cp.n_act == 0 || cp.sources.empty()) continue;
      const ApplyTabs<T> tb = tabs_of<T>(cp);
      CouplingArgs<T> a{};
      a.x = x; a.y = y; a.row_off = cp.off; a.npts = cp.npts; a.n_act = cp.n_act; a.act_pt = cp.act_pt;
      a.ns = (int)cp.sources.size(); a.nM = c->nM;
      const int RT = cp.r;
      for (int s = 0; s < a.ns; ++s) {
        const auto& src = c->comps[cp.sources[s].src];
        a.base[s] = cp.cpl_base + (int64_t)s * 3 * cp.n_act;
        a.val[s] = tb.cval + (int64_t)s * 3 * RT * cp.n_act;
        a.w[s] = tb.cw + (int64_t)s * c->nM * c->nM * cp.n_act;
        a.src_off[s] = src.off; a.src_npts[s] = src.npts;
        a.snx[s] = src.nx; a.sny[s] = src.ny; a.snz[s] = src.nz;
        if (staged) {
          a.stage[s] = reinterpret_cast<const T*>(c->ystage32 + src.ystage_off);
          a.snint[s] = src.ay.nint;
        }
      }
      a.sdir = 1;
      a.sq = cp.ay.q;
      {
        const int tk_ = timed ? prof_begin(c, FM_KERNEL_COUPLING) : -1;
        if constexpr (std::is_same<T, float>::value) {
          if (staged) {
            if (RT == 6) k_apply_coupling_staged<6><<<(cp.n_act + 127) / 128, 128, 0, c->stream>>>(a);
            else k_apply_coupling_staged<4><<<(cp.n_act + 127) / 128, 128, 0, c->stream>>>(a);
          } else if (RT == 6) {
            k_apply_coupling<6, T><<<(cp.n_act + 127) / 128, 128, 0, c->stream>>>(a);
          } else {
            k_apply_coupling<4, T><<<(cp.n_act + 127) / 128, 128, 0, c->stream>>>(a);
          }
        } else {
          if (RT == 6) k_apply_coupling<6, T><<<(cp.n_act + 127) / 128, 128, 0, c->stream>>>(a);
          else k_apply_coupling<4, T><<<(cp.n_act + 127) / 128, 128, 0, c->stream>>>(a);
        }
        // per (point, source): 2 (R^3 + R^2 + R) contraction flops per M'' and 2 n_M^2 for the weights
        const double cfl = 2.0 * (RT * RT * RT + RT * RT + RT);
        prof_end(c, tk_, (double)cp.n_act * a.ns * (cfl * c->nM + 2.0 * c->nM * c->nM),
                 (double)cp.n_act * (4.0 + 2.0 * c->nM * sizeof(T) + a.ns * (12.0 + (3.0 * RT + c->nM * c->nM) * sizeof(T))));
      }
      c->launches++;
    }
  }
  FM_CUDA(cudaGetLastError());
  return FM_OK;
}

int launch_apply(fm_ctx* c, double E, const double* x, double* y, bool only_S) {
  return apply_t<double>(c, E, x, y, only_S, c->P, c->Q, c->R, true);
}

int launch_apply32(fm_ctx* c, double E, const float* x, float* y, bool only_S) {
  return apply_t<float>(c, E, x, y, only_S, c->P32, c->Q32, c->R32, true);
}

// The operator apply with caller-chosen scratch planes (used by the entry point that allocates
// nothing, whose planes live in a fixed device array).  Same kernels and launch shapes as
// launch_apply; no per-kernel timing.
int launch_apply_scratch(fm_ctx* c, double E, const double* x, double* y, double* P, double* Q, double* R) {
  return apply_t<double>(c, E, x, y, false, P, Q, R, false);
}

// Banded y solves (Eq. prec-2 y stage with the M' chain) of the given components in one launch,
// in place on u[slab][j][i].
template <typename T>
static int ysolve_banded(fm_ctx* c, const std::vector<fmi::Comp*>& comps, T* u) {
  if (comps.empty()) return FM_OK;
  if (comps.size() > 3) return FM_ERR_ARG;
  const double ts = (double)sizeof(T);
  double yfl = 0.0, yby = 0.0;  // per line 2n(kl + ku + kl) + n flops; factor and vector bytes
  YBatch<T> yb;
  int maxn = 1, wring = 5, gx = 1, gy = 1;
  for (size_t q = 0; q < comps.size(); ++q) {
    const fmi::Comp& cp = *comps[q];
    for (int il = 0; il < cp.nl; ++il) {
      const int nc = cp.chain_n[il], n = nc * cp.ny, kl = band_kl(cp.ay, nc);
      yfl += (double)cp.nx * (2.0 * n * (3.0 * kl) + n);
      yby += (double)cp.nx * ((double)n * (3.0 * kl + 2.0) * ts + 2.0 * n * ts);
    }
    YArgs& ya = yb.a[q];
    ya.nx = cp.nx; ya.ny = cp.ny; ya.nz = cp.nz; ya.M0 = c->M0; ya.nl = cp.nl; ya.comp_off = cp.off;
    ya.kq = std::max(cp.ay.kl, cp.ay.ku);
    // the largest piece dividing the byte length of an x row and the component's byte offset (line rows
    // start at comp_off + multiple of n_x; factor rows at multiples of n_x); at least one element
    ya.pb = (int)sizeof(T);
    for (int pcand : {16, 8}) {
      if (pcand <= (int)sizeof(T)) break;
      if (((int64_t)cp.nx * (int64_t)sizeof(T)) % pcand == 0 && ((int64_t)cp.off * (int64_t)sizeof(T)) % pcand == 0) {
        ya.pb = pcand;
        break;
      }
    }
    ya.chain_lo = (const int*)cp.d_chain_lo; ya.chain_n = (const int*)cp.d_chain_n;
    ya.band_off = cp.d_band_off; ya.lmul_off = cp.d_lmul_off;
    int maxnc = 1;
    for (int v : cp.chain_n) maxnc = std::max(maxnc, v);
    ya.maxn = maxnc * cp.ny;
    yb.U[q] = std::is_same<T, double>::value ? (const T*)cp.yU : (const T*)cp.yU32;
    yb.L[q] = std::is_same<T, double>::value ? (const T*)cp.yL : (const T*)cp.yL32;
    int klmax = 2;
    for (int v : cp.chain_n) klmax = std::max(klmax, band_kl(cp.ay, v));
    maxn = std::max(maxn, ya.maxn);
    wring = std::max(wring, 2 * klmax + 1);
    gy = std::max(gy, cp.nl);
  }
  int maxnx = 1;
  for (auto* cp : comps) maxnx = std::max(maxnx, cp->nx);
  // Lines per CTA, and rows per ring half (factor slots plus the line value): the CTAs are latency-bound,
  // so the ring is sized for as many resident CTAs per SM as the grid can use (228 KB of shared memory per
  // SM), between 4 and 32 rows a half.
  auto plan = [&](int lpb, int* R, size_t* sm) -> bool {
    const size_t per_row = 2 * (size_t)(wring + 1) * lpb * sizeof(T);
    const int ctas = ((maxnx + lpb - 1) / lpb) * gy * (int)comps.size();
    const int per_sm = std::max(1, std::min(16, (ctas + 151) / 152));
    for (int want = per_sm; want >= 1; --want) {
      const size_t cap = std::min<size_t>(200 * 1024, 233472 / want - 1024);
      if (4 * per_row > cap) continue;
      *R = (int)std::min<size_t>(32, cap / per_row);
      *sm = (size_t)*R * per_row;
      return true;
    }
    return false;
  };
  const int tk_ = prof_begin(c, FM_KERNEL_YSOLVE);
  int R;
  size_t sm;
  if (plan(32, &R, &sm)) {
    gx = (maxnx + 31) / 32;
    k_ysolve<T, 32><<<dim3(gx, gy, (unsigned)comps.size()), 32, sm, c->stream>>>(yb, R, wring, maxn, u);
  } else if (plan(8, &R, &sm)) {
    gx = (maxnx + 7) / 8;
    k_ysolve<T, 8><<<dim3(gx, gy, (unsigned)comps.size()), 8, sm, c->stream>>>(yb, R, wring, maxn, u);
  } else {
    return FM_ERR_ARG;  // band too wide for the ring
  }
  prof_end(c, tk_, yfl, yby);
  c->launches++;
  FM_CUDA(cudaGetLastError());
  return FM_OK;
}

// y = P^{-1} x (Eq. prec-2), stage-major over the components: every component's z and x forward
// stages (and the diagonalised y stage for n_M = 1), then one launch with the banded y solves of
// all components that need them, then every component's x and z inverse stages.
template <typename T, typename TIO>
static int precond_impl(fm_ctx* c, const TIO* x, TIO* y, T* t) {
  const bool is32 = std::is_same<T, float>::value;
  const bool tc = is32 && c->tc_active;
  T* u = is32 ? (T*)c->u32 : (T*)c->u64;
  std::vector<fmi::Comp*> banded;
  int rc;
  if (tc) {  // z, x and y stages on the tensor cores
    if ((rc = fmi::precond_tc_front<TIO>(c, x, &banded))) return rc;
    if ((rc = ysolve_banded<T>(c, banded, u))) return rc;
    if ((rc = fmi::precond_tc_back<TIO>(c, y))) return rc;
    FM_CUDA(cudaGetLastError());
    return FM_OK;
  }
  for (auto& cp : c->comps) {
    const bool ymda = cp.ydiag_ok && (c->opts.y_solver == 2 || (c->opts.y_solver == 0 && is32));
    if (!ymda) banded.push_back(&cp);
    const int64_t nxy = (int64_t)cp.nx * cp.ny;
    const T* Wzb = std::is_same<T, double>::value ? (const T*)cp.Wzb : (const T*)cp.Wzb32;
    const T* Wxb = std::is_same<T, double>::value ? (const T*)cp.Wxb : (const T*)cp.Wxb32;
    const double ncomp = (double)nxy * cp.nz * c->nM;  // unknowns of this component
    const double ts = (double)sizeof(T);
    dim3 gz((unsigned)((nxy + 127) / 128), c->nM);
    const size_t smz = ((size_t)cp.nz * cp.nz + (size_t)cp.nz * 128) * sizeof(T);
    {
      const int tk_ = prof_begin(c, FM_KERNEL_ZMIX);
      k_zmix<TIO, T, T><<<gz, 128, smz, c->stream>>>(Wzb, x, t, cp.nz, nxy, cp.off);
      prof_end(c, tk_, 2.0 * cp.nz * ncomp, ncomp * (8.0 + ts));
    }
    dim3 gx((cp.ny + 63) / 64, (cp.nx + 63) / 64, c->nM * cp.nz);
    {
      const int tk_ = prof_begin(c, FM_KERNEL_XMIX);
      k_mix<T, false, true, false><<<gx, 256, 0, c->stream>>>(Wxb, t, u, cp.nx, cp.ny, cp.nz, cp.off, c->M0, nullptr, nullptr);
      prof_end(c, tk_, 2.0 * cp.nx * ncomp, 2.0 * ncomp * ts);
    }
    c->launches += 2;
    if (ymda) {
      // n_M = 1: per-l diagonalisation of (A_l, S_y): W_y (Lambda_y + lambda_x)^{-1} W-bar_y on transposed slabs
      const T* Wyb = is32 ? (const T*)cp.Wyb32 : (const T*)cp.Wyb64;
      const T* Wy = is32 ? (const T*)cp.Wy32 : (const T*)cp.Wy64;
      const T* dLy = is32 ? (const T*)cp.dLy32 : (const T*)cp.dLy64;
      const T* dLx = is32 ? (const T*)cp.dLx32 : (const T*)cp.dLx64;
      dim3 gyy((cp.nx + 63) / 64, (cp.ny + 63) / 64, c->nM * cp.nz);
      {
        const int tk_ = prof_begin(c, FM_KERNEL_YSOLVE);
        k_mix<T, false, false, true><<<gyy, 256, 0, c->stream>>>(Wyb, u, t, cp.ny, cp.nx, cp.nz, cp.off, c->M0, dLy, dLx);
        prof_end(c, tk_, 2.0 * cp.ny * ncomp, 2.0 * ncomp * ts);
      }
      {
        const int tk_ = prof_begin(c, FM_KERNEL_YSOLVE);
        k_mix<T, false, false, false><<<gyy, 256, 0, c->stream>>>(Wy, t, u, cp.ny, cp.nx, cp.nz, cp.off, c->M0, nullptr, nullptr);
        prof_end(c, tk_, 2.0 * cp.ny * ncomp, 2.0 * ncomp * ts);
      }
      c->launches += 2;
    }
  }
  if ((rc = ysolve_banded<T>(c, banded, u))) return rc;
  for (auto& cp : c->comps) {
    const int64_t nxy = (int64_t)cp.nx * cp.ny;
    const T* Wz = std::is_same<T, double>::value ? (const T*)cp.Wz : (const T*)cp.Wz32;
    const T* Wx = std::is_same<T, double>::value ? (const T*)cp.Wx : (const T*)cp.Wx32;
    const double ncomp = (double)nxy * cp.nz * c->nM;
    const double ts = (double)sizeof(T);
    dim3 gz((unsigned)((nxy + 127) / 128), c->nM);
    const size_t smz = ((size_t)cp.nz * cp.nz + (size_t)cp.nz * 128) * sizeof(T);
    dim3 gx((cp.ny + 63) / 64, (cp.nx + 63) / 64, c->nM * cp.nz);
    {
      const int tk_ = prof_begin(c, FM_KERNEL_XMIX);
      k_mix<T, true, false, false><<<gx, 256, 0, c->stream>>>(Wx, u, t, cp.nx, cp.ny, cp.nz, cp.off, c->M0, nullptr, nullptr);
      prof_end(c, tk_, 2.0 * cp.nx * ncomp, 2.0 * ncomp * ts);
    }
    {
      const int tk_ = prof_begin(c, FM_KERNEL_ZMIX);
      k_zmix<T, TIO, T><<<gz, 128, smz, c->stream>>>(Wz, t, y, cp.nz, nxy, cp.off);
      prof_end(c, tk_, 2.0 * cp.nz * ncomp, ncomp * (8.0 + ts));
    }
    c->launches += 2;
  }
  FM_CUDA(cudaGetLastError());
  return FM_OK;
}

int launch_precond(fm_ctx* c, const double* x, double* y) {
  if (c->opts.precision != FM_PREC_FP64) return precond_impl<float, double>(c, x, y, c->t32);
  return precond_impl<double, double>(c, x, y, c->t64);
}

int launch_precond32(fm_ctx* c, const float* x, float* y) { return precond_impl<float, float>(c, x, y, c->t32); }

int dot_many(fm_ctx* c, const double* V, int64_t ldv, int nv, const double* w, double* h_host) {
  return dot_many_x(c, V, ldv, nv, w, nullptr, h_host);
}

int dot_many_x(fm_ctx* c, const double* V, int64_t ldv, int nv, const double* w, const double* extra, double* h_host) {
  const int nt = nv + (extra ? 1 : 0);
  int rc;
  if ((rc = dot_many_dev(c, V, ldv, nv, w, extra, c->gsd))) return rc;
  FM_CUDA(cudaMemcpyAsync(c->red_host, c->gsd, nt * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  FM_CUDA(cudaStreamSynchronize(c->stream));
  std::memcpy(h_host, c->red_host, nt * sizeof(double));
  return prof_harvest(c);
}

// h_dev[j] = V[j] . w (j < nv), h_dev[nv] = extra . w when extra is given; stays on the device
int dot_many_dev(fm_ctx* c, const double* V, int64_t ldv, int nv, const double* w, const double* extra, double* h_dev,
                 bool lowp) {
  const int nb = c->red_blocks;
  const int nt = nv + (extra ? 1 : 0);
  if (nt > kGsMaxVec) return FM_ERR_ARG;
  // 16-byte element pairs when every vector starts on a 16-byte boundary, scalar loads otherwise (an odd
  // vector length puts every other basis vector on an 8-byte boundary)
  const uintptr_t al = reinterpret_cast<uintptr_t>(V) | reinterpret_cast<uintptr_t>(w) |
                       reinterpret_cast<uintptr_t>(extra) | (uintptr_t)(ldv * 8);
  const bool pairs = (al & 15u) == 0;
  const int tk_ = prof_begin(c, FM_KERNEL_DOT);
  if (pairs && lowp) k_dot_many<true><<<nb, kRedThreads, 0, c->stream>>>(V, ldv, nv, w, c->N, c->red, extra, c->gs_cnt, h_dev);
  else if (pairs) k_dot_many<false><<<nb, kRedThreads, 0, c->stream>>>(V, ldv, nv, w, c->N, c->red, extra, c->gs_cnt, h_dev);
  else if (lowp) k_dot_many_s<true><<<nb, kRedThreads, 0, c->stream>>>(V, ldv, nv, w, c->N, c->red, extra, c->gs_cnt, h_dev);
  else k_dot_many_s<false><<<nb, kRedThreads, 0, c->stream>>>(V, ldv, nv, w, c->N, c->red, extra, c->gs_cnt, h_dev);
  prof_end(c, tk_, 2.0 * nt * (double)c->N, (nt + 1.0) * 8.0 * (double)c->N);
  c->launches++;
  FM_CUDA(cudaGetLastError());
  return FM_OK;
}

int axpy_many(fm_ctx* c, const double* V, int64_t ldv, int nv, const double* h_host, double* w, double sign) {
  double* hd = c->red + (int64_t)c->red_blocks * 256 + 512;
  FM_CUDA(cudaMemcpyAsync(hd, h_host, nv * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  {
    const int tk_ = prof_begin(c, FM_KERNEL_AXPY);
    k_axpy_many<<<grid_for(c->N, 256), 256, 0, c->stream>>>(V, ldv, nv, hd, sign, w, c->N);
    prof_end(c, tk_, 2.0 * nv * (double)c->N, (nv + 2.0) * 8.0 * (double)c->N);
  }
  c->launches++;
  FM_CUDA(cudaGetLastError());
  return FM_OK;
}

// Classical Gram-Schmidt with one re-orthogonalisation (CGS2) of w against the orthonormal
// V[0..nv), all coefficients kept on the device:
//   h1 = V^T w;  w' = w - V h1;  h2 = V^T w';  vout = (w' - V h2) / nu,  nu^2 = ||w'||^2 - |h2|^2.
// Four launches and one host synchronisation.  On return h = h1 + h2 and *hn = ||w' - V h2||
// (nu times the measured norm of vout, which is renormalised if it is not 1 to rounding);
// *hn = 0 when w lies in span V to rounding (vout is then 0).  w is overwritten; vout may be w.
int gs_cgs2(fm_ctx* c, const double* V, int nv, double* w, double* vout, double* h, double* hn) {
  if (nv < 1 || nv > kGsMaxVec) return FM_ERR_ARG;
  const int64_t N = c->N;
  double* h1 = c->gsd;
  double* h2 = c->gsd + kGsMaxVec;
  double* sc = c->gsd + 3 * kGsMaxVec;  // [0] ||w'||^2, [1] ||vout||^2, [2] nu
  const int nb2 = 4 * c->red_blocks;
  int rc;
  // first pass: projections to about 1e-6, on the FP32 pipe; the float64 second pass removes what it leaves
  if ((rc = dot_many_dev(c, V, N, nv, w, nullptr, h1, true))) return rc;
  {
    const int tk_ = prof_begin(c, FM_KERNEL_AXPY);
    k_gs_axpy<0><<<nb2, kRedThreads, 0, c->stream>>>(V, N, nv, h1, nullptr, nullptr, w, nullptr, N, c->red, c->gs_cnt,
                                                     sc, nullptr);
    prof_end(c, tk_, (2.0 * nv + 2.0) * (double)N, (nv + 2.0) * 8.0 * (double)N);
  }
  if ((rc = dot_many_dev(c, V, N, nv, w, nullptr, h2))) return rc;
  {
    const int tk_ = prof_begin(c, FM_KERNEL_AXPY);
    k_gs_axpy<1><<<nb2, kRedThreads, 0, c->stream>>>(V, N, nv, h2, nullptr, nullptr, w, vout, N, c->red, c->gs_cnt,
                                                     sc + 1, sc);
    prof_end(c, tk_, (2.0 * nv + 2.0) * (double)N, (nv + 2.0) * 8.0 * (double)N);
  }
  c->launches += 2;
  FM_CUDA(cudaGetLastError());
  // one read-back: h1, h2 and the three scalars
  FM_CUDA(cudaMemcpyAsync(c->red_host, c->gsd, kGsRead * sizeof(double), cudaMemcpyDeviceToHost,
                          c->stream));
  FM_CUDA(cudaStreamSynchronize(c->stream));
  const double* hh = c->red_host;
  if (c->tc_active && reinterpret_cast<const int*>(hh + kGsFlag)[0] != 0) return FM_ERR_TIMEOUT;
  for (int i = 0; i < nv; ++i) h[i] = hh[i] + hh[kGsMaxVec + i];
  const double vn2 = hh[3 * kGsMaxVec + 1], nu = hh[3 * kGsMaxVec + 2];
  if (!(nu > 0.0) || !(vn2 > 0.0)) {
    *hn = std::isfinite(nu) && std::isfinite(vn2) ? 0.0 : nu + vn2;
    return prof_harvest(c);
  }
  const double vn = std::sqrt(vn2);
  *hn = nu * vn;
  if (std::fabs(vn - 1.0) > 1e-12)  // Pythagoras lost digits: rescale to unit norm
    if ((rc = scale_copy(c, vout, 1.0 / vn, vout))) return rc;
  return prof_harvest(c);
}

// Single-pass classical Gram-Schmidt in float64 with the DGKS re-orthogonalisation test: one multi-dot (with
// |w|^2 from the same pass), one update that normalises directly when |w - V h| >= |w| / sqrt(2); otherwise
// it keeps w - V h and a second float64 pass (multi-dot, closing update) follows.  One host synchronisation
// when no re-orthogonalisation is needed, two otherwise.  Same results as gs_cgs2 to rounding.
int gs_cgs1(fm_ctx* c, const double* V, int nv, double* w, double* vout, double* h, double* hn) {
  if (nv < 1 || nv + 1 > kGsMaxVec) return FM_ERR_ARG;
  const int64_t N = c->N;
  double* h1 = c->gsd;                  // [nv] V^T w, [nv] |w|^2
  double* h2 = c->gsd + kGsMaxVec;
  double* sc = c->gsd + 3 * kGsMaxVec;  // [1] |out|^2, [2] nu, [3] re-orthogonalise
  const int nb2 = 4 * c->red_blocks;
  int rc;
  if ((rc = dot_many_dev(c, V, N, nv, w, w, h1))) return rc;
  {
    const int tk_ = prof_begin(c, FM_KERNEL_AXPY);
    k_gs_axpy<2><<<nb2, kRedThreads, 0, c->stream>>>(V, N, nv, h1, nullptr, nullptr, w, vout, N, c->red, c->gs_cnt,
                                                     sc + 1, h1 + nv);
    prof_end(c, tk_, (2.0 * nv + 2.0) * (double)N, (nv + 2.0) * 8.0 * (double)N);
  }
  c->launches++;
  FM_CUDA(cudaGetLastError());
  FM_CUDA(cudaMemcpyAsync(c->red_host, c->gsd, kGsRead * sizeof(double), cudaMemcpyDeviceToHost,
                          c->stream));
  FM_CUDA(cudaStreamSynchronize(c->stream));
  const double* hh = c->red_host;
  if (c->tc_active && reinterpret_cast<const int*>(hh + kGsFlag)[0] != 0) return FM_ERR_TIMEOUT;
  for (int i = 0; i < nv; ++i) h[i] = hh[i];
  if (hh[3 * kGsMaxVec + 3] != 0.0) {  // cancellation: second float64 pass on w - V h
    if ((rc = dot_many_dev(c, V, N, nv, w, nullptr, h2))) return rc;
    {
      const int tk_ = prof_begin(c, FM_KERNEL_AXPY);
      k_gs_axpy<1><<<nb2, kRedThreads, 0, c->stream>>>(V, N, nv, h2, nullptr, nullptr, w, vout, N, c->red, c->gs_cnt,
                                                       sc + 1, sc + 1);
      prof_end(c, tk_, (2.0 * nv + 2.0) * (double)N, (nv + 2.0) * 8.0 * (double)N);
    }
    c->launches++;
    FM_CUDA(cudaGetLastError());
    FM_CUDA(cudaMemcpyAsync(c->red_host, c->gsd, kGsRead * sizeof(double), cudaMemcpyDeviceToHost,
                            c->stream));
    FM_CUDA(cudaStreamSynchronize(c->stream));
    if (c->tc_active && reinterpret_cast<const int*>(hh + kGsFlag)[0] != 0) return FM_ERR_TIMEOUT;
    for (int i = 0; i < nv; ++i) h[i] += hh[kGsMaxVec + i];
  }
  const double vn2 = hh[3 * kGsMaxVec + 1], nu = hh[3 * kGsMaxVec + 2];
  if (!(nu > 0.0) || !(vn2 > 0.0)) {
    *hn = std::isfinite(nu) && std::isfinite(vn2) ? 0.0 : nu + vn2;
    return prof_harvest(c);
  }
  const double vn = std::sqrt(vn2);
  *hn = nu * vn;
  if (std::fabs(vn - 1.0) > 1e-12)  // Pythagoras lost digits: rescale to unit norm
    if ((rc = scale_copy(c, vout, 1.0 / vn, vout))) return rc;
  return prof_harvest(c);
}

// float32 CGS2 (MIXED precision inner solves): as gs_cgs2 on float32 vectors, coefficients and norms
// in float64, one host synchronisation.
int gs_cgs2_32(fm_ctx* c, const float* V, int nv, float* w, float* vout, double* h, double* hn) {
  if (nv < 1 || nv > kGsMaxVec) return FM_ERR_ARG;
  const int64_t N = c->N;
  // 16-byte quads when every vector starts on a 16-byte boundary (N a multiple of 4), scalar loads otherwise
  const uintptr_t al = reinterpret_cast<uintptr_t>(V) | reinterpret_cast<uintptr_t>(w) | (uintptr_t)(N * 4);
  const bool quads = (al & 15u) == 0;
  double* h1 = c->gsd;
  double* h2 = c->gsd + kGsMaxVec;
  double* sc = c->gsd + 3 * kGsMaxVec;
  const int nb = c->red_blocks, nb2 = 4 * c->red_blocks;
  {
    const int tk_ = prof_begin(c, FM_KERNEL_DOT);
    if (quads) k_dot_many32v<<<nb, kRedThreads, 0, c->stream>>>(V, N, nv, w, N, c->red, c->gs_cnt, h1);
    else k_dot_many32<<<nb, kRedThreads, 0, c->stream>>>(V, N, nv, w, N, c->red, c->gs_cnt, h1);
    prof_end(c, tk_, 2.0 * nv * (double)N, (nv + 1.0) * 4.0 * (double)N);
  }
  {
    const int tk_ = prof_begin(c, FM_KERNEL_AXPY);
    k_gs_axpy32<0><<<nb2, kRedThreads, 0, c->stream>>>(V, N, nv, h1, w, nullptr, N, c->red, c->gs_cnt, sc, nullptr);
    prof_end(c, tk_, (2.0 * nv + 2.0) * (double)N, (nv + 2.0) * 4.0 * (double)N);
  }
  {
    const int tk_ = prof_begin(c, FM_KERNEL_DOT);
    if (quads) k_dot_many32v<<<nb, kRedThreads, 0, c->stream>>>(V, N, nv, w, N, c->red, c->gs_cnt, h2);
    else k_dot_many32<<<nb, kRedThreads, 0, c->stream>>>(V, N, nv, w, N, c->red, c->gs_cnt, h2);
    prof_end(c, tk_, 2.0 * nv * (double)N, (nv + 1.0) * 4.0 * (double)N);
  }
  {
    const int tk_ = prof_begin(c, FM_KERNEL_AXPY);
    k_gs_axpy32<1><<<nb2, kRedThreads, 0, c->stream>>>(V, N, nv, h2, w, vout, N, c->red, c->gs_cnt, sc + 1, sc);
    prof_end(c, tk_, (2.0 * nv + 2.0) * (double)N, (nv + 2.0) * 4.0 * (double)N);
  }
  c->launches += 4;
  FM_CUDA(cudaGetLastError());
  FM_CUDA(cudaMemcpyAsync(c->red_host, c->gsd, kGsRead * sizeof(double), cudaMemcpyDeviceToHost,
                          c->stream));
  FM_CUDA(cudaStreamSynchronize(c->stream));
  const double* hh = c->red_host;
  if (c->tc_active && reinterpret_cast<const int*>(hh + kGsFlag)[0] != 0) return FM_ERR_TIMEOUT;
  for (int i = 0; i < nv; ++i) h[i] = hh[i] + hh[kGsMaxVec + i];
  const double vn2 = hh[3 * kGsMaxVec + 1], nu = hh[3 * kGsMaxVec + 2];
  if (!(nu > 0.0) || !(vn2 > 0.0)) {
    *hn = std::isfinite(nu) && std::isfinite(vn2) ? 0.0 : nu + vn2;
    return prof_harvest(c);
  }
  const double vn = std::sqrt(vn2);
  *hn = nu * vn;
  int rc;
  if (std::fabs(vn - 1.0) > 1e-6)  // float32 vector: renormalise when Pythagoras lost digits
    if ((rc = axpby32(c, (float)(1.0 / vn), vout, 0.0f, vout))) return rc;
  return prof_harvest(c);
}

// z <- z - (W - U) G (U^T z) for the tuned preconditioner, G = (U^T W)^{-1} (k x k, on the device);
// no host synchronisation
int tuning_correct(fm_ctx* c, const double* U, const double* WmU, const double* Gdev, int k, double* z) {
  if (k <= 0) return FM_OK;
  if (k > kGsMaxVec) return FM_ERR_ARG;
  double* a = c->gsd + 2 * kGsMaxVec;
  int rc;
  if ((rc = dot_many_dev(c, U, c->N, k, z, nullptr, a))) return rc;
  const int tk_ = prof_begin(c, FM_KERNEL_AXPY);
  k_gs_axpy<0><<<4 * c->red_blocks, kRedThreads, 0, c->stream>>>(WmU, c->N, k, nullptr, Gdev, a, z, nullptr, c->N,
                                                                 c->red, c->gs_cnt, c->gsd + 3 * kGsMaxVec + 4,
                                                                 nullptr);
  prof_end(c, tk_, 2.0 * k * (double)c->N, (k + 2.0) * 8.0 * (double)c->N);
  c->launches++;
  FM_CUDA(cudaGetLastError());
  return FM_OK;
}

int scale_copy(fm_ctx* c, const double* x, double a, double* y) {
  {
    const int tk_ = prof_begin(c, FM_KERNEL_OTHER);
    k_axpby<<<grid_for(c->N, 256), 256, 0, c->stream>>>(a, x, 0.0, y, c->N);
    prof_end(c, tk_, 0.0, 0.0);
  }
  c->launches++;
  FM_CUDA(cudaGetLastError());
  return FM_OK;
}

int axpby(fm_ctx* c, double a, const double* x, double b, double* y) {
  {
    const int tk_ = prof_begin(c, FM_KERNEL_OTHER);
    k_axpby<<<grid_for(c->N, 256), 256, 0, c->stream>>>(a, x, b, y, c->N);
    prof_end(c, tk_, 0.0, 0.0);
  }
  c->launches++;
  FM_CUDA(cudaGetLastError());
  return FM_OK;
}

int combine(fm_ctx* c, const double* V, int64_t ldv, int nv, const double* Q_host, int nc, double* out, int64_t ldo) {
  double* qd = c->red + (int64_t)c->red_blocks * 256 + 512;
  if (nv * nc > 7680) return FM_ERR_ARG;
  FM_CUDA(cudaMemcpyAsync(qd, Q_host, (size_t)nv * nc * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  {
    const int tk_ = prof_begin(c, FM_KERNEL_OTHER);
    k_combine<<<grid_for(c->N, 256), 256, 0, c->stream>>>(V, ldv, nv, qd, nc, out, ldo, c->N);
    prof_end(c, tk_, 0.0, 0.0);
  }
  c->launches++;
  FM_CUDA(cudaGetLastError());
  FM_CUDA(cudaStreamSynchronize(c->stream));
  return FM_OK;
}

int absmax(fm_ctx* c, const double* x, double* val) {
  const int nb = c->red_blocks;
  double* pv = c->red;
  long long* pi = (long long*)(c->red + nb);
  {
    const int tk_ = prof_begin(c, FM_KERNEL_OTHER);
    k_absmax<<<nb, 256, 0, c->stream>>>(x, c->N, pv, pi);
    prof_end(c, tk_, 0.0, 0.0);
  }
  c->launches++;
  std::vector<double> hv(nb);
  std::vector<long long> hi(nb);
  FM_CUDA(cudaMemcpyAsync(hv.data(), pv, nb * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  FM_CUDA(cudaMemcpyAsync(hi.data(), pi, nb * sizeof(long long), cudaMemcpyDeviceToHost, c->stream));
  FM_CUDA(cudaStreamSynchronize(c->stream));
  double best = 0.0;
  long long bi = -1;
  for (int b = 0; b < nb; ++b) {
    if (hi[b] < 0) continue;
    if (bi < 0 || fabs(hv[b]) > fabs(best) || (fabs(hv[b]) == fabs(best) && hi[b] < bi)) { best = hv[b]; bi = hi[b]; }
  }
  *val = best;
  return FM_OK;
}

int prof_begin(fm_ctx* c, int cls) {
  if (!c->prof) return -1;
  cudaEvent_t a, b;
  for (cudaEvent_t* e : {&a, &b}) {
    if (!c->ev_free.empty()) {
      *e = c->ev_free.back();
      c->ev_free.pop_back();
    } else if (cudaEventCreate(e) != cudaSuccess) {
      return -1;
    }
  }
  cudaEventRecord(a, c->stream);
  c->recs.push_back({cls, a, b});
  return (int)c->recs.size() - 1;
}

void prof_end(fm_ctx* c, int token, double flops, double bytes) {
  if (token < 0 || token >= (int)c->recs.size()) return;
  cudaEventRecord(c->recs[token].b, c->stream);
  c->prof_flops[c->recs[token].cls] += flops;
  c->prof_bytes[c->recs[token].cls] += bytes;
}

int prof_harvest(fm_ctx* c) {
  if (c->recs.empty()) return FM_OK;
  std::vector<fm_ctx::ProfRec> keep;
  for (auto& r : c->recs) {
    if (cudaEventQuery(r.b) != cudaSuccess) {
      cudaGetLastError();
      keep.push_back(r);
      continue;
    }
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      c->prof_ms[r.cls] += ms;
      c->prof_n[r.cls] += 1;
    } else {
      cudaGetLastError();
    }
    c->ev_free.push_back(r.a);
    c->ev_free.push_back(r.b);
  }
  c->recs.swap(keep);
  return FM_OK;
}

int dot_many32(fm_ctx* c, const float* V, int64_t ldv, int nv, const float* w, double* h_host) {
  const int nb = c->red_blocks;
  if (nv > kGsMaxVec) return FM_ERR_ARG;
  {
    const int tk_ = prof_begin(c, FM_KERNEL_DOT);
    k_dot_many32<<<nb, kRedThreads, 0, c->stream>>>(V, ldv, nv, w, c->N, c->red, c->gs_cnt, c->gsd);
    prof_end(c, tk_, 2.0 * nv * (double)c->N, (nv + 1.0) * 4.0 * (double)c->N);
  }
  c->launches++;
  FM_CUDA(cudaGetLastError());
  FM_CUDA(cudaMemcpyAsync(c->red_host, c->gsd, nv * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  FM_CUDA(cudaStreamSynchronize(c->stream));
  std::memcpy(h_host, c->red_host, nv * sizeof(double));
  return prof_harvest(c);
}

int axpy_many_norm32(fm_ctx* c, const float* V, int64_t ldv, int nv, const double* h_host, float sign, float* w,
                     double* nrm2_out) {
  std::vector<float> hf(h_host, h_host + nv);
  float* hd = reinterpret_cast<float*>(c->red + (int64_t)c->red_blocks * 256 + 512);
  FM_CUDA(cudaMemcpyAsync(hd, hf.data(), nv * sizeof(float), cudaMemcpyHostToDevice, c->stream));
  const int nb = 4 * c->red_blocks;
  {
    const int tk_ = prof_begin(c, FM_KERNEL_AXPY);
    k_axpy_many_norm32<<<nb, kRedThreads, 0, c->stream>>>(V, ldv, nv, hd, sign, w, c->N, c->red, c->gs_cnt,
                                                          c->gsd + 3 * kGsMaxVec);
    prof_end(c, tk_, (2.0 * nv + 2.0) * (double)c->N, (nv + 2.0) * 4.0 * (double)c->N);
  }
  c->launches++;
  FM_CUDA(cudaGetLastError());
  if (nrm2_out) {
    FM_CUDA(cudaMemcpyAsync(c->red_host, c->gsd + 3 * kGsMaxVec, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    FM_CUDA(cudaStreamSynchronize(c->stream));
    *nrm2_out = c->red_host[0];
    return prof_harvest(c);
  }
  return FM_OK;
}

int to32(fm_ctx* c, const double* x, double a, float* y) {
  const int tk_ = prof_begin(c, FM_KERNEL_OTHER);
  k_to32<<<grid_for(c->N, 256), 256, 0, c->stream>>>(x, a, y, c->N);
  prof_end(c, tk_, 0.0, 0.0);
  c->launches++;
  FM_CUDA(cudaGetLastError());
  return FM_OK;
}

int add32(fm_ctx* c, const float* y, double a, double* x) {
  const int tk_ = prof_begin(c, FM_KERNEL_OTHER);
  k_add32<<<grid_for(c->N, 256), 256, 0, c->stream>>>(y, a, x, c->N);
  prof_end(c, tk_, 0.0, 0.0);
  c->launches++;
  FM_CUDA(cudaGetLastError());
  return FM_OK;
}

int axpby32(fm_ctx* c, float a, const float* x, float b, float* y) {
  const int tk_ = prof_begin(c, FM_KERNEL_OTHER);
  k_axpby32<<<grid_for(c->N, 256), 256, 0, c->stream>>>(a, x, b, y, c->N);
  prof_end(c, tk_, 0.0, 0.0);
  c->launches++;
  FM_CUDA(cudaGetLastError());
  return FM_OK;
}

// ---------------------------------------------------------------------------
// double-float inner solves (mixed_scheme 2)
// ---------------------------------------------------------------------------
int launch_apply_dd(fm_ctx* c, double E, const dd* x, dd* y, bool only_S) {
  // the float64 scratch planes, read as dd (the same 8 bytes per element; the float64 and dd applies never
  // overlap)
  return apply_t<dd>(c, E, x, y, only_S, reinterpret_cast<dd*>(c->P), reinterpret_cast<dd*>(c->Q),
                     reinterpret_cast<dd*>(c->R), true);
}

int launch_precond_dd(fm_ctx* c, const dd* x, dd* y) {
  int rc;
  {
    const int tk_ = prof_begin(c, FM_KERNEL_OTHER);
    k_dd_hi<<<grid_for(c->N, 256), 256, 0, c->stream>>>(x, c->d32, c->N);
    prof_end(c, tk_, 0.0, 12.0 * (double)c->N);
  }
  if ((rc = launch_precond32(c, c->d32, c->e32))) return rc;
  {
    const int tk_ = prof_begin(c, FM_KERNEL_OTHER);
    k_f_to_dd<<<grid_for(c->N, 256), 256, 0, c->stream>>>(c->e32, y, c->N);
    prof_end(c, tk_, 0.0, 12.0 * (double)c->N);
  }
  c->launches += 2;
  FM_CUDA(cudaGetLastError());
  return FM_OK;
}

int to_dd(fm_ctx* c, const double* x, double a, dd* y) {
  const int tk_ = prof_begin(c, FM_KERNEL_OTHER);
  k_to_dd<<<grid_for(c->N, 256), 256, 0, c->stream>>>(x, a, y, c->N);
  prof_end(c, tk_, 0.0, 16.0 * (double)c->N);
  c->launches++;
  FM_CUDA(cudaGetLastError());
  return FM_OK;
}

int add_dd(fm_ctx* c, const dd* y, double a, double* x) {
  const int tk_ = prof_begin(c, FM_KERNEL_OTHER);
  k_add_dd<<<grid_for(c->N, 256), 256, 0, c->stream>>>(y, a, x, c->N);
  prof_end(c, tk_, 0.0, 24.0 * (double)c->N);
  c->launches++;
  FM_CUDA(cudaGetLastError());
  return FM_OK;
}

int axpby_dd(fm_ctx* c, double a, const dd* x, double b, dd* y) {
  const int tk_ = prof_begin(c, FM_KERNEL_OTHER);
  k_axpby_dd<<<grid_for(c->N, 256), 256, 0, c->stream>>>(dd(a), x, dd(b), b == 0.0, y, c->N);
  prof_end(c, tk_, 0.0, 24.0 * (double)c->N);
  c->launches++;
  FM_CUDA(cudaGetLastError());
  return FM_OK;
}

int dot_many_dd(fm_ctx* c, const dd* V, int64_t ldv, int nv, const dd* w, double* h_host) {
  if (nv < 1 || nv > kGsMaxVec) return FM_ERR_ARG;
  {
    const int tk_ = prof_begin(c, FM_KERNEL_DOT);
    k_dot_many_dd<<<c->red_blocks, kRedThreads, 0, c->stream>>>(V, ldv, nv, w, c->N, c->red, c->gs_cnt, c->gsd);
    prof_end(c, tk_, 2.0 * nv * (double)c->N, (nv + 1.0) * 8.0 * (double)c->N);
  }
  c->launches++;
  FM_CUDA(cudaGetLastError());
  FM_CUDA(cudaMemcpyAsync(c->red_host, c->gsd, nv * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  FM_CUDA(cudaStreamSynchronize(c->stream));
  std::memcpy(h_host, c->red_host, nv * sizeof(double));
  return prof_harvest(c);
}

int axpy_many_dd(fm_ctx* c, const dd* V, int64_t ldv, int nv, const double* h_host, dd* w) {
  if (nv < 1 || nv > kGsMaxVec) return FM_ERR_ARG;
  double* hd = c->red + (int64_t)c->red_blocks * 256 + 512;
  FM_CUDA(cudaMemcpyAsync(hd, h_host, nv * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  {
    const int tk_ = prof_begin(c, FM_KERNEL_AXPY);
    k_gs_axpy_dd<2><<<4 * c->red_blocks, kRedThreads, 0, c->stream>>>(V, ldv, nv, hd, w, nullptr, c->N, nullptr,
                                                                      nullptr, nullptr, nullptr);
    prof_end(c, tk_, 2.0 * nv * (double)c->N, (nv + 2.0) * 8.0 * (double)c->N);
  }
  c->launches++;
  FM_CUDA(cudaGetLastError());
  return FM_OK;  // the next copy into hd is ordered after this kernel on the stream
}

// Two classical Gram-Schmidt passes in dd (dot products and updates accumulated in dd): w <- w - V h,
// vout = w / hn, as gs_cgs2_32 does in float32.
int gs_cgs2_dd(fm_ctx* c, const dd* V, int nv, dd* w, dd* vout, double* h, double* hn) {
  if (nv < 1 || nv > kGsMaxVec) return FM_ERR_ARG;
  const int64_t N = c->N;
  double* h1 = c->gsd;
  double* h2 = c->gsd + kGsMaxVec;
  double* sc = c->gsd + 3 * kGsMaxVec;
  const int nb = c->red_blocks, nb2 = 4 * c->red_blocks;
  {
    const int tk_ = prof_begin(c, FM_KERNEL_DOT);
    k_dot_many_dd<<<nb, kRedThreads, 0, c->stream>>>(V, N, nv, w, N, c->red, c->gs_cnt, h1);
    prof_end(c, tk_, 2.0 * nv * (double)N, (nv + 1.0) * 8.0 * (double)N);
  }
  {
    const int tk_ = prof_begin(c, FM_KERNEL_AXPY);
    k_gs_axpy_dd<0><<<nb2, kRedThreads, 0, c->stream>>>(V, N, nv, h1, w, nullptr, N, c->red, c->gs_cnt, sc, nullptr);
    prof_end(c, tk_, (2.0 * nv + 2.0) * (double)N, (nv + 2.0) * 8.0 * (double)N);
  }
  {
    const int tk_ = prof_begin(c, FM_KERNEL_DOT);
    k_dot_many_dd<<<nb, kRedThreads, 0, c->stream>>>(V, N, nv, w, N, c->red, c->gs_cnt, h2);
    prof_end(c, tk_, 2.0 * nv * (double)N, (nv + 1.0) * 8.0 * (double)N);
  }
  {
    const int tk_ = prof_begin(c, FM_KERNEL_AXPY);
    k_gs_axpy_dd<1><<<nb2, kRedThreads, 0, c->stream>>>(V, N, nv, h2, w, vout, N, c->red, c->gs_cnt, sc + 1, sc);
    prof_end(c, tk_, (2.0 * nv + 2.0) * (double)N, (nv + 2.0) * 8.0 * (double)N);
  }
  c->launches += 4;
  FM_CUDA(cudaGetLastError());
  FM_CUDA(cudaMemcpyAsync(c->red_host, c->gsd, kGsRead * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  FM_CUDA(cudaStreamSynchronize(c->stream));
  const double* hh = c->red_host;
  if (c->tc_active && reinterpret_cast<const int*>(hh + kGsFlag)[0] != 0) return FM_ERR_TIMEOUT;
  for (int i = 0; i < nv; ++i) h[i] = hh[i] + hh[kGsMaxVec + i];
  const double vn2 = hh[3 * kGsMaxVec + 1], nu = hh[3 * kGsMaxVec + 2];
  if (!(nu > 0.0) || !(vn2 > 0.0)) {
    *hn = std::isfinite(nu) && std::isfinite(vn2) ? 0.0 : nu + vn2;
    return prof_harvest(c);
  }
  const double vn = std::sqrt(vn2);
  *hn = nu * vn;
  int rc;
  if (std::fabs(vn - 1.0) > 1e-12)  // renormalise when Pythagoras lost digits
    if ((rc = axpby_dd(c, 1.0 / vn, vout, 0.0, vout))) return rc;
  return prof_harvest(c);
}

int* tc_flag_slot(fm_ctx* c) { return reinterpret_cast<int*>(c->gsd + kGsFlag); }

int kernels_init(fm_ctx* c) {
  (void)c;
  FM_CUDA(cudaFuncSetAttribute(k_apply_xy<8, 4, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  FM_CUDA(cudaFuncSetAttribute(k_apply_xy<8, 4, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  FM_CUDA(cudaFuncSetAttribute(k_apply_xy<8, 6, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  FM_CUDA(cudaFuncSetAttribute(k_apply_xy<8, 6, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  FM_CUDA(cudaFuncSetAttribute(k_apply_xy<8, 4, dd>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  FM_CUDA(cudaFuncSetAttribute(k_apply_xy<8, 6, dd>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  FM_CUDA(cudaFuncSetAttribute(k_zmix<double, double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  FM_CUDA(cudaFuncSetAttribute(k_zmix<double, float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  FM_CUDA(cudaFuncSetAttribute(k_zmix<float, double, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  FM_CUDA(cudaFuncSetAttribute(k_zmix<float, float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  FM_CUDA(cudaFuncSetAttribute(k_ysolve<double, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  FM_CUDA(cudaFuncSetAttribute(k_ysolve<double, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  FM_CUDA(cudaFuncSetAttribute(k_ysolve<float, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  FM_CUDA(cudaFuncSetAttribute(k_ysolve<float, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  return tc_kernels_init();
}

int fill_normal(fm_ctx* c, double* x, uint64_t seed) {
  {
    const int tk_ = prof_begin(c, FM_KERNEL_OTHER);
    k_fill_normal<<<grid_for(c->N, 256), 256, 0, c->stream>>>(x, c->N, seed);
    prof_end(c, tk_, 0.0, 0.0);
  }
  c->launches++;
  FM_CUDA(cudaGetLastError());
  return FM_OK;
}

}  // namespace fmi
