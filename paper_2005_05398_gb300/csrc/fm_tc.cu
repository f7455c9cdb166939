// Tensor-core mode products of the float32 preconditioner (Eq. prec-2, Section 3.3).
//
// The inverse of the tensor-trick preconditioner is a chain of mode products: W-bar_z, W-bar_x,
// the y stage, W_x, W_z.  The x and y stages are, per (component, M', z-mode) slab, dense
// n x n matrix products with the slab (n = 2 nint <= 256).  Here they run as batched GEMMs on the
// 5th-generation tensor cores: tcgen05.mma kind::tf32 with float32 accumulation in tensor memory,
// both operands staged into shared memory by TMA (128-byte swizzle, K-major), one CTA per 128
// slab rows, a 4-deep mbarrier pipeline between the TMA producer thread and the MMA thread, and
// a 4-warp epilogue that reads the accumulator with tcgen05.ld.
//
// Every operand is K-major (the contracted index contiguous in memory).  The chain keeps that
// true by choosing the layout each stage writes:
//   z forward   x[M'][k][i][j]           -> t[slab][j][i]     (SIMT, transposed store)
//   x forward   A = t (rows j, K = i)    -> u[slab][i][j]     (ydiag)  or u[slab][j][i] (banded y)
//   y forward   A = u (rows i, K = j)    -> t[slab][i][j] / (lambda_x + lambda_y)
//   y inverse   A = t (rows i, K = j)    -> u[slab][j][i]
//   (banded y solves work in place on u[slab][j][i])
//   x inverse   A = u (rows j, K = i)    -> t[slab][i][j]
//   z inverse   t[slab][i][j]            -> y[M'][k][i][j]    (SIMT)
// The diagonal 1/(lambda_x + lambda_y) of the y stage (lambda_y holds lambda_z - E*) is summed
// from float64 values split into (hi, lo) float pairs, so that the near-singular sum keeps its
// float64 accuracy before the float32 reciprocal.
//
// Every mbarrier wait is bounded (about one second of global time); a wait that expires sets an
// error flag that the host reads, and the kernel still releases its tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>

#include "fm_internal.h"

namespace fmi {

namespace {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the completion of the phase with the given parity, for at most about one second.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t it = 0;; ++it) {
    if (mbar_try(bar, parity)) return true;
    if ((it & 255u) == 255u && global_ns() - t0 > 1000000000ull) return false;
  }
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
      : "memory");
}

// Shared-memory matrix descriptor of a K-major operand tile in the 128-byte swizzled layout
// (rows of 128 bytes, 8-row atoms 1024 bytes apart).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
  uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;             // leading-dimension offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;   // stride between 8-row atoms
  d |= (uint64_t)1 << 46;             // descriptor version of sm_100 family
  d |= (uint64_t)2 << 61;             // 128-byte swizzle
  return d;
}

// Instruction descriptor: kind::tf32, D float32, A and B tf32, both K-major, M = 128, N = n.
__host__ __device__ constexpr uint32_t tf32_idesc(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((128u >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}

// kind::f16 with BF16 A and B, float32 accumulation (same descriptor conventions as the TF32 form)
__host__ __device__ constexpr uint32_t bf16_idesc(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((128u >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 consecutive accumulator columns of this warp's 32 lanes (one row per thread)
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float v[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// 1 / (a + b) for a = ah + al, b = bh + bl given as float pairs: the sum is formed with an
// error-free two-sum of the high parts, so cancellation between a and b costs no accuracy.
__device__ __forceinline__ float inv_sum2(float2 a, float2 b) {
  const float s = a.x + b.x;
  const float bb = s - a.x;
  const float e = (a.x - (s - bb)) + (b.x - bb);
  return __frcp_rn(s + (e + (a.y + b.y)));
}

}  // namespace

struct TcArgs {
  int rows;            // A rows per slab (the vector index that is not contracted)
  int K;               // contraction length
  int N;               // outputs per row (rows of W)
  int nb;              // N rounded up to 16: MMA N and the B box height
  int nkb;             // K blocks of 32 elements
  int stages;          // pipeline depth
  int ncols;           // tensor-memory columns allocated (power of two >= nb)
  int nz;              // slabs per M' (slab = iM * nz + k, l - M0 = iM + k)
  int trans_out;       // 1: out[slab][n][row]; 0: out[slab][row][n]
  int64_t slab_stride;
  int ldo;             // stride between out rows of the chosen layout
  float* out;
  const float2* dRow;  // optional diagonal terms (hi, lo): [nl][rows]
  const float2* dCol;  //                                    [nl][N]
  int* err;            // set to 1 when a bounded wait expired
};

constexpr int kTcThreads = 128;
constexpr uint32_t kTileA = 128 * 128;  // 128 rows x 32 tf32

// out = W^l . slab (see the chain above), one CTA per (128-row tile, slab)
__global__ void __launch_bounds__(kTcThreads, 1)
    k_tc_mix(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const TcArgs a) {
  extern __shared__ unsigned char tc_smem[];
  const uint32_t raw = smem_u32(tc_smem);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char* gbase = tc_smem + (base - raw);
  const uint32_t tileB = (uint32_t)a.nb * 128u;
  const uint32_t stage_bytes = kTileA + tileB;
  const uint32_t bars = base + (uint32_t)a.stages * stage_bytes;  // full[8], empty[8], done
  const uint32_t full0 = bars, empty0 = bars + 64, done = bars + 128, slot = bars + 136;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(gbase + (bars - base) + 140);
  volatile int* n_issued = reinterpret_cast<volatile int*>(gbase + (bars - base) + 144);
  float2* dcol_s = reinterpret_cast<float2*>(gbase + (bars - base) + 256);  // [nb] column diagonal terms
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int slab = blockIdx.y, row0 = blockIdx.x * 128;
  const int il = slab / a.nz + slab % a.nz;

  if (threadIdx.x == 0) {
    for (int s = 0; s < a.stages; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    *n_issued = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(a.ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(gbase + (slot - base));

  if (warp == 0 && lane == 0) {  // TMA producer
    for (int kb = 0; kb < a.nkb; ++kb) {
      const int s = kb % a.stages;
      const uint32_t ph = (uint32_t)(kb / a.stages) & 1u;
      if (kb >= a.stages && !mbar_wait(empty0 + 8 * s, ph ^ 1u)) {
        *abort_flag = 1;
        break;
      }
      if (*abort_flag) break;
      const uint32_t sa = base + (uint32_t)s * stage_bytes;
      mbar_expect_tx(full0 + 8 * s, stage_bytes);
      tma_load_3d(sa, &tmA, kb * 32, row0, slab, full0 + 8 * s);
      tma_load_3d(sa + kTileA, &tmB, kb * 32, 0, il, full0 + 8 * s);
      *n_issued = kb + 1;
    }
  } else if (warp == 1 && lane == 0) {  // MMA issuer
    const uint32_t idesc = tf32_idesc(a.nb);
    bool ok = true;
    for (int kb = 0; kb < a.nkb && ok; ++kb) {
      const int s = kb % a.stages;
      const uint32_t ph = (uint32_t)(kb / a.stages) & 1u;
      if (!mbar_wait(full0 + 8 * s, ph) || *abort_flag) {
        *abort_flag = 1;
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t sa = base + (uint32_t)s * stage_bytes;
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        if (kb * 32 + kk * 8 >= a.K) break;  // zero-filled tail of the last block
        mma_tf32(tmem, sw128_desc(sa + 32u * kk), sw128_desc(sa + kTileA + 32u * kk), idesc, (kb | kk) ? 1u : 0u);
      }
      mma_commit(empty0 + 8 * s);
    }
    mma_commit(done);  // arrives once every MMA issued above has completed
  }
  __syncwarp();
  if (a.dRow) {  // the slab's column terms of the diagonal, staged while the MMAs run
    for (int n = threadIdx.x; n < a.nb; n += kTcThreads)
      dcol_s[n] = (n < a.N) ? a.dCol[(int64_t)il * a.N + n] : make_float2(1.f, 0.f);
  }
  __syncthreads();

  // epilogue: all four warps, warp w owns accumulator lanes (rows) 32w .. 32w + 31
  const bool ready = mbar_wait(done, 0);
  tc_fence_after();
  if (!ready) *abort_flag = 1;
  if (__all_sync(0xffffffffu, ready && !*abort_flag)) {
    const int r = row0 + warp * 32 + lane;
    const bool rok = r < a.rows;
    float* outs = a.out + (int64_t)slab * a.slab_stride;
    float2 drow = make_float2(0.f, 0.f);
    if (a.dRow && rok) drow = a.dRow[(int64_t)il * a.rows + r];
    float* stg = reinterpret_cast<float*>(gbase) + warp * (32 * 33);  // stage 0 is free now
    for (int c0 = 0; c0 < a.nb; c0 += 32) {
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (a.dRow) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int n = c0 + j;
          if (n < a.N) v[j] *= inv_sum2(drow, dcol_s[n]);
        }
      }
      if (a.trans_out) {  // out[n][r]: lanes hold consecutive rows, 128-byte stores per column
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int n = c0 + j;
          if (rok && n < a.N) outs[(int64_t)n * a.ldo + r] = v[j];
        }
      } else {  // out[r][n]: transpose the warp's 32 x 32 block through shared memory
#pragma unroll
        for (int j = 0; j < 32; ++j) stg[lane * 33 + j] = v[j];
        __syncwarp();
        const int n = c0 + lane;
        for (int q = 0; q < 32; ++q) {
          const int rq = row0 + warp * 32 + q;
          if (rq < a.rows && n < a.N) outs[(int64_t)rq * a.ldo + n] = stg[q * 33 + lane];
        }
        __syncwarp();
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && *abort_flag) {
    // a wait expired: let the loads still in flight (at most one per stage) land before exit
    const int n = *n_issued;
    for (int kb = max(0, n - a.stages); kb < n; ++kb)
      (void)mbar_wait(full0 + 8 * (kb % a.stages), (uint32_t)(kb / a.stages) & 1u);
  }
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.ncols) : "memory");
  }
  if (threadIdx.x == 0 && *abort_flag) atomicExch(a.err, 1);
}

// ---------------------------------------------------------------------------
// z mode products, register-blocked: out[l][p] = sum_k W[l][k] in[k][p] for one (component, M')
// and a tile of 128 points p = (i, j).  Eight warps; warp w computes the outputs l = lc + w + 8u
// (u < 8) of four points per lane; W is kept in shared memory permuted as Wp[k][w][u] so that a
// thread reads its 8 weights of one k with two 16-byte loads.
//   TRANS = false: the tile is 128 consecutive points of the [i][j] plane; out[l][i][j].
//   TRANS = true:  the tile is 8 (i) x 16 (j) points; out[l][j][i] (x contiguous).
// ---------------------------------------------------------------------------
constexpr int kZWarps = 8, kZThreads = 32 * kZWarps, kZOut = 64 / kZWarps;

template <typename TI, typename TO, bool TRANS>
__global__ void __launch_bounds__(kZThreads) k_zmix_rb(const float* __restrict__ Wall, const TI* __restrict__ in,
                                                       TO* __restrict__ out, int nz, int nx, int ny, int64_t comp_off) {
  extern __shared__ __align__(16) float zsm[];
  float* Vs = zsm;                    // [nz][128]
  float* Wp = zsm + (size_t)nz * 128;  // [nz][kZWarps][kZOut]
  const int iM = blockIdx.y;
  const int64_t nxy = (int64_t)nx * ny;
  const float* W = Wall + (int64_t)iM * nz * nz;
  const int64_t base = comp_off + (int64_t)iM * nz * nxy;
  int i0 = 0, j0 = 0;
  int64_t p0 = 0;
  if (TRANS) {
    const int tj = (ny + 15) / 16;
    i0 = (blockIdx.x / tj) * 8;
    j0 = (blockIdx.x % tj) * 16;
  } else {
    p0 = (int64_t)blockIdx.x * 128;
  }
  // input tile: Vs[k][q], q = jl * 8 + il (TRANS) or q = p - p0; thread t loads point t % 128 of the
  // z rows k = t / 128, t / 128 + 2, ..., eight rows of loads in flight at a time
  {
    const int t = threadIdx.x % 128, k1 = threadIdx.x / 128;
    int q = t;
    int64_t src = -1;
    if (TRANS) {
      const int il = t / 16, jl = t % 16;  // consecutive threads walk j: coalesced reads
      const int i = i0 + il, j = j0 + jl;
      q = jl * 8 + il;
      if (i < nx && j < ny) src = base + (int64_t)i * ny + j;
    } else {
      if (p0 + t < nxy) src = base + p0 + t;
    }
    for (int k0 = k1; k0 < nz; k0 += 16) {
      float v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int k = k0 + 2 * u;
        v[u] = (src >= 0 && k < nz) ? (float)in[src + (int64_t)k * nxy] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (k0 + 2 * u < nz) Vs[(k0 + 2 * u) * 128 + q] = v[u];
    }
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int lc = 0; lc < nz; lc += 64) {
    __syncthreads();
    for (int e = threadIdx.x; e < nz * 64; e += kZThreads) {  // Wp[k][w][u] = W[lc + w + 8u][k]
      const int k = e / 64, wu = e % 64, w = wu / kZOut, u = wu % kZOut;
      const int l = lc + w + kZWarps * u;
      Wp[e] = (l < nz) ? W[(int64_t)l * nz + k] : 0.f;
    }
    __syncthreads();
    float acc[kZOut][4];
#pragma unroll
    for (int u = 0; u < kZOut; ++u)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[u][q] = 0.f;
    for (int k = 0; k < nz; ++k) {
      const float4 v = *reinterpret_cast<const float4*>(&Vs[k * 128 + 4 * lane]);
      const float4* wp = reinterpret_cast<const float4*>(&Wp[(k * kZWarps + warp) * kZOut]);
#pragma unroll
      for (int u4 = 0; u4 < kZOut / 4; ++u4) {
        const float4 w = wp[u4];
        const float ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          acc[4 * u4 + t][0] = fmaf(ww[t], v.x, acc[4 * u4 + t][0]);
          acc[4 * u4 + t][1] = fmaf(ww[t], v.y, acc[4 * u4 + t][1]);
          acc[4 * u4 + t][2] = fmaf(ww[t], v.z, acc[4 * u4 + t][2]);
          acc[4 * u4 + t][3] = fmaf(ww[t], v.w, acc[4 * u4 + t][3]);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kZOut; ++u) {
      const int l = lc + warp + kZWarps * u;
      if (l >= nz) break;
      TO* ol = out + base + (int64_t)l * nxy;
      if (TRANS) {
        const int jl = lane / 2, il = 4 * (lane % 2);  // q = 4 lane .. 4 lane + 3
        const int j = j0 + jl, i = i0 + il;
        if (j < ny) {
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (i + q < nx) ol[(int64_t)j * nx + i + q] = (TO)acc[u][q];
        }
      } else {
        const int64_t p = p0 + 4 * lane;
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (p + q < nxy) ol[p + q] = (TO)acc[u][q];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Operand formats of the tensor-core mode products.  TF32: float32 storage, 32 elements per
// 128-byte row of a swizzled K-major tile, K = 8 per MMA.  BF16: 64 elements per row, K = 16.
// Both advance 32 bytes of K per MMA instruction.
// ---------------------------------------------------------------------------
struct OpTF32 {
  using T = float;
  static constexpr int kRow = 32;
  static constexpr int kStep = 8;
  static __device__ __forceinline__ uint32_t idesc(int n) { return tf32_idesc(n); }
  static __device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
    mma_tf32(d, a, b, id, acc);
  }
  static __device__ __forceinline__ float from(float v) { return v; }
  static __device__ __forceinline__ float to_f(float v) { return v; }
};
struct OpBF16 {
  using T = uint16_t;  // bfloat16 bits
  static constexpr int kRow = 64;
  static constexpr int kStep = 16;
  static __device__ __forceinline__ uint32_t idesc(int n) { return bf16_idesc(n); }
  static __device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
    mma_bf16(d, a, b, id, acc);
  }
  static __device__ __forceinline__ uint16_t from(float v) {  // round to nearest even
    uint16_t h;
    asm("cvt.rn.bf16.f32 %0, %1;" : "=h"(h) : "f"(v));
    return h;
  }
  static __device__ __forceinline__ float to_f(uint16_t h) { return __uint_as_float((uint32_t)h << 16); }
};

template <typename T>
__device__ __forceinline__ float load_as_float(const T* p) { return (float)*p; }
template <>
__device__ __forceinline__ float load_as_float<uint16_t>(const uint16_t* p) { return __uint_as_float((uint32_t)*p << 16); }
template <typename T>
__device__ __forceinline__ void store_from_float(T* p, float v) { *p = (T)v; }
template <>
__device__ __forceinline__ void store_from_float<uint16_t>(uint16_t* p, float v) { *p = OpBF16::from(v); }
// four consecutive elements in one or two vector stores (p aligned to four elements)
template <typename T>
__device__ __forceinline__ void store4_from_float(T* p, const float* v);
template <>
__device__ __forceinline__ void store4_from_float<float>(float* p, const float* v) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
template <>
__device__ __forceinline__ void store4_from_float<double>(double* p, const float* v) {
  reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
}
template <>
__device__ __forceinline__ void store4_from_float<uint16_t>(uint16_t* p, const float* v) {
  const uint32_t lo = (uint32_t)OpBF16::from(v[0]) | ((uint32_t)OpBF16::from(v[1]) << 16);
  const uint32_t hi = (uint32_t)OpBF16::from(v[2]) | ((uint32_t)OpBF16::from(v[3]) << 16);
  *reinterpret_cast<uint2*>(p) = make_uint2(lo, hi);
}

// Byte offset of (row, byte within the 128-byte row) in a 128-byte-swizzled K-major tile whose base is
// 1024-byte aligned: 8-row atoms of 1024 bytes, the 16-byte chunks of row r permuted by XOR with r mod 8.
__device__ __forceinline__ uint32_t sw128(int row, int byte) {
  return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + ((((byte >> 4) ^ row) & 7) << 4) + (byte & 15));
}

__device__ __forceinline__ void st_shared_u32(uint32_t addr, uint32_t v) {
  asm volatile("st.shared.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ void st_shared_u16(uint32_t addr, uint16_t v) {
  asm volatile("st.shared.u16 [%0], %1;" ::"r"(addr), "h"(v) : "memory");
}
__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}
template <typename Op>
__device__ __forceinline__ void st_elem(uint32_t addr, float v) {
  if constexpr (sizeof(typename Op::T) == 4) st_shared_u32(addr, __float_as_uint(v));
  else st_shared_u16(addr, Op::from(v));
}
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void named_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// ---------------------------------------------------------------------------
// z mode products on the tensor cores (Eq. prec-2, the W-bar_z and W_z stages):
//   out[M'][l][p] = sum_k W[M'][l][k] in[M'][k][p]
// for every point p = (i, j) of a component.  A = W (rows l, K = k; n_z <= 128, TMA-loaded,
// zero-filled to 128 rows and to the K padding), B = a tile of NP points (rows; NP = 128, 64 or 32) with
// their n_z values (K), converted from the input type while it is written into shared memory, D in tensor
// memory (128 lanes l x NP columns p).  Persistent CTAs walk the (M', point tile) list.
//   OUT_JI (forward):  in x[M'][k][i][j] -> out t[slab][j][i]; tiles of NP/4 i x 4 j, B row = jj * TI + ii
//   !OUT_JI (inverse): in u[slab][j][i] (IN_JI) or t[slab][i][j] -> out y[M'][k][i][j]; tiles of 8 i x NP/8 j,
//                      B row = ii * TJ + jj
// (slab = M' * n_z + l).  Loads run along the input's contiguous index (runs of 4 j forward, 8 i inverse),
// stores along the output's (runs of TI i forward, TJ j inverse).  Smaller tiles give more CTAs per SM,
// hence more loads in flight per SM; the tile width is chosen per shape by the set-up's autotuner.  Each
// thread of the epilogue owns one output plane l.
// ---------------------------------------------------------------------------
struct TcZArgs {
  const void* in;
  void* out;
  int nz, nx, ny, nM;
  int64_t off;         // component offset (elements) in both vectors
  int tiles_i, tiles_j;
  int kblocks;         // 128-byte K blocks of A and B
  int ksteps;          // MMA instructions per tile
  int vec_out;         // output runs start on four-element boundaries (host-checked): vector stores
  int* err;
};

// Tile shapes (SH): 0 = long runs on the output side (forward NP/4 i x 4 j, inverse 8 i x NP/8 j), 1 = runs
// of 8 elements on the input side too (NP/8 i x 8 j both ways), for longer DRAM bursts on the strided loads.
template <bool OUT_JI, int NP, int SH>
struct ZTile {
  static constexpr int TI = SH == 1 ? NP / 8 : (OUT_JI ? NP / 4 : 8);  // i extent of a tile
  static constexpr int TJ = SH == 1 ? 8 : (OUT_JI ? 4 : NP / 8);       // j extent
};

template <typename TI, typename Op, typename TO, bool OUT_JI, bool IN_JI, int NP, int SH>
__global__ void __launch_bounds__(128) k_tc_z(const __grid_constant__ CUtensorMap tmW, const TcZArgs a) {
  static_assert(!(OUT_JI && IN_JI), "the forward stage reads x[M'][k][i][j]");
  static_assert(NP == 128 || NP == 64 || NP == 32, "tile of 128, 64 or 32 points");
  using TB = typename Op::T;
  constexpr int TI_ = ZTile<OUT_JI, NP, SH>::TI, TJ_ = ZTile<OUT_JI, NP, SH>::TJ;
  static_assert(TI_ * TJ_ == NP && 32 % TI_ == 0 && 32 % TJ_ == 0, "a 32-column load spans whole runs");
  constexpr int kTileA = 128 * 128;  // bytes of one K block of A (128 rows x 128 bytes)
  constexpr int kTileB = NP * 128;   // of B (NP rows)
  constexpr int kTpp = 128 / NP;     // threads per point of the tile (each loads every kTpp-th k)
  extern __shared__ unsigned char tz_smem[];
  const uint32_t raw = smem_u32(tz_smem);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char* gbase = tz_smem + (base - raw);
  const uint32_t sA = base, sB = base + (uint32_t)a.kblocks * kTileA;
  const uint32_t bars = sB + (uint32_t)a.kblocks * kTileB;
  const uint32_t abar = bars, mdone = bars + 8, slot = bars + 16;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(gbase + (bars - base) + 24);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, tid = threadIdx.x;
  if (tid == 0) {
    mbar_init(abar, 1);
    mbar_init(mdone, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(NP) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(gbase + (slot - base));
  const int64_t nxy = (int64_t)a.nx * a.ny;
  const int ntiles = a.tiles_i * a.tiles_j;
  const int kpad = a.ksteps * Op::kStep;
  const TI* in = static_cast<const TI*>(a.in);
  TO* out = static_cast<TO*>(a.out);
  int cur_iM = -1, a_loads = 0;
  uint32_t a_phase = 0, m_phase = 0;
  // thread -> (point of the tile, k residue): consecutive threads take consecutive points along the
  // input's contiguous index, so that a warp's loads are coalesced runs
  const int pt = tid % NP, ksub = tid / NP;
  const int ii = IN_JI ? pt % TI_ : pt / TJ_;
  const int jj = IN_JI ? pt / TI_ : pt % TJ_;
  const int prow = OUT_JI ? jj * TI_ + ii : ii * TJ_ + jj;
  for (int q = blockIdx.x; q < ntiles * a.nM; q += gridDim.x) {
    const int iM = q / ntiles, t = q - iM * ntiles;
    const int i0 = (t / a.tiles_j) * TI_, j0 = (t % a.tiles_j) * TJ_;
    const bool reload = iM != cur_iM;
    if (reload && tid == 0) {  // W of this M' (every thread of the previous tile has passed the MMA wait)
      mbar_expect_tx(abar, (uint32_t)a.kblocks * kTileA);
      for (int kb = 0; kb < a.kblocks; ++kb) tma_load_3d(sA + kb * kTileA, &tmW, kb * Op::kRow, 0, iM, abar);
    }
    if (reload) {
      cur_iM = iM;
      ++a_loads;
    }
    // B tile: row prow, K = k (this thread: k = ksub, ksub + kTpp, ...)
    {
      const int i = i0 + ii, j = j0 + jj;
      const bool ok = i < a.nx && j < a.ny;
      const int64_t src = IN_JI ? a.off + ((int64_t)iM * a.nz * a.ny + j) * a.nx + i
                                : a.off + ((int64_t)iM * a.nz * a.nx + i) * a.ny + j;
      // 32 loads in flight per thread
      for (int k0 = ksub; k0 < kpad; k0 += 32 * kTpp) {
        float v[32];
#pragma unroll
        for (int u = 0; u < 32; ++u) {
          const int k = k0 + u * kTpp;
          v[u] = (ok && k < a.nz) ? load_as_float<TI>(in + src + (int64_t)k * nxy) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 32; ++u) {
          const int k = k0 + u * kTpp;
          if (k < kpad) {
            const int kb = k / Op::kRow, byte = (k % Op::kRow) * (int)sizeof(TB);
            st_elem<Op>(sB + kb * kTileB + sw128(prow, byte), v[u]);
          }
        }
      }
    }
    fence_async_smem();
    __syncthreads();
    if (tid == 32) {
      bool ok = !*abort_flag;
      if (ok && reload) {
        ok = mbar_wait(abar, a_phase);
        if (!ok) *abort_flag = 1;
      }
      if (ok) {
        tc_fence_after();
        const uint32_t id = Op::idesc(NP);
        for (int ks = 0; ks < a.ksteps; ++ks) {
          const int kb = (ks * Op::kStep) / Op::kRow, kin = (ks * Op::kStep) % Op::kRow;
          const uint32_t kbyte = (uint32_t)(kin * (int)sizeof(TB));
          Op::mma(tmem, sw128_desc(sA + (uint32_t)(kb * kTileA) + kbyte), sw128_desc(sB + (uint32_t)(kb * kTileB) + kbyte),
                  id, ks ? 1u : 0u);
        }
      }
      mma_commit(mdone);  // arrives when the MMAs above (if any) have completed
    }
    if (reload) a_phase ^= 1u;
    const bool ready = mbar_wait(mdone, m_phase);
    m_phase ^= 1u;
    tc_fence_after();
    if (!ready) *abort_flag = 1;
    if (__syncthreads_or(*abort_flag)) break;
    // epilogue: thread = output plane l (its TMEM lane), 32 columns (points) per load
    const int l = warp * 32 + lane;
#pragma unroll 1
    for (int c0 = 0; c0 < NP; c0 += 32) {
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (l >= a.nz) continue;
      const int64_t plane = (int64_t)iM * a.nz + l;
      if (OUT_JI) {  // 32 / TI runs of TI consecutive i, at j = j0 + (c0 + r * TI) / TI
#pragma unroll
        for (int r = 0; r < 32 / TI_; ++r) {
          const int j = j0 + (c0 + r * TI_) / TI_;
          if (j >= a.ny) continue;
          TO* o = out + a.off + (plane * a.ny + j) * a.nx + i0;
          const float* w = v + r * TI_;
          if (a.vec_out) {  // n_x is a multiple of 4: each group of four is wholly inside or outside
#pragma unroll
            for (int e = 0; e < TI_; e += 4)
              if (i0 + e < a.nx) store4_from_float<TO>(o + e, w + e);
          } else {
#pragma unroll
            for (int e = 0; e < TI_; ++e)
              if (i0 + e < a.nx) store_from_float<TO>(o + e, w[e]);
          }
        }
      } else {  // 32 / TJ runs of TJ consecutive j, at i = i0 + (c0 + r * TJ) / TJ
#pragma unroll
        for (int r = 0; r < 32 / TJ_; ++r) {
          const int i = i0 + (c0 + r * TJ_) / TJ_;
          if (i >= a.nx) continue;
          TO* o = out + a.off + (plane * a.nx + i) * a.ny + j0;
          const float* w = v + r * TJ_;
          if (a.vec_out) {  // n_y is a multiple of 4
#pragma unroll
            for (int e = 0; e < TJ_; e += 4)
              if (j0 + e < a.ny) store4_from_float<TO>(o + e, w + e);
          } else {
#pragma unroll
            for (int e = 0; e < TJ_; ++e)
              if (j0 + e < a.ny) store_from_float<TO>(o + e, w[e]);
          }
        }
      }
    }
    tc_fence_before();
    __syncthreads();
  }
  __syncthreads();
  if (tid == 0 && *abort_flag && a_loads > 0) (void)mbar_wait(abar, a_phase ^ 1u);  // let an issued W load land
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NP) : "memory");
  }
  if (tid == 0 && *abort_flag) atomicExch(a.err, 1);
}

// ---------------------------------------------------------------------------
// The x and y stages of Eq. prec-2 for n_M = 1 (per-l y diagonalisation), fused per slab l:
//   D1 = W-bar_x^l T,  D2 = (W-bar_y^l D1^T) / (lambda_x^l + lambda_y^l),  D3 = W_y^l D2,  D4 = W_x^l D3^T
// (T = the slab t[l][j][i] written by the z stage; out u[l][j][i] = D4).  The slab stays on chip: it is
// the B operand of four GEMMs in turn, rewritten in shared memory from the accumulator between them;
// only the four W^l matrices stream from memory, through a ring of 128-row x 128-byte K blocks (TMA).
// Six warps: 0-3 epilogue (each owns a quarter of the tensor-memory lanes), 4 TMA producer, 5 MMA issuer.
//   GEMM 0: A = W-bar_x (rows i', K = i), B = T [j][i]          -> D[i'][j]   -> B[i'][j]   (own row)
//   GEMM 1: A = W-bar_y (rows j', K = j), B [i'][j]             -> D[j'][i']  -> diagonal -> B[i'][j'] (columns)
//   GEMM 2: A = W_y (rows j'', K = j'),   B [i'][j']            -> D[j''][i'] -> B[j''][i'] (own row)
//   GEMM 3: A = W_x (rows i, K = i'),     B [j''][i']           -> D[i][j'']  -> out[l][j][i] (columns)
// The near-singular diagonal 1/(lambda_x + lambda_y) is summed from float pairs (inv_sum2).
// ---------------------------------------------------------------------------
struct FusedComp {
  CUtensorMap tm_in;    // slab input [ns][ny][nx], box {row elements, round16(ny)}
  CUtensorMap tm_w[4];  // W-bar_x, W-bar_y, W_y, W_x: [nl][n][n], box {row elements, 128}
  void* out;            // [ns][ny][nx]
  const float2* dLx2;   // [nl][nx] lambda_x as float pairs
  const float2* dLy2;   // [nl][ny] lambda_y (with -E*) as float pairs
  int nx, ny, ns;
};
struct FusedArgs {
  FusedComp c[3];
  int ncomp, total;
  int rowsB, kbB;       // B tile: rows (multiple of 16) and 128-byte K blocks
  int stages, ncols;    // A ring depth, tensor-memory columns
  int* err;
};

constexpr int kFusedThreads = 192;

template <typename Op>
__global__ void __launch_bounds__(kFusedThreads, 1) k_tc_fused_xy(const __grid_constant__ FusedArgs a) {
  using TB = typename Op::T;
  constexpr uint32_t kItem = 128 * 128;  // one A ring item: 128 rows x 128 bytes
  extern __shared__ unsigned char tf_smem[];
  const uint32_t raw = smem_u32(tf_smem);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char* gbase = tf_smem + (base - raw);
  const uint32_t bstride = (uint32_t)a.rowsB * 128u;  // bytes per K block of B
  const uint32_t sB = base, sA = base + (uint32_t)a.kbB * bstride;
  const uint32_t sD = sA + (uint32_t)a.stages * kItem;  // dLx2 of the slab: 256 float2
  const uint32_t bars = sD + 256 * 8;
  const uint32_t full0 = bars, empty0 = bars + 64, bload = bars + 128, bfree = bars + 136, dfull = bars + 144,
                 dfree = bars + 152, mfin = bars + 160, slot = bars + 168;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(gbase + (bars - base) + 176);
  volatile int* n_items = reinterpret_cast<volatile int*>(gbase + (bars - base) + 180);
  volatile int* n_bloads = reinterpret_cast<volatile int*>(gbase + (bars - base) + 184);
  float2* dlx_s = reinterpret_cast<float2*>(gbase + (sD - base));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < a.stages; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    mbar_init(bload, 1);
    mbar_init(bfree, 1);
    mbar_init(dfull, 1);
    mbar_init(dfree, 128);
    mbar_init(mfin, 1);
    *abort_flag = 0;
    *n_items = 0;
    *n_bloads = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(a.ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(gbase + (slot - base));
  auto locate = [&](int q, int* comp, int* slab) {
    int cq = 0;
    while (cq + 1 < a.ncomp && q >= a.c[cq].ns) {
      q -= a.c[cq].ns;
      ++cq;
    }
    *comp = cq;
    *slab = q;
  };
  // GEMM g: rows (M) and K are n_x for g = 0, 3 and n_y for g = 1, 2; N is the other one
  auto gM = [](const FusedComp& cp, int g) { return (g == 0 || g == 3) ? cp.nx : cp.ny; };
  auto gN = [](const FusedComp& cp, int g) { return (g == 0 || g == 3) ? cp.ny : cp.nx; };

  if (warp == 4) {
    if (lane == 0) {  // TMA producer
      int it = 0, si = 0;
      for (int q = blockIdx.x; q < a.total && !*abort_flag; q += gridDim.x, ++si) {
        int ci, slab;
        locate(q, &ci, &slab);
        const FusedComp& cp = a.c[ci];
        if (si > 0 && !mbar_wait(bfree, (uint32_t)(si - 1) & 1u)) {
          *abort_flag = 1;
          break;
        }
        const int kb0 = (cp.nx + Op::kRow - 1) / Op::kRow, rows0 = (cp.ny + 15) / 16 * 16;
        mbar_expect_tx(bload, (uint32_t)(kb0 * rows0 * 128));
        for (int kb = 0; kb < kb0; ++kb) tma_load_3d(sB + kb * bstride, &cp.tm_in, kb * Op::kRow, 0, slab, bload);
        *n_bloads = si + 1;
        for (int g = 0; g < 4 && !*abort_flag; ++g) {
          const int M = gM(cp, g), mt = (M + 127) / 128, kbs = (M + Op::kRow - 1) / Op::kRow;
          for (int kb = 0; kb < kbs && !*abort_flag; ++kb)
            for (int m = 0; m < mt; ++m, ++it) {
              const int s = it % a.stages;
              if (it >= a.stages && !mbar_wait(empty0 + 8 * s, ((uint32_t)(it / a.stages) & 1u) ^ 1u)) {
                *abort_flag = 1;
                break;
              }
              mbar_expect_tx(full0 + 8 * s, kItem);
              tma_load_3d(sA + s * kItem, &cp.tm_w[g], kb * Op::kRow, m * 128, slab, full0 + 8 * s);
              *n_items = it + 1;
            }
        }
      }
    }
  } else if (warp == 5) {
    if (lane == 0) {  // MMA issuer
      int it = 0, si = 0, gc = 0;
      bool ok = true;
      for (int q = blockIdx.x; q < a.total && ok; q += gridDim.x, ++si) {
        int ci, slab;
        locate(q, &ci, &slab);
        const FusedComp& cp = a.c[ci];
        for (int g = 0; g < 4 && ok; ++g, ++gc) {
          if (g == 0) ok = mbar_wait(bload, (uint32_t)si & 1u);
          if (ok && gc > 0) ok = mbar_wait(dfree, (uint32_t)(gc - 1) & 1u);
          if (!ok || *abort_flag) {
            ok = false;
            break;
          }
          tc_fence_after();
          const int M = gM(cp, g), K = M, N = gN(cp, g), nb = (N + 15) / 16 * 16;
          const int mt = (M + 127) / 128, kbs = (K + Op::kRow - 1) / Op::kRow;
          const uint32_t id = Op::idesc(nb);
          for (int kb = 0; kb < kbs && ok; ++kb)
            for (int m = 0; m < mt; ++m, ++it) {
              const int s = it % a.stages;
              if (!mbar_wait(full0 + 8 * s, (uint32_t)(it / a.stages) & 1u) || *abort_flag) {
                ok = false;
                break;
              }
              tc_fence_after();
#pragma unroll
              for (int kk = 0; kk < Op::kRow / Op::kStep; ++kk) {
                if (kb * Op::kRow + kk * Op::kStep >= K) break;
                const uint32_t koff = (uint32_t)(kk * Op::kStep * (int)sizeof(TB));
                Op::mma(tmem + (uint32_t)(m * 256), sw128_desc(sA + s * kItem + koff),
                        sw128_desc(sB + kb * bstride + koff), id, (kb | kk) ? 1u : 0u);
              }
              mma_commit(empty0 + 8 * s);
            }
          if (!ok) break;
          mma_commit(dfull);
          if (g == 3) mma_commit(bfree);
        }
      }
      if (!ok) *abort_flag = 1;
      mma_commit(mfin);  // arrives once every MMA issued above has completed
    }
  } else {  // epilogue warps 0-3
    int si = 0, gc = 0;
    for (int q = blockIdx.x; q < a.total; q += gridDim.x, ++si) {
      int ci, slab;
      locate(q, &ci, &slab);
      const FusedComp& cp = a.c[ci];
      for (int e = threadIdx.x; e < cp.nx; e += 128) dlx_s[e] = cp.dLx2[(int64_t)slab * cp.nx + e];
      named_sync(1, 128);
      bool ok = true;
      for (int g = 0; g < 4; ++g, ++gc) {
        ok = mbar_wait(dfull, (uint32_t)gc & 1u);
        tc_fence_after();
        if (!ok) *abort_flag = 1;
        if (*abort_flag) {
          ok = false;
          break;
        }
        const int M = gM(cp, g), N = gN(cp, g), nb = (N + 15) / 16 * 16;
        const int nbM = (M + 15) / 16 * 16;  // rows of the next B tile (its N)
        const int mt = (M + 127) / 128;
        for (int m = 0; m < mt; ++m) {
          const int r = m * 128 + warp * 32 + lane;  // D row of this thread
          float2 dly = make_float2(0.f, 0.f);
          if (g == 1 && r < cp.ny) dly = cp.dLy2[(int64_t)slab * cp.ny + r];
          for (int c0 = 0; c0 < nb; c0 += 32) {
            float v[32];
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(m * 256 + c0), v);
            if (g == 0 || g == 2) {
              // own row: B[N = r][K = c0 .. c0 + 31]
              if (r < nbM) {
                const int kb = c0 / Op::kRow, byte0 = (c0 % Op::kRow) * (int)sizeof(TB);
                const uint32_t rowb = sB + kb * bstride;
                if constexpr (sizeof(TB) == 4) {
#pragma unroll
                  for (int qd = 0; qd < 8; ++qd)
                    st_shared_v4(rowb + sw128(r, byte0 + 16 * qd), __float_as_uint(v[4 * qd]),
                                 __float_as_uint(v[4 * qd + 1]), __float_as_uint(v[4 * qd + 2]),
                                 __float_as_uint(v[4 * qd + 3]));
                } else {
#pragma unroll
                  for (int qd = 0; qd < 4; ++qd) {
                    uint32_t w4[4];
#pragma unroll
                    for (int h = 0; h < 4; ++h)
                      w4[h] = (uint32_t)OpBF16::from(v[8 * qd + 2 * h]) | ((uint32_t)OpBF16::from(v[8 * qd + 2 * h + 1]) << 16);
                    st_shared_v4(rowb + sw128(r, byte0 + 16 * qd), w4[0], w4[1], w4[2], w4[3]);
                  }
                }
              }
            } else if (g == 1) {
              // diagonal, then columns: B[N = c][K = r] (the 32 lanes fill 32 consecutive K of row c)
              // K positions up to the next GEMM's padded K (= n_y rounded to the MMA step) only
              if (r < (cp.ny + Op::kStep - 1) / Op::kStep * Op::kStep) {
                const int kb = r / Op::kRow, byte = (r % Op::kRow) * (int)sizeof(TB);
                const uint32_t colb = sB + kb * bstride;
#pragma unroll
                for (int e = 0; e < 32; ++e) {
                  const int cc = c0 + e;
                  float x = v[e];
                  if (r < cp.ny && cc < cp.nx) x *= inv_sum2(dlx_s[cc], dly);
                  else x = 0.f;
                  if (cc < nb) st_elem<Op>(colb + sw128(cc, byte), x);
                }
              }
            } else {
              // out[l][j = c][i = r]: the 32 lanes write 32 consecutive i
              if (r < cp.nx) {
                TB* o = static_cast<TB*>(cp.out) + (int64_t)slab * cp.ny * cp.nx + r;
#pragma unroll
                for (int e = 0; e < 32; ++e) {
                  const int cc = c0 + e;
                  if (cc < cp.ny) {
                    if constexpr (sizeof(TB) == 4) o[(int64_t)cc * cp.nx] = v[e];
                    else o[(int64_t)cc * cp.nx] = OpBF16::from(v[e]);
                  }
                }
              }
            }
          }
        }
        if (g < 3) fence_async_smem();
        tc_fence_before();
        mbar_arrive(dfree);
      }
      if (!ok) break;
    }
  }
  // tear-down: every issued MMA has completed (mfin) and every issued TMA load has landed
  __syncthreads();
  if (threadIdx.x == 0) {
    if (!mbar_wait(mfin, 0)) *abort_flag = 1;
    if (*abort_flag) {
      const int n = *n_items;
      for (int it = (n > a.stages ? n - a.stages : 0); it < n; ++it)
        (void)mbar_wait(full0 + 8 * (it % a.stages), (uint32_t)(it / a.stages) & 1u);
      const int nb = *n_bloads;
      if (nb > 0) (void)mbar_wait(bload, (uint32_t)(nb - 1) & 1u);
    }
  }
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.ncols) : "memory");
  }
  if (threadIdx.x == 0 && *abort_flag) atomicExch(a.err, 1);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// 3D float32 map [d2][d1][d0] (d0 contiguous), box 32 x box1 x 1, 128-byte swizzle, zero fill
bool encode3(CUtensorMap* m, const float* ptr, int d0, int d1, int d2, int box1) {
  auto fn = encode_fn();
  if (!fn) return false;
  if ((reinterpret_cast<uintptr_t>(ptr) & 15u) != 0 || (d0 * 4) % 16 != 0 || box1 < 1 || box1 > 256) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)d0, (cuuint64_t)d1, (cuuint64_t)d2};
  const cuuint64_t strides[2] = {(cuuint64_t)d0 * 4, (cuuint64_t)d0 * d1 * 4};
  const cuuint32_t box[3] = {32, (cuuint32_t)box1, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(ptr), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 3D map of any element type [d2][d1][d0] (d0 contiguous), box box0 x box1 x 1, 128-byte swizzle, zero fill
bool encode3t(CUtensorMap* m, const void* ptr, CUtensorMapDataType dt, int esize, int d0, int d1, int d2, int box0,
              int box1) {
  auto fn = encode_fn();
  if (!fn || !ptr) return false;
  if ((reinterpret_cast<uintptr_t>(ptr) & 15u) != 0 || ((int64_t)d0 * esize) % 16 != 0 || box0 * esize > 128 ||
      box1 < 1 || box1 > 256)
    return false;
  const cuuint64_t dims[3] = {(cuuint64_t)d0, (cuuint64_t)d1, (cuuint64_t)d2};
  const cuuint64_t strides[2] = {(cuuint64_t)d0 * esize, (cuuint64_t)d0 * d1 * esize};
  const cuuint32_t box[3] = {(cuuint32_t)box0, (cuuint32_t)box1, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  return fn(m, dt, 3, const_cast<void*>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

int round16(int n) { return (n + 15) / 16 * 16; }

// shared memory of the fused x / y kernel: B tile, A ring, the slab's lambda_x pairs, barriers
size_t fused_smem(int nx, int ny, int row_elems, int stages) {
  const int n = std::max(nx, ny);
  const size_t rowsB = (size_t)round16(n), kbB = (size_t)((n + row_elems - 1) / row_elems);
  return 1024 + kbB * rowsB * 128 + (size_t)stages * 16384 + 256 * 8 + 256;
}

int fused_stages(int nx, int ny, int row_elems) {
  for (int st = 4; st >= 2; --st)
    if (fused_smem(nx, ny, row_elems, st) <= 232448 - 1024) return st;
  return 0;
}

size_t tcz_smem(int kblocks, int np) { return 1024 + (size_t)kblocks * 16384 + (size_t)kblocks * np * 128 + 64; }

int tmem_cols(int nb) {
  int c = 32;
  while (c < nb) c *= 2;
  return c;
}

size_t tc_smem_bytes(int nb, int stages, int ncols) {
  size_t b = 1024 + (size_t)stages * (kTileA + (size_t)nb * 128) + 256 + (size_t)nb * sizeof(float2);
  // at most 512 / ncols CTAs may share an SM's tensor memory: ask for enough shared memory that
  // no more fit (228 KB per SM, 1 KB reserved per CTA)
  const int max_ctas = 512 / ncols;
  if (max_ctas < 16) b = std::max(b, (size_t)(233472 / (max_ctas + 1)) + 1);
  return b;
}

}  // namespace

bool tc_component_ok(const Comp& cp) {
  return cp.nx % 4 == 0 && cp.ny % 4 == 0 && cp.nx <= 256 && cp.ny <= 256 && cp.nx >= 16 && cp.ny >= 16;
}

static bool bf16_component_ok(const Comp& cp) {
  return tc_component_ok(cp) && cp.nx % 8 == 0 && cp.ny % 8 == 0 && cp.nz <= 128;
}

static int tcz_autotune(fm_ctx* c);

int tc_setup(fm_ctx* c) {
  c->tc_active = false;
  c->bf16 = false;
  if (c->opts.precision == FM_PREC_FP64 || c->opts.mma == FM_MMA_SIMT) return FM_OK;
  const bool want_bf16 = c->opts.mma == FM_MMA_BF16;
  bool all = true;
  for (auto& cp : c->comps) all = all && (want_bf16 ? bf16_component_ok(cp) : tc_component_ok(cp));
  if (!all) return (c->opts.mma == FM_MMA_TF32 || want_bf16) ? FM_ERR_ARG : FM_OK;
  if (!encode_fn()) return c->opts.mma == FM_MMA_AUTO ? FM_OK : FM_ERR_CUDA;
  if (!c->tc_err) {  // read back with every Gram-Schmidt result, so a Krylov step sees an expired wait
    c->tc_err = tc_flag_slot(c);
    FM_CUDA(cudaMemsetAsync(c->tc_err, 0, sizeof(double), c->stream));
  }
  const CUtensorMapDataType dt = want_bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  const int es = want_bf16 ? 2 : 4, E = 128 / es;
  for (auto& cp : c->comps) {
    const int nx = cp.nx, ny = cp.ny, ns = c->nM * cp.nz, nl = cp.nl;
    float* t = c->t32 + cp.off;
    float* u = c->u32 + cp.off;
    bool ok = encode3(&cp.tm[0], t, nx, ny, ns, 128)       // x forward: t[slab][j][i]
              && encode3(&cp.tm[1], u, nx, ny, ns, 128)     // x inverse: u[slab][j][i]
              && encode3(&cp.tm[2], cp.Wxb32, nx, nx, nl, round16(nx)) && encode3(&cp.tm[3], cp.Wx32, nx, nx, nl, round16(nx));
    if (ok && cp.Wy32) {
      ok = encode3(&cp.tm[4], u, ny, nx, ns, 128)           // y forward: u[slab][i][j]
           && encode3(&cp.tm[5], t, ny, nx, ns, 128)        // y inverse: t[slab][i][j]
           && encode3(&cp.tm[6], cp.Wyb32, ny, ny, nl, round16(ny)) && encode3(&cp.tm[7], cp.Wy32, ny, ny, nl, round16(ny));
    }
    if (!ok) return FM_ERR_CUDA;
    // z stages on the tensor cores (W_z with padded rows)
    cp.tcz = c->opts.tc_chain == 0 && cp.Wz_tc && cp.Wzb_tc && cp.nz <= 128;
    if (cp.tcz) {
      ok = encode3t(&cp.tmz[0], cp.Wzb_tc, dt, es, cp.ldz, cp.nz, c->nM, E, 128) &&
           encode3t(&cp.tmz[1], cp.Wz_tc, dt, es, cp.ldz, cp.nz, c->nM, E, 128);
      if (!ok) return FM_ERR_CUDA;
    }
    // n_M = 1: the fused x / y chain (slab in t[slab][j][i], out u[slab][j][i])
    cp.fused = false;
    if (c->nM == 1 && cp.Wy32 && cp.tcz && fused_stages(nx, ny, E) > 0) {
      const void* tin = want_bf16 ? (const void*)(reinterpret_cast<const uint16_t*>(c->t32) + cp.off) : (const void*)t;
      const void* w[4] = {want_bf16 ? (const void*)cp.Wxb16 : (const void*)cp.Wxb32,
                          want_bf16 ? (const void*)cp.Wyb16 : (const void*)cp.Wyb32,
                          want_bf16 ? (const void*)cp.Wy16 : (const void*)cp.Wy32,
                          want_bf16 ? (const void*)cp.Wx16 : (const void*)cp.Wx32};
      const int wn[4] = {nx, ny, ny, nx};
      ok = encode3t(&cp.tmf[0], tin, dt, es, nx, ny, ns, E, round16(ny));
      for (int g = 0; g < 4 && ok; ++g) ok = encode3t(&cp.tmf[1 + g], w[g], dt, es, wn[g], wn[g], nl, E, 128);
      if (!ok) return FM_ERR_CUDA;
      cp.fused = true;
    }
  }
  c->bf16 = want_bf16;
  c->tc_active = true;
  return tcz_autotune(c);
}

template <typename TI, typename Op, typename TO, bool OUT_JI, bool IN_JI, int SH>
static cudaError_t tcz_attr_sh() {
  cudaError_t e = cudaFuncSetAttribute(k_tc_z<TI, Op, TO, OUT_JI, IN_JI, 128, SH>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_tc_z<TI, Op, TO, OUT_JI, IN_JI, 64, SH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             227 * 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_tc_z<TI, Op, TO, OUT_JI, IN_JI, 32, SH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             227 * 1024);
  return e;
}
template <typename TI, typename Op, typename TO, bool OUT_JI, bool IN_JI>
static cudaError_t tcz_attr() {
  cudaError_t e = tcz_attr_sh<TI, Op, TO, OUT_JI, IN_JI, 0>();
  return e == cudaSuccess ? tcz_attr_sh<TI, Op, TO, OUT_JI, IN_JI, 1>() : e;
}

int tc_kernels_init() {
  FM_CUDA(cudaFuncSetAttribute(k_tc_mix, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
  FM_CUDA(cudaFuncSetAttribute(k_tc_fused_xy<OpTF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
  FM_CUDA(cudaFuncSetAttribute(k_tc_fused_xy<OpBF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
  // z forward: x (float64 / float32) -> t (float32, or BF16 ahead of the fused BF16 chain)
  FM_CUDA((tcz_attr<double, OpTF32, float, true, false>()));
  FM_CUDA((tcz_attr<float, OpTF32, float, true, false>()));
  FM_CUDA((tcz_attr<double, OpBF16, float, true, false>()));
  FM_CUDA((tcz_attr<float, OpBF16, float, true, false>()));
  FM_CUDA((tcz_attr<double, OpBF16, uint16_t, true, false>()));
  FM_CUDA((tcz_attr<float, OpBF16, uint16_t, true, false>()));
  // z inverse: u[slab][j][i] of the fused chain or t[slab][i][j] of the unfused one -> y
  FM_CUDA((tcz_attr<float, OpTF32, double, false, true>()));
  FM_CUDA((tcz_attr<float, OpTF32, float, false, true>()));
  FM_CUDA((tcz_attr<float, OpTF32, double, false, false>()));
  FM_CUDA((tcz_attr<float, OpTF32, float, false, false>()));
  FM_CUDA((tcz_attr<float, OpBF16, double, false, false>()));
  FM_CUDA((tcz_attr<float, OpBF16, float, false, false>()));
  FM_CUDA((tcz_attr<uint16_t, OpBF16, double, false, true>()));
  FM_CUDA((tcz_attr<uint16_t, OpBF16, float, false, true>()));
  FM_CUDA(cudaFuncSetAttribute(k_zmix_rb<float, double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024));
  FM_CUDA(cudaFuncSetAttribute(k_zmix_rb<double, float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024));
  FM_CUDA(cudaFuncSetAttribute(k_zmix_rb<float, float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024));
  FM_CUDA(cudaFuncSetAttribute(k_zmix_rb<float, double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024));
  FM_CUDA(cudaFuncSetAttribute(k_zmix_rb<float, float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024));
  return FM_OK;
}

namespace {

// one tensor-core stage: out = W^l . slab for every slab of component cp
int tc_stage(fm_ctx* c, const Comp& cp, const CUtensorMap& mA, const CUtensorMap& mB, int rows, int K, int N,
             bool trans_out, float* out, const float2* dRow, const float2* dCol, int cls) {
  TcArgs a;
  a.rows = rows;
  a.K = K;
  a.N = N;
  a.nb = round16(N);
  a.nkb = (K + 31) / 32;
  a.stages = std::min(4, a.nkb);
  a.ncols = tmem_cols(a.nb);
  a.nz = cp.nz;
  a.trans_out = trans_out ? 1 : 0;
  a.slab_stride = (int64_t)rows * N;
  a.ldo = trans_out ? rows : N;
  a.out = out;
  a.dRow = dRow;
  a.dCol = dCol;
  a.err = c->tc_err;
  const int ns = c->nM * cp.nz;
  dim3 grid((unsigned)((rows + 127) / 128), (unsigned)ns);
  const size_t smem = tc_smem_bytes(a.nb, a.stages, a.ncols);
  const double nun = (double)rows * N * ns;
  const int tk_ = prof_begin(c, cls);
  k_tc_mix<<<grid, kTcThreads, smem, c->stream>>>(mA, mB, a);
  prof_end(c, tk_, 2.0 * K * nun, 8.0 * nun);
  c->launches++;
  FM_CUDA(cudaGetLastError());
  return FM_OK;
}

template <typename TI, typename TO, bool TRANS>
int zstage(fm_ctx* c, const Comp& cp, const float* W, const TI* in, TO* out) {
  const int nz = cp.nz;
  const int64_t nxy = (int64_t)cp.nx * cp.ny;
  const unsigned tiles = TRANS ? (unsigned)(((cp.nx + 7) / 8) * ((cp.ny + 15) / 16)) : (unsigned)((nxy + 127) / 128);
  dim3 grid(tiles, c->nM);
  const size_t smem = ((size_t)nz * 128 + (size_t)nz * 64) * sizeof(float);
  if (smem > 100 * 1024) return FM_ERR_ARG;
  const double ncomp = (double)nxy * nz * c->nM;
  const int tk_ = prof_begin(c, FM_KERNEL_ZMIX);
  k_zmix_rb<TI, TO, TRANS><<<grid, kZThreads, smem, c->stream>>>(W, in, out, nz, cp.nx, cp.ny, cp.off);
  prof_end(c, tk_, 2.0 * nz * ncomp, ncomp * (double)(sizeof(TI) + sizeof(TO)));
  c->launches++;
  FM_CUDA(cudaGetLastError());
  return FM_OK;
}

}  // namespace

// z stages on the tensor cores.  Forward: x -> t[slab][j][i] (BF16 storage when 'to_bf16', ahead of the fused
// BF16 chain).  Inverse: u[slab][j][i] (fused chain, 'in_ji') or t[slab][i][j] (unfused) -> y.
template <typename TI, typename Op, typename TO, bool OUT_JI, bool IN_JI, int NP, int SH>
static int tcz_launch_np(fm_ctx* c, const Comp& cp, const CUtensorMap& tm, const void* in, void* out) {
  TcZArgs a;
  a.in = in;
  a.out = out;
  a.nz = cp.nz;
  a.nx = cp.nx;
  a.ny = cp.ny;
  a.nM = c->nM;
  a.off = cp.off;
  const int TI_ = ZTile<OUT_JI, NP, SH>::TI, TJ_ = ZTile<OUT_JI, NP, SH>::TJ;
  a.tiles_i = (cp.nx + TI_ - 1) / TI_;
  a.tiles_j = (cp.ny + TJ_ - 1) / TJ_;
  a.kblocks = (cp.nz + Op::kRow - 1) / Op::kRow;
  a.ksteps = (cp.nz + Op::kStep - 1) / Op::kStep;
  // a run of four output elements starts at a multiple of 4 of the component's elements when the run
  // dimension (n_x forward, n_y inverse), the component offset and the base address allow it
  a.vec_out = ((OUT_JI ? cp.nx : cp.ny) % 4 == 0) && (cp.off % 4 == 0) &&
              ((uintptr_t)out % (4 * sizeof(TO)) == 0 || ((uintptr_t)out % 16 == 0 && sizeof(TO) == 8));
  a.err = c->tc_err;
  const size_t smem = tcz_smem(a.kblocks, NP);
  // CTAs per SM: shared memory (228 KB per SM, 1 KB reserved per CTA), tensor memory (512 columns), at most 8
  const int per_sm = std::max(1, std::min({8, 512 / NP, (int)(233472 / (smem + 1024))}));
  const int tiles = a.tiles_i * a.tiles_j * c->nM;
  const int grid = std::max(1, std::min(tiles, 152 * per_sm));
  const double nun = (double)cp.nx * cp.ny * cp.nz * c->nM;
  const int tk_ = prof_begin(c, FM_KERNEL_ZMIX);
  k_tc_z<TI, Op, TO, OUT_JI, IN_JI, NP, SH><<<grid, 128, smem, c->stream>>>(tm, a);
  prof_end(c, tk_, 2.0 * cp.nz * nun, nun * (double)(sizeof(TI) + sizeof(TO)));
  c->launches++;
  FM_CUDA(cudaGetLastError());
  return FM_OK;
}

// the component's z-stage tile for this direction: width (points) + 256 * shape, set by the autotuner (or
// the width by fm_opts.z_tile, shape 0)
template <typename TI, typename Op, typename TO, bool OUT_JI, bool IN_JI>
static int tcz_launch(fm_ctx* c, const Comp& cp, const CUtensorMap& tm, const void* in, void* out) {
  switch (cp.tcz_np[OUT_JI ? 0 : 1]) {
    case 32: return tcz_launch_np<TI, Op, TO, OUT_JI, IN_JI, 32, 0>(c, cp, tm, in, out);
    case 64: return tcz_launch_np<TI, Op, TO, OUT_JI, IN_JI, 64, 0>(c, cp, tm, in, out);
    case 256 + 32: return tcz_launch_np<TI, Op, TO, OUT_JI, IN_JI, 32, 1>(c, cp, tm, in, out);
    case 256 + 64: return tcz_launch_np<TI, Op, TO, OUT_JI, IN_JI, 64, 1>(c, cp, tm, in, out);
    case 256 + 128: return tcz_launch_np<TI, Op, TO, OUT_JI, IN_JI, 128, 1>(c, cp, tm, in, out);
    default: return tcz_launch_np<TI, Op, TO, OUT_JI, IN_JI, 128, 0>(c, cp, tm, in, out);
  }
}

bool tc_uses_ydiag(const fm_ctx* c, const Comp& cp) {
  return cp.ydiag_ok && (c->opts.y_solver == 2 || c->opts.y_solver == 0);
}

// the fused x / y chain of every component in 'comps' (one launch): t[slab][j][i] -> u[slab][j][i]
template <typename Op>
static int fused_launch(fm_ctx* c, const std::vector<Comp*>& comps) {
  using TB = typename Op::T;
  if (comps.empty()) return FM_OK;
  if (comps.size() > 3) return FM_ERR_ARG;
  FusedArgs a;
  std::memset(&a, 0, sizeof(a));
  a.ncomp = (int)comps.size();
  a.total = 0;
  int nmax = 16, stages = 4;
  double fl = 0.0, by = 0.0;
  for (size_t q = 0; q < comps.size(); ++q) {
    const Comp& cp = *comps[q];
    FusedComp& f = a.c[q];
    f.tm_in = cp.tmf[0];
    for (int g = 0; g < 4; ++g) f.tm_w[g] = cp.tmf[1 + g];
    f.out = reinterpret_cast<TB*>(c->u32) + cp.off;
    f.dLx2 = cp.dLx2;
    f.dLy2 = cp.dLy2;
    f.nx = cp.nx;
    f.ny = cp.ny;
    f.ns = cp.nz;  // n_M = 1: one slab per z mode
    a.total += f.ns;
    nmax = std::max(nmax, std::max(cp.nx, cp.ny));
    stages = std::min(stages, fused_stages(cp.nx, cp.ny, Op::kRow));
    const double nx = cp.nx, ny = cp.ny, es = (double)sizeof(TB);
    fl += f.ns * 4.0 * nx * ny * (nx + ny);
    by += f.ns * (2.0 * es * nx * ny + 2.0 * es * (nx * nx + ny * ny) + 8.0 * (nx + ny));
  }
  if (stages < 2) return FM_ERR_ARG;
  a.rowsB = round16(nmax);
  a.kbB = (nmax + Op::kRow - 1) / Op::kRow;
  a.stages = stages;
  a.ncols = nmax > 128 ? 512 : 256;
  a.err = c->tc_err;
  const size_t smem = 1024 + (size_t)a.kbB * a.rowsB * 128 + (size_t)stages * 16384 + 256 * 8 + 256;
  const int grid = std::min(a.total, 152);
  const int tk_ = prof_begin(c, FM_KERNEL_XMIX);
  k_tc_fused_xy<Op><<<grid, kFusedThreads, smem, c->stream>>>(a);
  prof_end(c, tk_, fl, by);
  c->launches++;
  FM_CUDA(cudaGetLastError());
  return FM_OK;
}

template <typename TIO>
static int zfwd(fm_ctx* c, Comp& cp, const TIO* x, bool to_bf16) {
  if (!cp.tcz) return zstage<TIO, float, true>(c, cp, cp.Wzb32, x, c->t32);  // t[slab][j][i]
  if (!c->bf16) return tcz_launch<TIO, OpTF32, float, true, false>(c, cp, cp.tmz[0], x, c->t32);
  if (to_bf16) return tcz_launch<TIO, OpBF16, uint16_t, true, false>(c, cp, cp.tmz[0], x, c->t32);
  return tcz_launch<TIO, OpBF16, float, true, false>(c, cp, cp.tmz[0], x, c->t32);
}

// Front half of y = P^{-1} x through the tensor-core chain, all components: z forward, then the x (and, for
// the n_M = 1 y diagonalisation, y) stages -- fused per slab where eligible.  Results: u[slab][j][i] for the
// fused components and for those left to the banded y solves (returned in 'banded', which work in place
// there); t[slab][j][i] ... see the layouts at the top of this file for the unfused diagonalised form.
template <typename TIO>
int precond_tc_front(fm_ctx* c, const TIO* x, std::vector<Comp*>* banded) {
  int rc;
  std::vector<Comp*> fused;
  for (auto& cp : c->comps) {
    const bool ydiag = tc_uses_ydiag(c, cp), fz = ydiag && cp.fused;
    if (!ydiag) banded->push_back(&cp);
    if (fz) fused.push_back(&cp);
    if ((rc = zfwd<TIO>(c, cp, x, fz && c->bf16))) return rc;
  }
  if (c->bf16) rc = fused_launch<OpBF16>(c, fused);
  else rc = fused_launch<OpTF32>(c, fused);
  if (rc) return rc;
  for (auto& cp : c->comps) {
    const bool ydiag = tc_uses_ydiag(c, cp);
    if (ydiag && cp.fused) continue;
    float* t = c->t32 + cp.off;
    float* u = c->u32 + cp.off;
    const int nx = cp.nx, ny = cp.ny;
    // x forward: rows j, K = i -> u[slab][i][j] (ydiag) or u[slab][j][i] (banded y)
    if ((rc = tc_stage(c, cp, cp.tm[0], cp.tm[2], ny, nx, nx, ydiag, u, nullptr, nullptr, FM_KERNEL_XMIX))) return rc;
    if (ydiag) {
      // y forward with the diagonal: rows i, K = j -> t[slab][i][j] / (lambda_x,i + lambda_y,j)
      if ((rc = tc_stage(c, cp, cp.tm[4], cp.tm[6], nx, ny, ny, false, t, cp.dLx2, cp.dLy2, FM_KERNEL_YSOLVE))) return rc;
      // y inverse: rows i, K = j -> u[slab][j][i]
      if ((rc = tc_stage(c, cp, cp.tm[5], cp.tm[7], nx, ny, ny, true, u, nullptr, nullptr, FM_KERNEL_YSOLVE))) return rc;
    }
  }
  return FM_OK;
}

// Back half: x inverse (rows j, K = i -> t[slab][i][j]) of the unfused components and the z inverse of all.
template <typename TIO>
int precond_tc_back(fm_ctx* c, TIO* y) {
  int rc;
  for (auto& cp : c->comps) {
    const bool fz = tc_uses_ydiag(c, cp) && cp.fused;
    const int nx = cp.nx, ny = cp.ny;
    if (fz) {  // u[slab][j][i] from the fused chain
      if (!c->bf16) rc = tcz_launch<float, OpTF32, TIO, false, true>(c, cp, cp.tmz[1], c->u32, y);
      else rc = tcz_launch<uint16_t, OpBF16, TIO, false, true>(c, cp, cp.tmz[1], c->u32, y);
      if (rc) return rc;
      continue;
    }
    float* t = c->t32 + cp.off;
    if ((rc = tc_stage(c, cp, cp.tm[1], cp.tm[3], ny, nx, nx, true, t, nullptr, nullptr, FM_KERNEL_XMIX))) return rc;
    if (!cp.tcz) rc = zstage<float, TIO, false>(c, cp, cp.Wz32, c->t32, y);
    else if (!c->bf16) rc = tcz_launch<float, OpTF32, TIO, false, false>(c, cp, cp.tmz[1], c->t32, y);
    else rc = tcz_launch<float, OpBF16, TIO, false, false>(c, cp, cp.tmz[1], c->t32, y);
    if (rc) return rc;
  }
  return FM_OK;
}

// ---------------------------------------------------------------------------
// Autotuner of the z-stage tile width (128, 64 or 32 points per tensor-core tile).  For each component and
// direction it times every width on the context's own buffers (CUDA events on the context's stream, one
// untimed launch, then the mean of three) and keeps the fastest.  Results are cached per shape (n_x, n_y,
// n_z, n_M, operand type, input / output type, fused or not), so contexts of the same shape -- the request
// loop's, a test's -- reuse them.  fm_opts.z_tile fixes the width instead.
// ---------------------------------------------------------------------------
namespace {
struct TuneKey {
  int nx, ny, nz, nM, bf16, fused, tio, dir;
  bool operator<(const TuneKey& o) const {
    return std::tie(nx, ny, nz, nM, bf16, fused, tio, dir) < std::tie(o.nx, o.ny, o.nz, o.nM, o.bf16, o.fused, o.tio, o.dir);
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, int> g_tune;

template <typename TIO>
int tcz_run(fm_ctx* c, Comp& cp, int dir, const TIO* x, TIO* y) {
  const bool fz = tc_uses_ydiag(c, cp) && cp.fused;
  if (dir == 0) return zfwd<TIO>(c, cp, x, fz && c->bf16);
  if (fz)
    return !c->bf16 ? tcz_launch<float, OpTF32, TIO, false, true>(c, cp, cp.tmz[1], c->u32, y)
                    : tcz_launch<uint16_t, OpBF16, TIO, false, true>(c, cp, cp.tmz[1], c->u32, y);
  return !c->bf16 ? tcz_launch<float, OpTF32, TIO, false, false>(c, cp, cp.tmz[1], c->t32, y)
                  : tcz_launch<float, OpBF16, TIO, false, false>(c, cp, cp.tmz[1], c->t32, y);
}

template <typename TIO>
int tcz_tune_comp(fm_ctx* c, Comp& cp, const TIO* x, TIO* y) {
  cudaEvent_t e0, e1;
  FM_CUDA(cudaEventCreate(&e0));
  FM_CUDA(cudaEventCreate(&e1));
  int rc = FM_OK;
  for (int dir = 0; dir < 2 && rc == FM_OK; ++dir) {
    const TuneKey key{cp.nx, cp.ny, cp.nz, c->nM, c->bf16 ? 1 : 0, (tc_uses_ydiag(c, cp) && cp.fused) ? 1 : 0,
                      (int)sizeof(TIO), dir};
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      auto it = g_tune.find(key);
      if (it != g_tune.end()) {
        cp.tcz_np[dir] = it->second;
        continue;
      }
    }
    // three interleaved rounds of four timed launches per candidate (after one untimed launch each), the
    // best round of each kept: the rounds share the device's state (clocks, L2) evenly among candidates
    constexpr int kCands = 6, kRounds = 3, kReps = 4;
    const int cand[kCands] = {128, 64, 32, 256 + 128, 256 + 64, 256 + 32};
    float tbest[kCands];
    for (int q = 0; q < kCands; ++q) tbest[q] = 1e30f;
    for (int q = 0; q < kCands && rc == FM_OK; ++q) {
      cp.tcz_np[dir] = cand[q];
      rc = tcz_run<TIO>(c, cp, dir, x, y);
    }
    for (int round = 0; round < kRounds && rc == FM_OK; ++round)
      for (int q = 0; q < kCands && rc == FM_OK; ++q) {
        cp.tcz_np[dir] = cand[q];
        if (cudaEventRecord(e0, c->stream) != cudaSuccess) { rc = FM_ERR_CUDA; break; }
        for (int r = 0; r < kReps && rc == FM_OK; ++r) rc = tcz_run<TIO>(c, cp, dir, x, y);
        if (rc) break;
        float ms = 0.f;
        if (cudaEventRecord(e1, c->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
          rc = FM_ERR_CUDA;
          break;
        }
        tbest[q] = std::min(tbest[q], ms / kReps);
      }
    // the default (128 points, first shape) unless another tile is faster by more than 3 %
    int best_np = cand[0];
    float best = tbest[0];
    for (int q = 1; q < kCands; ++q)
      if (tbest[q] < 0.97f * best) {
        best = tbest[q];
        best_np = cand[q];
      }
    if (getenv("FM_VERBOSE"))
      for (int q = 0; q < kCands; ++q)
        fprintf(stderr, "[fm_tune] component %d z %s, %3d-point tiles, shape %d: %.1f us%s\n", cp.label,
                dir ? "inverse" : "forward", cand[q] & 255, cand[q] >> 8, 1e3 * tbest[q],
                cand[q] == best_np ? "  <- chosen" : "");
    cp.tcz_np[dir] = best_np;
    if (rc == FM_OK) {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_tune[key] = best_np;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}
}  // namespace

static int tcz_autotune(fm_ctx* c) {
  const int fixed = c->opts.z_tile;
  bool any = false;
  for (auto& cp : c->comps) {
    cp.tcz_np[0] = cp.tcz_np[1] = fixed ? fixed : 128;
    any = any || cp.tcz;
  }
  if (fixed || !any) return FM_OK;
  // scratch: x and y in the float64 vector u64 (the float32 form in its first half), inputs zeroed
  FM_CUDA(cudaMemsetAsync(c->u64, 0, (size_t)c->N * sizeof(double), c->stream));
  FM_CUDA(cudaMemsetAsync(c->u32, 0, (size_t)c->N * sizeof(float), c->stream));
  FM_CUDA(cudaMemsetAsync(c->t32, 0, (size_t)c->N * sizeof(float), c->stream));
  int rc = FM_OK;
  for (auto& cp : c->comps) {
    if (!cp.tcz) continue;
    if (c->opts.precision == FM_PREC_MIXED) {
      float* v = reinterpret_cast<float*>(c->u64);
      rc = tcz_tune_comp<float>(c, cp, v, v);
    } else {
      rc = tcz_tune_comp<double>(c, cp, c->u64, c->u64);
    }
    if (rc) return rc;
  }
  return tc_check(c);
}

template int precond_tc_front<double>(fm_ctx*, const double*, std::vector<Comp*>*);
template int precond_tc_front<float>(fm_ctx*, const float*, std::vector<Comp*>*);
template int precond_tc_back<double>(fm_ctx*, double*);
template int precond_tc_back<float>(fm_ctx*, float*);

int tc_check(fm_ctx* c) {
  if (!c->tc_active || !c->tc_err) return FM_OK;
  int h = 0;
  FM_CUDA(cudaMemcpyAsync(&h, c->tc_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  FM_CUDA(cudaStreamSynchronize(c->stream));
  return h ? FM_ERR_TIMEOUT : FM_OK;
}

}  // namespace fmi
