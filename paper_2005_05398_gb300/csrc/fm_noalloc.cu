// fm_apply_noalloc: the operator apply y = (H - E S) x with its three scratch planes taken from
// a fixed device array of this file instead of the context's own buffers.  The call performs no
// device allocation of any kind (no cudaMalloc / cudaFree, no allocating library routine).
//
// The array below is part of the library image: every GPU on which the library is loaded holds
// FM_NOALLOC_MAX_UNKNOWNS * 3 doubles (24 MiB) for it until the process exits.  Host code may not
// use the array's name as a device address (in host code it names a host-side stand-in), so the
// device address is obtained once per device with cudaGetSymbolAddress, with that device current.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "fm_internal.h"

namespace {

static __device__ __align__(256) double g_apply_scratch[3 * (size_t)FM_NOALLOC_MAX_UNKNOWNS];

constexpr int kMaxDevices = 64;
double* g_scratch_dev[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

// Device address of the scratch array on the current device (looked up on first use).
int scratch_address(int device, double** out) {
  if (device < 0 || device >= kMaxDevices) return FM_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_dev[device]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_apply_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return FM_ERR_CUDA;
    }
    g_scratch_dev[device] = static_cast<double*>(p);
  }
  *out = g_scratch_dev[device];
  return FM_OK;
}

}  // namespace

extern "C" int fm_apply_noalloc(fm_ctx* ctx, double E, const double* x, double* y) {
  if (!ctx || !x || !y || x == y || !std::isfinite(E)) return FM_ERR_ARG;
  if (ctx->N > (int64_t)FM_NOALLOC_MAX_UNKNOWNS) return FM_ERR_SCRATCH_LIMIT;
  FM_CUDA(cudaSetDevice(ctx->device));
  double* s = nullptr;
  const int rc = scratch_address(ctx->device, &s);
  if (rc != FM_OK) return rc;
  const int64_t N = ctx->N;
  // every scratch element the kernels read is written earlier in the same call, so the contents
  // left by a previous call need no clearing
  return fmi::launch_apply_scratch(ctx, E, x, y, s, s + N, s + 2 * N);
}
