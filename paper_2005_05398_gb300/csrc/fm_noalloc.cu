// fm_apply_noalloc: the operator apply y = (H - E S) x with its three scratch planes taken from
// a fixed device array of this file instead of the context's own buffers.  The call performs no
// device allocation of any kind (no cudaMalloc / cudaFree, no allocating library routine).
//
// The array below is part of the library image: every GPU on which the library is loaded holds
// FM_NOALLOC_MAX_UNKNOWNS * 3 doubles (24 MiB) for it until the process exits.  Host code may not
// use the array's name as a device address (in host code it names a host-side stand-in), so the
// device address is obtained once per device with cudaGetSymbolAddress, with that device current.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "fm_internal.h"

namespace {

static __device__ __align__(256) double g_apply_scratch[3 * (size_t)FM_NOALLOC_MAX_UNKNOWNS];

constexpr int kMaxDevices = 64;
struct ScratchSlot {
  CUcontext ctx = nullptr;   // the context the address was looked up in
  double* addr = nullptr;
};
ScratchSlot g_scratch[kMaxDevices];
std::mutex g_scratch_mu;

using CtxGetCurrentFn = CUresult (*)(CUcontext*);

CtxGetCurrentFn ctx_get_current() {
  static std::once_flag once;
  static CtxGetCurrentFn fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<CtxGetCurrentFn>(p);
  });
  return fn;
}

// Device address of the scratch array in the current context of `device` (current on entry).  The
// address belongs to the module instance of that context: after a cudaDeviceReset, or when the primary
// context was released and made again, the context differs and the address is looked up anew.
int scratch_address(int device, double** out) {
  if (device < 0 || device >= kMaxDevices) return FM_ERR_ARG;
  CtxGetCurrentFn get = ctx_get_current();
  CUcontext cur = nullptr;
  if (!get || get(&cur) != CUDA_SUCCESS || !cur) return FM_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  ScratchSlot& slot = g_scratch[device];
  if (!slot.addr || slot.ctx != cur) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_apply_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      slot = ScratchSlot{};
      return FM_ERR_CUDA;
    }
    slot.ctx = cur;
    slot.addr = static_cast<double*>(p);
  }
  *out = slot.addr;
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
