// uot_sinkhorn_noalloc: uot_sinkhorn for callers that cannot allocate device
// memory.  The workspace is a fixed file-scope device array compiled into the
// library; this file only finds its device address (once per device) and
// hands it to uot_sinkhorn, which allocates nothing itself.
#include <mutex>

#include <cuda_runtime.h>

#include "uot_internal.h"

namespace {

// Scratch for uot_sinkhorn_noalloc.  In host code `g_noalloc_scratch` names a
// host-side stand-in, not device memory: kernels must be given the address
// from cudaGetSymbolAddress, taken with the device current.
static __device__ __align__(256) unsigned char g_noalloc_scratch[UOT_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the array on the current device, looked up once.
uot_status scratch_on_current_device(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return UOT_ERR_CUDA;
  if (dev >= kMaxDevices) return UOT_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return UOT_ERR_CUDA;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return UOT_OK;
}

}  // namespace

extern "C" uot_status uot_sinkhorn_noalloc(void* plan, int64_t ldp, const float* a,
                                           const float* b, int64_t n, int64_t m, float reg,
                                           float reg_m, int32_t iters, double tol,
                                           const uot_options* opt, void* stream,
                                           uot_result* out) {
  const size_t need = uot_workspace_size(n, m, opt);
  if (need == 0) return UOT_ERR_INVALID_ARG;
  if (need > UOT_STATIC_SCRATCH_BYTES) return UOT_ERR_WORKSPACE;
  void* scratch = nullptr;
  const uot_status st = scratch_on_current_device(&scratch);
  if (st != UOT_OK) return st;
  return uot_sinkhorn(plan, ldp, a, b, n, m, reg, reg_m, iters, tol, scratch,
                      UOT_STATIC_SCRATCH_BYTES, opt, stream, out);
}
