// uot_sinkhorn_noalloc: uot_sinkhorn for callers that cannot allocate device
// memory.  The workspace is a fixed file-scope device array compiled into the
// library; this file only finds its device address (once per CUDA context)
// and hands it to uot_sinkhorn, which allocates nothing itself.
#include <mutex>

#include <cuda.h>
#include <cuda_runtime.h>

#include "uot_internal.h"

namespace {

// Scratch for uot_sinkhorn_noalloc.  In host code `g_noalloc_scratch` names a
// host-side stand-in, not device memory: kernels must be given the address
// from cudaGetSymbolAddress, taken with the device current.
static __device__ __align__(256) unsigned char g_noalloc_scratch[UOT_STATIC_SCRATCH_BYTES];

// The address belongs to the copy of the module loaded in the current CUDA
// context, so it is cached per context (by the driver's unique context id):
// after cudaDeviceReset, or in a context the host application created, the
// id changes and the address is looked up again.  The two driver calls are
// fetched through the runtime, so the library does not link libcuda.
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

constexpr int kMaxContexts = 64;
struct CacheEntry {
  unsigned long long ctx_id;
  void* ptr;
};
std::mutex g_mu;
CacheEntry g_cache[kMaxContexts];
int g_used = 0, g_next = 0;
CtxGetCurrentFn g_get_current = nullptr;
CtxGetIdFn g_get_id = nullptr;

bool resolve_driver_calls() {
  if (g_get_current && g_get_id) return true;
  void* f0 = nullptr;
  void* f1 = nullptr;
  cudaDriverEntryPointQueryResult q0 = cudaDriverEntryPointSymbolNotFound, q1 = q0;
  if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f0, 12000, cudaEnableDefault, &q0) !=
          cudaSuccess ||
      cudaGetDriverEntryPointByVersion("cuCtxGetId", &f1, 12000, cudaEnableDefault, &q1) !=
          cudaSuccess ||
      q0 != cudaDriverEntryPointSuccess || q1 != cudaDriverEntryPointSuccess || !f0 || !f1)
    return false;
  g_get_current = reinterpret_cast<CtxGetCurrentFn>(f0);
  g_get_id = reinterpret_cast<CtxGetIdFn>(f1);
  return true;
}

// Id of the context current on this thread; false if there is none yet.
bool current_context_id(unsigned long long* id) {
  CUcontext ctx = nullptr;
  if (g_get_current(&ctx) != CUDA_SUCCESS || !ctx) return false;
  return g_get_id(ctx, id) == CUDA_SUCCESS;
}

// Device address of the array in the current context.
uot_status scratch_in_current_context(void** out) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (!resolve_driver_calls()) return UOT_ERR_CUDA;
  unsigned long long id = 0;
  if (current_context_id(&id)) {
    for (int i = 0; i < g_used; ++i)
      if (g_cache[i].ctx_id == id) {
        *out = g_cache[i].ptr;
        return UOT_OK;
      }
  }
  // Miss (or no context current on this thread yet): the runtime call makes
  // the device's primary context current if needed and loads the module.
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return UOT_ERR_CUDA;
  if (!current_context_id(&id)) return UOT_ERR_CUDA;
  const int slot = g_used < kMaxContexts ? g_used++ : (g_next++ % kMaxContexts);
  g_cache[slot] = CacheEntry{id, p};
  *out = p;
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
  const uot_status st = scratch_in_current_context(&scratch);
  if (st != UOT_OK) return st;
  return uot_sinkhorn(plan, ldp, a, b, n, m, reg, reg_m, iters, tol, scratch,
                      UOT_STATIC_SCRATCH_BYTES, opt, stream, out);
}
