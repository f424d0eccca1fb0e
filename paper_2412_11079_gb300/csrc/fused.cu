// Host side of the fused iteration pass: configuration choice, launch
// geometry (ring depth, CTAs per SM, cluster size) and launches, for both the
// in-place plan and the kernel form.  The kernel itself is in
// fused_kernel.cuh.
#include <cuda_runtime.h>

#include <mutex>

#include "fused_kernel.cuh"

namespace uot {

namespace {

const FusedEntry* table(bool kf) { return kf ? kKformTable : kInplaceTable; }

size_t elem_size(int dtype) { return dtype == UOT_F32 ? 4 : 2; }

size_t smem_bytes(const FusedConfig& c, int stages) {
  const size_t row = size_t(c.cols) * elem_size(c.dtype);
  const size_t red = 2 * MAX_CLUSTER * (c.threads / 32) * sizeof(float);
  const size_t slots = size_t(stages > 0 ? stages : 1);
  return size_t(stages) * row + red + slots * 8 + slots * 4 + 2 * sizeof(float);
}

// cudaFuncSetAttribute is set once per (device, kernel) and the launch
// geometry is cached per (device, form, config, cluster, rows): neither
// needs to be recomputed for each of the hundreds of passes of a solve.
constexpr int MAX_DEV = 64;
std::mutex g_mu;
size_t g_smem_set[MAX_DEV][2][kFusedConfigs][2];
bool g_cluster_set[MAX_DEV][2][kFusedConfigs][2];

struct GeoKey {
  int dev, kf, k, cs, n;
  bool operator==(const GeoKey& o) const {
    return dev == o.dev && kf == o.kf && k == o.k && cs == o.cs && n == o.n;
  }
};
struct GeoVal {
  int grid, stages;
  size_t smem;
};
constexpr int GEO_CACHE = 64;
GeoKey g_geo_key[GEO_CACHE];
GeoVal g_geo_val[GEO_CACHE];
int g_geo_used = 0, g_geo_next = 0;

cudaError_t ensure_attributes(int dev, bool kf, int k, bool tma, size_t smem, bool cluster) {
  if (dev < 0 || dev >= MAX_DEV) return cudaErrorInvalidDevice;
  const FusedEntry& e = table(kf)[k];
  const void* fn = tma ? e.fn_tma : e.fn_plain;
  std::lock_guard<std::mutex> lock(g_mu);
  if (g_smem_set[dev][kf][k][tma] < smem) {
    cudaError_t err =
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (err != cudaSuccess) return err;
    g_smem_set[dev][kf][k][tma] = smem;
  }
  if (cluster && !g_cluster_set[dev][kf][k][tma]) {
    cudaError_t err = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (err != cudaSuccess) return err;
    g_cluster_set[dev][kf][k][tma] = true;
  }
  return cudaSuccess;
}

}  // namespace

int fused_num_configs() { return kFusedConfigs; }

bool fused_config_info(int k, FusedConfig* out) {
  if (k < 0 || k >= kFusedConfigs) return false;
  *out = kInplaceTable[k].cfg;
  return true;
}

int fused_pick(int dtype, int64_t m, int tile) {
  if (tile > 0) {
    const int k = tile - 1;
    if (k >= kFusedConfigs || kInplaceTable[k].cfg.dtype != dtype) return -1;
    return k;
  }
  // Smallest CTA width that covers the row; otherwise the widest, split over
  // a cluster.
  int best = -1, widest = -1;
  for (int k = 0; k < kFusedConfigs; ++k) {
    const FusedConfig& c = kInplaceTable[k].cfg;
    if (c.dtype != dtype) continue;
    if (widest < 0 || c.cols > kInplaceTable[widest].cfg.cols) widest = k;
    if (c.cols >= m && (best < 0 || c.cols < kInplaceTable[best].cfg.cols)) best = k;
  }
  return best >= 0 ? best : widest;
}

cudaError_t fused_geometry(bool kf, int k, int cs, int n, int* grid, int* stages, size_t* smem) {
  const FusedEntry& e = table(kf)[k];
  int dev = 0, sms = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  const GeoKey key{dev, kf ? 1 : 0, k, cs, n};
  {
    std::lock_guard<std::mutex> lock(g_mu);
    for (int i = 0; i < g_geo_used; ++i)
      if (g_geo_key[i] == key) {
        *grid = g_geo_val[i].grid;
        *stages = g_geo_val[i].stages;
        *smem = g_geo_val[i].smem;
        return cudaSuccess;
      }
  }
  err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (err != cudaSuccess) return err;
  int optin = 0;
  err = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (err != cudaSuccess) return err;
  // Deepest ring that keeps the CTA count per SM of a two-slot ring.
  int occ2 = 0, best_s = 2;
  for (int s = 2; s <= 8; ++s) {
    const size_t b = smem_bytes(e.cfg, s);
    if (b > size_t(optin)) break;
    err = ensure_attributes(dev, kf, k, true, b, false);
    if (err != cudaSuccess) return err;
    int occ = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, e.fn_tma, e.cfg.threads, b);
    if (err != cudaSuccess) return err;
    if (s == 2) occ2 = occ;
    if (occ < occ2 || occ == 0) break;
    best_s = s;
  }
  if (occ2 == 0) return cudaErrorInvalidConfiguration;
  *stages = best_s;
  *smem = smem_bytes(e.cfg, best_s);
  int clusters = occ2 * sms;
  if (cs > 1) {
    err = ensure_attributes(dev, kf, k, true, *smem, true);
    if (err != cudaSuccess) return err;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(cs * occ2 * sms, 1, 1);
    cfg.blockDim = dim3(e.cfg.threads, 1, 1);
    cfg.dynamicSmemBytes = *smem;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nc = 0;
    err = cudaOccupancyMaxActiveClusters(&nc, e.fn_tma, &cfg);
    if (err != cudaSuccess) return err;
    if (nc <= 0) return cudaErrorInvalidConfiguration;
    clusters = nc;
  }
  // Keep at least two rows per cluster so the column flush stays small
  // (fewer, longer-lived CTAs measured slower for short rows: with one row in
  // flight per CTA, more CTAs per SM hide the per-row latency).
  const int cap = (n + 1) / 2;
  if (clusters > cap) clusters = cap > 0 ? cap : 1;
  *grid = clusters * cs;
  err = ensure_attributes(dev, kf, k, false, smem_bytes(e.cfg, 0), cs > 1);
  if (err != cudaSuccess) return err;
  err = ensure_attributes(dev, kf, k, true, *smem, cs > 1);
  if (err != cudaSuccess) return err;
  std::lock_guard<std::mutex> lock(g_mu);
  const int slot = g_geo_used < GEO_CACHE ? g_geo_used++ : (g_geo_next++ % GEO_CACHE);
  g_geo_key[slot] = key;
  g_geo_val[slot] = GeoVal{*grid, *stages, *smem};
  return cudaSuccess;
}

// Deterministic mode, after a pass: column j's sum of iteration t is the
// slots' partials added in slot order (each of the 8 warps of a CTA adds
// every 8th slot for 32 columns, then one warp adds the 8 results in warp
// order), so it does not depend on which CTA finished first.  The next
// factors follow as in the end-of-pass job of the pass kernel.  A pass that
// found the stopping rule already met leaves everything as it is.
constexpr int DR_WARPS = 8;

template <bool KF>
__global__ void __launch_bounds__(DR_WARPS * 32) det_reduce_kernel(const FusedArgs p,
                                                                   int groups) {
  __shared__ float part[DR_WARPS][32];
  if (p.track && *reinterpret_cast<volatile int32_t*>(&p.ctl->done)) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j = blockIdx.x * 32 + lane;
  float s = 0.0f;
  if (j < p.m)
    for (int g = warp; g < groups; g += DR_WARPS) s += __ldcg(p.part + size_t(g) * p.mpad + j);
  part[warp][lane] = s;
  __syncthreads();
  uint32_t st = 0;
  if (warp == 0 && j < p.m) {
    float c = 0.0f;
#pragma unroll
    for (int w = 0; w < DR_WARPS; ++w) c += part[w][lane];
    p.c_next[j] = c;
    if constexpr (KF) {
      const float inv_gauge = ldexpf(1.0f, -gauge_exponent(p.t, float(*p.log2k)));
      const float v = p.beta_out[j];
      const float cc = v * c * inv_gauge;
      const float v_new = p.pot ? rescale_factor(p.b_ws[j], c, p.fi, st)
                                : v * rescale_factor(p.b_ws[j], cc, p.fi, st) * inv_gauge;
      p.beta_out[j] = v_new;
      if (p.save_c) {
        p.save_c[j] = cc;
        p.save_V[j] = v_new;
      }
    } else {
      p.beta_out[j] = rescale_factor(p.b_ws[j], c, p.fi, st);
    }
  }
  if (p.track && blockIdx.x == 0 && threadIdx.x == 0) {
    double num = 0.0, den = 0.0;
    for (int g = 0; g < groups; ++g) {
      num += p.err_part[2 * g];
      den += p.err_part[2 * g + 1];
    }
    p.err_next[0] = num;
    p.err_next[1] = den;
  }
  if (st) atomicOr(&p.ctl->status, st);
}

cudaError_t det_reduce_launch(bool kf, int groups, const FusedArgs& args, cudaStream_t s) {
  const int blocks = (args.m + 31) / 32;
  if (kf)
    det_reduce_kernel<true><<<blocks, DR_WARPS * 32, 0, s>>>(args, groups);
  else
    det_reduce_kernel<false><<<blocks, DR_WARPS * 32, 0, s>>>(args, groups);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) count_launch();
  return e;
}

cudaError_t fused_launch(bool kf, int k, int cs, int grid, size_t smem, bool tma,
                         const FusedArgs& args, cudaStream_t s) {
  const FusedEntry& e = table(kf)[k];
  const void* fn = tma ? e.fn_tma : e.fn_plain;
  const size_t bytes = tma ? smem : smem_bytes(e.cfg, 0);
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(grid, 1, 1);
  cfg.blockDim = dim3(e.cfg.threads, 1, 1);
  cfg.dynamicSmemBytes = bytes;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = cs > 1 ? 1 : 0;
  FusedArgs a = args;
  void* kargs[] = {&a};
  cudaError_t err = cudaLaunchKernelExC(&cfg, fn, kargs);
  if (err == cudaSuccess) count_launch();
  return err;
}

}  // namespace uot
