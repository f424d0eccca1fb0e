// The three-way form of the iteration (the paper notes that the method
// applies to higher-dimensional tensors): a plan P of n1 x n2 x n3 entries
// with targets a, b, c; every iteration rescales along mode 1, then mode 2,
// then mode 3 by (target / marginal sum)^fi.
//
// One sweep per iteration, as Algorithm 1 does for the matrix.  Slice
// P[i, :, :] is a row of the mode-1 unfolding (n1 rows of n2 * n3 entries,
// column index j n3 + k), so the fused pass of the matrix iteration applies
// the pending mode-2 and mode-3 factors of iteration t-1 (beta_j gamma_k, one
// factor per unfolded column), forms the slice sum and alpha_i, rescales the
// slice and accumulates the unfolded column sums
//     M_jk = sum_i alpha_i x_ijk          (the mode-1-scaled plan over i).
// The rest of the iteration needs only M (n2 x n3, small next to the plan):
//     mode-2 sums   s2_j = sum_k M_jk,            beta_j  = (b_j / s2_j)^fi
//     mode-3 sums   s3_k = sum_j beta_j M_jk,     gamma_k = (c_k / s3_k)^fi
// (the mode-3 sums of the plan after its mode-2 step), and beta_j gamma_k is
// pending for the next pass; a last sweep applies it after the final pass.
#include <algorithm>
#include <cmath>

#include <cuda_runtime.h>

#include "uot_device.cuh"
#include "uot_internal.h"

namespace uot {

namespace {

constexpr int TB = 256;

struct Tensor3Layout {
  WsLayout L;        // of the n1 x (n2 n3) unfolding
  size_t beta2, gamma3, total;
};

Tensor3Layout tensor3_layout(int64_t n1, int64_t n2, int64_t n3) {
  Tensor3Layout T{};
  T.L = ws_layout(n1, n2 * n3);
  size_t off = T.L.total;
  T.beta2 = off; off = align256(off + size_t(n2) * 4);
  T.gamma3 = off; off = align256(off + size_t(n3) * 4);
  T.total = off;
  return T;
}

// beta_j = (b_j / sum_k M_jk)^fi, one warp per j.
__global__ void __launch_bounds__(TB) mode2_kernel(const float* M, int n2, int n3, const float* b,
                                                   float fi, float* beta, Control* ctl) {
  const int lane = threadIdx.x & 31;
  const int nw = gridDim.x * (TB / 32);
  uint32_t st = 0;
  for (int j = blockIdx.x * (TB / 32) + (threadIdx.x >> 5); j < n2; j += nw) {
    float s = 0.0f;
    for (int k = lane; k < n3; k += 32) s += M[size_t(j) * n3 + k];
    s = warp_sum(s);
    if (lane == 0) beta[j] = rescale_factor(b[j], s, fi, st);
  }
  if (st) atomicOr(&ctl->status, st);
}

// gamma_k = (c_k / sum_j beta_j M_jk)^fi and the pending factor
// beta_j gamma_k of every unfolded column for the next pass.  A CTA takes 32
// values of k (one per lane); its 32 warps add every 32nd j (a short chain
// of loads per warp: there are only n3 / 32 CTAs), and one warp adds the
// partial sums in warp order; then every warp writes 32 consecutive pending
// factors per row j.
constexpr int M3_THREADS = 1024;
constexpr int M3_WARPS = M3_THREADS / 32;

__global__ void __launch_bounds__(M3_THREADS) mode3_kernel(const float* M, int n2, int n3, const float* c,
                                                   float fi, const float* beta, float* gamma,
                                                   float* pending, Control* ctl, int t) {
  __shared__ float part[M3_WARPS][32];
  __shared__ float g_s[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int k = blockIdx.x * 32 + lane;
  if (blockIdx.x == 0 && threadIdx.x == 0) ctl->iters_done = t;
  float s = 0.0f;
  if (k < n3)
    for (int j = warp; j < n2; j += M3_WARPS) s = fmaf(beta[j], M[size_t(j) * n3 + k], s);
  part[warp][lane] = s;
  __syncthreads();
  if (warp == 0) {
    float tot = 0.0f;
#pragma unroll
    for (int w = 0; w < M3_WARPS; ++w) tot += part[w][lane];
    uint32_t st = 0;
    const float g = k < n3 ? rescale_factor(c[k], tot, fi, st) : 0.0f;
    if (k < n3) gamma[k] = g;
    g_s[lane] = g;
    if (st) atomicOr(&ctl->status, st);
  }
  __syncthreads();
  if (k < n3) {
    const float g = g_s[lane];
    for (int j = warp; j < n2; j += M3_WARPS) pending[size_t(j) * n3 + k] = beta[j] * g;
  }
}

}  // namespace

}  // namespace uot

using namespace uot;

extern "C" {

size_t uot_tensor3_workspace_size(int64_t n1, int64_t n2, int64_t n3) {
  if (n1 < 1 || n2 < 1 || n3 < 1 || n1 > (int64_t(1) << 30) || n2 > (int64_t(1) << 30) ||
      n3 > (int64_t(1) << 30) || n2 * n3 > (int64_t(1) << 30))
    return 0;
  return tensor3_layout(n1, n2, n3).total;
}

uot_status uot_sinkhorn_tensor3(void* P, int64_t n1, int64_t n2, int64_t n3, const float* a,
                                const float* b, const float* c, float reg, float reg_m,
                                int32_t iters, void* workspace, size_t ws_bytes,
                                const uot_options* opt, void* stream, uot_result* out) {
  uot_options o;
  uot_default_options(&o);
  if (opt) o = *opt;
  const size_t need = uot_tensor3_workspace_size(n1, n2, n3);
  if (!P || !a || !b || !c || need == 0 || iters < 0) return UOT_ERR_INVALID_ARG;
  if (o.dtype != UOT_F32 && o.dtype != UOT_BF16 && o.dtype != UOT_F16) return UOT_ERR_INVALID_ARG;
  if (!(reg > 0.0f) || !std::isfinite(reg) || !(reg_m > 0.0f) || o.reserved[0] != 0)
    return UOT_ERR_INVALID_ARG;
  if (o.cluster < 0 || o.cluster > 8 || o.tile < 0 || o.max_ctas < 0) return UOT_ERR_INVALID_ARG;
  if (o.algo != UOT_ALGO_FUSED || o.storage != UOT_STORAGE_INPLACE || o.deterministic ||
      o.rule != UOT_RULE_PAPER || o.schedule == UOT_SCHED_PERSISTENT)
    return UOT_ERR_UNSUPPORTED;
  const size_t es = o.dtype == UOT_F32 ? 4 : 2;
  if (reinterpret_cast<uintptr_t>(P) % es || reinterpret_cast<uintptr_t>(a) % 4 ||
      reinterpret_cast<uintptr_t>(b) % 4 || reinterpret_cast<uintptr_t>(c) % 4)
    return UOT_ERR_INVALID_ARG;
  if (!workspace || ws_bytes < need || reinterpret_cast<uintptr_t>(workspace) % 256)
    return UOT_ERR_WORKSPACE;
  const Tensor3Layout TL = tensor3_layout(n1, n2, n3);
  const WsLayout& L = TL.L;
  const int N = int(n1), M = int(n2 * n3), N2 = int(n2), N3 = int(n3);
  const int64_t ld = n2 * n3;
  int k = -1, cs = 1, grid = 0, stages = 0;
  size_t smem = 0;
  if (iters > 0) {
    k = fused_pick(o.dtype, M, o.tile);
    if (k < 0) return UOT_ERR_INVALID_ARG;
    FusedConfig cfg;
    fused_config_info(k, &cfg);
    cs = o.cluster > 0 ? o.cluster : int((M + cfg.cols - 1) / cfg.cols);
    if (cs > 8) return UOT_ERR_UNSUPPORTED;
    if (int64_t(cs) * cfg.cols < M) return UOT_ERR_INVALID_ARG;
    if (fused_geometry(false, k, cs, N, &grid, &stages, &smem) != cudaSuccess) return UOT_ERR_CUDA;
    if (o.max_ctas > 0 && grid > o.max_ctas) grid = std::max(cs, (o.max_ctas / cs) * cs);
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint8_t* ws = static_cast<uint8_t*>(workspace);
  const double fi_d = std::isinf(reg_m) ? 1.0 : double(reg_m) / (double(reg_m) + double(reg));
  const float fi = float(fi_d);
  // b of the unfolding is not used (the mode factors are formed here).
  if (launch_reset(ws, L, nullptr, M, s) != cudaSuccess) return UOT_ERR_CUDA;
  Control* ctl = reinterpret_cast<Control*>(ws + L.ctl);
  float* beta2 = reinterpret_cast<float*>(ws + TL.beta2);
  float* gamma3 = reinterpret_cast<float*>(ws + TL.gamma3);
  float* pending = reinterpret_cast<float*>(ws + L.beta);
  cudaEvent_t ev0 = static_cast<cudaEvent_t>(o.pass_events[0]);
  cudaEvent_t ev1 = static_cast<cudaEvent_t>(o.pass_events[1]);
  if (ev0 && cudaEventRecord(ev0, s) != cudaSuccess) return UOT_ERR_CUDA;
  if (iters > 0) {
    const bool tma = reinterpret_cast<uintptr_t>(P) % 16 == 0 && (uint64_t(ld) * es) % 16 == 0;
    FusedArgs A{};
    A.plan = P;
    A.ldp = ld;
    A.n = N;
    A.m = M;
    A.a = a;
    A.fi = fi;
    A.mpad = int(L.mpad);
    A.r_prev = reinterpret_cast<float*>(ws + L.r);
    A.ctl = ctl;
    A.stages = stages;
    A.b_ws = reinterpret_cast<const float*>(ws + L.bws);
    A.dynamic = 1;
    A.beta = pending;
    A.beta_out = pending;
    A.no_factors = 1;
    int* ctr = reinterpret_cast<int*>(ws + L.ctr);
    const int g2 = std::max(1, std::min((N2 + TB / 32 - 1) / (TB / 32), 1024));
    const int g3 = (N3 + 31) / 32;
    for (int t = 1; t <= iters; ++t) {
      float* cnext = reinterpret_cast<float*>(ws + L.c[t % 3]);
      A.t = t;
      A.first = t == 1;
      A.c_prev = reinterpret_cast<float*>(ws + L.c[(t - 1) % 3]);
      A.c_next = cnext;
      A.c_clear = reinterpret_cast<float*>(ws + L.c[(t + 1) % 3]);
      A.row_ctr = ctr + t % 3;
      A.ctr_clear = ctr + (t + 1) % 3;
      A.arrive = ctr + 3 + t % 3;
      A.arrive_clear = ctr + 3 + (t + 1) % 3;
      A.slice_ctr = ctr + 6 + t % 3;
      A.slice_clear = ctr + 6 + (t + 1) % 3;
      if (fused_launch(false, k, cs, grid, smem, tma, A, s) != cudaSuccess) return UOT_ERR_CUDA;
      mode2_kernel<<<g2, TB, 0, s>>>(cnext, N2, N3, b, fi, beta2, ctl);
      if (cudaGetLastError() != cudaSuccess) return UOT_ERR_CUDA;
      mode3_kernel<<<g3, M3_THREADS, 0, s>>>(cnext, N2, N3, c, fi, beta2, gamma3, pending, ctl, t);
      if (cudaGetLastError() != cudaSuccess) return UOT_ERR_CUDA;
      count_launch(2);
    }
    if (ev1 && cudaEventRecord(ev1, s) != cudaSuccess) return UOT_ERR_CUDA;
    if (launch_scale_cols(P, ld, N, M, o.dtype, pending, s) != cudaSuccess) return UOT_ERR_CUDA;
  } else if (ev1 && cudaEventRecord(ev1, s) != cudaSuccess) {
    return UOT_ERR_CUDA;
  }
  if (!out) return UOT_OK;
  return uot_read_result(workspace, n1, n2 * n3, &o, stream, out);
}

}  // extern "C"
