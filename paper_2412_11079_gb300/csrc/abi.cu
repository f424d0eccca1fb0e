// The extern "C" entry points of libuot (declared in include/uot.h): argument
// validation on the host, workspace layout, and the per-iteration launch
// sequence of the Sinkhorn-UOT iteration (Section 2.1 / Algorithm 1).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>

#include <cuda_runtime.h>

#include "uot_internal.h"

namespace uot {

static std::atomic<uint64_t> g_launches{0};
void count_launch(int k) { g_launches.fetch_add(uint64_t(k), std::memory_order_relaxed); }

static size_t esize(int dtype) { return dtype == UOT_F32 ? 4 : 2; }

static bool valid_dtype(int d) { return d == UOT_F32 || d == UOT_BF16 || d == UOT_F16; }

// Row and column indices and the per-pass row counters (which may run a few
// ring depths per CTA past n) are 32-bit in the kernels.
static bool valid_dims(int64_t n, int64_t m) {
  return n >= 1 && m >= 1 && n <= (int64_t(1) << 30) && m <= (int64_t(1) << 30);
}

static uot_options resolve(const uot_options* opt) {
  uot_options o;
  uot_default_options(&o);
  if (opt) o = *opt;
  if (o.check_every <= 0) o.check_every = 1;
  return o;
}

static bool reserved_zero(const uot_options& o) {
  for (int k = 0; k < 1; ++k)
    if (o.reserved[k] != 0) return false;
  return true;
}

static uot_status status_of(uint32_t dev) {
  if (dev & UOT_DEV_TIMEOUT) return UOT_ERR_TIMEOUT;
  if (dev & UOT_DEV_NONFINITE) return UOT_ERR_NONFINITE;
  if (dev & UOT_DEV_ZERO_SUM) return UOT_ERR_ZERO_SUM;
  return UOT_OK;
}

}  // namespace uot

using namespace uot;

extern "C" {

void uot_default_options(uot_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->dtype = UOT_F32;
  opt->algo = UOT_ALGO_FUSED;
  opt->check_every = 1;
}

const char* uot_status_string(uot_status s) {
  switch (s) {
    case UOT_OK: return "ok";
    case UOT_ERR_INVALID_ARG: return "invalid argument";
    case UOT_ERR_CUDA: return "CUDA error";
    case UOT_ERR_NONFINITE: return "non-finite sum or factor on the device";
    case UOT_ERR_ZERO_SUM: return "zero sum with a positive target on the device";
    case UOT_ERR_TIMEOUT: return "bounded device wait timed out";
    case UOT_ERR_UNSUPPORTED: return "unsupported configuration";
    case UOT_ERR_WORKSPACE: return "workspace missing, too small or misaligned";
  }
  return "unknown status";
}

size_t uot_workspace_size(int64_t n, int64_t m, const uot_options* opt) {
  if (!valid_dims(n, m)) return 0;
  return ws_layout(n, m, opt && opt->deterministic != 0).total;
}

uint64_t uot_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

uot_status uot_selftest_wait(const int32_t* counter_dev, int32_t target, int32_t complete,
                             double limit_s, uint32_t* status_dev, void* stream) {
  if (!counter_dev || !status_dev || !(limit_s > 0.0) || !(limit_s <= 10.0))
    return UOT_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(counter_dev) % 4 || reinterpret_cast<uintptr_t>(status_dev) % 4)
    return UOT_ERR_INVALID_ARG;
  const uint64_t limit_ns = uint64_t(limit_s * 1e9);
  cudaError_t e = launch_wait_selftest(counter_dev, target, complete ? 1 : 0, limit_ns, status_dev,
                                       static_cast<cudaStream_t>(stream));
  if (e == cudaSuccess) count_launch();
  return e == cudaSuccess ? UOT_OK : UOT_ERR_CUDA;
}

uot_status uot_selftest_factor(const float* target, const float* total, int64_t count, float fi,
                               float* out, uint32_t* status_dev, void* stream) {
  if (!target || !total || !out || !status_dev || count < 1 || count > (int64_t(1) << 30))
    return UOT_ERR_INVALID_ARG;
  if (!(fi > 0.0f) || !(fi <= 1.0f)) return UOT_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(target) % 4 || reinterpret_cast<uintptr_t>(total) % 4 ||
      reinterpret_cast<uintptr_t>(out) % 4 || reinterpret_cast<uintptr_t>(status_dev) % 4)
    return UOT_ERR_INVALID_ARG;
  cudaError_t e = launch_factor_selftest(target, total, count, fi, out, status_dev,
                                         static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? UOT_OK : UOT_ERR_CUDA;
}

uot_status uot_init_kernel(const float* C, int64_t ldc, void* plan, int64_t ldp, int64_t n,
                           int64_t m, float reg, const uot_options* opt, void* stream) {
  const uot_options o = resolve(opt);
  if (!C || !plan || !valid_dims(n, m) || ldc < m || ldp < m || !valid_dtype(o.dtype))
    return UOT_ERR_INVALID_ARG;
  if (!(reg > 0.0f) || !std::isfinite(reg)) return UOT_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(plan) % esize(o.dtype) || reinterpret_cast<uintptr_t>(C) % 4)
    return UOT_ERR_INVALID_ARG;
  cudaError_t e = launch_init(C, ldc, plan, ldp, int(n), int(m), reg, o.dtype, 1.0f,
                              static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? UOT_OK : UOT_ERR_CUDA;
}

uot_status uot_read_result(const void* workspace, int64_t n, int64_t m, const uot_options* opt,
                           void* stream, uot_result* out) {
  (void)opt;
  if (!workspace || !out || !valid_dims(n, m)) return UOT_ERR_INVALID_ARG;
  const WsLayout L = ws_layout(n, m);
  Control ctl;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(&ctl, static_cast<const uint8_t*>(workspace) + L.ctl, sizeof(ctl),
                      cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return UOT_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return UOT_ERR_CUDA;
  out->iters_done = ctl.iters_done;
  out->dev_status = ctl.status;
  out->err = ctl.err;
  return status_of(ctl.status);
}

}  // extern "C"

namespace uot {

// Validation, geometry and the launch sequence shared by the in-place plan
// (kf == false; `mat` is the plan) and the kernel form (kf == true; `mat` is
// K, read-only, and U / V receive the scalings).
static uot_status run_sinkhorn(bool kf, void* mat, int64_t ldm, const float* a, const float* b,
                               int64_t n, int64_t m, float reg, float reg_m, int32_t iters,
                               double tol, float k_log2_scale, float* U, float* V,
                               void* workspace, size_t ws_bytes, const uot_options* opt,
                               void* stream, uot_result* out, void* hist = nullptr,
                               size_t hist_bytes = 0) {
  const uot_options o = resolve(opt);
  if (!mat || !a || !b || !valid_dims(n, m) || ldm < m || !valid_dtype(o.dtype))
    return UOT_ERR_INVALID_ARG;
  if (!(reg > 0.0f) || !std::isfinite(reg) || !(reg_m > 0.0f) || iters < 0)
    return UOT_ERR_INVALID_ARG;
  if (std::isnan(tol) || std::isinf(tol) || !reserved_zero(o)) return UOT_ERR_INVALID_ARG;
  if (o.rule != UOT_RULE_PAPER && o.rule != UOT_RULE_POT) return UOT_ERR_INVALID_ARG;
  if (o.storage != UOT_STORAGE_INPLACE && o.storage != UOT_STORAGE_KFORM) return UOT_ERR_INVALID_ARG;
  if (o.deterministic != 0 && o.deterministic != 1) return UOT_ERR_INVALID_ARG;
  if (o.schedule < UOT_SCHED_AUTO || o.schedule > UOT_SCHED_PERSISTENT) return UOT_ERR_INVALID_ARG;
  if (o.algo != UOT_ALGO_FUSED && o.algo != UOT_ALGO_MULTIPASS) return UOT_ERR_INVALID_ARG;
  const bool det = o.deterministic == 1;
  // uot_sinkhorn with kernel-form storage: the plan buffer is K (read-only
  // during the iterations), U lives in the workspace, V in the factor buffer,
  // and a last sweep writes U_i K_ij V_j over the buffer.
  const bool kstore = !kf && o.storage == UOT_STORAGE_KFORM;
  const bool kfo = kf || kstore;  // the iterations run in kernel form
  if ((kstore || det) && o.algo != UOT_ALGO_FUSED) return UOT_ERR_UNSUPPORTED;
  // The scaling-vector rule needs the scalings (kernel form); the adjoint's
  // history is for the rule of Section 2.1.
  if (o.rule == UOT_RULE_POT && (!kfo || hist)) return UOT_ERR_UNSUPPORTED;
  const bool pot = o.rule == UOT_RULE_POT;
  if (o.cluster < 0 || o.cluster > 8 || o.tile < 0 || o.max_ctas < 0) return UOT_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(mat) % esize(o.dtype) ||
      reinterpret_cast<uintptr_t>(a) % 4 || reinterpret_cast<uintptr_t>(b) % 4)
    return UOT_ERR_INVALID_ARG;
  if (kf && (!U || !V || reinterpret_cast<uintptr_t>(U) % 4 || reinterpret_cast<uintptr_t>(V) % 4 ||
             !std::isfinite(k_log2_scale) || std::fabs(k_log2_scale) > 100.0f ||
             k_log2_scale != std::nearbyint(k_log2_scale) || o.algo != UOT_ALGO_FUSED))
    return UOT_ERR_INVALID_ARG;
  const WsLayout L = ws_layout(n, m, det);
  if (!workspace || ws_bytes < L.total || reinterpret_cast<uintptr_t>(workspace) % 256)
    return UOT_ERR_WORKSPACE;
  const HistLayout HL = hist_layout(n, m, iters);
  if (hist && (!kf || hist_bytes < HL.total || reinterpret_cast<uintptr_t>(hist) % 256 ||
               tol > 0.0))
    return UOT_ERR_INVALID_ARG;

  const double fi_d = std::isinf(reg_m) ? 1.0 : double(reg_m) / (double(reg_m) + double(reg));
  const float fi = float(fi_d);
  const bool track = tol > 0.0;
  if (o.algo == UOT_ALGO_MULTIPASS && track) return UOT_ERR_UNSUPPORTED;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint8_t* ws = static_cast<uint8_t*>(workspace);
  const int N = int(n), M = int(m);

  // Persistent schedule (every iteration in one launch, rows held in shared
  // memory) where the plan fits; decided before anything is enqueued.
  PersistPlan pp{};
  bool persist = false;
  if (o.schedule != UOT_SCHED_PASSES && iters > 0) {
    const bool eligible = o.algo == UOT_ALGO_FUSED && !det && !hist && o.tile == 0 &&
                          o.cluster == 0;
    if (eligible) {
      if (persistent_plan(o.dtype, kfo, N, M, o.max_ctas, &pp) != cudaSuccess) return UOT_ERR_CUDA;
      persist = pp.ok;
    }
    if (o.schedule == UOT_SCHED_PERSISTENT && !persist) return UOT_ERR_UNSUPPORTED;
  }

  // Fused-pass geometry, validated before anything is enqueued.
  int k = -1, cs = 1, grid = 0, stages = 0, pair = -1;
  size_t smem = 0;
  const bool tma_ok = reinterpret_cast<uintptr_t>(mat) % 16 == 0 &&
                      (uint64_t(ldm) * esize(o.dtype)) % 16 == 0;
  // Kernel form with bulk copies and no forced configuration: two rows per
  // step (kform_pair.cu); deterministic mode keeps the one-row pass.
  if (kfo && o.algo == UOT_ALGO_FUSED && iters > 0 && tma_ok && o.tile == 0 && o.cluster == 0 &&
      !det && !persist)
    pair = kform_pair_pick(o.dtype, m, &cs);
  if (pair >= 0) {
    if (kform_pair_geometry(pair, cs, N, &grid, &stages, &smem) != cudaSuccess) return UOT_ERR_CUDA;
    if (o.max_ctas > 0 && grid > o.max_ctas) grid = std::max(cs, (o.max_ctas / cs) * cs);
  } else if (o.algo == UOT_ALGO_FUSED && iters > 0 && !persist) {
    k = fused_pick(o.dtype, m, o.tile);
    if (k < 0) return UOT_ERR_INVALID_ARG;
    FusedConfig cfg;
    fused_config_info(k, &cfg);
    cs = o.cluster > 0 ? o.cluster : int((m + cfg.cols - 1) / cfg.cols);
    if (cs > 8) return UOT_ERR_UNSUPPORTED;
    if (int64_t(cs) * cfg.cols < m) return UOT_ERR_INVALID_ARG;
    if (fused_geometry(kfo, k, cs, N, &grid, &stages, &smem) != cudaSuccess) return UOT_ERR_CUDA;
    if (o.max_ctas > 0 && grid > o.max_ctas) grid = std::max(cs, (o.max_ctas / cs) * cs);
    // Deterministic mode: one slot of column partials per row group.
    if (det && grid > DET_SLOTS * cs) grid = DET_SLOTS * cs;
  }

  if (kstore) U = reinterpret_cast<float*>(ws + L.u);
  if (launch_reset(ws, L, b, M, s) != cudaSuccess) return UOT_ERR_CUDA;
  if (kfo && launch_kform_reset(U, N, std::ldexp(1.0f, -int(std::lround(k_log2_scale))),
                               reinterpret_cast<float*>(ws + L.beta), M, int(L.mpad), a, b, fi,
                               pot, reinterpret_cast<double*>(ws + L.log2k), s) != cudaSuccess)
    return UOT_ERR_CUDA;
  uint8_t* hb = static_cast<uint8_t*>(hist);
  if (hist && launch_hist_init(hb, N, M, iters, std::ldexp(1.0f, -int(std::lround(k_log2_scale))),
                               reinterpret_cast<const double*>(ws + L.log2k), s) != cudaSuccess)
    return UOT_ERR_CUDA;
  cudaEvent_t ev0 = static_cast<cudaEvent_t>(o.pass_events[0]);
  cudaEvent_t ev1 = static_cast<cudaEvent_t>(o.pass_events[1]);
  if (ev0 && cudaEventRecord(ev0, s) != cudaSuccess) return UOT_ERR_CUDA;

  if (o.algo == UOT_ALGO_MULTIPASS) {
    for (int t = 1; t <= iters; ++t) {
      if (launch_multipass_iter(mat, ldm, N, M, o.dtype, a, b, fi, t, tol, o.check_every, ws, L,
                                s, nullptr) != cudaSuccess)
        return UOT_ERR_CUDA;
    }
    if (ev1 && cudaEventRecord(ev1, s) != cudaSuccess) return UOT_ERR_CUDA;
  } else if (iters == 0) {
    if (ev1 && cudaEventRecord(ev1, s) != cudaSuccess) return UOT_ERR_CUDA;
  } else if (persist) {
    float* Vws = reinterpret_cast<float*>(ws + L.beta);
    if (persistent_launch(o.dtype, kfo, pp, mat, ldm, N, M, a, b, fi, iters, tol, o.check_every,
                          ws, L, U, Vws, pot ? 1 : 0,
                          std::ldexp(1.0f, int(std::lround(k_log2_scale))), !kf,
                          s) != cudaSuccess)
      return UOT_ERR_CUDA;
    if (ev1 && cudaEventRecord(ev1, s) != cudaSuccess) return UOT_ERR_CUDA;
    // The kernel form's entry point hands V back to the caller.
    if (kf && launch_kform_finish(V, M, iters, ws, L, tol, s) != cudaSuccess) return UOT_ERR_CUDA;
  } else {
    const bool tma = reinterpret_cast<uintptr_t>(mat) % 16 == 0 &&
                     (uint64_t(ldm) * esize(o.dtype)) % 16 == 0;

    FusedArgs A{};
    A.plan = mat;
    A.ldp = ldm;
    A.n = N;
    A.m = M;
    A.a = a;
    A.b = b;
    A.fi = fi;
    A.track = track ? 1 : 0;
    A.tol = tol;
    A.mpad = int(L.mpad);
    A.r_prev = reinterpret_cast<float*>(ws + L.r);
    A.ctl = reinterpret_cast<Control*>(ws + L.ctl);
    A.stages = stages;
    A.b_ws = reinterpret_cast<const float*>(ws + L.bws);
    A.dynamic = det ? 0 : 1;
    A.det = det ? 1 : 0;
    A.part = reinterpret_cast<float*>(ws + L.part);
    A.err_part = reinterpret_cast<double*>(ws + L.err_part);
    A.U = U;
    A.log2k = reinterpret_cast<const double*>(ws + L.log2k);
    A.beta = reinterpret_cast<const float*>(ws + L.beta);
    A.beta_out = reinterpret_cast<float*>(ws + L.beta);
    A.pot = pot ? 1 : 0;
    A.kscale = std::ldexp(1.0f, int(std::lround(k_log2_scale)));
    int* ctr = reinterpret_cast<int*>(ws + L.ctr);
    float* c[3];
    double* er[3];
    for (int q = 0; q < 3; ++q) {
      c[q] = reinterpret_cast<float*>(ws + L.c[q]);
      er[q] = reinterpret_cast<double*>(ws + L.err) + 2 * q;
    }
    for (int t = 1; t <= iters; ++t) {
      A.t = t;
      A.first = !kfo && t == 1;  // the kernel form starts from V = 1 in the buffer
      A.check_prev = track && (t - 1) >= 2 && ((t - 1) % o.check_every) == 0;
      A.c_prev = c[(t - 1) % 3];
      A.c_next = c[t % 3];
      A.c_clear = c[(t + 1) % 3];
      A.err_prev = er[(t - 1) % 3];
      A.err_next = er[t % 3];
      A.err_clear = er[(t + 1) % 3];
      A.row_ctr = ctr + t % 3;
      A.ctr_clear = ctr + (t + 1) % 3;
      A.arrive = ctr + 3 + t % 3;
      A.arrive_clear = ctr + 3 + (t + 1) % 3;
      A.slice_ctr = ctr + 6 + t % 3;
      A.slice_clear = ctr + 6 + (t + 1) % 3;
      if (hist) {
        A.save_r = reinterpret_cast<float*>(hb + HL.r + size_t(t) * HL.strideU);
        A.save_U = reinterpret_cast<float*>(hb + HL.U + size_t(t) * HL.strideU);
        A.save_c = reinterpret_cast<float*>(hb + HL.c + size_t(t) * HL.strideV);
        A.save_V = reinterpret_cast<float*>(hb + HL.V + size_t(t) * HL.strideV);
      }
      const cudaError_t le = pair >= 0 ? kform_pair_launch(pair, cs, grid, smem, A, s)
                                       : fused_launch(kfo, k, cs, grid, smem, tma, A, s);
      if (le != cudaSuccess) return UOT_ERR_CUDA;
      if (det && det_reduce_launch(kfo, grid / cs, A, s) != cudaSuccess) return UOT_ERR_CUDA;
    }
    if (ev1 && cudaEventRecord(ev1, s) != cudaSuccess) return UOT_ERR_CUDA;
    float* Vws = reinterpret_cast<float*>(ws + L.beta);
    cudaError_t e;
    if (kf) {
      e = launch_kform_finish(V, M, iters, ws, L, tol, s);
    } else if (kstore) {
      e = launch_kform_finish(Vws, M, iters, ws, L, tol, s);
      if (e == cudaSuccess) e = launch_kform_materialize(mat, ldm, o.dtype, U, Vws, N, M, s);
    } else {
      e = launch_finish(mat, ldm, N, M, o.dtype, b, fi, iters, ws, L, tol, o.check_every, true, s);
    }
    if (e != cudaSuccess) return UOT_ERR_CUDA;
  }
  if (!out) return UOT_OK;
  return uot_read_result(workspace, n, m, &o, stream, out);
}

}  // namespace uot

extern "C" {

uot_status uot_sinkhorn(void* plan, int64_t ldp, const float* a, const float* b, int64_t n,
                        int64_t m, float reg, float reg_m, int32_t iters, double tol,
                        void* workspace, size_t ws_bytes, const uot_options* opt, void* stream,
                        uot_result* out) {
  return run_sinkhorn(false, plan, ldp, a, b, n, m, reg, reg_m, iters, tol, 0.0f, nullptr,
                      nullptr, workspace, ws_bytes, opt, stream, out);
}

uot_status uot_sinkhorn_kform(const void* K, int64_t ldk, const float* a, const float* b,
                              int64_t n, int64_t m, float reg, float reg_m, int32_t iters,
                              double tol, float k_log2_scale, float* U, float* V,
                              void* workspace, size_t ws_bytes, const uot_options* opt,
                              void* stream, uot_result* out) {
  return run_sinkhorn(true, const_cast<void*>(K), ldk, a, b, n, m, reg, reg_m, iters, tol,
                      k_log2_scale, U, V, workspace, ws_bytes, opt, stream, out);
}

uot_status uot_sinkhorn_kform_save(const void* K, int64_t ldk, const float* a, const float* b,
                                   int64_t n, int64_t m, float reg, float reg_m, int32_t iters,
                                   float k_log2_scale, float* U, float* V, void* hist,
                                   size_t hist_bytes, void* workspace, size_t ws_bytes,
                                   const uot_options* opt, void* stream, uot_result* out) {
  if (!hist) return UOT_ERR_INVALID_ARG;
  return run_sinkhorn(true, const_cast<void*>(K), ldk, a, b, n, m, reg, reg_m, iters, 0.0,
                      k_log2_scale, U, V, workspace, ws_bytes, opt, stream, out, hist, hist_bytes);
}

uot_status uot_shard_pass(void* plan, int64_t ldp, const float* a, int64_t n, int64_t m,
                          float reg, float reg_m, int32_t t, const float* beta_in, float* colsum,
                          void* workspace, size_t ws_bytes, const uot_options* opt,
                          void* stream) {
  const uot_options o = resolve(opt);
  if (!plan || !a || !colsum || !valid_dims(n, m) || ldp < m || !valid_dtype(o.dtype) || t < 1)
    return UOT_ERR_INVALID_ARG;
  if (!(reg > 0.0f) || !std::isfinite(reg) || !(reg_m > 0.0f) || !reserved_zero(o))
    return UOT_ERR_INVALID_ARG;
  if (o.algo != UOT_ALGO_FUSED || o.storage != UOT_STORAGE_INPLACE || o.deterministic ||
      o.rule != UOT_RULE_PAPER || o.schedule == UOT_SCHED_PERSISTENT)
    return UOT_ERR_UNSUPPORTED;
  if (o.cluster < 0 || o.cluster > 8 || o.tile < 0 || o.max_ctas < 0) return UOT_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(plan) % esize(o.dtype) || reinterpret_cast<uintptr_t>(a) % 4 ||
      reinterpret_cast<uintptr_t>(colsum) % 4 || reinterpret_cast<uintptr_t>(beta_in) % 4)
    return UOT_ERR_INVALID_ARG;
  const WsLayout L = ws_layout(n, m);
  if (!workspace || ws_bytes < L.total || reinterpret_cast<uintptr_t>(workspace) % 256)
    return UOT_ERR_WORKSPACE;
  const int N = int(n), M = int(m);
  const int k = fused_pick(o.dtype, m, o.tile);
  if (k < 0) return UOT_ERR_INVALID_ARG;
  FusedConfig cfg;
  fused_config_info(k, &cfg);
  const int cs = o.cluster > 0 ? o.cluster : int((m + cfg.cols - 1) / cfg.cols);
  if (cs > 8) return UOT_ERR_UNSUPPORTED;
  if (int64_t(cs) * cfg.cols < m) return UOT_ERR_INVALID_ARG;
  int grid = 0, stages = 0;
  size_t smem = 0;
  if (fused_geometry(false, k, cs, N, &grid, &stages, &smem) != cudaSuccess) return UOT_ERR_CUDA;
  if (o.max_ctas > 0 && grid > o.max_ctas) grid = std::max(cs, (o.max_ctas / cs) * cs);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint8_t* ws = static_cast<uint8_t*>(workspace);
  const double fi_d = std::isinf(reg_m) ? 1.0 : double(reg_m) / (double(reg_m) + double(reg));
  if (launch_shard_prep(ws, L, beta_in, M, s) != cudaSuccess) return UOT_ERR_CUDA;
  FusedArgs A{};
  A.plan = plan;
  A.ldp = ldp;
  A.n = N;
  A.m = M;
  A.a = a;
  A.fi = float(fi_d);
  A.t = t;
  A.first = beta_in ? 0 : 1;
  A.mpad = int(L.mpad);
  A.c_prev = reinterpret_cast<float*>(ws + L.c[0]);
  A.c_next = reinterpret_cast<float*>(ws + L.c[0]);
  A.c_clear = reinterpret_cast<float*>(ws + L.c[1]);
  A.r_prev = reinterpret_cast<float*>(ws + L.r);
  A.ctl = reinterpret_cast<Control*>(ws + L.ctl);
  A.stages = stages;
  A.b_ws = reinterpret_cast<const float*>(ws + L.bws);
  int* ctr = reinterpret_cast<int*>(ws + L.ctr);
  A.row_ctr = ctr;
  A.ctr_clear = ctr + 1;
  A.arrive = ctr + 3;
  A.arrive_clear = ctr + 4;
  A.slice_ctr = ctr + 6;
  A.slice_clear = ctr + 7;
  A.dynamic = 1;
  A.beta = reinterpret_cast<const float*>(ws + L.beta);
  A.beta_out = reinterpret_cast<float*>(ws + L.beta);
  A.no_factors = 1;
  const bool tma = reinterpret_cast<uintptr_t>(plan) % 16 == 0 &&
                   (uint64_t(ldp) * esize(o.dtype)) % 16 == 0;
  if (fused_launch(false, k, cs, grid, smem, tma, A, s) != cudaSuccess) return UOT_ERR_CUDA;
  if (cudaMemcpyAsync(colsum, ws + L.c[0], size_t(M) * 4, cudaMemcpyDeviceToDevice, s) !=
      cudaSuccess)
    return UOT_ERR_CUDA;
  return UOT_OK;
}

uot_status uot_shard_factors(const float* colsum, const float* b, int64_t m, float reg,
                             float reg_m, float* beta, uint32_t* status_dev, void* stream) {
  if (!colsum || !b || !beta || !valid_dims(1, m)) return UOT_ERR_INVALID_ARG;
  if (!(reg > 0.0f) || !std::isfinite(reg) || !(reg_m > 0.0f)) return UOT_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(colsum) % 4 || reinterpret_cast<uintptr_t>(b) % 4 ||
      reinterpret_cast<uintptr_t>(beta) % 4 || reinterpret_cast<uintptr_t>(status_dev) % 4)
    return UOT_ERR_INVALID_ARG;
  const double fi_d = std::isinf(reg_m) ? 1.0 : double(reg_m) / (double(reg_m) + double(reg));
  return launch_shard_factors(colsum, b, int(m), float(fi_d), beta, status_dev,
                              static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? UOT_OK
             : UOT_ERR_CUDA;
}

uot_status uot_shard_finish(void* plan, int64_t ldp, int64_t n, int64_t m, int32_t dtype,
                            const float* beta, void* stream) {
  if (!plan || !beta || !valid_dims(n, m) || ldp < m || !valid_dtype(dtype))
    return UOT_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(plan) % esize(dtype) || reinterpret_cast<uintptr_t>(beta) % 4)
    return UOT_ERR_INVALID_ARG;
  return launch_scale_cols(plan, ldp, int(n), int(m), dtype, beta,
                           static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? UOT_OK
             : UOT_ERR_CUDA;
}

uot_status uot_init_kernel_scaled(const float* C, int64_t ldc, void* K, int64_t ldk, int64_t n,
                                  int64_t m, float reg, float log2_scale, const uot_options* opt,
                                  void* stream) {
  const uot_options o = resolve(opt);
  if (!C || !K || !valid_dims(n, m) || ldc < m || ldk < m || !valid_dtype(o.dtype))
    return UOT_ERR_INVALID_ARG;
  if (!(reg > 0.0f) || !std::isfinite(reg) || !std::isfinite(log2_scale) ||
      std::fabs(log2_scale) > 100.0f || log2_scale != std::nearbyint(log2_scale))
    return UOT_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(K) % esize(o.dtype) || reinterpret_cast<uintptr_t>(C) % 4)
    return UOT_ERR_INVALID_ARG;
  cudaError_t e = launch_init(C, ldc, K, ldk, int(n), int(m), reg, o.dtype,
                              std::ldexp(1.0f, int(log2_scale)), static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? UOT_OK : UOT_ERR_CUDA;
}

uot_status uot_kform_plan(const void* K, int64_t ldk, int32_t k_dtype, const float* U,
                          const float* V, int64_t n, int64_t m, void* plan, int64_t ldp,
                          int32_t plan_dtype, void* stream) {
  if (!K || !U || !V || !plan || !valid_dims(n, m) || ldk < m || ldp < m ||
      !valid_dtype(k_dtype) || !valid_dtype(plan_dtype))
    return UOT_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(K) % esize(k_dtype) ||
      reinterpret_cast<uintptr_t>(plan) % esize(plan_dtype))
    return UOT_ERR_INVALID_ARG;
  cudaError_t e = launch_kform_plan(K, ldk, k_dtype, U, V, int(n), int(m), plan, ldp, plan_dtype,
                                    static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? UOT_OK : UOT_ERR_CUDA;
}

uot_status uot_kform_cost(const void* K, int64_t ldk, int32_t k_dtype, const float* U,
                          const float* V, const float* C, int64_t ldc, int64_t n, int64_t m,
                          double* out_dev, void* stream) {
  if (!K || !U || !V || !C || !out_dev || !valid_dims(n, m) || ldk < m || ldc < m ||
      !valid_dtype(k_dtype))
    return UOT_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(K) % esize(k_dtype) || reinterpret_cast<uintptr_t>(out_dev) % 8)
    return UOT_ERR_INVALID_ARG;
  cudaError_t e = launch_kform_cost(K, ldk, k_dtype, U, V, C, ldc, int(n), int(m), out_dev,
                                    static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? UOT_OK : UOT_ERR_CUDA;
}

uot_status uot_cost(const void* plan, int64_t ldp, const float* C, int64_t ldc, int64_t n,
                    int64_t m, int32_t dtype, double* out_dev, void* stream) {
  if (!plan || !C || !out_dev || !valid_dims(n, m) || ldp < m || ldc < m || !valid_dtype(dtype))
    return UOT_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(plan) % esize(dtype) || reinterpret_cast<uintptr_t>(out_dev) % 8)
    return UOT_ERR_INVALID_ARG;
  cudaError_t e = launch_cost(plan, ldp, C, ldc, int(n), int(m), dtype, out_dev,
                              static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? UOT_OK : UOT_ERR_CUDA;
}

int32_t uot_fused_config(int32_t k, int32_t* dtype, int32_t* threads, int32_t* vecs,
                         int32_t* cols_per_cta) {
  FusedConfig c;
  if (k < 0 || !fused_config_info(k, &c)) return fused_num_configs();
  if (dtype) *dtype = c.dtype;
  if (threads) *threads = c.threads;
  if (vecs) *vecs = c.vecs;
  if (cols_per_cta) *cols_per_cta = c.cols;
  return fused_num_configs();
}

}  // extern "C"
