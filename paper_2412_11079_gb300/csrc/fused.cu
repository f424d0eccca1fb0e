// The fused MAP-UOT iteration pass (Section 4, Algorithm 1) on sm_103a.
//
// One launch performs one iteration.  The plan S stored before the pass is
// the plan after the row step of iteration t-1 with that iteration's column
// factor beta_{t-1} still pending.  For every row i the pass computes
//     x_ij = S_ij * beta_{t-1,j}           (column step of iteration t-1)
//     r_i  = sum_j x_ij,  alpha_i = (a_i / r_i)^fi
//     y_ij = x_ij * alpha_i                (row step of iteration t)
// stores y and accumulates c_j += y_ij, so the plan is read once and written
// once per iteration (Section 3.1 gives 2*N*M element transfers as the
// minimum).  beta_t = (b_j / c_j)^fi is applied by the next pass.
//
// GB300 mapping.  A cluster of `cs` CTAs owns one row at a time; CTA rank r
// covers columns [r*W, (r+1)*W) with W = threads * vecs * (16 / sizeof(T)).
// Rows of the CTA's column slice stream through a ring of `stages` shared-
// memory slots filled by 1-D bulk copies (cp.async.bulk, completion on an
// mbarrier); each thread keeps the pending column factors of its columns and
// its column partial sums in registers.  The row sum is reduced with warp
// shuffles and exchanged through distributed shared memory with one barrier
// per row (a plain CTA barrier when cs == 1).  The scaled row goes back with
// 16-byte streaming stores, and each CTA folds its column partials into the
// global column sums once, at the end of the pass, with vector reductions
// (red.global.add.v4.f32).  Clusters are persistent over rows: cluster g
// takes rows g, g + G, g + 2G, ...
//
// Column partial sums are combined with floating-point atomics, so their
// order (and the last bits of the column sums) can differ from run to run.
#include <cuda_runtime.h>

#include "uot_device.cuh"
#include "uot_internal.h"

namespace uot {

namespace {

constexpr int MAX_CLUSTER = 8;

template <typename T, int THREADS, int KV, bool TMA>
__global__ void __launch_bounds__(THREADS, 1) fused_pass_kernel(const FusedArgs p) {
  using E = Elem<T>;
  constexpr int VE = E::VE;
  constexpr int NW = THREADS / 32;
  constexpr int W = KV * VE * THREADS;
  constexpr int ROW_BYTES = W * int(sizeof(T));
  constexpr int RED = MAX_CLUSTER * NW;

  extern __shared__ __align__(128) unsigned char smem[];
  const int stages = TMA ? p.stages : 0;
  unsigned char* ring = smem;
  float* red = reinterpret_cast<float*>(smem + size_t(stages) * ROW_BYTES);
  uint64_t* bars = reinterpret_cast<uint64_t*>(red + 2 * RED);

  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const uint32_t cs = cluster_nctarank();
  const uint32_t cr = cluster_ctarank();
  const int cid = int(cluster_id_x());
  const int ncl = int(ncluster_x());
  Control* ctl = p.ctl;

  // Stopping rule (tol > 0): a previous pass may have stopped the iteration,
  // or iteration t-1 may satisfy it now.  Every CTA reads the same values and
  // takes the same decision, before touching any shared state.
  if (p.track) {
    if (*reinterpret_cast<volatile int32_t*>(&ctl->done)) return;
    if (p.check_prev) {
      const double num = p.err_prev[0], den = p.err_prev[1];
      const double e = den > 0.0 ? num / den : __longlong_as_double(0x7ff0000000000000ll);
      if (e <= p.tol) {
        if (blockIdx.x == 0 && tid == 0) {
          ctl->stop_iter = p.t - 1;
          ctl->err = e;
          __threadfence();
          ctl->done = 1;
        }
        return;
      }
    }
  }

  // Pending column factors of this thread's columns.
  const int m = p.m;
  const int col0 = int(cr) * W;
  uint32_t st = 0;
  float beta[KV][VE];
#pragma unroll
  for (int k = 0; k < KV; ++k) {
    const int cc = col0 + (k * THREADS + tid) * VE;
#pragma unroll
    for (int e = 0; e < VE; ++e) {
      const int j = cc + e;
      float bj = 0.0f;
      if (j < m) bj = p.first ? 1.0f : rescale_factor(__ldg(p.b + j), p.c_prev[j], p.fi, st);
      beta[k][e] = bj;
    }
  }

  // Clear the column-sum (and stopping-error) buffers of iteration t+1.
  {
    const int g = blockIdx.x * THREADS + tid;
    const int gs = gridDim.x * THREADS;
    for (int j = g; j < p.mpad; j += gs) p.c_clear[j] = 0.0f;
    if (p.track && blockIdx.x == 0 && tid < 2) p.err_clear[tid] = 0.0;
  }

  float cacc[KV][VE];
#pragma unroll
  for (int k = 0; k < KV; ++k)
#pragma unroll
    for (int e = 0; e < VE; ++e) cacc[k][e] = 0.0f;

  const int n = p.n;
  const int nq = cid < n ? (n - 1 - cid) / ncl + 1 : 0;
  const int valid = max(0, min(W, m - col0));
  const uint32_t copy_bytes = uint32_t((size_t(valid) * sizeof(T)) & ~size_t(15));
  T* plan = reinterpret_cast<T*>(p.plan);
  const int64_t ldp = p.ldp;
  uint64_t policy = 0;
  int issued = 0;  // copies issued (thread 0 only)

  if (TMA) {
    policy = policy_evict_first();
    if (tid == 0) {
      for (int s = 0; s < stages; ++s) mbar_init(&bars[s], 1);
      fence_mbar_init();
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
  }
  // All CTAs of the cluster must be running before distributed shared memory
  // is written; the same barrier publishes the mbarrier initialisation.
  if (cs > 1) cluster_sync(); else __syncthreads();

  auto issue = [&](int q) {
    const int row = cid + q * ncl;
    const int slot = q % stages;
    if (copy_bytes) {
      mbar_arrive_expect_tx(&bars[slot], copy_bytes);
      bulk_load(ring + size_t(slot) * ROW_BYTES, plan + int64_t(row) * ldp + col0, copy_bytes,
                &bars[slot], policy);
    } else {
      mbar_arrive(&bars[slot]);
    }
  };
  if (TMA && tid == 0) {
    const int first = min(stages, nq);
    for (int q = 0; q < first; ++q) issue(q);
    issued = first;
  }

  bool broken = false;
  double err_num = 0.0, err_den = 0.0;

  for (int q = 0; q < nq; ++q) {
    const int row = cid + q * ncl;
    const float arow = __ldg(p.a + row);
    T* grow = plan + int64_t(row) * ldp;
    float x[KV][VE];
    if (TMA) {
      const int slot = q % stages;
      if (!broken && !mbar_wait_bounded(&bars[slot], uint32_t(q / stages) & 1u, WAIT_LIMIT_NS)) {
        broken = true;
        st |= DEV_TIMEOUT;
      }
      const unsigned char* srow = ring + size_t(slot) * ROW_BYTES;
#pragma unroll
      for (int k = 0; k < KV; ++k) {
        const int li = k * THREADS + tid;
        const int cc = col0 + li * VE;
        if (cc + VE <= m) {
          E::unpack(ld_shared_v4(srow + size_t(li) * 16), x[k]);
        } else {
#pragma unroll
          for (int e = 0; e < VE; ++e) x[k][e] = (cc + e < m) ? E::load1(grow + cc + e) : 0.0f;
        }
      }
    } else {
#pragma unroll
      for (int k = 0; k < KV; ++k) {
        const int cc = col0 + (k * THREADS + tid) * VE;
#pragma unroll
        for (int e = 0; e < VE; ++e) x[k][e] = (cc + e < m) ? E::load1(grow + cc + e) : 0.0f;
      }
    }

    // Column step of iteration t-1 on this row, then its sum.
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < KV; ++k)
#pragma unroll
      for (int e = 0; e < VE; ++e) {
        x[k][e] = E::round(x[k][e] * beta[k][e]);
        s += x[k][e];
      }
    s = warp_sum(s);
    float* rb = red + (q & 1) * RED;
    if (lane == 0) {
      if (cs == 1) {
        rb[warp] = s;
      } else {
        for (uint32_t r = 0; r < cs; ++r) st_cluster_f32(map_shared_rank(rb + cr * NW + warp, r), s);
      }
    }
    if (cs > 1) cluster_sync(); else __syncthreads();
    // Every thread has finished reading this slot: refill it.
    if (TMA && tid == 0 && !broken && issued < nq) {
      issue(issued);
      ++issued;
    }
    float tot = 0.0f;
    for (uint32_t r = 0; r < cs; ++r)
#pragma unroll
      for (int w = 0; w < NW; ++w) tot += rb[r * NW + w];

    // Row step of iteration t.
    const float alpha = rescale_factor(arow, tot, p.fi, st);
#pragma unroll
    for (int k = 0; k < KV; ++k) {
      const int cc = col0 + (k * THREADS + tid) * VE;
      float y[VE];
#pragma unroll
      for (int e = 0; e < VE; ++e) {
        y[e] = E::round(x[k][e] * alpha);
        cacc[k][e] += y[e];
      }
      if (TMA && cc + VE <= m) {
        st_global_cs_v4(grow + cc, E::pack(y));
      } else {
#pragma unroll
        for (int e = 0; e < VE; ++e)
          if (cc + e < m) E::store1(grow + cc + e, y[e]);
      }
    }
    if (p.track && cr == 0 && tid == 0) {
      const double d = tot;
      if (p.t >= 2) err_num += fabs(d - double(p.r_prev[row]));
      err_den += d;
      p.r_prev[row] = tot;
    }
  }

  // Fold this CTA's column partials into the column sums of iteration t.
  if (nq > 0) {
#pragma unroll
    for (int k = 0; k < KV; ++k) {
      const int cc = col0 + (k * THREADS + tid) * VE;
      if (cc + VE <= m) {
#pragma unroll
        for (int e = 0; e < VE; e += 4)
          red_add_v4(p.c_next + cc + e, cacc[k][e], cacc[k][e + 1], cacc[k][e + 2], cacc[k][e + 3]);
      } else {
#pragma unroll
        for (int e = 0; e < VE; ++e)
          if (cc + e < m) atomicAdd(p.c_next + cc + e, cacc[k][e]);
      }
    }
  }
  if (p.track && cr == 0 && tid == 0 && nq > 0) {
    atomicAdd(&p.err_next[0], err_num);
    atomicAdd(&p.err_next[1], err_den);
  }
  if (st) atomicOr(&ctl->status, st);

  // After a timed-out wait, give copies still in flight a bounded chance to
  // land before the CTA (and its shared memory) goes away.
  if (TMA && tid == 0 && broken) {
    for (int q = max(0, issued - stages); q < issued; ++q)
      mbar_wait_bounded(&bars[q % stages], uint32_t(q / stages) & 1u, WAIT_LIMIT_NS);
  }
}

// ----------------------------------------------------------- config table
struct Entry {
  FusedConfig cfg;
  const void* fn_tma;
  const void* fn_plain;
};

#define UOT_ENTRY(T, DT, TH, KV)                                                         \
  Entry {                                                                                \
    FusedConfig{DT, TH, KV, KV * (16 / int(sizeof(T))) * TH, 1},                         \
        reinterpret_cast<const void*>(&fused_pass_kernel<T, TH, KV, true>),             \
        reinterpret_cast<const void*>(&fused_pass_kernel<T, TH, KV, false>)             \
  }

const Entry kTable[] = {
    UOT_ENTRY(float, UOT_F32, 512, 8),          UOT_ENTRY(float, UOT_F32, 512, 4),
    UOT_ENTRY(float, UOT_F32, 256, 4),          UOT_ENTRY(float, UOT_F32, 128, 4),
    UOT_ENTRY(float, UOT_F32, 128, 2),          UOT_ENTRY(float, UOT_F32, 64, 2),
    UOT_ENTRY(float, UOT_F32, 32, 2),           UOT_ENTRY(__nv_bfloat16, UOT_BF16, 512, 4),
    UOT_ENTRY(__nv_bfloat16, UOT_BF16, 256, 4), UOT_ENTRY(__nv_bfloat16, UOT_BF16, 128, 4),
    UOT_ENTRY(__nv_bfloat16, UOT_BF16, 128, 2), UOT_ENTRY(__nv_bfloat16, UOT_BF16, 64, 2),
    UOT_ENTRY(__nv_bfloat16, UOT_BF16, 32, 2),  UOT_ENTRY(__half, UOT_F16, 512, 4),
    UOT_ENTRY(__half, UOT_F16, 256, 4),         UOT_ENTRY(__half, UOT_F16, 128, 4),
    UOT_ENTRY(__half, UOT_F16, 128, 2),         UOT_ENTRY(__half, UOT_F16, 64, 2),
    UOT_ENTRY(__half, UOT_F16, 32, 2),
};
constexpr int kNum = int(sizeof(kTable) / sizeof(kTable[0]));

size_t elem_size(int dtype) { return dtype == UOT_F32 ? 4 : 2; }

size_t smem_bytes(const FusedConfig& c, int stages) {
  const size_t row = size_t(c.cols) * elem_size(c.dtype);
  const size_t red = 2 * MAX_CLUSTER * (c.threads / 32) * sizeof(float);
  return size_t(stages) * row + red + size_t(stages > 0 ? stages : 1) * 8;
}

}  // namespace

int fused_num_configs() { return kNum; }

bool fused_config_info(int k, FusedConfig* out) {
  if (k < 0 || k >= kNum) return false;
  *out = kTable[k].cfg;
  return true;
}

int fused_pick(int dtype, int64_t m, int tile) {
  if (tile > 0) {
    const int k = tile - 1;
    if (k >= kNum || kTable[k].cfg.dtype != dtype) return -1;
    return k;
  }
  // Smallest CTA width that covers the row; otherwise the widest, split over
  // a cluster.
  int best = -1, widest = -1;
  for (int k = 0; k < kNum; ++k) {
    const FusedConfig& c = kTable[k].cfg;
    if (c.dtype != dtype) continue;
    if (widest < 0 || c.cols > kTable[widest].cfg.cols) widest = k;
    if (c.cols >= m && (best < 0 || c.cols < kTable[best].cfg.cols)) best = k;
  }
  return best >= 0 ? best : widest;
}

cudaError_t fused_geometry(int k, int cs, int n, int* grid, int* stages, size_t* smem) {
  const Entry& e = kTable[k];
  int dev = 0, sms = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
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
    err = cudaFuncSetAttribute(e.fn_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, int(b));
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
  err = cudaFuncSetAttribute(e.fn_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, int(*smem));
  if (err != cudaSuccess) return err;
  int clusters = occ2 * sms;
  if (cs > 1) {
    err = cudaFuncSetAttribute(e.fn_tma, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
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
  // Keep at least two rows per cluster so the column flush stays small.
  const int cap = (n + 1) / 2;
  if (clusters > cap) clusters = cap > 0 ? cap : 1;
  *grid = clusters * cs;
  return cudaSuccess;
}

cudaError_t fused_launch(int k, int cs, int grid, size_t smem, bool tma, const FusedArgs& args,
                         cudaStream_t s) {
  const Entry& e = kTable[k];
  const void* fn = tma ? e.fn_tma : e.fn_plain;
  size_t bytes = tma ? smem : smem_bytes(e.cfg, 0);
  cudaError_t err = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
  if (err != cudaSuccess) return err;
  if (cs > 1) {
    err = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (err != cudaSuccess) return err;
  }
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
  err = cudaLaunchKernelExC(&cfg, fn, kargs);
  if (err == cudaSuccess) count_launch();
  return err;
}

}  // namespace uot
