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
// (red.global.add.v4.f32).
//
// Rows are scheduled dynamically when a row fits one CTA: CTAs take rows
// from a per-pass counter (the next index fetched one step ahead), so SMs
// that stream faster take more rows and the pass ends within about one row
// time on every SM; the direction alternates between passes so a pass starts
// on rows the previous pass wrote last.  The next pass's column factors are
// computed once: the last 16 CTAs to finish a pass each take 1/16 of the
// columns after all column partials have landed.  Clusters (rows wider than
// one CTA) and the path without bulk copies keep a static schedule: cluster
// g takes rows g, g + G, g + 2G, ...
//
// Column partial sums are combined with floating-point atomics, so their
// order (and the last bits of the column sums) can differ from run to run.
#include <cuda_runtime.h>

#include <mutex>

#include "uot_device.cuh"
#include "uot_internal.h"

namespace uot {

namespace {

constexpr int MAX_CLUSTER = 8;
constexpr int BETA_CTAS = 16;  // CTAs that compute the next column factors

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

  const int m = p.m;
  const int n = p.n;
  const int col0 = int(cr) * W;
  const int valid = max(0, min(W, m - col0));
  const uint32_t copy_bytes = uint32_t((size_t(valid) * sizeof(T)) & ~size_t(15));
  T* plan = reinterpret_cast<T*>(p.plan);
  const int64_t ldp = p.ldp;
  uint32_t st = 0;

  // Row schedule.  Dynamic (one CTA per row, bulk-copy path): CTAs take rows
  // from this pass's counter, so CTAs that stream faster take more rows and
  // all finish within about one row of each other.  Static (clusters, or the
  // path without bulk copies): cluster g takes rows g, g + G, g + 2G, ...
  const bool dyn = TMA && p.dynamic && cs == 1;
  const int nq = cid < n ? (n - 1 - cid) / ncl + 1 : 0;  // static rows
  int* slot_row = reinterpret_cast<int*>(bars + (TMA ? stages : 1));
  uint64_t policy = 0;
  int issued = 0;     // steps whose slot has been armed (thread 0 only)
  int next_row = n;   // dynamic: row index fetched one step ahead (thread 0)

  if constexpr (TMA) {
    // Evict-first loads and streaming stores measured fastest (evict-normal
    // loads/stores and evict-last stores for the rows the next pass reads
    // first were slower).
    policy = policy_evict_first();
    if (tid == 0) {
      for (int s2 = 0; s2 < stages; ++s2) mbar_init(&bars[s2], 1);
      fence_mbar_init();
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
  }
  // All CTAs of the cluster must be running before distributed shared memory
  // is written; the same barrier publishes the mbarrier initialisation.
  if (cs > 1) cluster_sync(); else __syncthreads();

  // Arms the slot of step q with `row` (row < 0 or >= n: end of the rows).
  // Dynamic rows alternate direction from pass to pass, so a pass starts on
  // the rows the previous pass wrote last, which are still in L2.
  const bool flip = dyn && (p.t & 1) == 0;
  auto arm = [&](int q, int row) {
    if constexpr (TMA) {
      const int slot = q % stages;
      if (row >= 0 && row < n) {
        if (flip) row = n - 1 - row;
        slot_row[slot] = row;
        if (copy_bytes) {
          mbar_arrive_expect_tx(&bars[slot], copy_bytes);
          bulk_load(ring + size_t(slot) * ROW_BYTES, plan + int64_t(row) * ldp + col0,
                    copy_bytes, &bars[slot], policy);
        } else {
          mbar_arrive(&bars[slot]);
        }
      } else {
        slot_row[slot] = -1;
        mbar_arrive(&bars[slot]);
      }
    }
  };
  if constexpr (TMA) {
    if (tid == 0) {
      if (dyn) {
        const int base = atomicAdd(p.row_ctr, stages);
        for (int q = 0; q < stages; ++q) arm(q, base + q);
        issued = stages;
        if (base + stages < n) next_row = atomicAdd(p.row_ctr, 1);
      } else {
        const int first = min(stages, nq);
        for (int q = 0; q < first; ++q) arm(q, cid + q * ncl);
        issued = first;
      }
    }
  }

  // Pending column factors of this thread's columns: beta_{t-1} was computed
  // once, at the end of the previous pass, by that pass's last CTAs.
  float beta[KV][VE];
#pragma unroll
  for (int k = 0; k < KV; ++k) {
    const int cc = col0 + (k * THREADS + tid) * VE;
    if (p.first) {
#pragma unroll
      for (int e = 0; e < VE; ++e) beta[k][e] = (cc + e < m) ? 1.0f : 0.0f;
    } else if (cc < m) {  // the factor buffer is zero-padded to a multiple of 64
#pragma unroll
      for (int e = 0; e < VE; e += 4) {
        const float4 b4 = __ldcg(reinterpret_cast<const float4*>(p.beta + cc + e));
        beta[k][e] = b4.x; beta[k][e + 1] = b4.y; beta[k][e + 2] = b4.z; beta[k][e + 3] = b4.w;
      }
    } else {
#pragma unroll
      for (int e = 0; e < VE; ++e) beta[k][e] = 0.0f;
    }
  }

  // Clear the column-sum, row-counter and stopping-error buffers of t+1.
  {
    const int g = blockIdx.x * THREADS + tid;
    const int gs = gridDim.x * THREADS;
    for (int j = g; j < p.mpad; j += gs) p.c_clear[j] = 0.0f;
    if (blockIdx.x == 0 && tid == 0) {
      *p.ctr_clear = 0;
      *p.arrive_clear = 0;
    }
    if (p.track && blockIdx.x == 0 && tid < 2) p.err_clear[tid] = 0.0;
  }

  float cacc[KV][VE];
#pragma unroll
  for (int k = 0; k < KV; ++k)
#pragma unroll
    for (int e = 0; e < VE; ++e) cacc[k][e] = 0.0f;

  bool broken = false;
  int done_rows = 0;
  double err_num = 0.0, err_den = 0.0;

  for (int q = 0;; ++q) {
    int row;
    float x[KV][VE];
    if constexpr (TMA) {
      if (!dyn && q >= nq) break;
      const int slot = q % stages;
      if (!broken && !mbar_wait_bounded(&bars[slot], uint32_t(q / stages) & 1u, WAIT_LIMIT_NS)) {
        broken = true;
        st |= DEV_TIMEOUT;
      }
      row = *reinterpret_cast<volatile int*>(&slot_row[slot]);
      if (row < 0 || row >= n) break;  // uniform: every thread reads the same slot
      const T* grow = plan + int64_t(row) * ldp;
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
      if (q >= nq) break;
      row = cid + q * ncl;
      const T* grow = plan + int64_t(row) * ldp;
#pragma unroll
      for (int k = 0; k < KV; ++k) {
        const int cc = col0 + (k * THREADS + tid) * VE;
#pragma unroll
        for (int e = 0; e < VE; ++e) x[k][e] = (cc + e < m) ? E::load1(grow + cc + e) : 0.0f;
      }
    }
    const float arow = __ldg(p.a + row);
    T* grow = plan + int64_t(row) * ldp;

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
    if (cs > 1) {
      cluster_sync();  // static rows: the loop is bounded by nq
    } else if (__syncthreads_or(broken ? 1 : 0)) {
      // A copy never completed: leave together (the data of this step is not
      // valid); copies still in flight are waited for below.
      broken = true;
      st |= DEV_TIMEOUT;
      break;
    }
    // Every thread has finished reading this slot: re-arm it.
    if constexpr (TMA) {
      if (tid == 0 && !broken) {
        if (dyn) {
          const int r2 = next_row;
          arm(issued, r2);
          ++issued;
          if (r2 < n) {
            next_row = atomicAdd(p.row_ctr, 1);
          }
        } else if (issued < nq) {
          arm(issued, cid + issued * ncl);
          ++issued;
        }
      }
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
    ++done_rows;
  }

  // Fold this CTA's column partials into the column sums of iteration t.
  if (done_rows > 0) {
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
  if (p.track && cr == 0 && tid == 0 && done_rows > 0) {
    atomicAdd(&p.err_next[0], err_num);
    atomicAdd(&p.err_next[1], err_den);
  }
  if (st) atomicOr(&ctl->status, st);

  // beta_t = (b_j / c_j)^fi for the next pass, computed once: the last K CTAs
  // to finish this pass each take 1/K of the columns, after waiting (bounded)
  // for every CTA's column partials to land.  Only CTAs already running are
  // waited for, so this needs no co-residency guarantee.
  __syncthreads();
  __shared__ int s_arrival;
  if (tid == 0) {
    __threadfence();
    s_arrival = atomicAdd(p.arrive, 1);
  }
  __syncthreads();
  const int G = int(gridDim.x);
  const int K = min(G, BETA_CTAS);
  const int slice = s_arrival - (G - K);
  if (slice >= 0) {
    if (tid == 0) {
      const uint64_t t0 = global_timer_ns();
      while (ld_acquire_gpu(p.arrive) < G) {
        if (global_timer_ns() - t0 > WAIT_LIMIT_NS) {
          atomicOr(&ctl->status, DEV_TIMEOUT);
          break;
        }
      }
    }
    __syncthreads();
    const int per = (m + K - 1) / K;
    const int j0 = slice * per, j1 = min(m, j0 + per);
    uint32_t st2 = 0;
    for (int j = j0 + tid; j < j1; j += THREADS)
      p.beta_out[j] = rescale_factor(__ldg(p.b_ws + j), __ldcg(p.c_next + j), p.fi, st2);
    if (st2) atomicOr(&ctl->status, st2);
  }

  // After a timed-out wait, give copies still in flight a bounded chance to
  // land before the CTA (and its shared memory) goes away.
  if constexpr (TMA) {
    if (tid == 0 && broken) {
      for (int q = max(0, issued - stages); q < issued; ++q)
        mbar_wait_bounded(&bars[q % stages], uint32_t(q / stages) & 1u, WAIT_LIMIT_NS);
    }
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
  const size_t slots = size_t(stages > 0 ? stages : 1);
  return size_t(stages) * row + red + slots * 8 + slots * 4;
}

// cudaFuncSetAttribute is a host call that can wait for running work on the
// device; re-issuing it before every iteration pass kept the host in lockstep
// with the GPU.  Attributes are therefore set once per (device, kernel) and
// the launch geometry is cached per (device, config, cluster, rows).
constexpr int MAX_DEV = 64;
std::mutex g_mu;
size_t g_smem_set[MAX_DEV][kNum][2];
bool g_cluster_set[MAX_DEV][kNum][2];

struct GeoKey {
  int dev, k, cs, n;
  bool operator==(const GeoKey& o) const {
    return dev == o.dev && k == o.k && cs == o.cs && n == o.n;
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

cudaError_t ensure_attributes(int dev, int k, bool tma, size_t smem, bool cluster) {
  if (dev < 0 || dev >= MAX_DEV) return cudaErrorInvalidDevice;
  const void* fn = tma ? kTable[k].fn_tma : kTable[k].fn_plain;
  std::lock_guard<std::mutex> lock(g_mu);
  if (g_smem_set[dev][k][tma] < smem) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    g_smem_set[dev][k][tma] = smem;
  }
  if (cluster && !g_cluster_set[dev][k][tma]) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    g_cluster_set[dev][k][tma] = true;
  }
  return cudaSuccess;
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
  const GeoKey key{dev, k, cs, n};
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
  err = ensure_attributes(dev, k, false, smem_bytes(e.cfg, 0), cs > 1);
  if (err != cudaSuccess) return err;
  err = ensure_attributes(dev, k, true, *smem, cs > 1);
  if (err != cudaSuccess) return err;
  std::lock_guard<std::mutex> lock(g_mu);
  const int slot = g_geo_used < GEO_CACHE ? g_geo_used++ : (g_geo_next++ % GEO_CACHE);
  g_geo_key[slot] = key;
  g_geo_val[slot] = GeoVal{*grid, *stages, *smem};
  return cudaSuccess;
}

cudaError_t fused_launch(int k, int cs, int grid, size_t smem, bool tma, const FusedArgs& args,
                         cudaStream_t s) {
  const Entry& e = kTable[k];
  const void* fn = tma ? e.fn_tma : e.fn_plain;
  size_t bytes = tma ? smem : smem_bytes(e.cfg, 0);
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
