// The fused MAP-UOT iteration pass (Section 4, Algorithm 1) on sm_103a:
// kernel template, instantiated by fused_inplace.cu and fused_kform.cu.
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
// Kernel form (KF): the plan is kept as diag(U) K diag(V) with K read-only
// (FP32, BF16 or FP16) and FP32 scalings.  The same pass reads K once, forms
// r_i = U_i sum_j K_ij V_j, updates U_i, and accumulates d_j = sum_i U_i K_ij;
// the last CTAs then set V_j <- V_j (b_j / (V_j d_j))^fi.  In real arithmetic
// this is the same iterate as the in-place plan; K is rounded only once.
//
// Column partial sums are combined with floating-point atomics, so their
// order (and the last bits of the column sums) can differ from run to run.
// Deterministic mode (p.det) keeps the static schedule for every row width,
// stores each row group's partials to a slot of its own instead, and leaves
// the next factors to a reduction launch that adds the slots in slot order
// (det_reduce_kernel): the same inputs then give the same bits.
#pragma once

#include <cuda_runtime.h>

#include "uot_device.cuh"
#include "uot_internal.h"

namespace uot {

constexpr int MAX_CLUSTER = 8;
constexpr int BETA_CTAS = 16;       // late CTAs that may help with the next factors
constexpr int BETA_SLICES = 64;     // column slices of that job
constexpr uint64_t HELP_LOOK_NS = 2000;  // how long a late CTA looks for the rest

template <typename T, int THREADS, int KV, bool TMA, bool KF>
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
      // err = num / den <= tol, decided without the (slow) FP64 division.
      const double num = p.err_prev[0], den = p.err_prev[1];
      if (den > 0.0 && num <= p.tol * den) {
        if (blockIdx.x == 0 && tid == 0) {
          ctl->stop_iter = p.t - 1;
          ctl->err = num / den;
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
  // Kernel form: the scalings drift as U ~ k^t, V ~ k^-t (at the fixed point
  // every row factor tends to k and every column factor to 1/k), which leaves
  // FP32's range within a few hundred iterations.  The plan U K V does not
  // change if U is multiplied by 2^e and V by 2^-e, so each pass applies the
  // exact power-of-two gauge 2^e_t (gauge_exponent).
  float gauge = 1.0f, inv_gauge = 1.0f;
  if constexpr (KF) {
    const int e = gauge_exponent(p.t, float(*p.log2k));
    gauge = ldexpf(1.0f, e);
    inv_gauge = ldexpf(1.0f, -e);
  }
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
  float* uf = reinterpret_cast<float*>(slot_row + (TMA ? stages : 1));  // [2] row factor
  // The thread that forms a row's factor in the kernel form: in the last
  // warp, away from thread 0's refills.
  constexpr int ftid = KF ? THREADS - 1 : 0;
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
  // once, at the end of the previous pass, by that pass's last CTAs.  In the
  // kernel form the same registers hold the cumulative column scaling V.
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
      *p.slice_clear = 0;
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
  // Stopping-rule sums of this CTA's rows (FP32 with compensation; folded
  // into the FP64 totals once per CTA).
  float err_num = 0.0f, err_den = 0.0f, err_num_c = 0.0f, err_den_c = 0.0f;

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
    // Kernel form: one thread (ftid) forms the row factor; in place, every
    // thread scales the row and needs a_i.
    float arow = 0.0f, u_old = 1.0f;
    if (!KF || tid == ftid) arow = __ldg(p.a + row);
    if constexpr (KF) {
      if (tid == ftid) u_old = __ldcg(p.U + row);
    }
    T* grow = plan + int64_t(row) * ldp;

    // Column step of iteration t-1 on this row, then its sum.  Kernel form:
    // the row sum of U_i K_ij V_j is U_i sum_j K_ij V_j; K stays in x.
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < KV; ++k)
#pragma unroll
      for (int e = 0; e < VE; ++e) {
        if constexpr (KF) {
          s = fmaf(x[k][e], beta[k][e], s);
        } else {
          x[k][e] = E::round(x[k][e] * beta[k][e]);
          s += x[k][e];
        }
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
    if (!KF || tid == ftid) {
      for (uint32_t r = 0; r < cs; ++r)
#pragma unroll
        for (int w = 0; w < NW; ++w) tot += rb[r * NW + w];
    }

    // Row step of iteration t.
    if constexpr (KF) {
      // Kernel form: U_i <- U_i alpha_i 2^e_t, formed once per row (one power
      // per row rather than one per thread) and handed over through shared
      // memory; column partials of U_i K_ij (the column sums are V_j 2^-e_t
      // times these).
      float* ufq = uf + (q & 1);
      if (tid == ftid) {
        const float s_kv = tot;  // sum_j K_ij V_j (K as stored)
        tot *= u_old;            // r_i, the row sum of the plan
        // Scaling-vector rule: u_i <- (a_i / (K v)_i)^fi with K = stored K / kscale
        // and U = u / kscale; no gauge.
        const float u_new = p.pot ? rescale_factor(arow * p.kscale, s_kv, p.fi, st) / p.kscale
                                  : u_old * rescale_factor(arow, tot, p.fi, st) * gauge;
        *ufq = u_new;
        if (cr == 0) {
          p.U[row] = u_new;
          if (p.save_r) {  // history for the adjoint: r_t and U_t of this row
            p.save_r[row] = tot;
            p.save_U[row] = u_new;
          }
        }
      }
      __syncthreads();
      const float u_new = *ufq;
#pragma unroll
      for (int k = 0; k < KV; ++k)
#pragma unroll
        for (int e = 0; e < VE; ++e) cacc[k][e] = fmaf(u_new, x[k][e], cacc[k][e]);
    } else {
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
    }
    if (p.track && cr == 0 && tid == ftid) {
      auto kahan = [](float& sum, float& comp, float v) {
        const float y = v - comp;
        const float t2 = sum + y;
        comp = (t2 - sum) - y;
        sum = t2;
      };
      if (p.t >= 2) kahan(err_num, err_num_c, fabsf(tot - p.r_prev[row]));
      kahan(err_den, err_den_c, tot);
      p.r_prev[row] = tot;
    }
    ++done_rows;
  }

  // Fold this CTA's column partials into the column sums of iteration t:
  // with vector reductions, or, in deterministic mode, by storing them (zeros
  // included) to this row group's slot, which a reduction launch adds to the
  // other slots in slot order.
  if (p.det) {
    float* slot = p.part + size_t(cid) * size_t(p.mpad);
#pragma unroll
    for (int k = 0; k < KV; ++k) {
      const int cc = col0 + (k * THREADS + tid) * VE;
      if (cc + VE <= m) {
#pragma unroll
        for (int e = 0; e < VE; e += 4)
          *reinterpret_cast<float4*>(slot + cc + e) =
              make_float4(cacc[k][e], cacc[k][e + 1], cacc[k][e + 2], cacc[k][e + 3]);
      } else {
#pragma unroll
        for (int e = 0; e < VE; ++e)
          if (cc + e < m) slot[cc + e] = cacc[k][e];
      }
    }
    if (cr == 0 && tid == ftid) {
      p.err_part[2 * cid] = double(err_num) - double(err_num_c);
      p.err_part[2 * cid + 1] = double(err_den) - double(err_den_c);
    }
  } else if (done_rows > 0) {
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
  if (p.track && !p.det && cr == 0 && tid == ftid && done_rows > 0) {
    atomicAdd(&p.err_next[0], double(err_num) - double(err_num_c));
    atomicAdd(&p.err_next[1], double(err_den) - double(err_den_c));
  }
  if (st) atomicOr(&ctl->status, st);

  // beta_t = (b_j / c_j)^fi for the next pass (kernel form: V <- V beta_t),
  // computed once per column by the CTAs that finish last, in slices, after
  // every CTA's column partials have landed (deterministic mode: by the
  // reduction launch that follows the pass; a row-sharded pass leaves the
  // column sums to be reduced across processes first).
  if (!p.det && !p.no_factors) {
    const int nsl = BETA_SLICES;
    const int per = (m + nsl - 1) / nsl;
    uint32_t st2 = 0;
    finish_pass_job(p.arrive, p.slice_ctr, nsl, BETA_CTAS, HELP_LOOK_NS, [&](int sl) {
      const int j0 = sl * per, j1 = min(m, j0 + per);
      for (int j = j0 + tid; j < j1; j += THREADS) {
        if constexpr (KF) {
          // V_j <- V_j (b_j / c_j)^fi 2^-e_t with c_j = V_j 2^-e_t sum_i U_i K_ij;
          // scaling-vector rule: v_j <- (b_j / sum_i U_i K_ij)^fi.
          const float v = __ldcg(p.beta_out + j);
          const float d = __ldcg(p.c_next + j);
          const float c = v * d * inv_gauge;
          const float v_new = p.pot ? rescale_factor(__ldg(p.b_ws + j), d, p.fi, st2)
                                    : v * rescale_factor(__ldg(p.b_ws + j), c, p.fi, st2) * inv_gauge;
          p.beta_out[j] = v_new;
          if (p.save_c) {  // history for the adjoint: c_t and V_t of this column
            p.save_c[j] = c;
            p.save_V[j] = v_new;
          }
        } else {
          p.beta_out[j] = rescale_factor(__ldg(p.b_ws + j), __ldcg(p.c_next + j), p.fi, st2);
        }
      }
    });
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

struct FusedEntry {
  FusedConfig cfg;
  const void* fn_tma;
  const void* fn_plain;
};

#define UOT_FUSED_ENTRY(T, DT, TH, KV, KFORM)                                             \
  FusedEntry {                                                                            \
    FusedConfig{DT, TH, KV, KV * (16 / int(sizeof(T))) * TH, 1},                          \
        reinterpret_cast<const void*>(&fused_pass_kernel<T, TH, KV, true, KFORM>),       \
        reinterpret_cast<const void*>(&fused_pass_kernel<T, TH, KV, false, KFORM>)       \
  }

#define UOT_FUSED_TABLE(KFORM)                                                            \
  {                                                                                       \
    UOT_FUSED_ENTRY(float, UOT_F32, 512, 8, KFORM),                                       \
    UOT_FUSED_ENTRY(float, UOT_F32, 512, 4, KFORM),                                       \
    UOT_FUSED_ENTRY(float, UOT_F32, 256, 4, KFORM),                                       \
    UOT_FUSED_ENTRY(float, UOT_F32, 128, 4, KFORM),                                       \
    UOT_FUSED_ENTRY(float, UOT_F32, 128, 2, KFORM),                                       \
    UOT_FUSED_ENTRY(float, UOT_F32, 64, 2, KFORM),                                        \
    UOT_FUSED_ENTRY(float, UOT_F32, 32, 2, KFORM),                                        \
    UOT_FUSED_ENTRY(__nv_bfloat16, UOT_BF16, 512, 4, KFORM),                              \
    UOT_FUSED_ENTRY(__nv_bfloat16, UOT_BF16, 256, 4, KFORM),                              \
    UOT_FUSED_ENTRY(__nv_bfloat16, UOT_BF16, 128, 4, KFORM),                              \
    UOT_FUSED_ENTRY(__nv_bfloat16, UOT_BF16, 128, 2, KFORM),                              \
    UOT_FUSED_ENTRY(__nv_bfloat16, UOT_BF16, 64, 2, KFORM),                               \
    UOT_FUSED_ENTRY(__nv_bfloat16, UOT_BF16, 32, 2, KFORM),                               \
    UOT_FUSED_ENTRY(__half, UOT_F16, 512, 4, KFORM),                                      \
    UOT_FUSED_ENTRY(__half, UOT_F16, 256, 4, KFORM),                                      \
    UOT_FUSED_ENTRY(__half, UOT_F16, 128, 4, KFORM),                                      \
    UOT_FUSED_ENTRY(__half, UOT_F16, 128, 2, KFORM),                                      \
    UOT_FUSED_ENTRY(__half, UOT_F16, 64, 2, KFORM),                                       \
    UOT_FUSED_ENTRY(__half, UOT_F16, 32, 2, KFORM),                                       \
  }

constexpr int kFusedConfigs = 19;
extern const FusedEntry kInplaceTable[kFusedConfigs];
extern const FusedEntry kKformTable[kFusedConfigs];

}  // namespace uot
