// Kernel-form pass, two rows per step.
//
// The same iteration as fused_pass_kernel<T, ..., KF = true> (the plan kept
// as diag(U) K diag(V), K read-only, FP32 scalings; one pass per iteration of
// Section 2.1's rule, Algorithm 1's single sweep) for K in FP32, BF16 or FP16
// when bulk copies apply.  With one row per step the fixed latency of a step
// (barrier, the row factor's power, the refill) bounds a read-only pass well
// below HBM bandwidth.  Here each step takes two rows: both row sums share one
// barrier, two threads of the last warp form the two row factors, and a
// second barrier hands them to every thread.  With HOLD each thread keeps
// its part of both rows in registers as packed 16-byte vectors for the
// column partials, so the first barrier already shows the slot fully read and
// it is refilled at once: every slot of the ring is loading while a step
// computes.  Without HOLD (where those registers would spill) the rows are
// read from shared memory a second time and a slot is refilled one step
// later, so one slot of the ring is held through each step.
//
// A row wider than one CTA is split over a cluster of cs CTAs (CTA rank r on
// columns [r W, (r+1) W)); the row partial sums go to every CTA of the
// cluster through distributed shared memory before a cluster barrier, and
// every CTA forms the same two factors.  With cs == 1 rows are taken in pairs
// from the pass's counter (the next pair fetched one step ahead), alternating
// direction between passes; clusters take pairs g, g + G, g + 2G, ...  The
// column factors of the next pass are formed by the CTAs that finish last
// (finish_pass_job).  The stopping rule's row sums are accumulated by the two
// factor threads of rank 0; so is the adjoint's history when it is kept.
#include <cuda_runtime.h>

#include <mutex>

#include "fused_kernel.cuh"

namespace uot {

namespace {

template <typename T, int THREADS, int KV, bool CL, bool HOLD>
__global__ void __launch_bounds__(THREADS, 1) kform_pair_kernel(const FusedArgs p) {
  using E = Elem<T>;
  constexpr int VE = E::VE;  // elements per 16-byte vector
  constexpr int NW = THREADS / 32;
  constexpr int W = KV * VE * THREADS;
  constexpr int ROW_BYTES = W * int(sizeof(T));
  constexpr int SLOT_BYTES = 2 * ROW_BYTES;
  constexpr int RQ = 2 * MAX_CLUSTER * NW;  // partials of one step: [row][rank][warp]

  extern __shared__ __align__(128) unsigned char smem[];
  const int stages = p.stages;
  unsigned char* ring = smem;
  float* red = reinterpret_cast<float*>(smem + size_t(stages) * SLOT_BYTES);  // [2][RQ]
  float* uf = red + 2 * RQ;                                                    // [2][2]
  uint64_t* bars = reinterpret_cast<uint64_t*>(uf + 4);
  int* slot_rows = reinterpret_cast<int*>(bars + stages);  // [stages][2]

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // CL: launched in clusters (a row split over cs CTAs).
  const uint32_t cs = CL ? cluster_nctarank() : 1u;
  const uint32_t cr = CL ? cluster_ctarank() : 0u;
  const int cid = CL ? int(cluster_id_x()) : int(blockIdx.x);
  const int ncl = CL ? int(ncluster_x()) : int(gridDim.x);
  Control* ctl = p.ctl;
  if (p.track) {
    if (*reinterpret_cast<volatile int32_t*>(&ctl->done)) return;
    if (p.check_prev) {
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

  const int m = p.m, n = p.n;
  const int col0 = int(cr) * W;
  float gauge = 1.0f, inv_gauge = 1.0f;
  {
    const int e = gauge_exponent(p.t, float(*p.log2k));
    gauge = ldexpf(1.0f, e);
    inv_gauge = ldexpf(1.0f, -e);
  }
  const int valid = max(0, min(W, m - col0));
  const uint32_t copy_bytes = uint32_t((size_t(valid) * sizeof(T)) & ~size_t(15));
  const T* plan = reinterpret_cast<const T*>(p.plan);
  const int64_t ldp = p.ldp;
  uint32_t st = 0;
  const uint64_t policy = policy_evict_first();
  const bool dyn = !CL;
  const int npairs = (n + 1) / 2;
  const int nq = cid < npairs ? (npairs - 1 - cid) / ncl + 1 : 0;  // static pairs
  int issued = 0, next_base = n;

  if (tid == 0) {
    for (int s2 = 0; s2 < stages; ++s2) mbar_init(&bars[s2], 1);
    fence_mbar_init();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  // All CTAs of the cluster run before distributed shared memory is written.
  if constexpr (CL) cluster_sync(); else __syncthreads();

  const bool flip = dyn && (p.t & 1) == 0;
  // Whole rows stored back to back: a step's two rows (adjacent, the lower
  // first) come in one bulk copy, and the second row follows the first in
  // the slot.  A bulk copy has a fixed cost of about 0.3 us on an SM's copy
  // engine, which caps copies of one 8 KB row each at ~27 GB/s per SM.
  const bool joint = !CL && size_t(m) * sizeof(T) == copy_bytes && ldp == m;
  const uint32_t rowb_off = joint ? copy_bytes : uint32_t(ROW_BYTES);
  // Arms the slot of step q with the rows base, base + 1 (those below n).
  auto arm = [&](int q, int base) {
    const int slot = q % stages;
    if (base >= 0 && base < n) {
      int ra = base, rb = base + 1 < n ? base + 1 : -1;
      if (flip) {
        ra = n - 1 - ra;
        if (rb >= 0) {  // keep the lower row first
          rb = ra;
          ra = ra - 1;
        }
      }
      slot_rows[2 * slot] = ra;
      slot_rows[2 * slot + 1] = rb;
      if (copy_bytes && joint && rb >= 0) {
        mbar_arrive_expect_tx(&bars[slot], 2u * copy_bytes);
        bulk_load(ring + size_t(slot) * SLOT_BYTES, plan + int64_t(ra) * ldp, 2u * copy_bytes,
                  &bars[slot], policy);
      } else if (copy_bytes) {
        mbar_arrive_expect_tx(&bars[slot], copy_bytes * (rb >= 0 ? 2u : 1u));
        bulk_load(ring + size_t(slot) * SLOT_BYTES, plan + int64_t(ra) * ldp + col0, copy_bytes,
                  &bars[slot], policy);
        if (rb >= 0)
          bulk_load(ring + size_t(slot) * SLOT_BYTES + rowb_off, plan + int64_t(rb) * ldp + col0,
                    copy_bytes, &bars[slot], policy);
      } else {
        mbar_arrive(&bars[slot]);
      }
    } else {
      slot_rows[2 * slot] = -1;
      mbar_arrive(&bars[slot]);
    }
  };
  auto static_base = [&](int q) { return q < nq ? 2 * (cid + q * ncl) : -1; };
  if (tid == 0) {
    if (dyn) {
      const int base = atomicAdd(p.row_ctr, 2 * stages);
      for (int q = 0; q < stages; ++q) arm(q, base + 2 * q);
      if (base + 2 * stages < n) next_base = atomicAdd(p.row_ctr, 2);
    } else {
      for (int q = 0; q < stages; ++q) arm(q, static_base(q));
    }
    issued = stages;
  }

  // Column scalings V of this thread's columns (zero-padded buffer).
  float V[KV][VE];
#pragma unroll
  for (int k = 0; k < KV; ++k) {
    const int cc = col0 + (k * THREADS + tid) * VE;
    if (cc < m) {
#pragma unroll
      for (int e = 0; e < VE; e += 4) {
        const float4 b4 = __ldcg(reinterpret_cast<const float4*>(p.beta + cc + e));
        V[k][e] = b4.x; V[k][e + 1] = b4.y; V[k][e + 2] = b4.z; V[k][e + 3] = b4.w;
      }
    } else {
#pragma unroll
      for (int e = 0; e < VE; ++e) V[k][e] = 0.0f;
    }
  }
  {
    const int g = blockIdx.x * THREADS + tid, gs = gridDim.x * THREADS;
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

  // Two factor threads in the last warp: THREADS-1 for the first row of a
  // step, THREADS-2 for the second.
  const int fh = THREADS - 1 - tid;  // 0 or 1 for the factor threads
  const bool factor_thread = fh == 0 || fh == 1;
  const bool writer = factor_thread && cr == 0;  // U, history and stopping sums
  float err_num = 0.0f, err_den = 0.0f, err_num_c = 0.0f, err_den_c = 0.0f;
  bool broken = false;
  int done_steps = 0;

  // Chunk k of a row as a packed 16-byte vector: the bulk-copied part from
  // the slot, the rest from global memory, columns >= m as zeros.
  auto load_raw = [&](const unsigned char* srow, int row, int k) -> uint4 {
    const int li = k * THREADS + tid;
    const int cc = li * VE;
    if ((cc + VE) * int(sizeof(T)) <= int(copy_bytes)) return ld_shared_v4(srow + size_t(li) * 16);
    float f[VE];
#pragma unroll
    for (int e = 0; e < VE; ++e)
      f[e] = (col0 + cc + e < m) ? E::load1(plan + int64_t(row) * ldp + col0 + cc + e) : 0.0f;
    return E::pack(f);  // exact: the values are elements of T
  };

  for (int q = 0;; ++q) {
    if (CL && q >= nq) break;
    const int slot = q % stages;
    if (!broken && !mbar_wait_bounded(&bars[slot], uint32_t(q / stages) & 1u, WAIT_LIMIT_NS)) {
      broken = true;
      st |= DEV_TIMEOUT;
    }
    const int ra = *reinterpret_cast<volatile int*>(&slot_rows[2 * slot]);
    if (ra < 0 || ra >= n) break;  // uniform: every thread reads the same slot
    const int rb = *reinterpret_cast<volatile int*>(&slot_rows[2 * slot + 1]);
    const bool lb = rb >= 0;
    const unsigned char* sbase = ring + size_t(slot) * SLOT_BYTES;
    // Row data of the factor threads' rows, loaded before the barrier.
    const int frow = fh == 0 ? ra : rb;
    float arow = 0.0f, u_old = 1.0f;
    if (factor_thread && frow >= 0) {
      arow = __ldg(p.a + frow);
      u_old = __ldcg(p.U + frow);
    }
    uint4 xa[KV], xb[KV];
#pragma unroll
    for (int k = 0; k < KV; ++k) {
      xa[k] = load_raw(sbase, ra, k);
      xb[k] = lb ? load_raw(sbase + rowb_off, rb, k) : make_uint4(0u, 0u, 0u, 0u);
    }
    // Row sums of K V: even and odd columns in the two lanes of a packed
    // FMA, added at the end.
    float2 pa = make_float2(0.0f, 0.0f), pb = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int k = 0; k < KV; ++k) {
      float fa[VE], fb[VE];
      E::unpack(xa[k], fa);
      E::unpack(xb[k], fb);
#pragma unroll
      for (int e = 0; e < VE; e += 2) {
        const float2 v2 = make_float2(V[k][e], V[k][e + 1]);
        pa = ffma2(make_float2(fa[e], fa[e + 1]), v2, pa);
        pb = ffma2(make_float2(fb[e], fb[e + 1]), v2, pb);
      }
    }
    float sa = warp_sum(pa.x + pa.y);
    float sb = warp_sum(pb.x + pb.y);
    float* rq = red + (q & 1) * RQ;
    if (lane == 0) {
      if constexpr (!CL) {
        rq[warp] = sa;
        rq[MAX_CLUSTER * NW + warp] = sb;
      } else {
        for (uint32_t r = 0; r < cs; ++r) {
          st_cluster_f32(map_shared_rank(rq + cr * NW + warp, r), sa);
          st_cluster_f32(map_shared_rank(rq + (MAX_CLUSTER + cr) * NW + warp, r), sb);
        }
      }
    }
    if constexpr (CL) {
      cluster_sync();  // static pairs: the loop is bounded by nq
    } else if (__syncthreads_or(broken ? 1 : 0)) {
      broken = true;
      st |= DEV_TIMEOUT;
      break;
    }
    auto refill = [&]() {
      if (dyn) {
        const int b2 = next_base;
        arm(issued, b2);
        if (b2 < n) next_base = atomicAdd(p.row_ctr, 2);
      } else {
        arm(issued, static_base(issued));
      }
      ++issued;
    };
    // HOLD: every thread of this CTA has its part of this step's rows in
    // registers (their sums are posted), so the slot is free.
    if (HOLD && tid == 0) refill();
    float* uq = uf + (q & 1) * 2;
    if (factor_thread && frow >= 0) {
      float s_kv = 0.0f;
      if constexpr (!CL) {
#pragma unroll
        for (int w = 0; w < NW; ++w) s_kv += rq[fh * MAX_CLUSTER * NW + w];
      } else {
        for (uint32_t r = 0; r < cs; ++r)
#pragma unroll
          for (int w = 0; w < NW; ++w) s_kv += rq[(fh * MAX_CLUSTER + int(r)) * NW + w];
      }
      const float rsum = u_old * s_kv;
      const float u_new = p.pot ? rescale_factor(arow * p.kscale, s_kv, p.fi, st) / p.kscale
                                : u_old * rescale_factor(arow, rsum, p.fi, st) * gauge;
      uq[fh] = u_new;
      if (writer) {
        p.U[frow] = u_new;
        if (p.save_r) {  // history for the adjoint: r_t and U_t of this row
          p.save_r[frow] = rsum;
          p.save_U[frow] = u_new;
        }
        if (p.track) {
          auto kahan = [](float& sum, float& comp, float v) {
            const float y = v - comp;
            const float t2 = sum + y;
            comp = (t2 - sum) - y;
            sum = t2;
          };
          if (p.t >= 2) kahan(err_num, err_num_c, fabsf(rsum - p.r_prev[frow]));
          kahan(err_den, err_den_c, rsum);
          p.r_prev[frow] = rsum;
        }
      }
    }
    __syncthreads();
    // Without HOLD the previous step's slot is no longer read by anyone
    // (every thread has passed this barrier after its second read of it).
    if (!HOLD && tid == 0 && q > 0) refill();
    const float ua = uq[0], ub = lb ? uq[1] : 0.0f;
#pragma unroll
    for (int k = 0; k < KV; ++k) {
      float fa[VE], fb[VE];
      if constexpr (HOLD) {
        E::unpack(xa[k], fa);
        E::unpack(xb[k], fb);
      } else {
        E::unpack(load_raw(sbase, ra, k), fa);
        E::unpack(lb ? load_raw(sbase + rowb_off, rb, k) : make_uint4(0u, 0u, 0u, 0u), fb);
      }
      const float2 ua2 = make_float2(ua, ua), ub2 = make_float2(ub, ub);
#pragma unroll
      for (int e = 0; e < VE; e += 2) {
        float2 c2 = make_float2(cacc[k][e], cacc[k][e + 1]);
        c2 = ffma2(ub2, make_float2(fb[e], fb[e + 1]), ffma2(ua2, make_float2(fa[e], fa[e + 1]), c2));
        cacc[k][e] = c2.x;
        cacc[k][e + 1] = c2.y;
      }
    }
    ++done_steps;
  }

  if (done_steps > 0) {
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
  if (p.track && writer && done_steps > 0) {
    atomicAdd(&p.err_next[0], double(err_num) - double(err_num_c));
    atomicAdd(&p.err_next[1], double(err_den) - double(err_den_c));
  }
  if (st) atomicOr(&ctl->status, st);

  // V_t for the next pass, once per column by the CTAs that finish last.
  {
    const int nsl = BETA_SLICES;
    const int per = (m + nsl - 1) / nsl;
    uint32_t st2 = 0;
    finish_pass_job(p.arrive, p.slice_ctr, nsl, BETA_CTAS, HELP_LOOK_NS, [&](int sl) {
      const int j0 = sl * per, j1 = min(m, j0 + per);
      for (int j = j0 + tid; j < j1; j += THREADS) {
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
      }
    });
    if (st2) atomicOr(&ctl->status, st2);
  }

  if (tid == 0 && broken) {
    for (int q = max(0, issued - stages); q < issued; ++q)
      mbar_wait_bounded(&bars[q % stages], uint32_t(q / stages) & 1u, WAIT_LIMIT_NS);
  }
}

struct PairEntry {
  int dtype, threads, kv;
  const void* fn;     // one CTA per row
  const void* fn_cl;  // rows split over a cluster
};

#define UOT_PAIR_ENTRY(T, DT, TH, KV, H)                                                \
  PairEntry {                                                                           \
    DT, TH, KV, reinterpret_cast<const void*>(&kform_pair_kernel<T, TH, KV, false, H>), \
        reinterpret_cast<const void*>(&kform_pair_kernel<T, TH, KV, true, H>)             \
  }

// Configurations whose two-row slot leaves room for a ring of three.  Rows
// are held in registers (HOLD) except in the 16-bit configuration of 16384
// columns, where V, the column partials and two rows would need more than
// the 128 registers a thread of a 512-thread CTA may have.
// 16-bit rows of up to 8192 columns take 512 x 2 with HOLD (45 us per pass
// at 8192^2, against 65 us for 256 x 4 re-reading its rows).
const PairEntry kPairTable[] = {
    UOT_PAIR_ENTRY(float, UOT_F32, 512, 4, true),
    UOT_PAIR_ENTRY(float, UOT_F32, 256, 4, true),
    UOT_PAIR_ENTRY(float, UOT_F32, 128, 4, true),
    UOT_PAIR_ENTRY(float, UOT_F32, 128, 2, true),
    UOT_PAIR_ENTRY(float, UOT_F32, 64, 2, true),
    UOT_PAIR_ENTRY(float, UOT_F32, 32, 2, true),
    UOT_PAIR_ENTRY(__nv_bfloat16, UOT_BF16, 512, 4, false),
    UOT_PAIR_ENTRY(__nv_bfloat16, UOT_BF16, 512, 2, true),
    UOT_PAIR_ENTRY(__nv_bfloat16, UOT_BF16, 128, 4, true),
    UOT_PAIR_ENTRY(__nv_bfloat16, UOT_BF16, 128, 2, true),
    UOT_PAIR_ENTRY(__nv_bfloat16, UOT_BF16, 64, 2, true),
    UOT_PAIR_ENTRY(__nv_bfloat16, UOT_BF16, 32, 2, true),
    UOT_PAIR_ENTRY(__half, UOT_F16, 512, 4, false),
    UOT_PAIR_ENTRY(__half, UOT_F16, 512, 2, true),
    UOT_PAIR_ENTRY(__half, UOT_F16, 128, 4, true),
    UOT_PAIR_ENTRY(__half, UOT_F16, 128, 2, true),
    UOT_PAIR_ENTRY(__half, UOT_F16, 64, 2, true),
    UOT_PAIR_ENTRY(__half, UOT_F16, 32, 2, true),
};
constexpr int kPairConfigs = int(sizeof(kPairTable) / sizeof(kPairTable[0]));

size_t pair_smem(const PairEntry& e, int stages) {
  const size_t row = size_t(e.kv) * 16 * e.threads;
  return size_t(stages) * 2 * row + (2 * 2 * MAX_CLUSTER * (e.threads / 32) + 4) * sizeof(float) +
         size_t(stages) * 8 + size_t(stages) * 2 * sizeof(int);
}

int pair_cols(const PairEntry& e) {
  return e.threads * e.kv * (e.dtype == UOT_F32 ? 4 : 8);
}

std::mutex g_pair_mu;
constexpr int PAIR_MAX_DEV = 64;
size_t g_pair_smem_set[PAIR_MAX_DEV][kPairConfigs][2];
bool g_pair_cluster_set[PAIR_MAX_DEV][kPairConfigs];
struct PairGeo {
  int dev, k, cs, n, grid, stages;
  size_t smem;
};
PairGeo g_pair_geo[32];
int g_pair_geo_used = 0, g_pair_geo_next = 0;

cudaError_t pair_attributes(int dev, int i, size_t smem, bool cluster) {
  const PairEntry& e = kPairTable[i];
  const void* fn = cluster ? e.fn_cl : e.fn;
  std::lock_guard<std::mutex> lock(g_pair_mu);
  if (g_pair_smem_set[dev][i][cluster] < smem) {
    cudaError_t err = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (err != cudaSuccess) return err;
    g_pair_smem_set[dev][i][cluster] = smem;
  }
  if (cluster && !g_pair_cluster_set[dev][i]) {
    cudaError_t err = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (err != cudaSuccess) return err;
    g_pair_cluster_set[dev][i] = true;
  }
  return cudaSuccess;
}

}  // namespace

int kform_pair_pick(int dtype, int64_t m, int* cs) {
  // The narrowest configuration that covers the row, else the widest one
  // split over a cluster.
  int best = -1, widest = -1;
  for (int i = 0; i < kPairConfigs; ++i) {
    const PairEntry& e = kPairTable[i];
    if (e.dtype != dtype) continue;
    if (widest < 0 || pair_cols(e) > pair_cols(kPairTable[widest])) widest = i;
    if (pair_cols(e) >= m && (best < 0 || pair_cols(e) < pair_cols(kPairTable[best]))) best = i;
  }
  if (best >= 0) {
    *cs = 1;
    return best;
  }
  // Wider FP32 rows measured faster with the one-row pass of 16384 columns
  // per CTA than split over clusters of two-row CTAs of 8192; wider 16-bit
  // rows faster over clusters of the 16384-column configuration than of the
  // 8192-column one that holds its rows (540 against 833 us at 32768^2).
  if (widest < 0 || dtype == UOT_F32) return -1;
  const int64_t c = (m + pair_cols(kPairTable[widest]) - 1) / pair_cols(kPairTable[widest]);
  if (c > MAX_CLUSTER) return -1;
  *cs = int(c);
  return widest;
}

cudaError_t kform_pair_geometry(int i, int cs, int n, int* grid, int* stages, size_t* smem) {
  const PairEntry& e = kPairTable[i];
  int dev = 0, sms = 0, optin = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  if (dev < 0 || dev >= PAIR_MAX_DEV) return cudaErrorInvalidDevice;
  {
    std::lock_guard<std::mutex> lock(g_pair_mu);
    for (int j = 0; j < g_pair_geo_used; ++j) {
      const PairGeo& g = g_pair_geo[j];
      if (g.dev == dev && g.k == i && g.cs == cs && g.n == n) {
        *grid = g.grid;
        *stages = g.stages;
        *smem = g.smem;
        return cudaSuccess;
      }
    }
  }
  err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (err != cudaSuccess) return err;
  err = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (err != cudaSuccess) return err;
  // Deepest ring that keeps the CTA count per SM of a two-slot ring.
  int occ2 = 0, best_s = 2;
  for (int s = 2; s <= 8; ++s) {
    const size_t b = pair_smem(e, s);
    if (b > size_t(optin)) break;
    err = pair_attributes(dev, i, b, cs > 1);
    if (err != cudaSuccess) return err;
    int occ = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, cs > 1 ? e.fn_cl : e.fn, e.threads, b);
    if (err != cudaSuccess) return err;
    if (s == 2) occ2 = occ;
    if (occ < occ2 || occ == 0) break;
    best_s = s;
  }
  if (occ2 == 0) return cudaErrorInvalidConfiguration;
  *stages = best_s;
  *smem = pair_smem(e, best_s);
  int clusters = occ2 * sms;
  if (cs > 1) {
    err = pair_attributes(dev, i, *smem, true);
    if (err != cudaSuccess) return err;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(cs * occ2 * sms, 1, 1);
    cfg.blockDim = dim3(e.threads, 1, 1);
    cfg.dynamicSmemBytes = *smem;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nc = 0;
    err = cudaOccupancyMaxActiveClusters(&nc, e.fn_cl, &cfg);
    if (err != cudaSuccess) return err;
    if (nc <= 0) return cudaErrorInvalidConfiguration;
    clusters = nc;
  }
  const int cap = (n + 3) / 4;  // at least two pairs of rows per cluster
  if (clusters > cap) clusters = cap > 0 ? cap : 1;
  *grid = clusters * cs;
  std::lock_guard<std::mutex> lock(g_pair_mu);
  const int slot = g_pair_geo_used < 32 ? g_pair_geo_used++ : (g_pair_geo_next++ % 32);
  g_pair_geo[slot] = PairGeo{dev, i, cs, n, *grid, *stages, *smem};
  return cudaSuccess;
}

cudaError_t kform_pair_launch(int i, int cs, int grid, size_t smem, const FusedArgs& args,
                              cudaStream_t s) {
  const PairEntry& e = kPairTable[i];
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(grid, 1, 1);
  cfg.blockDim = dim3(e.threads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = cs > 1 ? 1 : 0;
  FusedArgs a = args;
  void* kargs[] = {&a};
  cudaError_t err = cudaLaunchKernelExC(&cfg, cs > 1 ? e.fn_cl : e.fn, kargs);
  if (err == cudaSuccess) count_launch();
  return err;
}

}  // namespace uot
