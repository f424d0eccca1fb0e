// Batched Sinkhorn-UOT, streaming form: many independent problems of uneven
// size in one persistent launch (the rule of Section 2.1 with Algorithm 1's
// single sweep per iteration).  Each problem runs in kernel form: during the
// iterations the plan buffer holds the initial plan K read-only and only the
// FP32 scalings change (plan = diag(U) K diag(V)); the final sweep writes
// the plan over K.  Compared with rescaling the plan in place this reads 4
// instead of moving 8 bytes per element per iteration, and no plan entry
// accumulates two roundings per iteration.  (Problems small enough for the
// shared memory of a cluster run in the on-chip engine instead.)
//
// Scheduling.  Problems are sorted into size classes; class c is served by
// teams of G_c CTAs (G_c a power of two, larger for larger problems).  Teams
// are aligned blocks of G_c consecutive CTAs, and a CTA walks the classes
// from the largest team size down: while its team of the current class is
// complete, the team leader takes the next problem of that class from a
// largest-first queue (an atomic cursor) and hands it to the members through
// a mailbox.  When a class queue runs dry the team splits into the teams of
// the next class.  The host picks the classes (the autotuner varies the
// target work per CTA and the ring depth).
//
// Per problem.  CTA r of a team owns the contiguous rows [r nb, (r+1) nb),
// nb = ceil(N / G), for all iterations, and keeps their scalings U and
// marginals a in shared memory.  Each step moves 2R rows (R = 256 / GT row
// groups of GT threads, GT the smallest power of two with 16 GT >= M; at most
// 32 KB) into a ring slot with 1-D bulk copies issued by one warp; each
// thread covers 4 16-byte chunks of two rows, holding its columns' scalings V
// and column partial sums in registers.  A step: partial row sums (shuffles,
// one partial per warp), barrier, one thread per row forms the row factor
// (one power per row rather than one per thread), barrier, column partials
// of U_i K_ij.  Once per iteration the row groups'
// partials are combined in shared memory and folded into the problem's
// column sums with vector reductions, the team meets at a software barrier
// (bounded spin), and the CTA updates V for all columns (one thread per
// column).  The final sweep writes diag(U) K diag(V).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "batched_internal.h"
#include "uot_device.cuh"
#include "uot_internal.h"

namespace uot {

namespace {

constexpr int BT = 256;           // threads per CTA
constexpr int BKV = 4;            // 16-byte vectors per thread per row
constexpr int BW = BT * BKV * 4;  // widest row (FP32 columns)
constexpr int MAX_CLASSES = 8;
constexpr int MAX_RES_CLASSES = 5;  // on-chip cluster sizes 1, 2, 4, 8, 16
constexpr int CURSORS = MAX_CLASSES + MAX_RES_CLASSES;
constexpr int MAX_STAGES = 6;
constexpr int SLOT_BYTES = 2 * BT * BKV * 16;  // two rows per row group
constexpr int ROWS_MAX = 1024;                 // rows one CTA owns

struct BatchSched {
  int nprob;
  int nclass;
  int stages;
  int class_g[MAX_CLASSES];
  int class_begin[MAX_CLASSES];
  int class_end[MAX_CLASSES];
  int team_base[MAX_CLASSES];  // offset of this class's teams in the team arrays
  const BatchProblem* probs;
  const int* order;      // problem indices, by class, largest first
  int* cursor;           // [MAX_CLASSES] queue positions
  int* mailbox;          // [teams] problem handed to the team
  int* bar;              // [teams][2] barrier arrival count, unused
};

struct BatchHeader {  // at the start of the batched workspace (for inspection)
  int nprob;
  int teams;
  int64_t probs_off, order_off, cursor_off, mailbox_off, bar_off, sched_off;
  int64_t total;
};

// Team barrier over G CTAs (G > 1), bounded: one monotonic arrival counter
// per team; the e-th barrier of a team completes when the counter reaches
// e * G.  The release reduction publishes the CTA's earlier writes (ordered
// before it by the CTA barrier), the acquire loads see the other CTAs'.
__device__ bool team_barrier(int* count, int G, int& epoch, uint32_t& st) {
  __syncthreads();
  bool ok = true;
  ++epoch;
  if (threadIdx.x == 0) {
    const int target = epoch * G;
    red_release_gpu_add(count, 1);
    const uint64_t t0 = global_timer_ns();
    while (ld_acquire_gpu(count) < target) {
      if (global_timer_ns() - t0 > WAIT_LIMIT_NS) {
        st |= DEV_TIMEOUT;
        ok = false;
        break;
      }
    }
  }
  return __syncthreads_and(ok ? 1 : 0) != 0;
}

__device__ __forceinline__ float4 lds4(const void* p) {
  return *reinterpret_cast<const float4*>(p);
}

// One sweep over this CTA's rows [r0, r0 + nloc) of problem P.  The plan
// buffer holds K during the iterations; U (Us) and a (As) of the rows are in
// shared memory, V in registers.  Iteration sweep: r_i = U_i sum_j K_ij V_j,
// U_i <- U_i alpha_i gauge, column partials of U_i K_ij into c_next.  Final
// sweep: P_ij = (K_ij V_j) U_i written over K.
__device__ void sweep(const BatchProblem& P, bool finish, const float (&V)[BKV][4], float gauge,
                      int r0, int nloc, float* c_next, float* Us, const float* As, int stages,
                      unsigned char* ring, uint64_t* full, float* rp, float* uf, int& qbase,
                      uint32_t& st, bool& broken) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int m = P.m;
  const int ldk = (m + 3) & ~3, c4 = ldk >> 2;
  int gt = 1;
  while (gt * BKV < c4) gt <<= 1;  // threads per row
  const int R = BT / gt, RS = 2 * R;
  const int g = tid / gt, l = tid - g * gt;
  const int wr = gt < 32 ? gt : 32;  // lanes of one row within a warp
  const int wpg = gt > 32 ? gt >> 5 : 1;  // warps per row group
  const int wg = warp % wpg;              // this warp's place in its group
  const uint32_t row_bytes = uint32_t(ldk) * 4;  // 16-byte multiple; padding lies in ldp
  const int nsteps = (nloc + RS - 1) / RS;
  const int64_t ldp = P.ldp;
  float* plan = P.plan;
  const float fi = P.fi;

  float cacc[BKV][4];
#pragma unroll
  for (int k = 0; k < BKV; ++k)
#pragma unroll
    for (int e = 0; e < 4; ++e) cacc[k][e] = 0.0f;

  // The ring was last written through the generic proxy (column sums, V);
  // order that before the bulk copies that refill it.
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  // Warp 0 fills ring slots: one expect-tx arrival, then a bulk copy per row
  // spread over the lanes.  Steps are numbered across sweeps (qbase) so the
  // mbarrier phases continue.
  const uint64_t policy = policy_evict_normal();
  // Rows stored without padding beyond the 16-byte rounding are contiguous:
  // one copy per step.
  const bool packed = ldp == ldk;
  auto arm = [&](int ql) {
    const int slot = (qbase + ql) % stages;
    const int rb = ql * RS;
    const int rows = min(RS, nloc - rb);
    unsigned char* dst = ring + size_t(slot) * SLOT_BYTES;
    const float* src = plan + int64_t(r0 + rb) * ldp;
    if (packed) {
      if (lane == 0) {
        mbar_arrive_expect_tx(&full[slot], uint32_t(rows) * row_bytes);
        bulk_load(dst, src, uint32_t(rows) * row_bytes, &full[slot], policy);
      }
      return;
    }
    if (lane == 0) mbar_arrive_expect_tx(&full[slot], uint32_t(rows) * row_bytes);
    __syncwarp();
    for (int r = lane; r < rows; r += 32)
      bulk_load(dst + size_t(r) * row_bytes, src + int64_t(r) * ldp, row_bytes, &full[slot], policy);
  };
  int armed = min(stages, nsteps);
  if (warp == 0)
    for (int ql = 0; ql < armed; ++ql) arm(ql);

  const bool ragged = (m & 3) != 0;
  int ql = 0;
  for (; ql < nsteps; ++ql) {
    const int q = qbase + ql;
    const int slot = q % stages;
    if (!broken && !mbar_wait_bounded(&full[slot], uint32_t(q / stages) & 1u, WAIT_LIMIT_NS)) {
      broken = true;
      st |= DEV_TIMEOUT;
    }
    const int ia = ql * RS + g, ib = ia + R;  // local rows of this group
    const bool la = ia < nloc, lb = ib < nloc;
    const unsigned char* sa_ = ring + size_t(slot) * SLOT_BYTES + size_t(g) * row_bytes;
    const unsigned char* sb_ = sa_ + size_t(R) * row_bytes;
    float xa[BKV][4], xb[BKV][4];
    float pa = 0.0f, pb = 0.0f;
#pragma unroll
    for (int k = 0; k < BKV; ++k) {
      const int ch = l + k * gt;
      const bool cv = ch < c4;
      const float4 va = (cv && la) ? lds4(sa_ + size_t(ch) * 16) : make_float4(0.f, 0.f, 0.f, 0.f);
      const float4 vb = (cv && lb) ? lds4(sb_ + size_t(ch) * 16) : make_float4(0.f, 0.f, 0.f, 0.f);
      xa[k][0] = va.x; xa[k][1] = va.y; xa[k][2] = va.z; xa[k][3] = va.w;
      xb[k][0] = vb.x; xb[k][1] = vb.y; xb[k][2] = vb.z; xb[k][3] = vb.w;
      if (ragged && ch == c4 - 1) {  // the copy ran past column m - 1 into padding
#pragma unroll
        for (int e = 1; e < 4; ++e)
          if (ch * 4 + e >= m) {
            xa[k][e] = 0.0f;
            xb[k][e] = 0.0f;
          }
      }
      pa = fmaf(xa[k][3], V[k][3], fmaf(xa[k][2], V[k][2], fmaf(xa[k][1], V[k][1], fmaf(xa[k][0], V[k][0], pa))));
      pb = fmaf(xb[k][3], V[k][3], fmaf(xb[k][2], V[k][2], fmaf(xb[k][1], V[k][1], fmaf(xb[k][0], V[k][0], pb))));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      if (o < wr) {
        pa += __shfl_xor_sync(0xffffffffu, pa, o);
        pb += __shfl_xor_sync(0xffffffffu, pb, o);
      }
    }
    // One partial per warp and row of the step.
    if ((lane & (wr - 1)) == 0) {
      rp[g * wpg + wg] = pa;
      rp[(g + R) * wpg + wg] = pb;
    }
    if (__syncthreads_or(broken ? 1 : 0)) {
      broken = true;
      st |= DEV_TIMEOUT;
      break;
    }
    // Every thread holds this slot's rows in registers: refill it.  Every
    // thread counts the armed steps (the phase bookkeeping of later sweeps).
    if (ql + stages < nsteps) {
      if (warp == 0) arm(ql + stages);
      ++armed;
    }
    // Row factors, one thread per row of the step: U_i <- U_i alpha_i gauge
    // with r_i = U_i sum_j K_ij V_j (the final sweep only reads U_i).  The
    // threads are counted from the last warp, so that warp 0's refill and
    // the factors' latency overlap.
    for (int r = BT - 1 - tid; r >= 0 && r < RS; r += BT) {
      const int i = ql * RS + r;
      if (i < nloc) {
        const float u_old = Us[i];
        if (finish) {
          uf[r] = u_old;
        } else {
          float sum = 0.0f;
          for (int w = 0; w < wpg; ++w) sum += rp[r * wpg + w];
          const float u_new = P.pot ? rescale_factor(As[i], sum, fi, st)
                                    : u_old * rescale_factor(As[i], u_old * sum, fi, st) * gauge;
          Us[i] = u_new;
          uf[r] = u_new;
        }
      }
    }
    __syncthreads();
    const float fa = la ? uf[g] : 0.0f, fb = lb ? uf[g + R] : 0.0f;
    if (finish) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const bool live = h == 0 ? la : lb;
        if (!live) continue;
        const float u = h == 0 ? fa : fb;
        float* grow = plan + int64_t(r0 + (h == 0 ? ia : ib)) * ldp;
#pragma unroll
        for (int k = 0; k < BKV; ++k) {
          const int cc = (l + k * gt) * 4;
          if (cc >= m) continue;
          float y[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) y[e] = ((h == 0 ? xa[k][e] : xb[k][e]) * V[k][e]) * u;
          if (cc + 4 <= m) {
            st_global_cs_v4(grow + cc, Elem<float>::pack(y));
          } else {
#pragma unroll
            for (int e = 0; e < 4; ++e)
              if (cc + e < m) grow[cc + e] = y[e];
          }
        }
      }
      continue;
    }
#pragma unroll
    for (int k = 0; k < BKV; ++k)
#pragma unroll
      for (int e = 0; e < 4; ++e) cacc[k][e] = fmaf(fb, xb[k][e], fmaf(fa, xa[k][e], cacc[k][e]));
  }
  if (broken) {
    // Copies of abandoned steps: wait for them (bounded) before the ring
    // may be reused or the CTA exits.
    for (int q2 = qbase + ql; q2 < qbase + armed; ++q2)
      mbar_wait_bounded(&full[q2 % stages], uint32_t(q2 / stages) & 1u, WAIT_LIMIT_NS);
  }
  qbase += armed;
  if (finish || broken) return;
  // Combine the R row groups' column partials (they cover the same columns)
  // in the idle ring: groups [R/2, R) hand theirs to groups [0, R/2), then
  // one thread per 4 columns sums the R/2 pair sums into the column sums.
  __syncthreads();
  float* W = reinterpret_cast<float*>(ring);
  const int half = R / 2;
  if (half == 0) {
#pragma unroll
    for (int k = 0; k < BKV; ++k) {
      const int ch = l + k * gt;
      if (ch < c4)
        *reinterpret_cast<float4*>(W + ch * 4) =
            make_float4(cacc[k][0], cacc[k][1], cacc[k][2], cacc[k][3]);
    }
  } else {
    if (g >= half) {
#pragma unroll
      for (int k = 0; k < BKV; ++k) {
        const int ch = l + k * gt;
        if (ch < c4)
          *reinterpret_cast<float4*>(W + size_t(g - half) * ldk + ch * 4) =
              make_float4(cacc[k][0], cacc[k][1], cacc[k][2], cacc[k][3]);
      }
    }
    __syncthreads();
    if (g < half) {
#pragma unroll
      for (int k = 0; k < BKV; ++k) {
        const int ch = l + k * gt;
        if (ch < c4) {
          float4* w = reinterpret_cast<float4*>(W + size_t(g) * ldk + ch * 4);
          const float4 o = *w;
          *w = make_float4(cacc[k][0] + o.x, cacc[k][1] + o.y, cacc[k][2] + o.z, cacc[k][3] + o.w);
        }
      }
    }
  }
  __syncthreads();
  const int copies = half > 0 ? half : 1;
  for (int ch = tid; ch < c4; ch += BT) {
    float4 s4 = lds4(W + ch * 4);
    for (int u = 1; u < copies; ++u) {
      const float4 o = lds4(W + size_t(u) * ldk + ch * 4);
      s4.x += o.x;
      s4.y += o.y;
      s4.z += o.z;
      s4.w += o.w;
    }
    const int cc = ch * 4;
    if (cc + 4 <= m) {
      red_add_v4(c_next + cc, s4.x, s4.y, s4.z, s4.w);
    } else {
      const float v4[4] = {s4.x, s4.y, s4.z, s4.w};
      for (int e = 0; e < 4; ++e)
        if (cc + e < m) atomicAdd(c_next + cc + e, v4[e]);
    }
  }
}

__global__ void __launch_bounds__(BT, 2) batched_kernel(const BatchSched S) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int stages = S.stages;
  unsigned char* ring = smem;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + size_t(stages) * SLOT_BYTES);
  float* Us = reinterpret_cast<float*>(full + MAX_STAGES);
  float* As = Us + ROWS_MAX;
  float* rp = As + ROWS_MAX;  // row-sum partials of a step (rows x warps per row)
  float* uf = rp + 2 * BT;    // row factors of a step
  __shared__ int s_prob;
  const int tid = threadIdx.x;
  uint32_t st = 0;
  bool broken = false;
  int qbase = 0;  // ring steps consumed so far (mbarrier phase bookkeeping)

  if (tid == 0) {
    for (int s = 0; s < MAX_STAGES; ++s) mbar_init(&full[s], 1);
    fence_mbar_init();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();

  for (int c = 0; c < S.nclass && !broken; ++c) {
    const int G = S.class_g[c];
    const int team = blockIdx.x / G;
    if ((team + 1) * G > int(gridDim.x)) continue;  // incomplete team
    const int rank = blockIdx.x % G;
    int* bar = S.bar + 2 * (S.team_base[c] + team);
    int epoch = 0;  // barriers of this team passed so far
    int* mbox = S.mailbox + S.team_base[c] + team;
    while (true) {
      // The leader takes the next problem of this class and hands it over.
      if (rank == 0 && tid == 0) {
        const int pos = atomicAdd(S.cursor + c, 1);
        const int idx = S.class_begin[c] + pos < S.class_end[c] ? S.order[S.class_begin[c] + pos] : -1;
        if (G > 1) *reinterpret_cast<volatile int*>(mbox) = idx;
        s_prob = idx;
      }
      if (G > 1) {
        if (!team_barrier(bar, G, epoch, st)) { broken = true; break; }
        if (tid == 0) s_prob = ld_acquire_gpu(mbox);
      }
      __syncthreads();
      const int pi = s_prob;
      if (pi < 0) break;
      const BatchProblem P = S.probs[pi];
      const int m = P.m;
      const int ldk = (m + 3) & ~3, c4 = ldk >> 2;
      int gt = 1;
      while (gt * BKV < c4) gt <<= 1;
      const int l = tid % gt;
      // This CTA's rows, their scalings and marginals.
      const int nb = (P.n + G - 1) / G;
      const int r0 = min(P.n, rank * nb);
      const int nloc = max(0, min(P.n - r0, nb));
      for (int i = tid; i < nloc; i += BT) {
        Us[i] = 1.0f;
        As[i] = __ldg(P.a + r0 + i);
      }
      // Column scalings V of this thread's columns, in registers (every row
      // group and every CTA of the team holds the same values).
      float V[BKV][4];
#pragma unroll
      for (int k = 0; k < BKV; ++k)
#pragma unroll
        for (int e = 0; e < 4; ++e) V[k][e] = ((l + k * gt) * 4 + e < m) ? 1.0f : 0.0f;
      const float Lf = float(*P.log2k);
      float gauge = 1.0f, inv_gauge = 1.0f;
      for (int t = 1; t <= P.iters + 1 && !broken; ++t) {
        const bool finish = t == P.iters + 1;
        if (t > 1) {
          // V_j <- V_j (b_j / c_j)^fi 2^-e_{t-1}, c_j = V_j 2^-e_{t-1} sum_i U_i K_ij:
          // one thread per column, through the idle ring.
          float* Vsm = reinterpret_cast<float*>(ring);
          if (tid < gt) {
#pragma unroll
            for (int k = 0; k < BKV; ++k) {
              const int ch = l + k * gt;
              if (ch < c4)
                *reinterpret_cast<float4*>(Vsm + ch * 4) = make_float4(V[k][0], V[k][1], V[k][2], V[k][3]);
            }
          }
          __syncthreads();
          const float* cprev = P.c + size_t((t - 1) % 3) * P.mpad;
          constexpr int VB = 8;  // columns per thread in flight
          for (int j0 = tid; j0 < m; j0 += VB * BT) {
            float cv[VB], bv[VB];
#pragma unroll
            for (int u = 0; u < VB; ++u) {
              const int j = j0 + u * BT;
              cv[u] = j < m ? __ldcg(cprev + j) : 0.0f;
              bv[u] = j < m ? __ldg(P.b + j) : 0.0f;
            }
#pragma unroll
            for (int u = 0; u < VB; ++u) {
              const int j = j0 + u * BT;
              if (j < m) {
                const float v = Vsm[j];
                const float cj = v * cv[u] * inv_gauge;
                Vsm[j] = P.pot ? rescale_factor(bv[u], cv[u], P.fi, st)
                               : v * rescale_factor(bv[u], cj, P.fi, st) * inv_gauge;
              }
            }
          }
          __syncthreads();
#pragma unroll
          for (int k = 0; k < BKV; ++k) {
            const int ch = l + k * gt;
            if (ch < c4) {
              const float4 v4 = lds4(Vsm + ch * 4);
              V[k][0] = v4.x;
              V[k][1] = v4.y;
              V[k][2] = v4.z;
              V[k][3] = v4.w;
            }
          }
        }
        if (!finish) {
          const int ex = gauge_exponent(t, Lf);
          gauge = ldexpf(1.0f, ex);
          inv_gauge = ldexpf(1.0f, -ex);
        }
        // Clear the column sums of iteration t + 1 (leader CTA).
        if (rank == 0) {
          float* cl = P.c + size_t((t + 1) % 3) * P.mpad;
          for (int j = tid; j < P.mpad; j += BT) cl[j] = 0.0f;
        }
        sweep(P, finish, V, gauge, r0, nloc, P.c + size_t(t % 3) * P.mpad, Us, As, stages, ring,
              full, rp, uf, qbase, st, broken);
        if (G > 1) {
          if (!team_barrier(bar, G, epoch, st)) { broken = true; break; }
        } else {
          __syncthreads();
        }
      }
      if (rank == 0 && tid == 0) P.ctl->iters_done = broken ? 0 : P.iters;
      if (st && tid == 0) atomicOr(&P.ctl->status, st);
      st = 0;
    }
  }
}

__global__ void batched_reset_kernel(const BatchProblem* probs, int nprob, int* cursor,
                                     int* mailbox, int* bar, int nteams) {
  const int p = blockIdx.x;
  if (p < nprob) {
    const BatchProblem P = probs[p];
    for (int j = threadIdx.x; j < 3 * P.mpad; j += blockDim.x) P.c[j] = 0.0f;
    if (threadIdx.x < 3) P.ctr[threadIdx.x] = 0;
    for (int i = threadIdx.x; i < P.n; i += blockDim.x) P.U[i] = 1.0f;
    // log2 k, k = (sum a / sum b)^(fi / (2 - fi)): the fixed-point row factor.
    __shared__ double part[2][32];
    double sa = 0.0, sb = 0.0;
    for (int i = threadIdx.x; i < P.n; i += blockDim.x) sa += P.a[i];
    for (int j = threadIdx.x; j < P.m; j += blockDim.x) sb += P.b[j];
    sa = warp_sum_d(sa);
    sb = warp_sum_d(sb);
    if ((threadIdx.x & 31) == 0) {
      part[0][threadIdx.x >> 5] = sa;
      part[1][threadIdx.x >> 5] = sb;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double ta = 0.0, tb = 0.0;
      for (int w = 0; w < int(blockDim.x >> 5); ++w) {
        ta += part[0][w];
        tb += part[1][w];
      }
      const double f = double(P.fi);
      const double Lk = (f / (2.0 - f)) * log2(ta / tb);
      *P.log2k = (!P.pot && ta > 0.0 && tb > 0.0 && isfinite(Lk)) ? Lk : 0.0;
    }
    if (threadIdx.x == 0) {
      P.ctl->status = 0;
      P.ctl->done = 0;
      P.ctl->stop_iter = 0;
      P.ctl->iters_done = 0;
      P.ctl->err = __longlong_as_double(0x7ff0000000000000ll);
    }
  }
  if (p == 0) {
    for (int i = threadIdx.x; i < CURSORS; i += blockDim.x) cursor[i] = 0;
    for (int i = threadIdx.x; i < nteams; i += blockDim.x) {
      mailbox[i] = -1;
      bar[2 * i] = 0;
      bar[2 * i + 1] = 0;
    }
  }
}

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

size_t batched_smem(int stages) {
  return size_t(stages) * SLOT_BYTES + MAX_STAGES * 8 + 2 * ROWS_MAX * 4 + 2 * (2 * BT) * 4;
}

}  // namespace

// ---------------------------------------------------------------- host side
// Workspace layout: header | BatchSched | problems | order | cursor | mailbox
// | bar | Control[nprob] | per-problem regions (3 x mpad column sums, counters).

static size_t per_problem_bytes(int64_t n, int64_t m) {
  const int64_t mpad = (m + 63) & ~int64_t(63);
  return a256(size_t(3 * mpad) * 4) + 256 + a256(size_t(n) * 4) + 256;
}

// What a launch needs on the host, recorded by uot_batched_prepare for its
// workspace (a launch may be captured in a CUDA graph, so it cannot read the
// device copy back).
struct ResClass {
  int cs, begin, count, grid;
  size_t smem;
};
struct HostPlan {
  const void* ws;
  int grid, stages, nprob, teams;
  size_t probs_off, order_off, cursor_off, mailbox_off, bar_off, ctl_off;
  BatchSched sched;
  int nres;
  ResClass res[MAX_RES_CLASSES];
  std::vector<int8_t> placement;  // per problem: on-chip cluster size, 0 = streaming
  std::vector<int16_t> team;      // per problem: streaming team size class, 0 = on chip
};
static std::mutex g_plan_mu;
static std::vector<HostPlan> g_plans;

static bool find_plan(const void* ws, HostPlan* out) {
  std::lock_guard<std::mutex> lock(g_plan_mu);
  for (const HostPlan& h : g_plans)
    if (h.ws == ws) {
      *out = h;
      return true;
    }
  return false;
}

static int64_t max_teams_bound(int nprob) { return int64_t(nprob) + 4096; }

}  // namespace uot

using namespace uot;

extern "C" {

size_t uot_batched_workspace_size(const uot_problem* probs, int32_t nprob, const uot_options* opt) {
  (void)opt;
  if (!probs || nprob <= 0) return 0;
  size_t total = a256(sizeof(BatchHeader)) + a256(sizeof(BatchSched)) +
                 a256(size_t(nprob) * sizeof(BatchProblem)) + a256(size_t(nprob) * 4) +
                 a256(CURSORS * 4) + a256(size_t(max_teams_bound(nprob)) * 4) +
                 a256(size_t(max_teams_bound(nprob)) * 8) + a256(size_t(nprob) * sizeof(Control));
  for (int i = 0; i < nprob; ++i) {
    if (probs[i].n < 1 || probs[i].m < 1) return 0;
    total += per_problem_bytes(probs[i].n, probs[i].m);
  }
  return total;
}

uot_status uot_batched_prepare(const uot_problem* probs, int32_t nprob, const uot_options* opt,
                               const uot_batch_tuning* tuning, void* workspace, size_t ws_bytes,
                               void* stream) {
  if (!probs || nprob <= 0) return UOT_ERR_INVALID_ARG;
  uot_options o;
  uot_default_options(&o);
  if (opt) o = *opt;
  if (o.dtype != UOT_F32 || o.algo != UOT_ALGO_FUSED) return UOT_ERR_UNSUPPORTED;
  const size_t need = uot_batched_workspace_size(probs, nprob, opt);
  if (need == 0) return UOT_ERR_INVALID_ARG;
  if (!workspace || ws_bytes < need || reinterpret_cast<uintptr_t>(workspace) % 256)
    return UOT_ERR_WORKSPACE;
  for (int i = 0; i < nprob; ++i) {
    const uot_problem& q = probs[i];
    if (!q.plan || !q.a || !q.b || q.m > BW || q.n > INT32_MAX || q.ldp < q.m || q.iters < 0 ||
        (q.rule != UOT_RULE_PAPER && q.rule != UOT_RULE_POT) ||
        !(q.reg > 0.0f) || !std::isfinite(q.reg) || !(q.reg_m > 0.0f) ||
        reinterpret_cast<uintptr_t>(q.plan) % 16 || (q.ldp % 4) != 0 ||
        reinterpret_cast<uintptr_t>(q.a) % 4 || reinterpret_cast<uintptr_t>(q.b) % 4)
      return UOT_ERR_INVALID_ARG;
  }
  uot_batch_tuning tu;
  uot_batch_default_tuning(&tu);
  if (tuning) tu = *tuning;
  if (tu.stages < 2 || tu.stages > MAX_STAGES || tu.target_elems <= 0 || tu.max_team < 1 ||
      tu.max_team > 1024 || (tu.max_team & (tu.max_team - 1)) || tu.resident_max_cluster < 0 ||
      tu.resident_max_cluster > RESIDENT_MAX_CLUSTER ||
      (tu.resident_max_cluster & (tu.resident_max_cluster - 1)) || tu.reserved[0] ||
      tu.reserved[1] || tu.reserved[2])
    return UOT_ERR_INVALID_ARG;

  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return UOT_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return UOT_ERR_CUDA;
  const size_t smem = batched_smem(tu.stages);
  if (cudaFuncSetAttribute(batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           int(smem)) != cudaSuccess)
    return UOT_ERR_CUDA;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batched_kernel, BT, smem) !=
          cudaSuccess ||
      occ < 1)
    return UOT_ERR_CUDA;
  const int grid = occ * sms;

  // On chip: the smallest cluster (up to resident_max_cluster) whose shared
  // memory holds the problem; rescls[i] = index of that cluster size, or -1.
  std::vector<double> work(nprob);
  for (int i = 0; i < nprob; ++i)
    work[i] = double(probs[i].n) * double(probs[i].m) * double(probs[i].iters + 1);
  std::vector<int> rescls(nprob, -1);
  int res_clusters[MAX_RES_CLASSES] = {0, 0, 0, 0, 0};
  size_t res_cap = 0;
  if (tu.resident_max_cluster > 0) {
    if (resident_smem_cap(&res_cap) != cudaSuccess) return UOT_ERR_CUDA;
    for (int c = 0; c < MAX_RES_CLASSES && (1 << c) <= tu.resident_max_cluster; ++c)
      if (resident_max_clusters(1 << c, res_cap, &res_clusters[c]) != cudaSuccess)
        return UOT_ERR_CUDA;
    for (int i = 0; i < nprob; ++i)
      for (int c = 0; c < MAX_RES_CLASSES && (1 << c) <= tu.resident_max_cluster; ++c)
        if (res_clusters[c] > 0 &&
            resident_smem_need(probs[i].n, probs[i].m, 1 << c) <= res_cap) {
          rescls[i] = c;
          break;
        }
  }

  // Streaming classes: team size = clamp(next power of two of N*M*iters /
  // target), so every CTA of a team gets about `target_elems`
  // element-iterations.
  std::vector<int> gsize(nprob, 0);
  for (int i = 0; i < nprob; ++i) {
    if (rescls[i] >= 0) continue;
    int g = 1;
    while (g < tu.max_team && g * 2 <= grid && double(g) * tu.target_elems < work[i]) g <<= 1;
    // A CTA keeps the scalings of at most ROWS_MAX rows.
    while (g < grid && int64_t(g) * ROWS_MAX < probs[i].n) g <<= 1;
    if (int64_t(g) * ROWS_MAX < probs[i].n || g > grid) return UOT_ERR_UNSUPPORTED;
    gsize[i] = g;
  }
  std::vector<int> classes;
  const int gmax = nprob > 0 ? *std::max_element(gsize.begin(), gsize.end()) : 1;
  for (int g = gmax; g >= 1; g >>= 1)
    for (int i = 0; i < nprob; ++i)
      if (gsize[i] == g) {
        classes.push_back(g);
        break;
      }
  if (int(classes.size()) > MAX_CLASSES) {  // merge the smallest classes into size 1
    for (int i = 0; i < nprob; ++i)
      if (gsize[i] > 0 && gsize[i] < classes[MAX_CLASSES - 1]) gsize[i] = classes[MAX_CLASSES - 1];
    classes.resize(MAX_CLASSES);
  }

  uint8_t* ws = static_cast<uint8_t*>(workspace);
  std::vector<uint8_t> host(need, 0);
  size_t off = 0;
  BatchHeader* H = reinterpret_cast<BatchHeader*>(host.data());
  off = a256(sizeof(BatchHeader));
  const size_t sched_off = off;
  off += a256(sizeof(BatchSched));
  const size_t probs_off = off;
  off += a256(size_t(nprob) * sizeof(BatchProblem));
  const size_t order_off = off;
  off += a256(size_t(nprob) * 4);
  const size_t cursor_off = off;
  off += a256(CURSORS * 4);
  const size_t mailbox_off = off;
  off += a256(size_t(max_teams_bound(nprob)) * 4);
  const size_t bar_off = off;
  off += a256(size_t(max_teams_bound(nprob)) * 8);
  const size_t ctl_off = off;
  off += a256(size_t(nprob) * sizeof(Control));

  BatchProblem* P = reinterpret_cast<BatchProblem*>(host.data() + probs_off);
  for (int i = 0; i < nprob; ++i) {
    const uot_problem& q = probs[i];
    BatchProblem& d = P[i];
    d.plan = static_cast<float*>(q.plan);
    d.ldp = q.ldp;
    d.n = int(q.n);
    d.m = int(q.m);
    d.a = q.a;
    d.b = q.b;
    const double fi = std::isinf(q.reg_m) ? 1.0
                                          : double(q.reg_m) / (double(q.reg_m) + double(q.reg));
    d.fi = float(fi);
    d.iters = q.iters;
    d.pot = q.rule == UOT_RULE_POT ? 1 : 0;
    d.mpad = int((q.m + 63) & ~int64_t(63));
    d.ctl = reinterpret_cast<Control*>(ws + ctl_off) + i;
    d.c = reinterpret_cast<float*>(ws + off);
    off += a256(size_t(3) * d.mpad * 4);
    d.ctr = reinterpret_cast<int*>(ws + off);
    off += 256;
    d.U = reinterpret_cast<float*>(ws + off);
    off += a256(size_t(q.n) * 4);
    d.log2k = reinterpret_cast<double*>(ws + off);
    off += 256;
  }
  int* order = reinterpret_cast<int*>(host.data() + order_off);
  BatchSched S{};
  S.nprob = nprob;
  S.nclass = int(classes.size());
  S.stages = tu.stages;
  int pos = 0, teams = 0;
  for (int c = 0; c < S.nclass; ++c) {
    const int g = classes[c];
    std::vector<int> idx;
    for (int i = 0; i < nprob; ++i)
      if (gsize[i] == g) idx.push_back(i);
    std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return work[x] > work[y]; });
    S.class_g[c] = g;
    S.class_begin[c] = pos;
    for (int i : idx) order[pos++] = i;
    S.class_end[c] = pos;
    S.team_base[c] = teams;
    teams += grid / g;
  }
  if (teams > max_teams_bound(nprob)) return UOT_ERR_UNSUPPORTED;
  // On-chip classes, after the streaming ones in `order`.
  ResClass res[MAX_RES_CLASSES];
  int nres = 0;
  for (int c = 0; c < MAX_RES_CLASSES; ++c) {
    std::vector<int> idx;
    size_t smem = 0;
    for (int i = 0; i < nprob; ++i)
      if (rescls[i] == c) {
        idx.push_back(i);
        smem = std::max(smem, resident_smem_need(probs[i].n, probs[i].m, 1 << c));
      }
    if (idx.empty()) continue;
    std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return work[x] > work[y]; });
    ResClass& rc = res[nres++];
    rc.cs = 1 << c;
    rc.begin = pos;
    rc.count = int(idx.size());
    for (int i : idx) order[pos++] = i;
    int nc = 0;
    if (resident_max_clusters(rc.cs, smem, &nc) != cudaSuccess) return UOT_ERR_CUDA;
    if (nc <= 0) return UOT_ERR_UNSUPPORTED;
    rc.grid = std::min(nc, rc.count) * rc.cs;
    rc.smem = smem;
  }
  S.probs = reinterpret_cast<const BatchProblem*>(ws + probs_off);
  S.order = reinterpret_cast<const int*>(ws + order_off);
  S.cursor = reinterpret_cast<int*>(ws + cursor_off);
  S.mailbox = reinterpret_cast<int*>(ws + mailbox_off);
  S.bar = reinterpret_cast<int*>(ws + bar_off);
  std::memcpy(host.data() + sched_off, &S, sizeof(S));
  H->nprob = nprob;
  H->teams = teams;
  H->probs_off = int64_t(probs_off);
  H->order_off = int64_t(order_off);
  H->cursor_off = int64_t(cursor_off);
  H->mailbox_off = int64_t(mailbox_off);
  H->bar_off = int64_t(bar_off);
  H->sched_off = int64_t(sched_off);
  H->total = int64_t(off);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(ws, host.data(), off, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return UOT_ERR_CUDA;
  // The host copy must outlive the asynchronous transfer.
  if (cudaStreamSynchronize(s) != cudaSuccess) return UOT_ERR_CUDA;
  HostPlan hp{workspace, grid,        tu.stages,   nprob,   teams, probs_off, order_off,
              cursor_off, mailbox_off, bar_off,     ctl_off, S,     nres,      {}};
  for (int c = 0; c < nres; ++c) hp.res[c] = res[c];
  hp.placement.resize(size_t(nprob));
  for (int i = 0; i < nprob; ++i) hp.placement[i] = int8_t(rescls[i] >= 0 ? 1 << rescls[i] : 0);
  hp.team.assign(gsize.begin(), gsize.end());
  std::lock_guard<std::mutex> lock(g_plan_mu);
  for (HostPlan& h : g_plans)
    if (h.ws == workspace) {
      h = hp;
      return UOT_OK;
    }
  g_plans.push_back(hp);
  return UOT_OK;
}

uot_status uot_sinkhorn_batched(void* workspace, void* stream) {
  HostPlan hp;
  if (!workspace || !find_plan(workspace, &hp)) return UOT_ERR_WORKSPACE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint8_t* ws = static_cast<uint8_t*>(workspace);
  batched_reset_kernel<<<std::max(hp.nprob, 1), 256, 0, s>>>(
      reinterpret_cast<const BatchProblem*>(ws + hp.probs_off), hp.nprob,
      reinterpret_cast<int*>(ws + hp.cursor_off), reinterpret_cast<int*>(ws + hp.mailbox_off),
      reinterpret_cast<int*>(ws + hp.bar_off), hp.teams);
  if (cudaGetLastError() != cudaSuccess) return UOT_ERR_CUDA;
  count_launch();
  for (int c = 0; c < hp.nres; ++c) {
    const ResClass& rc = hp.res[c];
    if (resident_launch(reinterpret_cast<const BatchProblem*>(ws + hp.probs_off),
                        reinterpret_cast<const int*>(ws + hp.order_off) + rc.begin, rc.count,
                        reinterpret_cast<int*>(ws + hp.cursor_off) + MAX_CLASSES + c, rc.cs,
                        rc.grid, rc.smem, s) != cudaSuccess)
      return UOT_ERR_CUDA;
  }
  if (hp.sched.nclass == 0) return UOT_OK;
  // All CTAs must be resident at once (team barriers): the grid is the
  // occupancy recorded at preparation, re-checked here.
  int dev = 0, sms = 0, occ = 0;
  const size_t smem = batched_smem(hp.stages);
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batched_kernel, BT, smem) != cudaSuccess)
    return UOT_ERR_CUDA;
  if (occ * sms < hp.grid) return UOT_ERR_UNSUPPORTED;
  // Team barriers need every CTA resident at once: a cooperative launch
  // guarantees it (or fails) even when other work shares the GPU.
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.gridDim = dim3(hp.grid);
  cfg.blockDim = dim3(BT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  BatchSched S = hp.sched;
  void* kargs[] = {&S};
  if (cudaLaunchKernelExC(&cfg, reinterpret_cast<const void*>(batched_kernel), kargs) !=
      cudaSuccess)
    return UOT_ERR_CUDA;
  count_launch();
  return UOT_OK;
}

uot_status uot_batched_results(const void* workspace, int32_t nprob, uot_result* out,
                               void* stream) {
  HostPlan hp;
  if (!workspace || !out || !find_plan(workspace, &hp) || nprob != hp.nprob)
    return UOT_ERR_INVALID_ARG;
  std::vector<Control> ctl(static_cast<size_t>(nprob));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(ctl.data(), static_cast<const uint8_t*>(workspace) + hp.ctl_off,
                      size_t(nprob) * sizeof(Control), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return UOT_ERR_CUDA;
  uint32_t any = 0;
  for (int i = 0; i < nprob; ++i) {
    out[i].iters_done = ctl[i].iters_done;
    out[i].dev_status = ctl[i].status;
    out[i].err = ctl[i].err;
    any |= ctl[i].status;
  }
  if (any & UOT_DEV_TIMEOUT) return UOT_ERR_TIMEOUT;
  if (any & UOT_DEV_NONFINITE) return UOT_ERR_NONFINITE;
  if (any & UOT_DEV_ZERO_SUM) return UOT_ERR_ZERO_SUM;
  return UOT_OK;
}

int32_t uot_batched_placement(const void* workspace, int32_t nprob, int32_t* cluster,
                              int32_t* team) {
  HostPlan hp;
  if (!workspace || !find_plan(workspace, &hp)) return -1;
  for (int i = 0; i < std::min(nprob, hp.nprob); ++i) {
    if (cluster) cluster[i] = hp.placement[i];
    if (team) team[i] = hp.team[i];
  }
  return hp.nprob;
}

void uot_batch_default_tuning(uot_batch_tuning* t) {
  if (!t) return;
  std::memset(t, 0, sizeof(*t));
  t->stages = 4;
  t->max_team = 32;
  t->target_elems = 4.0e7;
  t->resident_max_cluster = RESIDENT_MAX_CLUSTER;
}

}  // extern "C"
