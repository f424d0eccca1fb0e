// Adjoint of the unrolled Sinkhorn-UOT iteration (the rule of Section 2.1):
// gradients of L = <P_T, C> with respect to C, a and b, from the history a
// kernel-form forward solve saved (scalings U_t, V_t and sums r_t, c_t).
//
// In log space (l = -C/reg, f_t = log U_t, g_t = log V_t) the forward steps
// are f_t = f_{t-1} + fi (log a - log r_t) and g_t = g_{t-1} + fi (log b -
// log c_t) with r_t = rowsum(R_t), R_t = exp(l + f_{t-1} (+) g_{t-1}), and
// c_t = colsum(Q_t), Q_t = exp(l + f_t (+) g_{t-1}).  Reverse mode from
// dl = P_T * C, F = rowsum(dl), G = colsum(dl), for t = T .. 1:
//   column step: w = -fi G / c_t, db += fi G / b, F += Q_t w,
//                dl += Q_t * w, G = (1 - fi) G;
//   row step:    z = -fi F / r_t, da += fi F / a, G += R_t^T z,
//                dl += R_t * z, F = (1 - fi) F;
// and dC = P_T - dl / reg.  Each reverse step is one read-only sweep over
// the rows of K with the same structure as the forward pass: Q_t and R_t are
// recomputed per row from K and the saved scalings (never stored), the row
// reduction (Q_t w)_i gives z_i, and R_t^T z is accumulated per column.  The
// last CTAs of a step fold the column partials into G and prepare w for the
// next step.
//
// dl is never updated in place.  Every step adds K (x) (q_t v_t w_t^T +
// pz_t v_t^T) with per-step vectors q_t = U_t 2^-e_t, pz_t = U_{t-1} z_t
// (rows) and v_t = V_{t-1}, v_t w_t (columns), so after all steps
//     dl = P_T * C + K * (A B^T),  A = [q_1..q_T, pz_1..pz_T] (n x 2T),
//                                  B = [v_1 w_1..v_T w_T, v_1..v_T] (m x 2T):
// the steps record the 2T vectors (4 bytes per element of K per step instead
// of reading and writing dl as well, 12), and one tiled FP32 contraction of
// depth 2T with the final scaling fused (bw_gemm_kernel) writes dC at the
// end.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "uot_device.cuh"
#include "uot_internal.h"

namespace uot {

namespace {

constexpr int BW_BETA_CTAS = 16;

struct BwArgs {
  const float* K;
  int64_t ldk;
  int n, m, mpad;
  const float* a;
  const float* b;
  float fi;
  int t;           // reverse step (iteration index)
  const double* log2k;  // gauge of the forward solve: Q_t = K U'_t V'_{t-1} 2^-e_t
  const float* q;  // U'_t (n)
  const float* pr; // U'_{t-1} (n)
  const float* v;  // V'_{t-1} (mpad)
  const float* r;  // r_t (n)
  const float* c_prev;  // c_{t-1} (mpad), for the next step's w (t > 1)
  float* F;        // row adjoints (n)
  float* da;       // (n)
  float* w;        // (mpad): w of this step, overwritten with the next step's
  float* Gs;       // (mpad): (1 - fi) G entering this step's row part
  float* db;       // (mpad)
  float* h_next;   // (mpad) column partials R_t^T z, pre-zeroed
  float* h_clear;  // buffer to clear for the next step
  int* row_ctr;
  int* ctr_clear;
  int* arrive;
  int* arrive_clear;
  int* slice_ctr;
  int* slice_clear;
  Control* ctl;
  int stages;
  float* Aq;       // (n): q_t = U_t 2^-e_t of this step's rows
  float* Az;       // (n): pz_t = U_{t-1} z_t
  float* Bw;       // (m): v_t w_t of this step's columns
};

template <int THREADS, int KV>
__global__ void __launch_bounds__(THREADS, 1) reverse_pass_kernel(const BwArgs p) {
  constexpr int VE = 4;
  constexpr int NW = THREADS / 32;
  constexpr int W = KV * VE * THREADS;
  constexpr int ROW_BYTES = W * 4;
  extern __shared__ __align__(128) unsigned char smem[];
  const int stages = p.stages;
  unsigned char* ring = smem;  // per slot: one row of K
  float* red = reinterpret_cast<float*>(smem + size_t(stages) * ROW_BYTES);
  uint64_t* bars = reinterpret_cast<uint64_t*>(red + 2 * NW);
  int* slot_row = reinterpret_cast<int*>(bars + stages);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n = p.n, m = p.m;
  const float qscale = ldexpf(1.0f, -gauge_exponent(p.t, float(*p.log2k)));
  const uint32_t copy_bytes = uint32_t((size_t(m) * 4) & ~size_t(15));
  uint32_t st = 0;

  if (tid == 0) {
    for (int s = 0; s < stages; ++s) mbar_init(&bars[s], 1);
    fence_mbar_init();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  const uint64_t policy = policy_evict_first();
  // Static schedule: CTA g owns the contiguous rows [g R, (g+1) R), so the
  // ring is armed without a shared counter and the rows' scalars are loaded
  // in coalesced chunks ahead of use (a row here is only m floats of K; the
  // per-row round trips of a dynamic schedule would bound the step).
  const int R = (n + int(gridDim.x) - 1) / int(gridDim.x);
  const int r0 = int(blockIdx.x) * R;
  const int nrows = max(0, min(n, r0 + R) - r0);
  int issued = 0;
  auto arm = [&](int q, int row) {
    const int slot = q % stages;
    if (row >= 0 && row < n) {
      slot_row[slot] = row;
      if (copy_bytes) {
        mbar_arrive_expect_tx(&bars[slot], copy_bytes);
        bulk_load(ring + size_t(slot) * ROW_BYTES, p.K + int64_t(row) * p.ldk, copy_bytes,
                  &bars[slot], policy);
      } else {
        mbar_arrive(&bars[slot]);
      }
    } else {
      slot_row[slot] = -1;
      mbar_arrive(&bars[slot]);
    }
  };
  if (tid == 0) {
    for (int q = 0; q < stages; ++q) arm(q, q < nrows ? r0 + q : -1);
    issued = stages;
  }

  // This step's column values: V'_{t-1} and w.
  float v[KV][VE], w[KV][VE], h[KV][VE];
#pragma unroll
  for (int k = 0; k < KV; ++k) {
    const int cc = (k * THREADS + tid) * VE;
#pragma unroll
    for (int e = 0; e < VE; ++e) {
      v[k][e] = cc + e < m ? __ldcg(p.v + cc + e) : 0.0f;
      w[k][e] = cc + e < m ? __ldcg(p.w + cc + e) : 0.0f;
      h[k][e] = 0.0f;
    }
  }
  // This step's column vector v_t w_t of the final contraction (every CTA
  // covers all columns; one stores it).
  if (blockIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < KV; ++k) {
      const int cc = (k * THREADS + tid) * VE;
#pragma unroll
      for (int e = 0; e < VE; ++e)
        if (cc + e < m) p.Bw[cc + e] = v[k][e] * w[k][e];
    }
  }
  {
    const int g = blockIdx.x * THREADS + tid, gs = gridDim.x * THREADS;
    for (int j = g; j < p.mpad; j += gs) p.h_clear[j] = 0.0f;
    if (blockIdx.x == 0 && tid == 0) {
      *p.ctr_clear = 0;
      *p.arrive_clear = 0;
      *p.slice_clear = 0;
    }
  }

  bool broken = false;
  int done_rows = 0;
  // Per-row values (q, pr, r, a, F) of the CTA's rows, a chunk of RCH rows at
  // a time.
  constexpr int RCH = 64;
  __shared__ float sc[5][RCH];
  for (int q = 0;; ++q) {
    if (q % RCH == 0 && q < nrows) {  // uniform for the CTA
      __syncthreads();  // every thread is done with the previous chunk
      for (int i = tid; i < min(RCH, nrows - q); i += THREADS) {
        const int row = r0 + q + i;
        sc[0][i] = __ldcg(p.q + row);
        sc[1][i] = __ldcg(p.pr + row);
        sc[2][i] = __ldcg(p.r + row);
        sc[3][i] = __ldg(p.a + row);
        sc[4][i] = __ldcg(p.F + row);
      }
      __syncthreads();
    }
    const int slot = q % stages;
    if (!broken && !mbar_wait_bounded(&bars[slot], uint32_t(q / stages) & 1u, WAIT_LIMIT_NS)) {
      broken = true;
      st |= DEV_TIMEOUT;
    }
    const int row = *reinterpret_cast<volatile int*>(&slot_row[slot]);
    if (row < 0 || row >= n) break;
    const int ci = q % RCH;
    const float qi = sc[0][ci] * qscale;
    const float pi = sc[1][ci];
    const float ri = sc[2][ci];
    const float ai = sc[3][ci];
    const float Fi = sc[4][ci];
    const unsigned char* sK = ring + size_t(slot) * ROW_BYTES;
    const float* gK = p.K + int64_t(row) * p.ldk;
    float x[KV][VE];
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < KV; ++k) {
      const int li = k * THREADS + tid;
      const int cc = li * VE;
      if (cc + VE <= m) {
        Elem<float>::unpack(ld_shared_v4(sK + size_t(li) * 16), x[k]);
      } else {
#pragma unroll
        for (int e = 0; e < VE; ++e) x[k][e] = cc + e < m ? gK[cc + e] : 0.0f;
      }
#pragma unroll
      for (int e = 0; e < VE; ++e) s = fmaf(x[k][e] * v[k][e], w[k][e], s);
    }
    s = warp_sum(s);
    float* rb = red + (q & 1) * NW;
    if (lane == 0) rb[warp] = s;
    if (__syncthreads_or(broken ? 1 : 0)) {
      broken = true;
      st |= DEV_TIMEOUT;
      break;
    }
    if (tid == 0 && !broken) {
      arm(issued, issued < nrows ? r0 + issued : -1);
      ++issued;
    }
    float S1 = 0.0f;
#pragma unroll
    for (int k = 0; k < NW; ++k) S1 += rb[k];
    // Column step: F += (Q_t w)_i; row step: z, da, F.
    const float Fn = Fi + qi * S1;
    const float z = -p.fi * Fn / ri;
    const float pz = pi * z;
    if (tid == 0) {
      p.da[row] += p.fi * Fn / ai;
      p.F[row] = (1.0f - p.fi) * Fn;
      p.Aq[row] = qi;  // this step's row vectors of the final contraction
      p.Az[row] = pz;
    }
#pragma unroll
    for (int k = 0; k < KV; ++k)
#pragma unroll
      for (int e = 0; e < VE; ++e) h[k][e] = fmaf(x[k][e] * v[k][e], pz, h[k][e]);
    ++done_rows;
  }
  if (done_rows > 0) {
#pragma unroll
    for (int k = 0; k < KV; ++k) {
      const int cc = (k * THREADS + tid) * VE;
      if (cc + VE <= m) {
        red_add_v4(p.h_next + cc, h[k][0], h[k][1], h[k][2], h[k][3]);
      } else {
#pragma unroll
        for (int e = 0; e < VE; ++e)
          if (cc + e < m) atomicAdd(p.h_next + cc + e, h[k][e]);
      }
    }
  }
  if (st) atomicOr(&p.ctl->status, st);
  // The CTAs that finish last: G = (1 - fi) G_prev + R_t^T z; db and the next
  // step's w (claimed in column slices once every CTA's partials landed).
  {
    const int nsl = 64;
    const int per = (m + nsl - 1) / nsl;
    finish_pass_job(p.arrive, p.slice_ctr, nsl, BW_BETA_CTAS, 2000, [&](int sl) {
      const int j0 = sl * per, j1 = min(m, j0 + per);
      for (int j = j0 + tid; j < j1; j += THREADS) {
        const float Gj = p.Gs[j] + __ldcg(p.h_next + j);
        if (p.t > 1) {
          p.db[j] += p.fi * Gj / __ldg(p.b + j);
          p.w[j] = -p.fi * Gj / __ldcg(p.c_prev + j);
          p.Gs[j] = (1.0f - p.fi) * Gj;
        }
      }
    });
  }
  if (tid == 0 && broken) {
    for (int q = max(0, issued - stages); q < issued; ++q)
      mbar_wait_bounded(&bars[q % stages], uint32_t(q / stages) & 1u, WAIT_LIMIT_NS);
  }
}

constexpr int TB = 256;

// dl = P_T * C with P_T = (U_i K_ij) V_j; F = rowsum(dl) (one warp per row).
__global__ void __launch_bounds__(TB) bw_init_kernel(const float* K, int64_t ldk, const float* C,
                                                     int64_t ldc, const float* U, const float* V,
                                                     float* D, int64_t ldd, int n, int m,
                                                     float* F, float* da) {
  const int warp = (blockIdx.x * TB + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int nw = (gridDim.x * TB) >> 5;
  for (int i = warp; i < n; i += nw) {
    float s = 0.0f;
    const float u = U[i];
    for (int j = lane; j < m; j += 32) {
      const float dl = (u * K[int64_t(i) * ldk + j]) * V[j] * C[int64_t(i) * ldc + j];
      D[int64_t(i) * ldd + j] = dl;
      s += dl;
    }
    s = warp_sum(s);
    if (lane == 0) {
      F[i] = s;
      da[i] = 0.0f;
    }
  }
}

// G0 = colsum(dl): a column per thread over a stride of rows, then atomics.
__global__ void __launch_bounds__(TB) bw_colsum_kernel(const float* D, int64_t ldd, int n, int m,
                                                       float* G0) {
  const int j = blockIdx.x * TB + threadIdx.x;
  if (j >= m) return;
  float s = 0.0f;
  for (int i = blockIdx.y; i < n; i += gridDim.y) s += D[int64_t(i) * ldd + j];
  atomicAdd(G0 + j, s);
}

// w_T = -fi G0 / c_T, db = fi G0 / b, Gs = (1 - fi) G0.
__global__ void bw_cols_kernel(const float* G0, const float* cT, const float* b, float fi, int m,
                               float* w, float* db, float* Gs) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m) return;
  const float G = G0[j];
  w[j] = -fi * G / cT[j];
  db[j] = fi * G / b[j];
  Gs[j] = (1.0f - fi) * G;
}

// The final contraction: acc = A B^T over the 2T recorded step vectors
// (A_s = q_t or pz_t of the rows, B_s = v_t w_t or v_t of the columns), then
//     dl = P_T * C + K * acc,   dC = g (P_T - dl / reg),
// with g = grad_out times the optional device scalar (read here, so the
// caller need not synchronise).  FP32 on the CUDA cores (the depth-2T sum
// needs FP32 accuracy): 128 x 128 tiles, 16 steps of depth per stage in
// shared memory, 8 x 8 outputs per thread.
constexpr int GB = 128, GKD = 16, GT = 256;

struct BwGemmArgs {
  const float* K;
  int64_t ldk;
  const float* C;
  int64_t ldc;
  float* D;
  int64_t ldd;
  const float* UT;  // U_T (n)
  const float* VT;  // V_T (m)
  const float* Aq;  // q_t at Aq + (t-1) sn
  const float* Az;  // pz_t at Az + (t-1) sn
  const float* Bw;  // v_t w_t at Bw + (t-1) sm
  const float* Vh;  // V_{t-1} at Vh + (t-1) sv (the history)
  int64_t sn, sm, sv;
  int n, m, T;
  float inv_reg;
  double g_host;
  const double* g_dev;
};

__global__ void __launch_bounds__(GT) bw_gemm_kernel(const BwGemmArgs p) {
  __shared__ __align__(16) float As[GKD][GB];
  __shared__ __align__(16) float Bs[GKD][GB];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int i0 = blockIdx.y * GB, j0 = blockIdx.x * GB;
  const int S = 2 * p.T;
  float acc[8][8];
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[r][c] = 0.0f;
  const int lk = threadIdx.x / 16, l8 = (threadIdx.x % 16) * 8;  // loader: depth row, 8 entries
  for (int s0 = 0; s0 < S; s0 += GKD) {
    {
      const int sidx = s0 + lk;
      const float* arow = nullptr;
      const float* brow = nullptr;
      if (sidx < p.T) {
        arow = p.Aq + sidx * p.sn;
        brow = p.Bw + sidx * p.sm;
      } else if (sidx < S) {
        arow = p.Az + (sidx - p.T) * p.sn;
        brow = p.Vh + (sidx - p.T) * p.sv;
      }
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int i = i0 + l8 + e, j = j0 + l8 + e;
        As[lk][l8 + e] = (arow && i < p.n) ? __ldg(arow + i) : 0.0f;
        Bs[lk][l8 + e] = (brow && j < p.m) ? __ldg(brow + j) : 0.0f;
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GKD; ++kk) {
      float a[8], b[8];
      const float4 a0 = *reinterpret_cast<const float4*>(&As[kk][ty * 8]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[kk][ty * 8 + 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[kk][tx * 8]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[kk][tx * 8 + 4]);
      a[0] = a0.x; a[1] = a0.y; a[2] = a0.z; a[3] = a0.w;
      a[4] = a1.x; a[5] = a1.y; a[6] = a1.z; a[7] = a1.w;
      b[0] = b0.x; b[1] = b0.y; b[2] = b0.z; b[3] = b0.w;
      b[4] = b1.x; b[5] = b1.y; b[6] = b1.z; b[7] = b1.w;
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[r][c] = fmaf(a[r], b[c], acc[r][c]);
    }
    __syncthreads();
  }
  const float g = float(p.g_dev ? p.g_host * *p.g_dev : p.g_host);
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int i = i0 + ty * 8 + r;
    if (i >= p.n) continue;
    const float u = p.UT[i];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int j = j0 + tx * 8 + c;
      if (j >= p.m) continue;
      const float k = p.K[int64_t(i) * p.ldk + j];
      const float P = (u * k) * p.VT[j];
      const float dl = fmaf(k, acc[r][c], P * p.C[int64_t(i) * p.ldc + j]);
      p.D[int64_t(i) * p.ldd + j] = g * (P - dl * p.inv_reg);
    }
  }
}

// da *= g, db *= g.
__global__ void bw_scale_kernel(float* da, int n, float* db, int m, double g_host,
                                const double* g_dev) {
  const float g = float(g_dev ? g_host * *g_dev : g_host);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < max(n, m); i += gridDim.x * blockDim.x) {
    if (i < n) da[i] *= g;
    if (i < m) db[i] *= g;
  }
}

__global__ void bw_hist_init_kernel(uint8_t* hist, HistLayout L, int n, int m, int iters,
                                    float u0, const double* log2k) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  const int gs = gridDim.x * blockDim.x;
  float* U0 = reinterpret_cast<float*>(hist + L.U);
  float* V0 = reinterpret_cast<float*>(hist + L.V);
  for (int i = g; i < n; i += gs) U0[i] = u0;
  for (int j = g; j < m; j += gs) V0[j] = 1.0f;
  if (g == 0) {
    HistHeader* H = reinterpret_cast<HistHeader*>(hist);
    H->log2k = *log2k;
    H->n = n;
    H->m = m;
    H->iters = iters;
    H->k_scale_inv = u0;
  }
}

struct BwEntry {
  int threads, kv;
  const void* fn;
};
#define BW_ENTRY(TH, KV) \
  BwEntry { TH, KV, reinterpret_cast<const void*>(&reverse_pass_kernel<TH, KV>) }
// Four vectors per thread (four warps for rows of 2048 columns, four CTAs
// per SM): a reverse step's CTA barrier per row is cheapest with few warps,
// and the per-row latency is hidden by CTAs side by side rather than by wider
// CTAs (512 x 1: 69 ms, 256 x 2: 55 ms, 128 x 4: 48 ms per gradient step).
const BwEntry kBw[] = {BW_ENTRY(512, 4), BW_ENTRY(256, 4), BW_ENTRY(128, 4),
                       BW_ENTRY(128, 2), BW_ENTRY(64, 2),  BW_ENTRY(32, 2)};
constexpr int kBwNum = int(sizeof(kBw) / sizeof(kBw[0]));

size_t bw_smem(const BwEntry& e, int stages) {
  const size_t row = size_t(e.threads) * e.kv * 16;
  return size_t(stages) * row + 2 * (e.threads / 32) * 4 + size_t(stages) * 12;
}

// Backward workspace: the adjoint state (cleared at the start of a call),
// then the step vectors of the final contraction (T rows each, written
// before they are read).
struct BwLayout {
  size_t ctl, F, da, w, Gs, G0, h[3], ctr, state_end, Aq, Az, Bw, total;
  size_t npad, mpad;  // floats
};
BwLayout bw_layout(int64_t n, int64_t m, int T) {
  BwLayout L{};
  L.npad = size_t((n + 63) & ~int64_t(63));
  L.mpad = size_t((m + 63) & ~int64_t(63));
  const size_t npad = L.npad * 4, mpad = L.mpad * 4;
  size_t off = 0;
  L.ctl = off; off = align256(off + sizeof(Control));
  L.F = off; off = align256(off + npad);
  L.da = off; off = align256(off + npad);
  L.w = off; off = align256(off + mpad);
  L.Gs = off; off = align256(off + mpad);
  L.G0 = off; off = align256(off + mpad);
  for (int k = 0; k < 3; ++k) { L.h[k] = off; off = align256(off + mpad); }
  L.ctr = off; off = align256(off + 9 * sizeof(int));
  L.state_end = off;
  L.Aq = off; off = align256(off + size_t(T) * npad);
  L.Az = off; off = align256(off + size_t(T) * npad);
  L.Bw = off; off = align256(off + size_t(T) * mpad);
  L.total = off;
  return L;
}

std::mutex g_bw_mu;
size_t g_bw_smem_set[64][kBwNum];

}  // namespace

cudaError_t launch_hist_init(uint8_t* hist, int n, int m, int iters, float u0, const double* log2k,
                             cudaStream_t s) {
  const HistLayout L = hist_layout(n, m, iters);
  bw_hist_init_kernel<<<(std::max(n, m) + 255) / 256, 256, 0, s>>>(hist, L, n, m, iters, u0, log2k);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) count_launch();
  return e;
}

}  // namespace uot

using namespace uot;

extern "C" {

size_t uot_grad_hist_size(int64_t n, int64_t m, int32_t iters) {
  if (n < 1 || m < 1 || iters < 0 || n > INT32_MAX || m > INT32_MAX / 2) return 0;
  return hist_layout(n, m, iters).total;
}

size_t uot_backward_workspace_size(int64_t n, int64_t m, int32_t iters) {
  if (n < 1 || m < 1 || iters < 0 || n > INT32_MAX || m > INT32_MAX / 2) return 0;
  return bw_layout(n, m, iters).total;
}

uot_status uot_sinkhorn_backward(const float* K, int64_t ldk, const float* C, int64_t ldc,
                                 const float* a, const float* b, int64_t n, int64_t m, float reg,
                                 float reg_m, int32_t iters, const void* hist, size_t hist_bytes,
                                 double grad_out, const double* grad_out_dev, float* dC,
                                 int64_t lddc, float* da, float* db, void* workspace,
                                 size_t ws_bytes, const uot_options* opt, void* stream) {
  const int max_ctas = opt ? opt->max_ctas : 0;
  if (max_ctas < 0) return UOT_ERR_INVALID_ARG;
  if (!K || !C || !a || !b || !hist || !dC || !da || !db || n < 1 || m < 1 || n > INT32_MAX ||
      m > INT32_MAX / 2 || ldk < m || ldc < m || lddc < m)
    return UOT_ERR_INVALID_ARG;
  if (!(reg > 0.0f) || !std::isfinite(reg) || !(reg_m > 0.0f) || !std::isfinite(grad_out))
    return UOT_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(grad_out_dev) % 8) return UOT_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(K) % 16 || reinterpret_cast<uintptr_t>(dC) % 16 ||
      ldk % 4 || lddc % 4)
    return UOT_ERR_INVALID_ARG;  // rows of K and dC are fetched with bulk copies
  if (iters < 0) return UOT_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int T = iters, N = int(n), M = int(m);
  const HistLayout HL = hist_layout(n, m, T);
  if (hist_bytes < HL.total) return UOT_ERR_INVALID_ARG;
  const BwLayout L = bw_layout(n, m, T);
  if (!workspace || ws_bytes < L.total || reinterpret_cast<uintptr_t>(workspace) % 256)
    return UOT_ERR_WORKSPACE;
  int k = -1;
  for (int i = 0; i < kBwNum; ++i)
    if (kBw[i].threads * kBw[i].kv * 4 >= M && (k < 0 || kBw[i].threads * kBw[i].kv < kBw[k].threads * kBw[k].kv))
      k = i;
  if (k < 0) return UOT_ERR_UNSUPPORTED;  // rows wider than one CTA (8192 columns)

  const double fi_d = std::isinf(reg_m) ? 1.0 : double(reg_m) / (double(reg_m) + double(reg));
  const float fi = float(fi_d);
  uint8_t* ws = static_cast<uint8_t*>(workspace);
  const uint8_t* hb = static_cast<const uint8_t*>(hist);
  auto U_t = [&](int t) { return reinterpret_cast<const float*>(hb + HL.U + size_t(t) * HL.strideU); };
  auto V_t = [&](int t) { return reinterpret_cast<const float*>(hb + HL.V + size_t(t) * HL.strideV); };
  auto r_t = [&](int t) { return reinterpret_cast<const float*>(hb + HL.r + size_t(t) * HL.strideU); };
  auto c_t = [&](int t) { return reinterpret_cast<const float*>(hb + HL.c + size_t(t) * HL.strideV); };
  float* F = reinterpret_cast<float*>(ws + L.F);
  float* w = reinterpret_cast<float*>(ws + L.w);
  float* Gs = reinterpret_cast<float*>(ws + L.Gs);
  float* G0 = reinterpret_cast<float*>(ws + L.G0);
  int* ctr = reinterpret_cast<int*>(ws + L.ctr);
  Control* ctl = reinterpret_cast<Control*>(ws + L.ctl);

  if (cudaMemsetAsync(ws, 0, L.state_end, s) != cudaSuccess) return UOT_ERR_CUDA;
  float* Aq = reinterpret_cast<float*>(ws + L.Aq);
  float* Az = reinterpret_cast<float*>(ws + L.Az);
  float* Bw = reinterpret_cast<float*>(ws + L.Bw);
  {
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    bw_init_kernel<<<sms * 8, TB, 0, s>>>(K, ldk, C, ldc, U_t(T), V_t(T), dC, lddc, N, M, F, da);
    if (cudaGetLastError() != cudaSuccess) return UOT_ERR_CUDA;
    count_launch();
    const int gx = (M + TB - 1) / TB;
    const int gy = std::max(1, std::min(std::min(N, 65535), (sms * 8 + gx - 1) / gx));
    bw_colsum_kernel<<<dim3(gx, gy), TB, 0, s>>>(dC, lddc, N, M, G0);
    if (cudaGetLastError() != cudaSuccess) return UOT_ERR_CUDA;
    count_launch();
  }
  if (T > 0) {
    bw_cols_kernel<<<(M + 255) / 256, 256, 0, s>>>(G0, c_t(T), b, fi, M, w, db, Gs);
    if (cudaGetLastError() != cudaSuccess) return UOT_ERR_CUDA;
    count_launch();
  } else {
    if (cudaMemsetAsync(db, 0, size_t(M) * 4, s) != cudaSuccess) return UOT_ERR_CUDA;
  }

  // Geometry of the reverse pass.
  const BwEntry& e = kBw[k];
  int dev = 0, sms = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return UOT_ERR_CUDA;
  int stages = 2, occ = 0;
  for (int st = 8; st >= 2; --st)
    if (bw_smem(e, st) <= size_t(optin)) {
      stages = st;
      break;
    }
  // Prefer more CTAs per SM over a deeper ring once two slots fit.
  int best_occ = 0, best_st = stages;
  for (int st = 2; st <= stages; ++st) {
    const size_t b2 = bw_smem(e, st);
    {
      std::lock_guard<std::mutex> lock(g_bw_mu);
      if (dev < 64 && g_bw_smem_set[dev][k] < b2) {
        if (cudaFuncSetAttribute(e.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(b2)) !=
            cudaSuccess)
          return UOT_ERR_CUDA;
        g_bw_smem_set[dev][k] = b2;
      }
    }
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, e.fn, e.threads, b2) != cudaSuccess)
      return UOT_ERR_CUDA;
    if (occ == 0) break;
    if (st == 2) best_occ = occ;
    if (occ < best_occ) break;
    best_st = st;
  }
  if (best_occ == 0) return UOT_ERR_CUDA;
  const size_t smem = bw_smem(e, best_st);
  int grid = best_occ * sms;
  if (grid > (N + 1) / 2) grid = std::max(1, (N + 1) / 2);
  if (max_ctas > 0 && grid > max_ctas) grid = max_ctas;

  BwArgs A{};
  A.K = K;
  A.ldk = ldk;
  A.n = N;
  A.m = M;
  A.mpad = int((m + 63) & ~int64_t(63));
  A.a = a;
  A.b = b;
  A.fi = fi;
  A.F = F;
  A.da = da;
  A.w = w;
  A.Gs = Gs;
  A.db = db;
  A.ctl = ctl;
  A.stages = best_st;
  for (int t = T; t >= 1; --t) {
    const int q = T - t;  // pass counter for the rings
    A.t = t;
    A.log2k = reinterpret_cast<const double*>(hb);  // HistHeader::log2k
    A.q = U_t(t);
    A.pr = U_t(t - 1);
    A.v = V_t(t - 1);
    A.r = r_t(t);
    A.c_prev = t > 1 ? c_t(t - 1) : c_t(t);
    A.h_next = reinterpret_cast<float*>(ws + L.h[q % 3]);
    A.h_clear = reinterpret_cast<float*>(ws + L.h[(q + 1) % 3]);
    A.row_ctr = ctr + q % 3;
    A.ctr_clear = ctr + (q + 1) % 3;
    A.arrive = ctr + 3 + q % 3;
    A.arrive_clear = ctr + 3 + (q + 1) % 3;
    A.slice_ctr = ctr + 6 + q % 3;
    A.slice_clear = ctr + 6 + (q + 1) % 3;
    A.Aq = Aq + size_t(t - 1) * L.npad;
    A.Az = Az + size_t(t - 1) * L.npad;
    A.Bw = Bw + size_t(t - 1) * L.mpad;
    void* kargs[] = {&A};
    if (cudaLaunchKernel(e.fn, dim3(grid), dim3(e.threads), kargs, smem, s) != cudaSuccess)
      return UOT_ERR_CUDA;
    count_launch();
  }
  {
    BwGemmArgs G{};
    G.K = K;
    G.ldk = ldk;
    G.C = C;
    G.ldc = ldc;
    G.D = dC;
    G.ldd = lddc;
    G.UT = U_t(T);
    G.VT = V_t(T);
    G.Aq = Aq;
    G.Az = Az;
    G.Bw = Bw;
    G.Vh = V_t(0);
    G.sn = int64_t(L.npad);
    G.sm = int64_t(L.mpad);
    G.sv = int64_t(HL.strideV / 4);
    G.n = N;
    G.m = M;
    G.T = T;
    G.inv_reg = 1.0f / reg;
    G.g_host = grad_out;
    G.g_dev = grad_out_dev;
    const dim3 gg((M + GB - 1) / GB, (N + GB - 1) / GB);
    bw_gemm_kernel<<<gg, GT, 0, s>>>(G);
    if (cudaGetLastError() != cudaSuccess) return UOT_ERR_CUDA;
    bw_scale_kernel<<<std::max(1, std::min((std::max(N, M) + 255) / 256, sms * 4)), 256, 0, s>>>(
        da, N, db, M, grad_out, grad_out_dev);
    if (cudaGetLastError() != cudaSuccess) return UOT_ERR_CUDA;
    count_launch(2);
  }
  return UOT_OK;
}

}  // extern "C"
