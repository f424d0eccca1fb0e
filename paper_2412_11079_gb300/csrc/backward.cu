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
// next step's CTAs fold those column partials into G as they start (each
// forms w for its own columns; every column's db and G are written by one of
// them).
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

// A uniform batch: problem k's data sits at fixed strides from problem 0's.
struct BwBatch {
  int64_t sK, sC, sD;  // elements between problems' K, C and dC
  size_t sH, sW;       // bytes between problems' histories and workspaces
};

// Programmatic dependent launch: a reverse step may start while the
// previous one drains; it waits for that grid (complete, memory visible)
// before it touches the adjoint state.
__device__ __forceinline__ void grid_dependency_wait() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}
__device__ __forceinline__ void allow_dependent_launch() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename P>
__device__ __forceinline__ P* at_bytes(P* x, size_t off) {  // x advanced by off bytes
  return reinterpret_cast<P*>(reinterpret_cast<uintptr_t>(x) + off);
}

// One reverse step of every problem of the batch; problem 0's pointers.
struct BwArgs {
  BwBatch B;
  const float* K;
  int64_t ldk;
  int n, m, mpad;
  int cpp;         // CTAs per problem (the grid is batch x cpp)
  const float* a;  // [batch][n]
  const float* b;  // [batch][m]
  float fi;
  int t;           // reverse step (iteration index)
  int first;       // t = T: db is assigned rather than accumulated
  const double* log2k;  // gauge of the forward solve: Q_t = K U'_t V'_{t-1} 2^-e_t
  const float* q;  // U'_t (n)
  const float* pr; // U'_{t-1} (n)
  const float* v;  // V'_{t-1} (mpad)
  const float* r;  // r_t (n)
  const float* c;  // c_t (mpad), for this step's w
  float* F;        // row adjoints (n)
  float* da;       // [batch][n]
  const float* Gs_in;   // (mpad): (1 - fi) G after the previous step's column step
  const float* h_prev;  // (mpad): R^T z of the previous step (colsum(dl) at t = T)
  float* Gs_out;   // (mpad): (1 - fi) G after this step's column step
  float* db;       // [batch][m]
  float* h_next;   // (mpad) column partials R_t^T z, pre-zeroed
  float* h_clear;  // buffer to clear for the next step
  Control* ctl;
  int stages;
  float* Aq;       // (n): q_t = U_t 2^-e_t of this step's rows
  float* Az;       // (n): pz_t = U_{t-1} z_t
  float* Bw;       // (m): v_t w_t of this step's columns
};

// CTA (k, g) of the grid takes problem k's contiguous rows [g R, (g+1) R).
// Each thread holds VE * KV columns: vw = v w for the row reductions
// (Q_t w)_i = U_t,i sum_j K_ij v_j w_j and the column partials
// hh_j = sum_i K_ij pz_i (h = v hh once the block is done).  The row loop is
// software-pipelined: after the barrier that publishes row q's reduction,
// every thread loads row q+1 from the ring and reduces it while it finishes
// row q (pz_q and its column partials), so one barrier per row carries both
// and the two dependency chains overlap.  A row's scalars come from a
// shared chunk loaded 64 rows at a time, and its outputs (F, da, the step
// vectors) are written back per chunk, coalesced: nothing on a row's path
// waits on global memory.
template <int THREADS, int KV, bool TAIL>
__global__ void __launch_bounds__(THREADS, (512 / THREADS > 1 ? 512 / THREADS : 1))
    reverse_pass_kernel(const BwArgs p) {
  constexpr int VE = 4;
  constexpr int NW = THREADS / 32;
  constexpr int W = KV * VE * THREADS;
  constexpr int ROW_BYTES = W * 4;
  constexpr int RCH = 64;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ float sc[6][RCH];  // q 2^-e, U_{t-1}, r, a, F, da of the chunk's rows
  __shared__ float so[2][RCH];  // F + (Q_t w)_i and pz of the chunk's rows
  const int stages = p.stages;
  unsigned char* ring = smem;  // per slot: one row of K
  float* red = reinterpret_cast<float*>(smem + size_t(stages) * ROW_BYTES);  // [2][NW]
  uint64_t* bars = reinterpret_cast<uint64_t*>(red + 2 * NW);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n = p.n, m = p.m;
  const int prob = int(blockIdx.x) / p.cpp, lb = int(blockIdx.x) - prob * p.cpp;
  const size_t oh = size_t(prob) * p.B.sH, ow = size_t(prob) * p.B.sW;
  const float* K = p.K + int64_t(prob) * p.B.sK;
  const float* av = p.a + int64_t(prob) * n;
  const float* bv = p.b + int64_t(prob) * m;
  float* da = p.da + int64_t(prob) * n;
  float* db = p.db + int64_t(prob) * m;
  const float* qv = at_bytes(p.q, oh);
  const float* prv = at_bytes(p.pr, oh);
  const float* vv = at_bytes(p.v, oh);
  const float* rv = at_bytes(p.r, oh);
  float* F = at_bytes(p.F, ow);
  float* h_next = at_bytes(p.h_next, ow);
  float* Aq = at_bytes(p.Aq, ow);
  float* Az = at_bytes(p.Az, ow);
  Control* ctl = at_bytes(p.ctl, ow);
  const uint32_t copy_bytes = uint32_t((size_t(m) * 4) & ~size_t(15));
  uint32_t st = 0;

  allow_dependent_launch();  // the next step's CTAs fill SMs as this grid's leave
  if (tid == 0) {
    for (int s = 0; s < stages; ++s) mbar_init(&bars[s], 1);
    fence_mbar_init();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  const uint64_t policy = policy_evict_first();
  const int R = (n + p.cpp - 1) / p.cpp;
  const int r0 = lb * R;
  const int nrows = max(0, min(n, r0 + R) - r0);
  int armed = 0;  // rows armed so far (thread 0)
  auto arm = [&](int q) {  // row q of the block into slot q % stages
    if (q >= nrows) return;
    const int slot = q % stages;
    if (copy_bytes) {
      mbar_arrive_expect_tx(&bars[slot], copy_bytes);
      bulk_load(ring + size_t(slot) * ROW_BYTES, K + int64_t(r0 + q) * p.ldk, copy_bytes,
                &bars[slot], policy);
    } else {
      mbar_arrive(&bars[slot]);
    }
    armed = q + 1;
  };
  if (tid == 0)
    for (int q = 0; q < stages; ++q) arm(q);  // K is read-only: fetched before the wait
  grid_dependency_wait();
  const float qscale =
      ldexpf(1.0f, -gauge_exponent(p.t, float(*at_bytes(p.log2k, oh))));

  // Column step: G = (1 - fi) G + R^T z of the previous step, w = -fi G / c_t,
  // db += fi G / b; the CTA that owns column j (j / ceil(m / cpp) == its
  // index) writes db_j and (1 - fi) G_j for the next step.
  float vw[KV][VE], hh[KV][VE];
  {
    const float* gin = at_bytes(p.Gs_in, ow);
    const float* hprev = at_bytes(p.h_prev, ow);
    const float* ct = at_bytes(p.c, oh);
    float* gout = at_bytes(p.Gs_out, ow);
    const int own = (m + p.cpp - 1) / p.cpp;
#pragma unroll
    for (int k = 0; k < KV; ++k) {
      const int cc = (k * THREADS + tid) * VE;
#pragma unroll
      for (int e = 0; e < VE; ++e) {
        const int j = cc + e;
        hh[k][e] = 0.0f;
        vw[k][e] = 0.0f;
        if (j < m) {
          const float G = __ldcg(gin + j) + __ldcg(hprev + j);
          vw[k][e] = __ldcg(vv + j) * (-p.fi * G / __ldcg(ct + j));
          if (j / own == lb) {
            db[j] = (p.first ? 0.0f : db[j]) + p.fi * G / __ldg(bv + j);
            gout[j] = (1.0f - p.fi) * G;
          }
        }
      }
    }
  }
  // This step's column vector v_t w_t of the final contraction (every CTA of
  // the problem holds all columns; its first one stores them).
  if (lb == 0) {
    float* Bw = at_bytes(p.Bw, ow);
#pragma unroll
    for (int k = 0; k < KV; ++k) {
      const int cc = (k * THREADS + tid) * VE;
#pragma unroll
      for (int e = 0; e < VE; ++e)
        if (cc + e < m) Bw[cc + e] = vw[k][e];
    }
  }
  {
    float* h_clear = at_bytes(p.h_clear, ow);
    for (int j = lb * THREADS + tid; j < p.mpad; j += p.cpp * THREADS) h_clear[j] = 0.0f;
  }

  auto load_chunk = [&](int q0) {
    for (int i = tid; i < min(RCH, nrows - q0); i += THREADS) {
      const int row = r0 + q0 + i;
      const float qi = __ldcg(qv + row) * qscale;
      sc[0][i] = qi;
      sc[1][i] = __ldcg(prv + row);
      sc[2][i] = __ldcg(rv + row);
      sc[3][i] = __ldg(av + row);
      sc[4][i] = __ldcg(F + row);
      sc[5][i] = __ldcg(da + row);
      Aq[row] = qi;  // this step's row vectors of the final contraction
    }
  };
  // Column step: F += (Q_t w)_i; row step: z, da += fi F / a, F = (1 - fi) F.
  auto flush = [&](int q0, int cnt) {
    for (int i = tid; i < cnt; i += THREADS) {
      const int row = r0 + q0 + i;
      const float Fn = so[0][i];
      da[row] = sc[5][i] + p.fi * Fn / sc[3][i];
      F[row] = (1.0f - p.fi) * Fn;
      Az[row] = so[1][i];
    }
  };
  bool broken = false;
  auto load_row = [&](int q, float (&x)[KV][VE]) {
    const int slot = q % stages;
    if (!broken && !mbar_wait_bounded(&bars[slot], uint32_t(q / stages) & 1u, WAIT_LIMIT_NS)) {
      broken = true;
      st |= DEV_TIMEOUT;
    }
    const unsigned char* sK = ring + size_t(slot) * ROW_BYTES;
    const float* gK = K + int64_t(r0 + q) * p.ldk;
#pragma unroll
    for (int k = 0; k < KV; ++k) {
      const int li = k * THREADS + tid;
      const int cc = li * VE;
      if (!TAIL || cc + VE <= m) {  // without TAIL every vector is in the slot
        Elem<float>::unpack(ld_shared_v4(sK + size_t(li) * 16), x[k]);
      } else {
#pragma unroll
        for (int e = 0; e < VE; ++e) x[k][e] = cc + e < m ? gK[cc + e] : 0.0f;
      }
    }
  };
  auto dot = [&](const float (&x)[KV][VE]) {
    float s4[VE];
#pragma unroll
    for (int e = 0; e < VE; ++e) s4[e] = 0.0f;
#pragma unroll
    for (int k = 0; k < KV; ++k)
#pragma unroll
      for (int e = 0; e < VE; ++e) s4[e] = fmaf(x[k][e], vw[k][e], s4[e]);
    return warp_sum((s4[0] + s4[1]) + (s4[2] + s4[3]));
  };
  auto finish_row = [&](int q, const float (&x)[KV][VE]) {
    const float* rb = red + (q & 1) * NW;
    float S1 = 0.0f;
#pragma unroll
    for (int k = 0; k < NW; ++k) S1 += rb[k];
    const int ci = q % RCH;
    const float Fn = sc[4][ci] + sc[0][ci] * S1;
    const float pz = sc[1][ci] * (-p.fi * Fn / sc[2][ci]);
    if (tid == 0) {
      so[0][ci] = Fn;
      so[1][ci] = pz;
    }
#pragma unroll
    for (int k = 0; k < KV; ++k)
#pragma unroll
      for (int e = 0; e < VE; ++e) hh[k][e] = fmaf(x[k][e], pz, hh[k][e]);
  };

  if (nrows > 0) {
    load_chunk(0);
    float xc[KV][VE];
    load_row(0, xc);
    {
      const float s0 = dot(xc);
      if (lane == 0) red[warp] = s0;
    }
    bool stop = __syncthreads_or(broken ? 1 : 0) != 0;
    if (!stop) {
      if (tid == 0) arm(stages);  // row 0 is in every thread's registers
      // Row q is in xc, row q + 1 goes to xn; the next step swaps the roles
      // (the loop is unrolled by two, so no registers are copied).
      auto step = [&](int q, const float (&xc)[KV][VE], float (&xn)[KV][VE]) {
        if (q > 0 && q % RCH == 0) {  // uniform; rows < q are finished
          flush(q - RCH, RCH);
          __syncthreads();
          load_chunk(q);
          __syncthreads();
        }
        const bool nx = q + 1 < nrows;
        float sn = 0.0f;
        if (nx) {
          load_row(q + 1, xn);
          sn = dot(xn);
        }
        finish_row(q, xc);
        if (nx && lane == 0) red[((q + 1) & 1) * NW + warp] = sn;
        if (__syncthreads_or(broken ? 1 : 0)) return false;
        if (nx && tid == 0) arm(q + 1 + stages);
        return true;
      };
      float xd[KV][VE];
      for (int q = 0; q < nrows; q += 2) {
        if (!step(q, xc, xd)) {
          stop = true;
          break;
        }
        if (q + 1 < nrows && !step(q + 1, xd, xc)) {
          stop = true;
          break;
        }
      }
    }
    if (stop) {
      broken = true;
      st |= DEV_TIMEOUT;
    } else {
      const int q0 = ((nrows - 1) / RCH) * RCH;
      flush(q0, nrows - q0);  // the last barrier published so[] of every row
    }
#pragma unroll
    for (int k = 0; k < KV; ++k) {
      const int cc = (k * THREADS + tid) * VE;
      if (cc + VE <= m) {
        red_add_v4(h_next + cc, __ldcg(vv + cc) * hh[k][0], __ldcg(vv + cc + 1) * hh[k][1],
                   __ldcg(vv + cc + 2) * hh[k][2], __ldcg(vv + cc + 3) * hh[k][3]);
      } else {
#pragma unroll
        for (int e = 0; e < VE; ++e)
          if (cc + e < m) atomicAdd(h_next + cc + e, __ldcg(vv + cc + e) * hh[k][e]);
      }
    }
  }
  if (st) atomicOr(&ctl->status, st);
  if (tid == 0 && broken) {  // let the copies in flight land before exiting
    for (int q = max(0, armed - stages); q < armed; ++q)
      mbar_wait_bounded(&bars[q % stages], uint32_t(q / stages) & 1u, WAIT_LIMIT_NS);
  }
}

constexpr int TB = 256;

// Clears the adjoint state of every problem's workspace (grid.y = problem).
__global__ void __launch_bounds__(TB) bw_zero_kernel(unsigned char* ws, size_t bytes, size_t sW) {
  uint4* z = reinterpret_cast<uint4*>(ws + size_t(blockIdx.y) * sW);
  for (size_t i = blockIdx.x * size_t(TB) + threadIdx.x; i < bytes / 16; i += size_t(gridDim.x) * TB)
    z[i] = make_uint4(0u, 0u, 0u, 0u);
}

// The adjoint's start, one read of K and C: dl = P_T * C with P_T =
// (U_i K_ij) V_j (not stored: the final contraction forms it again),
// F = rowsum(dl) and G0 = colsum(dl), da = 0.  A thread takes four
// consecutive columns of a block of rows: its column sums stay in registers
// (one atomic each at the end) and each row's sum is reduced over the CTA
// (one atomic per row and CTA).  grid = (column blocks, row blocks, problem).
constexpr int ST_ROWS = 32;
__global__ void __launch_bounds__(TB) bw_start_kernel(const float* K, int64_t ldk, const float* C,
                                                      int64_t ldc, const float* U, const float* V,
                                                      int n, int m, float* F, float* G0,
                                                      float* da, BwBatch B) {
  __shared__ float part[TB / 32][ST_ROWS];
  const int k = blockIdx.z;
  K += int64_t(k) * B.sK;
  C += int64_t(k) * B.sC;
  U = at_bytes(U, size_t(k) * B.sH);
  V = at_bytes(V, size_t(k) * B.sH);
  F = at_bytes(F, size_t(k) * B.sW);
  G0 = at_bytes(G0, size_t(k) * B.sW);
  da += int64_t(k) * n;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j = (blockIdx.x * TB + threadIdx.x) * 4;
  const int r0 = blockIdx.y * ST_ROWS, r1 = min(n, r0 + ST_ROWS);
  float v[4], g[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
  for (int e = 0; e < 4; ++e) v[e] = j + e < m ? V[j + e] : 0.0f;
  for (int i = r0; i < r1; ++i) {
    const float u = U[i];
    float s = 0.0f;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      if (j + e < m) {
        const float dl = (u * __ldg(K + int64_t(i) * ldk + j + e)) * v[e] *
                         __ldg(C + int64_t(i) * ldc + j + e);
        g[e] += dl;
        s += dl;
      }
    }
    s = warp_sum(s);
    if (lane == 0) part[warp][i - r0] = s;
  }
  __syncthreads();
  if (warp == 0) {
    for (int i = r0 + lane; i < r1; i += 32) {
      float s = 0.0f;
#pragma unroll
      for (int w = 0; w < TB / 32; ++w) s += part[w][i - r0];
      atomicAdd(F + i, s);
      if (blockIdx.x == 0) da[i] = 0.0f;
    }
  }
#pragma unroll
  for (int e = 0; e < 4; ++e)
    if (j + e < m && r1 > r0) atomicAdd(G0 + j + e, g[e]);
}

// The final contraction: acc = A B^T over the 2T recorded step vectors
// (A_s = q_t or pz_t of the rows, B_s = v_t w_t or v_t of the columns), then
//     dl = P_T * C + K * acc,   dC = g (P_T - dl / reg),
// with g = grad_out times the optional device scalar (read here, so the
// caller need not synchronise).  FP32 on the CUDA cores (the depth-2T sum
// needs FP32 accuracy): 128 x 128 tiles of 256 threads, 8 x 8 outputs per
// thread (rows ty*4 + {0..3} and 64 + ty*4 + {0..3}, columns likewise with
// tx, so the 16-byte shared loads of a warp hit distinct banks), slabs of 16
// depth steps in two shared buffers: the next slab is fetched into
// registers (16-byte loads) while the current one is used, one barrier per
// slab, and the FMAs packed in pairs.  The step vectors are padded to 128
// entries (the workspace layout), so a tile's loads stay inside them.
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
  const double* g_dev;  // one per problem, or NULL
  BwBatch B;
};

__global__ void __launch_bounds__(GT, 2) bw_gemm_kernel(BwGemmArgs p) {
  {  // problem blockIdx.z of the batch
    const int k = blockIdx.z;
    const size_t oh = size_t(k) * p.B.sH, ow = size_t(k) * p.B.sW;
    p.K += int64_t(k) * p.B.sK;
    p.C += int64_t(k) * p.B.sC;
    p.D += int64_t(k) * p.B.sD;
    p.UT = at_bytes(p.UT, oh);
    p.VT = at_bytes(p.VT, oh);
    p.Vh = at_bytes(p.Vh, oh);
    p.Aq = at_bytes(p.Aq, ow);
    p.Az = at_bytes(p.Az, ow);
    p.Bw = at_bytes(p.Bw, ow);
    if (p.g_dev) p.g_dev += k;
  }
  __shared__ __align__(16) float As[2][GKD][GB];
  __shared__ __align__(16) float Bs[2][GKD][GB];
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int i0 = blockIdx.y * GB, j0 = blockIdx.x * GB;
  const int S = 2 * p.T;
  // Loader: float4 number f = tid + 256 h (h = 0, 1) of a slab's 16 x 32.
  float4 ra[2], rb[2];
  auto fetch = [&](int s0) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int f = tid + h * GT, row = f / 32, c4 = (f % 32) * 4;
      const int sidx = s0 + row;
      ra[h] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      rb[h] = ra[h];
      if (sidx < p.T) {
        ra[h] = __ldg(reinterpret_cast<const float4*>(p.Aq + sidx * p.sn + i0 + c4));
        rb[h] = __ldg(reinterpret_cast<const float4*>(p.Bw + sidx * p.sm + j0 + c4));
      } else if (sidx < S) {
        ra[h] = __ldg(reinterpret_cast<const float4*>(p.Az + (sidx - p.T) * p.sn + i0 + c4));
        rb[h] = __ldg(reinterpret_cast<const float4*>(p.Vh + (sidx - p.T) * p.sv + j0 + c4));
      }
    }
  };
  auto stash = [&](int buf) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int f = tid + h * GT, row = f / 32, c4 = (f % 32) * 4;
      *reinterpret_cast<float4*>(&As[buf][row][c4]) = ra[h];
      *reinterpret_cast<float4*>(&Bs[buf][row][c4]) = rb[h];
    }
  };
  float2 acc[8][4];  // rows r, column pairs
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = make_float2(0.0f, 0.0f);
  if (S > 0) {
    fetch(0);
    stash(0);
  }
  __syncthreads();
  int cur = 0;
  for (int s0 = 0; s0 < S; s0 += GKD) {
    const bool more = s0 + GKD < S;
    if (more) fetch(s0 + GKD);
#pragma unroll
    for (int kk = 0; kk < GKD; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[cur][kk][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[cur][kk][64 + ty * 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[cur][kk][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[cur][kk][64 + tx * 4]);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float2 b[4] = {make_float2(b0.x, b0.y), make_float2(b0.z, b0.w),
                           make_float2(b1.x, b1.y), make_float2(b1.z, b1.w)};
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = ffma2(make_float2(a[r], a[r]), b[c], acc[r][c]);
    }
    if (more) stash(cur ^ 1);
    __syncthreads();
    cur ^= 1;
  }
  const float g = float(p.g_dev ? p.g_host * *p.g_dev : p.g_host);
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int i = i0 + (r < 4 ? ty * 4 + r : 64 + ty * 4 + r - 4);
    if (i >= p.n) continue;
    const float u = p.UT[i];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int j = j0 + (c < 4 ? tx * 4 + c : 64 + tx * 4 + c - 4);
      if (j >= p.m) continue;
      const float k = p.K[int64_t(i) * p.ldk + j];
      const float P = (u * k) * p.VT[j];
      const float a = (c & 1) ? acc[r][c / 2].y : acc[r][c / 2].x;
      const float dl = fmaf(k, a, P * p.C[int64_t(i) * p.ldc + j]);
      p.D[int64_t(i) * p.ldd + j] = g * (P - dl * p.inv_reg);
    }
  }
}

// da *= g, db *= g (grid.y = problem).
__global__ void bw_scale_kernel(float* da, int n, float* db, int m, double g_host,
                                const double* g_dev) {
  da += int64_t(blockIdx.y) * n;
  db += int64_t(blockIdx.y) * m;
  const float g = float(g_dev ? g_host * g_dev[blockIdx.y] : g_host);
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
  const void* fn[2];  // [rows of a multiple of 4 columns, any width]
};
#define BW_ENTRY(TH, KV)                                                        \
  BwEntry {                                                                      \
    TH, KV, {reinterpret_cast<const void*>(&reverse_pass_kernel<TH, KV, false>), \
             reinterpret_cast<const void*>(&reverse_pass_kernel<TH, KV, true>)}  \
  }
// Four vectors per thread (four warps for rows of 2048 columns, four CTAs
// per SM): a reverse step's CTA barrier per row is cheapest with few warps,
// and the per-row latency is hidden by CTAs side by side rather than by wider
// CTAs (measured with one launch per problem and step: 512 x 1 69 ms,
// 256 x 2 55 ms, 128 x 4 48 ms per gradient step; a fifth CTA per SM, at
// 96 registers, made the batched launches slower).
const BwEntry kBw[] = {BW_ENTRY(512, 4), BW_ENTRY(256, 4), BW_ENTRY(128, 4),
                       BW_ENTRY(128, 2), BW_ENTRY(64, 2),  BW_ENTRY(32, 2)};
constexpr int kBwNum = int(sizeof(kBw) / sizeof(kBw[0]));

size_t bw_smem(const BwEntry& e, int stages) {
  const size_t row = size_t(e.threads) * e.kv * 16;
  return size_t(stages) * row + 2 * (e.threads / 32) * 4 + size_t(stages) * 8;
}

// Backward workspace: the adjoint state (cleared at the start of a call),
// then the step vectors of the final contraction (T rows each, written
// before they are read).
struct BwLayout {
  size_t ctl, F, Gs[2], G0, h[3], state_end, Aq, Az, Bw, total;
  size_t npad, mpad;  // floats
};
BwLayout bw_layout(int64_t n, int64_t m, int T) {
  BwLayout L{};
  L.npad = size_t((n + 127) & ~int64_t(127));  // step vectors of whole 128-entry tiles
  L.mpad = size_t((m + 127) & ~int64_t(127));
  const size_t npad = L.npad * 4, mpad = L.mpad * 4;
  size_t off = 0;
  L.ctl = off; off = align256(off + sizeof(Control));
  L.F = off; off = align256(off + npad);
  for (int k = 0; k < 2; ++k) { L.Gs[k] = off; off = align256(off + mpad); }
  L.G0 = off; off = align256(off + mpad);
  for (int k = 0; k < 3; ++k) { L.h[k] = off; off = align256(off + mpad); }
  L.state_end = off;
  L.Aq = off; off = align256(off + size_t(T) * npad);
  L.Az = off; off = align256(off + size_t(T) * npad);
  L.Bw = off; off = align256(off + size_t(T) * mpad);
  L.total = off;
  return L;
}

std::mutex g_bw_mu;
size_t g_bw_smem_set[64][kBwNum][2];

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

}  // extern "C"

namespace {

// The adjoint of `batch` problems of one shape; problem k's arrays at the
// given strides from problem 0's (a, b, da, db packed: n or m apart).
uot_status backward_run(int32_t batch, const float* K, int64_t ldk, int64_t sK, const float* C,
                        int64_t ldc, int64_t sC, const float* a, const float* b, int64_t n,
                        int64_t m, float reg, float reg_m, int32_t iters, const void* hist,
                        size_t hist_bytes, size_t sH, double grad_out,
                        const double* grad_out_dev, float* dC, int64_t lddc, int64_t sD,
                        float* da, float* db, void* workspace, size_t ws_bytes,
                        const uot_options* opt, void* stream) {
  const int max_ctas = opt ? opt->max_ctas : 0;
  if (max_ctas < 0 || batch < 1 || batch > 65535) return UOT_ERR_INVALID_ARG;
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
  const int T = iters, N = int(n), M = int(m);
  const HistLayout HL = hist_layout(n, m, T);
  if (hist_bytes < HL.total) return UOT_ERR_INVALID_ARG;
  if (batch > 1) {  // problems neither overlap nor lose the alignment of problem 0
    if (sK < (n - 1) * ldk + m || sC < (n - 1) * ldc + m || sD < (n - 1) * lddc + m ||
        sK % 4 || sD % 4 || sH < HL.total || sH % 256 ||
        reinterpret_cast<uintptr_t>(hist) % 256)
      return UOT_ERR_INVALID_ARG;
  }
  const BwLayout L = bw_layout(n, m, T);
  if (!workspace || ws_bytes / size_t(batch) < L.total ||
      reinterpret_cast<uintptr_t>(workspace) % 256)
    return UOT_ERR_WORKSPACE;
  int k = -1;
  for (int i = 0; i < kBwNum; ++i)
    if (kBw[i].threads * kBw[i].kv * 4 >= M &&
        (k < 0 || kBw[i].threads * kBw[i].kv < kBw[k].threads * kBw[k].kv))
      k = i;
  if (k < 0) return UOT_ERR_UNSUPPORTED;  // rows wider than one CTA (8192 columns)
  if ((N + GB - 1) / GB > 65535) return UOT_ERR_UNSUPPORTED;

  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const BwBatch Bt{sK, sC, sD, sH, L.total};
  const double fi_d = std::isinf(reg_m) ? 1.0 : double(reg_m) / (double(reg_m) + double(reg));
  const float fi = float(fi_d);
  uint8_t* ws = static_cast<uint8_t*>(workspace);
  const uint8_t* hb = static_cast<const uint8_t*>(hist);
  auto U_t = [&](int t) { return reinterpret_cast<const float*>(hb + HL.U + size_t(t) * HL.strideU); };
  auto V_t = [&](int t) { return reinterpret_cast<const float*>(hb + HL.V + size_t(t) * HL.strideV); };
  auto r_t = [&](int t) { return reinterpret_cast<const float*>(hb + HL.r + size_t(t) * HL.strideU); };
  auto c_t = [&](int t) { return reinterpret_cast<const float*>(hb + HL.c + size_t(t) * HL.strideV); };
  float* F = reinterpret_cast<float*>(ws + L.F);
  float* G0 = reinterpret_cast<float*>(ws + L.G0);
  Control* ctl = reinterpret_cast<Control*>(ws + L.ctl);
  float* Aq = reinterpret_cast<float*>(ws + L.Aq);
  float* Az = reinterpret_cast<float*>(ws + L.Az);
  float* Bw = reinterpret_cast<float*>(ws + L.Bw);

  int dev = 0, sms = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return UOT_ERR_CUDA;
  const int per_prob = std::max(1, sms * 8 / batch);  // blocks of the one-off kernels
  bw_zero_kernel<<<dim3(std::max(1, std::min(per_prob, int(L.state_end / (16 * TB)) + 1)), batch),
                   TB, 0, s>>>(ws, L.state_end, L.total);
  if (cudaGetLastError() != cudaSuccess) return UOT_ERR_CUDA;
  if ((N + ST_ROWS - 1) / ST_ROWS > 65535) return UOT_ERR_UNSUPPORTED;
  bw_start_kernel<<<dim3((M + 4 * TB - 1) / (4 * TB), (N + ST_ROWS - 1) / ST_ROWS, batch), TB, 0,
                    s>>>(K, ldk, C, ldc, U_t(T), V_t(T), N, M, F, G0, da, Bt);
  if (cudaGetLastError() != cudaSuccess) return UOT_ERR_CUDA;
  count_launch(2);
  if (T == 0 && cudaMemsetAsync(db, 0, size_t(batch) * size_t(M) * 4, s) != cudaSuccess)
    return UOT_ERR_CUDA;

  // Geometry of the reverse pass: as many CTAs as fit on the GPU at once,
  // shared evenly among the problems (at least two rows each).
  const BwEntry& e = kBw[k];
  const int tail = M % 4 ? 1 : 0;
  const void* fn = e.fn[tail];
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
      if (dev < 64 && g_bw_smem_set[dev][k][tail] < b2) {
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(b2)) !=
            cudaSuccess)
          return UOT_ERR_CUDA;
        g_bw_smem_set[dev][k][tail] = b2;
      }
    }
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, e.threads, b2) != cudaSuccess)
      return UOT_ERR_CUDA;
    if (occ == 0) break;
    if (st == 2) best_occ = occ;
    if (occ < best_occ) break;
    best_st = st;
  }
  if (best_occ == 0) return UOT_ERR_CUDA;
  const size_t smem = bw_smem(e, best_st);
  int total = best_occ * sms;
  if (max_ctas > 0 && total > max_ctas) total = max_ctas;
  const int cpp = std::max(1, std::min(total / batch, (N + 1) / 2));

  BwArgs A{};
  A.B = Bt;
  A.K = K;
  A.ldk = ldk;
  A.n = N;
  A.m = M;
  A.mpad = int(L.mpad);
  A.cpp = cpp;
  A.a = a;
  A.b = b;
  A.fi = fi;
  A.F = F;
  A.da = da;
  A.db = db;
  A.ctl = ctl;
  A.stages = best_st;
  A.log2k = reinterpret_cast<const double*>(hb);  // HistHeader::log2k
  for (int t = T; t >= 1; --t) {
    const int q = T - t;  // pass counter for the rings
    A.t = t;
    A.first = q == 0;
    A.q = U_t(t);
    A.pr = U_t(t - 1);
    A.v = V_t(t - 1);
    A.r = r_t(t);
    A.c = c_t(t);
    // G enters step T as colsum(dl) (Gs zero); later steps fold the previous
    // step's partials.  h cycles through three buffers: the previous step's
    // (read), this step's (accumulated) and the next step's (cleared).
    A.Gs_in = reinterpret_cast<const float*>(ws + L.Gs[q % 2]);
    A.Gs_out = reinterpret_cast<float*>(ws + L.Gs[(q + 1) % 2]);
    A.h_prev = q == 0 ? G0 : reinterpret_cast<const float*>(ws + L.h[(q + 2) % 3]);
    A.h_next = reinterpret_cast<float*>(ws + L.h[q % 3]);
    A.h_clear = reinterpret_cast<float*>(ws + L.h[(q + 1) % 3]);
    A.Aq = Aq + size_t(t - 1) * L.npad;
    A.Az = Az + size_t(t - 1) * L.npad;
    A.Bw = Bw + size_t(t - 1) * L.mpad;
    void* kargs[] = {&A};
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(batch * cpp);
    cfg.blockDim = dim3(e.threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelExC(&cfg, fn, kargs) != cudaSuccess) return UOT_ERR_CUDA;
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
    G.B = Bt;
    const dim3 gg((M + GB - 1) / GB, (N + GB - 1) / GB, batch);
    bw_gemm_kernel<<<gg, GT, 0, s>>>(G);
    if (cudaGetLastError() != cudaSuccess) return UOT_ERR_CUDA;
    bw_scale_kernel<<<dim3(std::max(1, std::min((std::max(N, M) + 255) / 256, per_prob)), batch),
                      256, 0, s>>>(da, N, db, M, grad_out, grad_out_dev);
    if (cudaGetLastError() != cudaSuccess) return UOT_ERR_CUDA;
    count_launch(2);
  }
  return UOT_OK;
}

}  // namespace

extern "C" {

uot_status uot_sinkhorn_backward(const float* K, int64_t ldk, const float* C, int64_t ldc,
                                 const float* a, const float* b, int64_t n, int64_t m, float reg,
                                 float reg_m, int32_t iters, const void* hist, size_t hist_bytes,
                                 double grad_out, const double* grad_out_dev, float* dC,
                                 int64_t lddc, float* da, float* db, void* workspace,
                                 size_t ws_bytes, const uot_options* opt, void* stream) {
  return backward_run(1, K, ldk, 0, C, ldc, 0, a, b, n, m, reg, reg_m, iters, hist, hist_bytes, 0,
                      grad_out, grad_out_dev, dC, lddc, 0, da, db, workspace, ws_bytes, opt,
                      stream);
}

size_t uot_backward_batch_workspace_size(int32_t batch, int64_t n, int64_t m, int32_t iters) {
  const size_t one = uot_backward_workspace_size(n, m, iters);
  if (one == 0 || batch < 1 || batch > 65535 || one > SIZE_MAX / size_t(batch)) return 0;
  return one * size_t(batch);
}

uot_status uot_sinkhorn_backward_batch(int32_t batch, const float* K, int64_t ldk,
                                       int64_t stride_k, const float* C, int64_t ldc,
                                       int64_t stride_c, const float* a, const float* b,
                                       int64_t n, int64_t m, float reg, float reg_m,
                                       int32_t iters, const void* hist, size_t hist_stride,
                                       double grad_out, const double* grad_out_dev, float* dC,
                                       int64_t lddc, int64_t stride_dc, float* da, float* db,
                                       void* workspace, size_t ws_bytes, const uot_options* opt,
                                       void* stream) {
  return backward_run(batch, K, ldk, stride_k, C, ldc, stride_c, a, b, n, m, reg, reg_m, iters,
                      hist, hist_stride, hist_stride, grad_out, grad_out_dev, dC, lddc, stride_dc,
                      da, db, workspace, ws_bytes, opt, stream);
}

}  // extern "C"
