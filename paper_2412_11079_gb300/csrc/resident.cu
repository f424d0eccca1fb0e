// Batched Sinkhorn-UOT, on-chip form.  A problem whose initial plan fits in
// the shared memory of one CTA, or of a cluster of up to 16 CTAs, runs all
// its iterations (the rule of Section 2.1 with Algorithm 1's single sweep per
// iteration, in kernel form: plan = diag(U) K diag(V)) with K held in shared
// memory.  K is read from global memory once and the plan written once; each
// iteration reads only shared memory, so these problems are bound by shared
// memory bandwidth and barrier latency rather than by HBM.
//
// Layout.  CTA r of a cluster of cs holds rows [r nb, (r + 1) nb) of K,
// nb = ceil(N / cs), with row stride ldk = M rounded up to 4 (padding
// zeroed); U and a of those rows; a copy of the column scalings V; and, for
// the contiguous slice of columns it owns, b and the column partials pushed
// to it by every CTA of the cluster.
//
// Iteration t, in phases over the CTA's rows; each thread covers 4 16-byte
// chunks of a row, gt threads per row (the smallest power of two with
// 16 gt >= M), R = 512 / gt rows at a time:
//   (a) sums of K_ij V_j per row (partials per warp);
//   (b) one thread per row: U_i <- U_i alpha_i 2^e_t with
//       r_i = U_i sum_j K_ij V_j (one power per row, not one per thread);
//   (c) column partials of U_i K_ij in registers (K read a second time),
//       combined over the CTA's units (warps sharing columns are combined by
//       shuffles, the rest by a two-level shared-memory sum);
//   (d) cs > 1: each CTA pushes the partials of every column slice to the
//       slice's owner (distributed shared memory stores), cluster barrier;
//   (e) each owner sums the partials in rank order and forms
//       V_j <- V_j (b_j / c_j)^fi 2^-e_t with c_j = V_j 2^-e_t sum_i U_i K_ij,
//       writing V_j into every CTA's copy; barrier (cluster barrier if cs > 1).
// After the last iteration each CTA writes its rows of diag(U) K diag(V)
// over the initial plan.  2^e_t is the exact power-of-two gauge of the
// kernel form (the scalings drift as U ~ k^t, V ~ k^-t when the masses
// differ).
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "batched_internal.h"
#include "uot_device.cuh"

namespace uot {

namespace {

constexpr int RT = 512;                   // threads per CTA
constexpr int RKV = 4;                    // 16-byte chunks per thread per row
constexpr int RMAX_M = RT / 2 * RKV * 4;  // widest row: two row groups per CTA

struct ResidentArgs {
  const BatchProblem* probs;
  const int* order;
  int count;
  int* cursor;
};

__device__ __forceinline__ void cta_or_cluster_sync(int cs) {
  if (cs > 1)
    cluster_sync();
  else
    __syncthreads();
}

// Threads per row and partial-sum units for a row width of c4 chunks: units
// are warps when several rows share a warp (gt < 32), else row groups.
struct ResGeom {
  int gt, R, units, wpg;
};
__host__ __device__ __forceinline__ ResGeom res_geom(int c4) {
  int gt = 1;
  while (gt * RKV < c4) gt <<= 1;
  ResGeom g;
  g.gt = gt;
  g.R = RT / gt;
  g.units = gt < 32 ? RT / 32 : RT / gt;
  g.wpg = gt > 32 ? gt / 32 : 1;
  return g;
}

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, const float4& v) { *reinterpret_cast<float4*>(p) = v; }

__global__ void __launch_bounds__(RT, 1) resident_kernel(const ResidentArgs A) {
  extern __shared__ __align__(128) float smem[];
  __shared__ int s_prob;
  const int cs = int(cluster_nctarank());
  const int rank = int(cluster_ctarank());
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  while (true) {
    // Rank 0 takes the next problem of the queue and hands it to the cluster.
    if (rank == 0 && tid == 0) {
      const int pos = atomicAdd(A.cursor, 1);
      const int idx = pos < A.count ? A.order[pos] : -1;
      if (cs > 1) {
        for (int r = 0; r < cs; ++r) st_cluster_s32(map_shared_rank(&s_prob, uint32_t(r)), idx);
      } else {
        s_prob = idx;
      }
    }
    cta_or_cluster_sync(cs);
    const int pi = s_prob;
    // Every CTA has read the index before rank 0 may write the next one.
    cta_or_cluster_sync(cs);
    if (pi < 0) break;

    const BatchProblem P = A.probs[pi];
    const int n = P.n, m = P.m;
    const int ldk = (m + 3) & ~3, c4 = ldk >> 2;
    const int nb = (n + cs - 1) / cs;
    const int i0 = rank * nb;
    const int nloc = max(0, min(n - i0, nb));
    const int mb4 = (c4 + cs - 1) / cs;  // chunks of columns owned per CTA
    const int slice = mb4 * 4;
    const int ch0 = rank * mb4, ch1 = min(c4, ch0 + mb4);  // owned chunks
    const ResGeom G = res_geom(c4);
    const int gt = G.gt, R = G.R, g = tid / gt, l = tid - g * gt;
    const int wpg = G.wpg, wg = warp % wpg;
    // Partial-sum unit of this thread, and whether it holds the unit's values.
    const int unit = gt < 32 ? warp : g;
    const bool holder = gt >= 32 || lane < gt;
    const int half = G.units / 2;
    float* Ks = smem;
    float* Vs = Ks + size_t(nb) * ldk;
    float* W = Vs + ldk;                 // half x ldk unit partials
    float* bs = W + size_t(half) * ldk;  // b of the owned slice
    float* recv = bs + slice;            // cs x slice partials pushed by every CTA
    float* rsp = recv + (cs > 1 ? cs * slice : 0);  // wpg x nb partial row sums
    float* Ul = rsp + wpg * nb;
    float* al = Ul + nb;

    // Load this CTA's rows of K (16-byte chunks; rows start 16-byte aligned
    // and the leading dimension covers the last chunk), zero the padding.
    for (int idx = tid; idx < nloc * c4; idx += RT) {
      const int r = idx / c4, ch = idx - r * c4;
      float4 v = __ldcs(reinterpret_cast<const float4*>(P.plan + int64_t(i0 + r) * P.ldp) + ch);
      const int cc = ch * 4;
      if (cc + 1 >= m) v.y = 0.0f;  // cc < m: only the last chunk is partial
      if (cc + 2 >= m) v.z = 0.0f;
      if (cc + 3 >= m) v.w = 0.0f;
      st4(Ks + size_t(r) * ldk + cc, v);
    }
    for (int j = tid; j < ldk; j += RT) Vs[j] = j < m ? 1.0f : 0.0f;
    for (int j = ch0 * 4 + tid; j < min(m, ch1 * 4); j += RT) bs[j - ch0 * 4] = __ldg(P.b + j);
    for (int r = tid; r < nloc; r += RT) {
      Ul[r] = 1.0f;
      al[r] = __ldg(P.a + i0 + r);
    }
    __syncthreads();

    float V[RKV][4];
    auto load_v = [&]() {
#pragma unroll
      for (int k = 0; k < RKV; ++k) {
        const int ch = l + k * gt;
        const float4 v4 = ch < c4 ? ld4(Vs + ch * 4) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        V[k][0] = v4.x;
        V[k][1] = v4.y;
        V[k][2] = v4.z;
        V[k][3] = v4.w;
      }
    };
    load_v();

    const float Lf = float(*P.log2k);
    const float fi = P.fi;
    uint32_t st = 0;
    const int wr = gt < 32 ? gt : 32;  // lanes of one row within a warp
    for (int t = 1; t <= P.iters; ++t) {
      const int ex = gauge_exponent(t, Lf);
      const float gauge = ldexpf(1.0f, ex), inv_gauge = ldexpf(1.0f, -ex);

      // (a) Row sums of K_ij V_j, two rows per group at a time, reduced over
      // the row's lanes in each warp; one partial per warp of the group.
      // The trip count is the same for every thread (rows past the block
      // join the shuffles with zeros).
      for (int base = 0; base < nloc; base += 2 * R) {
        const int ia = base + g, ib = base + R + g;
        const bool la = ia < nloc, lb = ib < nloc;
        float pa[RKV], pb[RKV];
#pragma unroll
        for (int k = 0; k < RKV; ++k) {
          const int ch = l + k * gt;
          pa[k] = 0.0f;
          pb[k] = 0.0f;
          if (ch < c4) {
            if (la) {
              const float4 v4 = ld4(Ks + size_t(ia) * ldk + ch * 4);
              pa[k] = fmaf(v4.w, V[k][3], fmaf(v4.z, V[k][2], fmaf(v4.y, V[k][1], v4.x * V[k][0])));
            }
            if (lb) {
              const float4 v4 = ld4(Ks + size_t(ib) * ldk + ch * 4);
              pb[k] = fmaf(v4.w, V[k][3], fmaf(v4.z, V[k][2], fmaf(v4.y, V[k][1], v4.x * V[k][0])));
            }
          }
        }
        float sa = (pa[0] + pa[1]) + (pa[2] + pa[3]);
        float sb = (pb[0] + pb[1]) + (pb[2] + pb[3]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          if (o < wr) {
            sa += __shfl_xor_sync(0xffffffffu, sa, o);
            sb += __shfl_xor_sync(0xffffffffu, sb, o);
          }
        }
        if ((lane & (wr - 1)) == 0) {
          if (la) rsp[wg * nb + ia] = sa;
          if (lb) rsp[wg * nb + ib] = sb;
        }
      }
      __syncthreads();
      // (b) Row factors, one thread per row: U_i <- U_i alpha_i 2^e_t with
      // r_i = U_i sum_j K_ij V_j.
      for (int i = tid; i < nloc; i += RT) {
        float sum = 0.0f;
        for (int w = 0; w < wpg; ++w) sum += rsp[w * nb + i];
        const float u_old = Ul[i];
        Ul[i] = P.pot ? rescale_factor(al[i], sum, fi, st)
                      : u_old * rescale_factor(al[i], u_old * sum, fi, st) * gauge;
      }
      __syncthreads();
      // (c) Column partials of U_i K_ij over this CTA's rows.
      float cacc[RKV][4];
#pragma unroll
      for (int k = 0; k < RKV; ++k)
#pragma unroll
        for (int e = 0; e < 4; ++e) cacc[k][e] = 0.0f;
      for (int i = g; i < nloc; i += R) {
        const float u = Ul[i];
        const float* krow = Ks + size_t(i) * ldk;
#pragma unroll
        for (int k = 0; k < RKV; ++k) {
          const int ch = l + k * gt;
          if (ch < c4) {
            const float4 v4 = ld4(krow + ch * 4);
            cacc[k][0] = fmaf(u, v4.x, cacc[k][0]);
            cacc[k][1] = fmaf(u, v4.y, cacc[k][1]);
            cacc[k][2] = fmaf(u, v4.z, cacc[k][2]);
            cacc[k][3] = fmaf(u, v4.w, cacc[k][3]);
          }
        }
      }
      // Rows sharing a warp hold the same columns: combine them by shuffles.
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        if (o >= gt) {
#pragma unroll
          for (int k = 0; k < RKV; ++k)
#pragma unroll
            for (int e = 0; e < 4; ++e) cacc[k][e] += __shfl_xor_sync(0xffffffffu, cacc[k][e], o);
        }
      }
      // Units [half, units) hand their partials to units [0, half), which
      // store the pair sums; the column sums are then over `half` copies.
      if (holder && unit >= half) {
#pragma unroll
        for (int k = 0; k < RKV; ++k) {
          const int ch = l + k * gt;
          if (ch < c4)
            st4(W + size_t(unit - half) * ldk + ch * 4,
                make_float4(cacc[k][0], cacc[k][1], cacc[k][2], cacc[k][3]));
        }
      }
      __syncthreads();
      if (holder && unit < half) {
#pragma unroll
        for (int k = 0; k < RKV; ++k) {
          const int ch = l + k * gt;
          if (ch < c4) {
            float* w = W + size_t(unit) * ldk + ch * 4;
            const float4 o4 = ld4(w);
            st4(w, make_float4(cacc[k][0] + o4.x, cacc[k][1] + o4.y, cacc[k][2] + o4.z,
                               cacc[k][3] + o4.w));
          }
        }
      }
      __syncthreads();
      auto chunk_sum = [&](int ch) {
        float4 s4 = ld4(W + ch * 4);
        for (int u = 1; u < half; ++u) {
          const float4 o4 = ld4(W + size_t(u) * ldk + ch * 4);
          s4.x += o4.x;
          s4.y += o4.y;
          s4.z += o4.z;
          s4.w += o4.w;
        }
        return s4;
      };
      // Column step on 4 columns: V_j <- V_j (b_j / c_j)^fi 2^-e_t.
      auto column_step = [&](int ch, const float4& c4sum) {
        const float4 v4 = ld4(Vs + ch * 4);
        const float vv[4] = {v4.x, v4.y, v4.z, v4.w};
        const float cc[4] = {c4sum.x, c4sum.y, c4sum.z, c4sum.w};
        float vn[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int j = ch * 4 + e;
          if (j < m) {
            const float cj = vv[e] * cc[e] * inv_gauge;
            vn[e] = P.pot ? rescale_factor(bs[j - ch0 * 4], cc[e], fi, st)
                          : vv[e] * rescale_factor(bs[j - ch0 * 4], cj, fi, st) * inv_gauge;
          } else {
            vn[e] = 0.0f;
          }
        }
        return make_float4(vn[0], vn[1], vn[2], vn[3]);
      };
      if (cs == 1) {
        for (int ch = tid; ch < c4; ch += RT) st4(Vs + ch * 4, column_step(ch, chunk_sum(ch)));
        __syncthreads();
      } else {
        // (d) Push every chunk's partial to the owner of its slice.
        for (int ch = tid; ch < c4; ch += RT) {
          const int owner = ch / mb4;
          st_cluster_v4(map_shared_rank(recv + rank * slice + (ch - owner * mb4) * 4,
                                        uint32_t(owner)),
                        chunk_sum(ch));
        }
        cluster_sync();
        // (e) Owned chunks: partials of every CTA in rank order.
        for (int ch = ch0 + tid; ch < ch1; ch += RT) {
          float4 s4 = ld4(recv + (ch - ch0) * 4);
          for (int r = 1; r < cs; ++r) {
            const float4 o4 = ld4(recv + r * slice + (ch - ch0) * 4);
            s4.x += o4.x;
            s4.y += o4.y;
            s4.z += o4.z;
            s4.w += o4.w;
          }
          const float4 vn = column_step(ch, s4);
          for (int r = 0; r < cs; ++r) st_cluster_v4(map_shared_rank(Vs + ch * 4, uint32_t(r)), vn);
        }
        cluster_sync();
      }
      load_v();
    }

    // The plan diag(U) K diag(V) over the initial plan.
    for (int i = g; i < nloc; i += R) {
      const float u = Ul[i];
      const float* krow = Ks + size_t(i) * ldk;
      float* grow = P.plan + int64_t(i0 + i) * P.ldp;
#pragma unroll
      for (int k = 0; k < RKV; ++k) {
        const int ch = l + k * gt;
        if (ch >= c4) continue;
        const float4 v4 = ld4(krow + ch * 4);
        const float xv[4] = {v4.x, v4.y, v4.z, v4.w};
        float y[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) y[e] = (xv[e] * V[k][e]) * u;
        const int cc = ch * 4;
        if (cc + 4 <= m) {
          st_global_cs_v4(grow + cc, Elem<float>::pack(y));
        } else {
#pragma unroll
          for (int e = 0; e < 4; ++e)
            if (cc + e < m) grow[cc + e] = y[e];
        }
      }
    }
    if (st) atomicOr(&P.ctl->status, st);
    if (rank == 0 && tid == 0) P.ctl->iters_done = P.iters;
  }
}

std::mutex g_res_mu;
bool g_res_attr_set[64];

cudaError_t ensure_resident_attributes(int dev, size_t cap) {
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_res_mu);
  if (g_res_attr_set[dev]) return cudaSuccess;
  cudaError_t err = cudaFuncSetAttribute(resident_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, int(cap));
  if (err != cudaSuccess) return err;
  err = cudaFuncSetAttribute(resident_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (err != cudaSuccess) return err;
  g_res_attr_set[dev] = true;
  return cudaSuccess;
}

}  // namespace

size_t resident_smem_need(int64_t n, int64_t m, int cs) {
  if (n < 1 || m < 1 || m > RMAX_M || cs < 1) return ~size_t(0);
  const int64_t ldk = (m + 3) & ~int64_t(3), c4 = ldk / 4;
  const int64_t nb = (n + cs - 1) / cs;
  const int64_t slice = (c4 + cs - 1) / cs * 4;
  const ResGeom G = res_geom(int(c4));
  const int64_t floats = nb * ldk + ldk + int64_t(G.units / 2) * ldk + slice +
                         (cs > 1 ? cs * slice : 0) + int64_t(G.wpg) * nb + 2 * nb;
  return size_t(floats) * sizeof(float);
}

cudaError_t resident_smem_cap(size_t* cap) {
  int dev = 0, optin = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  err = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (err != cudaSuccess) return err;
  cudaFuncAttributes fa;
  err = cudaFuncGetAttributes(&fa, resident_kernel);
  if (err != cudaSuccess) return err;
  const size_t stat = fa.sharedSizeBytes;
  *cap = size_t(optin) > stat ? size_t(optin) - stat : 0;
  return ensure_resident_attributes(dev, *cap);
}

cudaError_t resident_max_clusters(int cs, size_t smem, int* clusters) {
  *clusters = 0;
  int dev = 0, sms = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  size_t cap = 0;
  err = resident_smem_cap(&cap);
  if (err != cudaSuccess) return err;
  if (smem > cap) return cudaSuccess;
  if (cs == 1) {
    err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (err != cudaSuccess) return err;
    int occ = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, resident_kernel, RT, smem);
    if (err != cudaSuccess) return err;
    *clusters = occ * sms;
    return cudaSuccess;
  }
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(cs, 1, 1);
  cfg.blockDim = dim3(RT, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int nc = 0;
  err = cudaOccupancyMaxActiveClusters(&nc, resident_kernel, &cfg);
  if (err != cudaSuccess) {
    // Cluster size not supported with this footprint: report none.
    cudaGetLastError();
    return cudaSuccess;
  }
  *clusters = nc;
  return cudaSuccess;
}

cudaError_t resident_launch(const BatchProblem* probs, const int* order, int count, int* cursor,
                            int cs, int grid, size_t smem, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(grid, 1, 1);
  cfg.blockDim = dim3(RT, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = cs > 1 ? 1 : 0;
  ResidentArgs a{probs, order, count, cursor};
  void* kargs[] = {&a};
  cudaError_t err = cudaLaunchKernelExC(&cfg, reinterpret_cast<const void*>(resident_kernel), kargs);
  if (err == cudaSuccess) count_launch();
  return err;
}

}  // namespace uot
