// The whole iteration of Section 2.1 in one persistent launch, for plans
// that fit in the shared memory of the GPU's CTAs (one CTA per SM): the
// per-iteration launch and its fixed cost disappear, and the plan never
// leaves the chip between the first load and the final store.
//
// CTA g owns the rows [g R, (g+1) R) for the whole solve and keeps them in
// shared memory.  One iteration (Algorithm 1's single sweep, per CTA):
//   row step     one warp per row: x_ij = S_ij beta_j (the column step of
//                the previous iteration), r_i = sum_j x_ij by lane partials
//                and shuffles, alpha_i = (a_i / r_i)^fi, S_ij = x_ij alpha_i;
//   column sums  one thread per chunk of columns adds them over the CTA's
//                rows and folds the partials into the column sums of
//                iteration t (a ring of three buffers in the workspace) with
//                vector reductions; CTA g adds into replica g % 4 of the
//                buffer, so fewer reductions meet at one address (rows of at
//                most 8192 columns);
//   grid barrier every CTA has added its partials (a release/acquire counter,
//                bounded: a wait that gives up sets UOT_DEV_TIMEOUT);
//   next factors every CTA adds the replicas in replica order and forms
//                beta_t = (b_j / c_j)^fi for all columns into its shared
//                memory, and the stopping rule is decided
//                from the same FP64 totals by every CTA alike.
// The entries are rounded exactly as by the fused pass (fl(fl(S beta) alpha)
// in the plan's dtype); only the order of the column partial sums differs.
// Kernel form (KF): the rows hold K, read-only; U of the owned rows and all
// of V stay in shared memory, with the power-of-two gauge of the fused pass;
// the last step writes U_i K_ij V_j.
#include <algorithm>

#include <cuda_runtime.h>

#include "uot_device.cuh"
#include "uot_internal.h"

namespace uot {

namespace {

__host__ __device__ constexpr size_t align_up(size_t x) { return (x + 15) & ~size_t(15); }

constexpr int PT = 512;           // threads per CTA
constexpr int PNW = PT / 32;      // warps per CTA
constexpr size_t SMEM_CAP = 220 * 1024;

struct PersistArgs {
  void* plan;
  int64_t ldp;
  int n, m, rows, ldm;  // rows per CTA; shared-memory row stride (elements)
  const float* a;
  const float* b;
  float fi;
  int iters;
  int track, check_every;
  double tol;
  float* c[3];          // column sums of iteration t in c[t % 3], nrep replicas each
  int nrep;             // replicas (CTA g adds into replica g % nrep)
  int rep_stride;       // elements between replicas
  double* err;          // [3][2] stopping-error sums, ring of 3
  int* bar;             // grid barrier counter (zero at launch)
  Control* ctl;
  float* U;             // kernel form: row scalings (read and written back)
  float* V;             // kernel form: column scalings (workspace, read and written back)
  const double* log2k;  // kernel form: the gauge's log2 k
  int pot;
  float kscale;
  int write_plan;       // 1: store the rows back (kernel form: U_i K_ij V_j); 0: K stays
};

// Grid barrier number `epoch` (1, 2, ...): every CTA adds one to the counter
// after its writes; the barrier completes when the counter reaches
// epoch * gridDim.x (compared modulo 2^32, so the count may wrap on very long
// solves).  Returns false if the wait gave up.
__device__ __forceinline__ bool reached(const int* bar, uint32_t target) {
  return int32_t(uint32_t(ld_acquire_gpu(bar)) - target) >= 0;
}

__device__ __forceinline__ bool grid_barrier(int* bar, int epoch, bool& broken) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    if (!broken) {
      // The release reduction is cumulative: it orders every write the CTA
      // barrier above made visible to this thread (the column partials of all
      // warps) before the arrival, so no separate fence is needed.
      red_release_gpu_add(bar, 1);
      const uint32_t target = uint32_t(epoch) * gridDim.x;
      if (!reached(bar, target)) {
        const uint64_t t0 = global_timer_ns();
        while (!reached(bar, target)) {
          if (global_timer_ns() - t0 > WAIT_LIMIT_NS) {
            ok = 0;
            break;
          }
        }
      }
    } else {
      ok = 0;
    }
    s_ok = ok;
  }
  __syncthreads();
  if (!s_ok) broken = true;
  return s_ok != 0;
}

// Elements of a row moved as one unit: a 16-byte vector when the row width
// is a multiple of it (VEC), else one element.
template <typename T, bool VEC>
struct Chunk {
  static constexpr int N = VEC ? Elem<T>::VE : 1;
  static __device__ __forceinline__ void load(const T* p, float* f) {
    if constexpr (VEC)
      Elem<T>::unpack(ld_shared_v4(p), f);
    else
      f[0] = Elem<T>::load1(p);
  }
  static __device__ __forceinline__ void store(T* p, const float* f) {
    if constexpr (VEC)
      *reinterpret_cast<uint4*>(p) = Elem<T>::pack(f);
    else
      Elem<T>::store1(p, f[0]);
  }
  static __device__ __forceinline__ void load_f32(const float* p, float* f) {
    if constexpr (VEC) {
#pragma unroll
      for (int e = 0; e < N; e += 4) {
        const float4 q = *reinterpret_cast<const float4*>(p + e);
        f[e] = q.x; f[e + 1] = q.y; f[e + 2] = q.z; f[e + 3] = q.w;
      }
    } else {
      f[0] = *p;
    }
  }
};

template <typename T, bool KF, bool VEC>
__global__ void __launch_bounds__(PT, 1) persistent_kernel(const PersistArgs p) {
  using E = Elem<T>;
  using CH = Chunk<T, VEC>;
  constexpr int VE = CH::N;
  extern __shared__ __align__(16) unsigned char smem[];
  const int m = p.m, ldm = p.ldm;
  const int nv = m / VE;  // chunks per row (m % VE == 0 when VEC)
  T* S = reinterpret_cast<T*>(smem);
  float* beta = reinterpret_cast<float*>(smem + align_up(size_t(p.rows) * ldm * sizeof(T)));
  float* rprev = beta + ((m + 3) & ~3);
  float* urow = rprev + ((p.rows + 3) & ~3);  // kernel form: U of the owned rows
  __shared__ float s_num[PNW], s_den[PNW], s_part[PNW];
  __shared__ int s_stop;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int row0 = blockIdx.x * p.rows;
  const int nr = max(0, min(p.rows, p.n - row0));
  T* plan = reinterpret_cast<T*>(p.plan);
  uint32_t st = 0;
  bool broken = false;
  // Warps per row: a power of two that spreads the CTA's rows over all its
  // warps (one round of rows when nr <= 16); the row's chunks are strided
  // over the group's lanes.
  int wpr = 1;
  while (wpr * 2 <= PNW && wpr * 2 * nr <= PNW) wpr *= 2;
  const int ng = PNW / wpr, grp = warp / wpr, wig = warp % wpr;
  const int li = wig * 32 + lane, lstride = wpr * 32;
  const int rounds = (nr + ng - 1) / ng;

  // Load the owned rows; beta = 1 (kernel form: V from the workspace).
  for (int r = 0; r < nr; ++r)
    for (int j = tid; j < m; j += PT) S[r * ldm + j] = plan[int64_t(row0 + r) * p.ldp + j];
  for (int j = tid; j < m; j += PT) beta[j] = KF ? p.V[j] : 1.0f;
  if constexpr (KF) {
    for (int r = tid; r < nr; r += PT) urow[r] = p.U[row0 + r];
  }
  __syncthreads();

  int t_done = 0;
  for (int t = 1; t <= p.iters; ++t) {
    float* cnext = p.c[t % 3];
    float* cmine = cnext + size_t(blockIdx.x % p.nrep) * p.rep_stride;
    // Clear the buffers of iteration t+1 (last read in iteration t-2).
    {
      float* cc = p.c[(t + 1) % 3];
      for (int q = 0; q < p.nrep; ++q)
        for (int j = blockIdx.x * PT + tid; j < m; j += gridDim.x * PT)
          cc[size_t(q) * p.rep_stride + j] = 0.0f;
      if (p.track && blockIdx.x == 0 && tid < 2) p.err[((t + 1) % 3) * 2 + tid] = 0.0;
    }
    float gauge = 1.0f, inv_gauge = 1.0f;
    if constexpr (KF) {
      const int e = gauge_exponent(t, float(*p.log2k));
      gauge = ldexpf(1.0f, e);
      inv_gauge = ldexpf(1.0f, -e);
    }
    // Row step: group grp of wpr warps takes rows grp, grp + ng, ...
    float num = 0.0f, den = 0.0f;
    for (int k = 0; k < rounds; ++k) {
      const int r = grp + k * ng;
      const bool have = r < nr;
      T* row = S + r * ldm;
      float s = 0.0f;
      if (have) {
#pragma unroll 4
        for (int v = li; v < nv; v += lstride) {
          float f[VE], bb[VE];
          CH::load(row + v * VE, f);
          CH::load_f32(beta + v * VE, bb);
          if constexpr (KF) {
#pragma unroll
            for (int e = 0; e < VE; ++e) s = fmaf(f[e], bb[e], s);
          } else {
#pragma unroll
            for (int e = 0; e < VE; ++e) {
              f[e] = E::round(f[e] * bb[e]);
              s += f[e];
            }
            CH::store(row + v * VE, f);  // exact: x is representable in T
          }
        }
      }
      s = warp_sum(s);
      if (wpr > 1) {  // uniform for the CTA
        if (lane == 0) s_part[warp] = s;
        __syncthreads();
        s = 0.0f;
        for (int w = grp * wpr; w < (grp + 1) * wpr; ++w) s += s_part[w];
      }
      if (have) {
        const int i = row0 + r;
        float tot;
        if constexpr (KF) {
          const float u_old = urow[r];
          tot = s * u_old;
          const float u_new = p.pot
              ? rescale_factor(__ldg(p.a + i) * p.kscale, s, p.fi, st) / p.kscale
              : u_old * rescale_factor(__ldg(p.a + i), tot, p.fi, st) * gauge;
          if (wig == 0 && lane == 0) urow[r] = u_new;
        } else {
          tot = s;
          const float alpha = rescale_factor(__ldg(p.a + i), tot, p.fi, st);
#pragma unroll 4
          for (int v = li; v < nv; v += lstride) {
            float f[VE];
            CH::load(row + v * VE, f);
#pragma unroll
            for (int e = 0; e < VE; ++e) f[e] = E::round(f[e] * alpha);
            CH::store(row + v * VE, f);
          }
        }
        if (p.track && wig == 0 && lane == 0) {
          if (t >= 2) num += fabsf(tot - rprev[r]);
          den += tot;
          rprev[r] = tot;
        }
      }
      if (wpr > 1) __syncthreads();  // s_part is reused by the next round
    }
    if (p.track && lane == 0) {
      s_num[warp] = num;
      s_den[warp] = den;
    }
    __syncthreads();
    // Column partial sums over the owned rows (kernel form: of U_i K_ij),
    // one chunk of columns per thread, folded in with vector reductions.
    if (nr > 0) {
      for (int v = tid; v < nv; v += PT) {
        float c[VE];
#pragma unroll
        for (int e = 0; e < VE; ++e) c[e] = 0.0f;
        for (int r = 0; r < nr; ++r) {
          float f[VE];
          CH::load(S + r * ldm + v * VE, f);
          if constexpr (KF) {
            const float u = urow[r];
#pragma unroll
            for (int e = 0; e < VE; ++e) c[e] = fmaf(u, f[e], c[e]);
          } else {
#pragma unroll
            for (int e = 0; e < VE; ++e) c[e] += f[e];
          }
        }
        if constexpr (VEC) {
#pragma unroll
          for (int e = 0; e < VE; e += 4)
            red_add_v4(cmine + v * VE + e, c[e], c[e + 1], c[e + 2], c[e + 3]);
        } else {
          atomicAdd(cmine + v, c[0]);
        }
      }
    }
    if (p.track && tid == 0 && nr > 0) {
      double dn = 0.0, dd = 0.0;
      for (int w = 0; w < PNW; ++w) {
        dn += s_num[w];
        dd += s_den[w];
      }
      atomicAdd(p.err + (t % 3) * 2, dn);
      atomicAdd(p.err + (t % 3) * 2 + 1, dd);
    }
    if (!grid_barrier(p.bar, t, broken)) break;
    // Next column factors for every column (kernel form: the new V).
    for (int v = tid; v < nv; v += PT) {
      // The replicas added in replica order.
      float c[VE];
#pragma unroll
      for (int e = 0; e < VE; ++e) c[e] = 0.0f;
      for (int q = 0; q < p.nrep; ++q) {
        const float* cq = cnext + size_t(q) * p.rep_stride;
        if constexpr (VEC) {
#pragma unroll
          for (int e = 0; e < VE; e += 4) {
            const float4 w = __ldcg(reinterpret_cast<const float4*>(cq + v * VE + e));
            c[e] += w.x; c[e + 1] += w.y; c[e + 2] += w.z; c[e + 3] += w.w;
          }
        } else {
          c[0] += __ldcg(cq + v);
        }
      }
#pragma unroll
      for (int e = 0; e < VE; ++e) {
        const int j = v * VE + e;
        if constexpr (KF) {
          const float vj = beta[j];
          beta[j] = p.pot ? rescale_factor(__ldg(p.b + j), c[e], p.fi, st)
                          : vj * rescale_factor(__ldg(p.b + j), vj * c[e] * inv_gauge, p.fi, st) *
                                inv_gauge;
        } else {
          beta[j] = rescale_factor(__ldg(p.b + j), c[e], p.fi, st);
        }
      }
    }
    t_done = t;
    if (tid == 0) {
      int stop = 0;
      if (p.track && t >= 2 && t % p.check_every == 0) {
        const double dn = __ldcg(p.err + (t % 3) * 2), dd = __ldcg(p.err + (t % 3) * 2 + 1);
        stop = dd > 0.0 && dn <= p.tol * dd;
        if (stop && blockIdx.x == 0) {
          p.ctl->stop_iter = t;
          p.ctl->done = 1;
          p.ctl->err = dn / dd;
        }
      }
      s_stop = stop;
    }
    __syncthreads();
    if (s_stop) break;
  }

  // Apply the last column factor and store the rows (kernel form: write
  // U_i K_ij V_j when the buffer is to become the plan, and hand U and V
  // back).
  for (int r = 0; r < (p.write_plan ? nr : 0); ++r)
    for (int j = tid; j < m; j += PT) {
      float v;
      if constexpr (KF)
        v = (urow[r] * E::load1(S + r * ldm + j)) * beta[j];
      else
        v = E::load1(S + r * ldm + j) * beta[j];
      E::store1(plan + int64_t(row0 + r) * p.ldp + j, v);
    }
  if constexpr (KF) {
    for (int r = tid; r < nr; r += PT) p.U[row0 + r] = urow[r];
    if (blockIdx.x == 0)
      for (int j = tid; j < m; j += PT) p.V[j] = beta[j];
  }
  if (broken) st |= DEV_TIMEOUT;
  if (st) atomicOr(&p.ctl->status, st);
  if (blockIdx.x == 0 && tid == 0) {
    p.ctl->iters_done = t_done;
    if (p.track && !p.ctl->done && t_done >= 2) {
      const double dn = __ldcg(p.err + (t_done % 3) * 2);
      const double dd = __ldcg(p.err + (t_done % 3) * 2 + 1);
      p.ctl->err = dd > 0.0 ? dn / dd : __longlong_as_double(0x7ff0000000000000ll);
    }
  }
}

// The kernel for a dtype, form and row width.
template <typename T>
const void* persistent_fn(bool kf, int m) {
  const bool vec = m % Elem<T>::VE == 0;
  if (kf)
    return vec ? reinterpret_cast<const void*>(&persistent_kernel<T, true, true>)
               : reinterpret_cast<const void*>(&persistent_kernel<T, true, false>);
  return vec ? reinterpret_cast<const void*>(&persistent_kernel<T, false, true>)
             : reinterpret_cast<const void*>(&persistent_kernel<T, false, false>);
}

template <typename T>
size_t persist_smem(int rows, int m, int ldm) {
  return align_up(size_t(rows) * ldm * sizeof(T)) + size_t((m + 3) & ~3) * 4 +
         2 * size_t((rows + 3) & ~3) * 4;
}

template <typename F>
cudaError_t with_dtype(int dtype, F&& f) {
  switch (dtype) {
    case UOT_F32: return f(float());
    case UOT_BF16: return f(__nv_bfloat16());
    case UOT_F16: return f(__half());
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t persistent_plan(int dtype, bool kf, int n, int m, int max_ctas, PersistPlan* out) {
  int dev = 0, sms = 0, optin = 0, coop = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) !=
          cudaSuccess ||
      (e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev)) != cudaSuccess)
    return e;
  out->ok = false;
  if (!coop) return cudaSuccess;
  const int gmax = max_ctas > 0 ? std::min(max_ctas, sms) : sms;
  const int rows = (n + gmax - 1) / gmax;
  const int grid = (n + rows - 1) / rows;
  const int ldm = (m + 7) & ~7;
  return with_dtype(dtype, [&](auto z) {
    using T = decltype(z);
    const size_t smem = persist_smem<T>(rows, m, ldm);
    if (smem > std::min<size_t>(size_t(optin), SMEM_CAP)) return cudaSuccess;
    const void* fn = persistent_fn<T>(kf, m);
    cudaError_t err = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           int(smem));
    if (err != cudaSuccess) return err;
    int occ = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, PT, smem);
    if (err != cudaSuccess) return err;
    if (occ * sms < grid) return cudaSuccess;
    out->ok = true;
    out->grid = grid;
    out->rows = rows;
    out->ldm = ldm;
    out->smem = smem;
    return cudaSuccess;
  });
}

cudaError_t persistent_launch(int dtype, bool kf, const PersistPlan& pl, void* plan, int64_t ldp,
                              int n, int m, const float* a, const float* b, float fi, int iters,
                              double tol, int check_every, uint8_t* ws, const WsLayout& L,
                              float* U, float* V, int pot, float kscale, bool write_plan,
                              cudaStream_t s) {
  PersistArgs A{};
  A.write_plan = write_plan ? 1 : 0;
  A.plan = plan;
  A.ldp = ldp;
  A.n = n;
  A.m = m;
  A.rows = pl.rows;
  A.ldm = pl.ldm;
  A.a = a;
  A.b = b;
  A.fi = fi;
  A.iters = iters;
  A.track = tol > 0.0 ? 1 : 0;
  A.check_every = check_every;
  A.tol = tol;
  if (L.mpad <= PERSIST_REP_MAX_M) {
    A.nrep = PERSIST_REPS;
    A.rep_stride = int(L.mpad);
    for (int q = 0; q < 3; ++q)
      A.c[q] = reinterpret_cast<float*>(ws + L.crep) + size_t(q) * PERSIST_REPS * size_t(L.mpad);
  } else {
    A.nrep = 1;
    A.rep_stride = 0;
    for (int q = 0; q < 3; ++q) A.c[q] = reinterpret_cast<float*>(ws + L.c[q]);
  }
  A.err = reinterpret_cast<double*>(ws + L.err);
  A.bar = reinterpret_cast<int*>(ws + L.ctr);
  A.ctl = reinterpret_cast<Control*>(ws + L.ctl);
  A.U = U;
  A.V = V;
  A.log2k = reinterpret_cast<const double*>(ws + L.log2k);
  A.pot = pot;
  A.kscale = kscale;
  return with_dtype(dtype, [&](auto z) {
    using T = decltype(z);
    const void* fn = persistent_fn<T>(kf, m);
    // Every CTA must be resident at once (grid barrier): a cooperative launch
    // guarantees it or fails.
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.gridDim = dim3(pl.grid);
    cfg.blockDim = dim3(PT);
    cfg.dynamicSmemBytes = pl.smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    void* kargs[] = {&A};
    cudaError_t e = cudaLaunchKernelExC(&cfg, fn, kargs);
    if (e == cudaSuccess) count_launch();
    return e;
  });
}

}  // namespace uot
