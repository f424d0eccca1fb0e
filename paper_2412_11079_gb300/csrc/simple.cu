// Simple streaming kernels of libuot: the initial plan, the finishing sweep
// that applies the last pending column factor, the transport cost, the
// workspace reset, and the plain multi-pass form of one iteration (separate
// row-sum, row-scale, column-sum and column-scale sweeps, the baseline form
// of Section 2.1 that Section 3.1 analyses).
#include <algorithm>

#include <cuda_runtime.h>

#include "uot_device.cuh"
#include "uot_internal.h"

namespace uot {

namespace {

constexpr int TB = 256;

// exp(-c/reg) without the error of rounding the exponent to FP32 first: with
// hi = fl(-c/reg), the residual -c - hi*reg is exact in FP32 (it is the
// remainder of a correctly rounded division), so -c/reg = hi + e/reg and
// exp(-c/reg) = expf(hi) * exp(e/reg), where |e/reg| <= |hi| 2^-24 lets the
// second factor be taken to first order.
__device__ __forceinline__ float gibbs(float c, float reg) {
  const float hi = -c / reg;
  const float e = fmaf(-hi, reg, -c);
  const float x = expf(hi);
  return fmaf(x, e / reg, x);
}

// P = exp(-C/reg) * scale; scale is a power of two (FP16 kernels are stored
// scaled into FP16's normal range).
template <typename T>
__global__ void __launch_bounds__(TB) init_kernel(const float* __restrict__ C, int64_t ldc,
                                                  T* __restrict__ P, int64_t ldp, int n, int m,
                                                  float reg, float scale) {
  const int j = blockIdx.x * TB + threadIdx.x;
  if (j >= m) return;
  for (int i = blockIdx.y; i < n; i += gridDim.y) {
    const float c = C[int64_t(i) * ldc + j];
    Elem<T>::store1(P + int64_t(i) * ldp + j, gibbs(c, reg) * scale);
  }
}

// Compensated accumulation in a pair of floats (hi + lo): Dekker's exact
// product through fma, Knuth's TwoSum for the addition.  About 2^-44 relative
// accuracy for sums of non-negative terms, without the FP64 pipe.
struct Acc2 {
  float hi = 0.0f, lo = 0.0f;
  __device__ __forceinline__ void add_product(float x, float y) {
    const float p = x * y;
    const float pe = fmaf(x, y, -p);
    const float s = hi + p;
    const float bb = s - hi;
    const float se = (hi - (s - bb)) + (p - bb);
    hi = s;
    lo += se + pe;
  }
  __device__ __forceinline__ double value() const { return double(hi) + double(lo); }
};

__device__ __forceinline__ void block_add_double(double v, double* out) {
  __shared__ double part[TB / 32];
  v = warp_sum_d(v);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < TB / 32; ++w) t += part[w];
    atomicAdd(out, t);
  }
}

// Applies beta_j = (b_j / c_j)^fi of the last completed iteration and records
// the iteration count and the last stopping error.
template <typename T>
__global__ void __launch_bounds__(TB) finish_kernel(T* __restrict__ P, int64_t ldp, int n, int m,
                                                    const float* __restrict__ b, float fi,
                                                    int iters, const float* c0, const float* c1,
                                                    const float* c2, const double* err_ring,
                                                    Control* ctl, double tol, int check_every,
                                                    const float* beta_ready) {
  const int done = ctl->done;
  const int t = done ? ctl->stop_iter : iters;
  const float* c = (t % 3 == 0) ? c0 : (t % 3 == 1) ? c1 : c2;
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
    ctl->iters_done = t;
    if (!done && tol > 0.0 && t >= 2) {
      const double num = err_ring[(t % 3) * 2], den = err_ring[(t % 3) * 2 + 1];
      ctl->err = den > 0.0 ? num / den : __longlong_as_double(0x7ff0000000000000ll);
    }
  }
  const int j = blockIdx.x * TB + threadIdx.x;
  if (j >= m) return;
  uint32_t st = 0;
  // The fused passes leave beta_t ready (its status was recorded there).
  const float beta = beta_ready ? beta_ready[j] : rescale_factor(b[j], c[j], fi, st);
  if (st && blockIdx.y == 0) atomicOr(&ctl->status, st);
  for (int i = blockIdx.y; i < n; i += gridDim.y) {
    T* q = P + int64_t(i) * ldp + j;
    Elem<T>::store1(q, Elem<T>::load1(q) * beta);
  }
}

template <typename T>
__global__ void __launch_bounds__(TB) cost_kernel(const T* __restrict__ P, int64_t ldp,
                                                  const float* __restrict__ C, int64_t ldc, int n,
                                                  int m, double* out) {
  const int j = blockIdx.x * TB + threadIdx.x;
  Acc2 acc;
  if (j < m)
    for (int i = blockIdx.y; i < n; i += gridDim.y)
      acc.add_product(Elem<T>::load1(P + int64_t(i) * ldp + j), C[int64_t(i) * ldc + j]);
  block_add_double(acc.value(), out);
}

// <diag(U) K diag(V), C>: each term (U_i K_ij) V_j is formed in FP32 (two
// roundings) and accumulated as above.
template <typename T>
__global__ void __launch_bounds__(TB) kform_cost_kernel(const T* __restrict__ K, int64_t ldk,
                                                        const float* __restrict__ U,
                                                        const float* __restrict__ V,
                                                        const float* __restrict__ C, int64_t ldc,
                                                        int n, int m, double* out) {
  const int j = blockIdx.x * TB + threadIdx.x;
  Acc2 acc;
  if (j < m) {
    const float v = V[j];
    for (int i = blockIdx.y; i < n; i += gridDim.y)
      acc.add_product(U[i] * Elem<T>::load1(K + int64_t(i) * ldk + j) * v,
                      C[int64_t(i) * ldc + j]);
  }
  block_add_double(acc.value(), out);
}

// P = diag(U) K diag(V) in the plan's dtype.
template <typename TK, typename TP>
__global__ void __launch_bounds__(TB) kform_plan_kernel(const TK* __restrict__ K, int64_t ldk,
                                                        const float* __restrict__ U,
                                                        const float* __restrict__ V, int n, int m,
                                                        TP* __restrict__ P, int64_t ldp) {
  const int j = blockIdx.x * TB + threadIdx.x;
  if (j >= m) return;
  const float v = V[j];
  for (int i = blockIdx.y; i < n; i += gridDim.y)
    Elem<TP>::store1(P + int64_t(i) * ldp + j, U[i] * Elem<TK>::load1(K + int64_t(i) * ldk + j) * v);
}

// uot_sinkhorn's kernel-form storage, last sweep: the buffer holds K, and
// every entry becomes (U_i K_ij) V_j in place (the product in the order of
// kform_plan_kernel).
template <typename T>
__global__ void __launch_bounds__(TB) kform_materialize_kernel(T* P, int64_t ldp,
                                                               const float* __restrict__ U,
                                                               const float* __restrict__ V,
                                                               int n, int m) {
  const int j = blockIdx.x * TB + threadIdx.x;
  if (j >= m) return;
  const float v = V[j];
  for (int i = blockIdx.y; i < n; i += gridDim.y) {
    T* q = P + int64_t(i) * ldp + j;
    Elem<T>::store1(q, U[i] * Elem<T>::load1(q) * v);
  }
}

// Kernel form: U = u0 (the inverse of K's storage scale), V = 1 (zero-padded).
__global__ void kform_reset_kernel(float* U, int n, float u0, float* V_ws, int m, int mpad) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  const int gs = gridDim.x * blockDim.x;
  for (int i = g; i < n; i += gs) U[i] = u0;
  for (int j = g; j < mpad; j += gs) V_ws[j] = j < m ? 1.0f : 0.0f;
}

// Kernel form: log2 k, k = (m_a / m_b)^(fi / (2 - fi)) the row factor at the
// fixed point of the row-then-column rule (0 when a mass is 0 or not finite).
__global__ void __launch_bounds__(1024) kform_gauge_kernel(const float* a, int n, const float* b,
                                                           int m, float fi, bool pot,
                                                           double* log2k) {
  __shared__ double part[2][32];
  double sa = 0.0, sb = 0.0;
  for (int i = threadIdx.x; i < n; i += 1024) sa += a[i];
  for (int j = threadIdx.x; j < m; j += 1024) sb += b[j];
  sa = warp_sum_d(sa);
  sb = warp_sum_d(sb);
  if ((threadIdx.x & 31) == 0) {
    part[0][threadIdx.x >> 5] = sa;
    part[1][threadIdx.x >> 5] = sb;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double ta = 0.0, tb = 0.0;
    for (int w = 0; w < 32; ++w) {
      ta += part[0][w];
      tb += part[1][w];
    }
    const double f = double(fi);
    const double L = (f / (2.0 - f)) * log2(ta / tb);
    // The scaling-vector rule converges in (U, V) itself: no drift, no gauge.
    *log2k = (!pot && ta > 0.0 && tb > 0.0 && isfinite(L)) ? L : 0.0;
  }
}

// Kernel form: iteration count, last stopping error, V to the caller.
__global__ void kform_finish_kernel(float* V, const float* V_ws, int m, int iters,
                                    const double* err_ring, Control* ctl, double tol) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g == 0) {
    const int done = ctl->done;
    const int t = done ? ctl->stop_iter : iters;
    ctl->iters_done = t;
    if (!done && tol > 0.0 && t >= 2) {
      const double num = err_ring[(t % 3) * 2], den = err_ring[(t % 3) * 2 + 1];
      ctl->err = den > 0.0 ? num / den : __longlong_as_double(0x7ff0000000000000ll);
    }
  }
  for (int j = g; j < m; j += gridDim.x * blockDim.x) V[j] = V_ws[j];
}

__global__ void reset_kernel(Control* ctl, double* err_ring, float* c1, int mpad, const float* b,
                             float* b_ws, int m, int* ctr, float* beta, float* crep1,
                             int crep_len) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g == 0) {
    ctl->status = 0;
    ctl->done = 0;
    ctl->stop_iter = 0;
    ctl->iters_done = 0;
    ctl->err = __longlong_as_double(0x7ff0000000000000ll);
  }
  if (g < 6) err_ring[g] = 0.0;
  if (g < 9) ctr[g] = 0;
  for (int j = g; j < mpad; j += gridDim.x * blockDim.x) {
    c1[j] = 0.0f;
    b_ws[j] = (b && j < m) ? b[j] : 0.0f;  // no b: a pass that forms no column factors
    beta[j] = 0.0f;
  }
  for (int j = g; j < crep_len; j += gridDim.x * blockDim.x) crep1[j] = 0.0f;
}

// ---- multi-pass iteration: 5 launches, 3 reads + 2 writes of the plan ----

// One warp per row: r_i = sum_j P_ij, f_i = (a_i / r_i)^fi.  Also clears the
// column-sum buffer for this iteration.
template <typename T>
__global__ void __launch_bounds__(TB) mp_row_factor(const T* __restrict__ P, int64_t ldp, int n,
                                                    int m, const float* __restrict__ a, float fi,
                                                    float* f, float* c, int mpad, Control* ctl) {
  const int g = blockIdx.x * TB + threadIdx.x;
  for (int j = g; j < mpad; j += gridDim.x * TB) c[j] = 0.0f;
  const int warp = g >> 5, lane = threadIdx.x & 31;
  const int nw = (gridDim.x * TB) >> 5;
  uint32_t st = 0;
  for (int i = warp; i < n; i += nw) {
    const T* row = P + int64_t(i) * ldp;
    float s = 0.0f;
    for (int j = lane; j < m; j += 32) s += Elem<T>::load1(row + j);
    s = warp_sum(s);
    if (lane == 0) f[i] = rescale_factor(a[i], s, fi, st);
  }
  if (st) atomicOr(&ctl->status, st);
}

template <typename T>
__global__ void __launch_bounds__(TB) mp_scale_rows(T* __restrict__ P, int64_t ldp, int n, int m,
                                                    const float* __restrict__ f) {
  const int j = blockIdx.x * TB + threadIdx.x;
  if (j >= m) return;
  for (int i = blockIdx.y; i < n; i += gridDim.y) {
    T* q = P + int64_t(i) * ldp + j;
    Elem<T>::store1(q, Elem<T>::load1(q) * f[i]);
  }
}

template <typename T>
__global__ void __launch_bounds__(TB) mp_col_sums(const T* __restrict__ P, int64_t ldp, int n,
                                                  int m, float* c) {
  const int j = blockIdx.x * TB + threadIdx.x;
  if (j >= m) return;
  float s = 0.0f;
  for (int i = blockIdx.y; i < n; i += gridDim.y) s += Elem<T>::load1(P + int64_t(i) * ldp + j);
  atomicAdd(c + j, s);
}

__global__ void __launch_bounds__(TB) mp_col_factor(const float* __restrict__ b, const float* c,
                                                    float fi, float* g, int m, Control* ctl) {
  const int j = blockIdx.x * TB + threadIdx.x;
  if (j >= m) return;
  uint32_t st = 0;
  g[j] = rescale_factor(b[j], c[j], fi, st);
  if (st) atomicOr(&ctl->status, st);
}

template <typename T>
__global__ void __launch_bounds__(TB) mp_scale_cols(T* __restrict__ P, int64_t ldp, int n, int m,
                                                    const float* __restrict__ g, Control* ctl,
                                                    int t) {
  const int j = blockIdx.x * TB + threadIdx.x;
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) ctl->iters_done = t;
  if (j >= m) return;
  const float gj = g[j];
  for (int i = blockIdx.y; i < n; i += gridDim.y) {
    T* q = P + int64_t(i) * ldp + j;
    Elem<T>::store1(q, Elem<T>::load1(q) * gj);
  }
}

int sm_count() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

// 2-D grid for the column-parallel kernels: blockIdx.x over columns,
// blockIdx.y over row strides, about 8 resident CTAs per SM in total.
dim3 col_grid(int n, int m) {
  const int gx = (m + TB - 1) / TB;
  int gy = (sm_count() * 8 + gx - 1) / gx;
  if (gy > n) gy = n;
  if (gy > 65535) gy = 65535;
  if (gy < 1) gy = 1;
  return dim3(gx, gy, 1);
}

template <typename F>
cudaError_t by_dtype(int dtype, F&& f) {
  switch (dtype) {
    case UOT_F32: return f(float());
    case UOT_BF16: return f(__nv_bfloat16());
    case UOT_F16: return f(__half());
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t last(int k = 1) {
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) count_launch(k);
  return e;
}

}  // namespace

cudaError_t launch_init(const float* C, int64_t ldc, void* P, int64_t ldp, int n, int m,
                        float reg, int dtype, float scale, cudaStream_t s) {
  return by_dtype(dtype, [&](auto z) {
    using T = decltype(z);
    init_kernel<T><<<col_grid(n, m), TB, 0, s>>>(C, ldc, reinterpret_cast<T*>(P), ldp, n, m, reg,
                                                 scale);
    return last();
  });
}

cudaError_t launch_kform_reset(float* U, int n, float u0, float* V_ws, int m, int mpad,
                               const float* a, const float* b, float fi, bool pot, double* log2k,
                               cudaStream_t s) {
  const int blocks = (max(n, mpad) + TB - 1) / TB;
  kform_reset_kernel<<<blocks, TB, 0, s>>>(U, n, u0, V_ws, m, mpad);
  cudaError_t e = last();
  if (e != cudaSuccess) return e;
  kform_gauge_kernel<<<1, 1024, 0, s>>>(a, n, b, m, fi, pot, log2k);
  return last();
}

cudaError_t launch_kform_finish(float* V, int m, int iters, const uint8_t* ws, WsLayout L,
                                double tol, cudaStream_t s) {
  uint8_t* w = const_cast<uint8_t*>(ws);
  kform_finish_kernel<<<(m + TB - 1) / TB, TB, 0, s>>>(
      V, reinterpret_cast<const float*>(w + L.beta), m, iters,
      reinterpret_cast<const double*>(w + L.err), reinterpret_cast<Control*>(w + L.ctl), tol);
  return last();
}

cudaError_t launch_kform_plan(const void* K, int64_t ldk, int k_dtype, const float* U,
                              const float* V, int n, int m, void* P, int64_t ldp, int p_dtype,
                              cudaStream_t s) {
  return by_dtype(k_dtype, [&](auto zk) {
    using TK = decltype(zk);
    return by_dtype(p_dtype, [&](auto zp) {
      using TP = decltype(zp);
      kform_plan_kernel<TK, TP><<<col_grid(n, m), TB, 0, s>>>(
          reinterpret_cast<const TK*>(K), ldk, U, V, n, m, reinterpret_cast<TP*>(P), ldp);
      return last();
    });
  });
}

cudaError_t launch_kform_materialize(void* P, int64_t ldp, int dtype, const float* U,
                                     const float* V, int n, int m, cudaStream_t s) {
  return by_dtype(dtype, [&](auto z) {
    using T = decltype(z);
    kform_materialize_kernel<T><<<col_grid(n, m), TB, 0, s>>>(reinterpret_cast<T*>(P), ldp, U, V,
                                                              n, m);
    return last();
  });
}

cudaError_t launch_kform_cost(const void* K, int64_t ldk, int k_dtype, const float* U,
                              const float* V, const float* C, int64_t ldc, int n, int m,
                              double* out, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double), s);
  if (e != cudaSuccess) return e;
  return by_dtype(k_dtype, [&](auto z) {
    using T = decltype(z);
    kform_cost_kernel<T><<<col_grid(n, m), TB, 0, s>>>(reinterpret_cast<const T*>(K), ldk, U, V,
                                                       C, ldc, n, m, out);
    return last();
  });
}

cudaError_t launch_finish(void* P, int64_t ldp, int n, int m, int dtype, const float* b, float fi,
                          int iters, const uint8_t* ws, WsLayout L, double tol, int check_every,
                          bool beta_ready, cudaStream_t s) {
  uint8_t* w = const_cast<uint8_t*>(ws);
  return by_dtype(dtype, [&](auto z) {
    using T = decltype(z);
    finish_kernel<T><<<col_grid(n, m), TB, 0, s>>>(
        reinterpret_cast<T*>(P), ldp, n, m, b, fi, iters, reinterpret_cast<const float*>(w + L.c[0]),
        reinterpret_cast<const float*>(w + L.c[1]), reinterpret_cast<const float*>(w + L.c[2]),
        reinterpret_cast<const double*>(w + L.err), reinterpret_cast<Control*>(w + L.ctl), tol,
        check_every, beta_ready ? reinterpret_cast<const float*>(w + L.beta) : nullptr);
    return last();
  });
}

cudaError_t launch_cost(const void* P, int64_t ldp, const float* C, int64_t ldc, int n, int m,
                        int dtype, double* out, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double), s);
  if (e != cudaSuccess) return e;
  return by_dtype(dtype, [&](auto z) {
    using T = decltype(z);
    cost_kernel<T><<<col_grid(n, m), TB, 0, s>>>(reinterpret_cast<const T*>(P), ldp, C, ldc, n, m,
                                                 out);
    return last();
  });
}

// Self-test of the bounded waits: one thread waits on an mbarrier phase with
// the helper every bulk-copy ring uses (mbar_wait_bounded), then spins on a
// global counter with an acquire load until it reaches `target`, the pattern
// of the inter-CTA barriers, each wait giving up after limit_ns.  Unless
// `complete` is set nothing arrives on the barrier.  Each outcome goes to
// status[0] (barrier) and status[1] (counter): DEV_TIMEOUT or 0.
__global__ void wait_selftest_kernel(const int* counter, int target, int complete,
                                     uint64_t limit_ns, uint32_t* status) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  if (complete) mbar_arrive(&bar);
  status[0] = mbar_wait_bounded(&bar, 0u, limit_ns) ? 0u : DEV_TIMEOUT;
  uint32_t st = 0;
  const uint64_t t0 = global_timer_ns();
  while (ld_acquire_gpu(counter) < target) {
    if (global_timer_ns() - t0 > limit_ns) {
      st = DEV_TIMEOUT;
      break;
    }
  }
  status[1] = st;
}

// Self-test of the rescaling factor: out[k] = rescale_factor(target[k],
// total[k], fi), the same device function every pass uses, with the
// degenerate-case status bits OR-ed into *status.
__global__ void factor_selftest_kernel(const float* target, const float* total, int64_t count,
                                       float fi, float* out, uint32_t* status) {
  uint32_t st = 0;
  for (int64_t k = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; k < count;
       k += int64_t(gridDim.x) * blockDim.x)
    out[k] = rescale_factor(target[k], total[k], fi, st);
  if (st) atomicOr(status, st);
}

cudaError_t launch_factor_selftest(const float* target, const float* total, int64_t count,
                                   float fi, float* out, uint32_t* status, cudaStream_t s) {
  const int64_t blocks = std::min<int64_t>((count + TB - 1) / TB, int64_t(sm_count()) * 8);
  factor_selftest_kernel<<<int(std::max<int64_t>(blocks, 1)), TB, 0, s>>>(target, total, count,
                                                                          fi, out, status);
  return last();
}

// Row-sharded pass set-up: the previous column factors into the zero-padded
// factor buffer (ones when there are none yet, and then the status word is
// cleared too: a new solve), the column sums of this pass and the pass
// counters cleared.
__global__ void shard_prep_kernel(const float* beta_in, int m, int mpad, float* beta_ws,
                                  float* c_next, int* ctr, Control* ctl) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  const int gs = gridDim.x * blockDim.x;
  if (g == 0 && !beta_in) {
    ctl->status = 0;
    ctl->done = 0;
  }
  for (int j = g; j < mpad; j += gs) {
    beta_ws[j] = j < m ? (beta_in ? beta_in[j] : 1.0f) : 0.0f;
    c_next[j] = 0.0f;
  }
  if (g < 9) ctr[g] = 0;
}

// beta_j = (b_j / c_j)^fi from the reduced column sums.
__global__ void shard_factors_kernel(const float* c, const float* b, int m, float fi, float* beta,
                                     uint32_t* status) {
  uint32_t st = 0;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x)
    beta[j] = rescale_factor(b[j], c[j], fi, st);
  if (st && status) atomicOr(status, st);
}

template <typename T>
__global__ void __launch_bounds__(TB) scale_cols_kernel(T* P, int64_t ldp, int n, int m,
                                                        const float* __restrict__ beta) {
  const int j = blockIdx.x * TB + threadIdx.x;
  if (j >= m) return;
  const float g = beta[j];
  for (int i = blockIdx.y; i < n; i += gridDim.y) {
    T* q = P + int64_t(i) * ldp + j;
    Elem<T>::store1(q, Elem<T>::load1(q) * g);
  }
}

cudaError_t launch_shard_prep(uint8_t* ws, WsLayout L, const float* beta_in, int m, cudaStream_t s) {
  const int blocks = int((L.mpad + TB - 1) / TB);
  shard_prep_kernel<<<blocks, TB, 0, s>>>(beta_in, m, int(L.mpad),
                                          reinterpret_cast<float*>(ws + L.beta),
                                          reinterpret_cast<float*>(ws + L.c[0]),
                                          reinterpret_cast<int*>(ws + L.ctr),
                                          reinterpret_cast<Control*>(ws + L.ctl));
  return last();
}

cudaError_t launch_shard_factors(const float* c, const float* b, int m, float fi, float* beta,
                                 uint32_t* status, cudaStream_t s) {
  const int blocks = std::min((m + TB - 1) / TB, sm_count() * 8);
  shard_factors_kernel<<<blocks, TB, 0, s>>>(c, b, m, fi, beta, status);
  return last();
}

cudaError_t launch_scale_cols(void* P, int64_t ldp, int n, int m, int dtype, const float* beta,
                              cudaStream_t s) {
  return by_dtype(dtype, [&](auto z) {
    using T = decltype(z);
    scale_cols_kernel<T><<<col_grid(n, m), TB, 0, s>>>(reinterpret_cast<T*>(P), ldp, n, m, beta);
    return last();
  });
}

cudaError_t launch_wait_selftest(const int* counter, int target, int complete, uint64_t limit_ns,
                                 uint32_t* status, cudaStream_t s) {
  wait_selftest_kernel<<<1, 32, 0, s>>>(counter, target, complete, limit_ns, status);
  return last();
}

cudaError_t launch_reset(uint8_t* ws, WsLayout L, const float* b, int m, cudaStream_t s) {
  const int blocks = int((L.mpad + TB - 1) / TB);
  // Ring slot 1 of the persistent schedule's column-sum replicas (when the
  // workspace has them) starts at zero too.
  const int crep_len = L.mpad <= PERSIST_REP_MAX_M ? PERSIST_REPS * int(L.mpad) : 0;
  reset_kernel<<<blocks, TB, 0, s>>>(reinterpret_cast<Control*>(ws + L.ctl),
                                     reinterpret_cast<double*>(ws + L.err),
                                     reinterpret_cast<float*>(ws + L.c[1]), int(L.mpad), b,
                                     reinterpret_cast<float*>(ws + L.bws), m,
                                     reinterpret_cast<int*>(ws + L.ctr),
                                     reinterpret_cast<float*>(ws + L.beta),
                                     reinterpret_cast<float*>(ws + L.crep) +
                                         size_t(PERSIST_REPS) * size_t(L.mpad),
                                     crep_len);
  return last();
}

cudaError_t launch_multipass_iter(void* P, int64_t ldp, int n, int m, int dtype, const float* a,
                                  const float* b, float fi, int t, double tol, int check_every,
                                  uint8_t* ws, WsLayout L, cudaStream_t s, int* launches) {
  (void)tol;
  (void)check_every;
  Control* ctl = reinterpret_cast<Control*>(ws + L.ctl);
  float* f = reinterpret_cast<float*>(ws + L.f);
  float* g = reinterpret_cast<float*>(ws + L.g);
  float* c = reinterpret_cast<float*>(ws + L.c[0]);
  return by_dtype(dtype, [&](auto z) {
    using T = decltype(z);
    T* plan = reinterpret_cast<T*>(P);
    const int rows_blocks = sm_count() * 8;
    mp_row_factor<T><<<rows_blocks, TB, 0, s>>>(plan, ldp, n, m, a, fi, f, c, int(L.mpad), ctl);
    cudaError_t e = last();
    if (e != cudaSuccess) return e;
    const dim3 gg = col_grid(n, m);
    mp_scale_rows<T><<<gg, TB, 0, s>>>(plan, ldp, n, m, f);
    if ((e = last()) != cudaSuccess) return e;
    mp_col_sums<T><<<gg, TB, 0, s>>>(plan, ldp, n, m, c);
    if ((e = last()) != cudaSuccess) return e;
    mp_col_factor<<<(m + TB - 1) / TB, TB, 0, s>>>(b, c, fi, g, m, ctl);
    if ((e = last()) != cudaSuccess) return e;
    mp_scale_cols<T><<<gg, TB, 0, s>>>(plan, ldp, n, m, g, ctl, t);
    e = last();
    if (launches) *launches += 5;
    return e;
  });
}

}  // namespace uot
