// Internal declarations of libuot shared by its translation units: the
// workspace layout, kernel argument blocks and the launchers.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "uot.h"

namespace uot {

constexpr uint32_t DEV_ZERO_SUM = UOT_DEV_ZERO_SUM;
constexpr uint32_t DEV_NONFINITE = UOT_DEV_NONFINITE;
constexpr uint32_t DEV_TIMEOUT = UOT_DEV_TIMEOUT;

// A bounded device wait gives up after this long (nanoseconds).
constexpr uint64_t WAIT_LIMIT_NS = 1000000000ull;

// Control block at the start of the workspace.
struct Control {
  uint32_t status;     // DEV_* bits
  int32_t done;        // 1 once the stopping rule fired
  int32_t stop_iter;   // iteration at which it fired
  int32_t iters_done;  // written by the finishing sweep
  double err;          // last stopping error (+inf if none)
  double pad[5];
};

// Deterministic mode: at most this many row groups (one per CTA, or per
// cluster when a row spans several CTAs) in a pass, each with its own slot of
// column partial sums.
constexpr int DET_SLOTS = 304;

// Persistent schedule: CTAs add their column partials into one of this many
// replicas of the column sums (fewer reductions meeting at one address),
// for rows of at most PERSIST_REP_MAX_M columns.
constexpr int PERSIST_REPS = 4;
constexpr int64_t PERSIST_REP_MAX_M = 8192;

// Offsets (bytes) of the workspace regions for an n x m problem.
struct WsLayout {
  size_t ctl;     // Control
  size_t err;     // double[3][2]: per-pass (sum |r_t - r_{t-1}|, sum r_t), ring of 3
  size_t c[3];    // float[mpad]: column sums, ring of 3 (read / accumulate / clear)
  size_t r;       // float[npad]: previous row sums (stopping rule)
  size_t f;       // float[npad]: row factors (multi-pass algorithm)
  size_t g;       // float[mpad]: column factors (multi-pass algorithm)
  size_t bws;     // float[mpad]: copy of b, zero-padded (aligned vector loads)
  size_t ctr;     // int32[9]: per-pass row, arrival and slice counters, rings of 3
  size_t beta;    // float[mpad]: column factors of the last completed pass
  size_t log2k;   // double: log2 of the fixed-point row factor (kernel-form gauge)
  size_t u;       // float[npad]: row scalings U of uot_sinkhorn's kernel-form storage
  size_t crep;    // float[3][PERSIST_REPS][mpad] when mpad <= PERSIST_REP_MAX_M: the
                  // persistent schedule's column sums, in replicas (else it uses c[3])
  size_t part;    // float[DET_SLOTS][mpad]: deterministic mode, column partials per slot
  size_t err_part;// double[DET_SLOTS][2]: deterministic mode, stopping-error partials
  size_t total;
  int64_t mpad, npad;
};

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

inline WsLayout ws_layout(int64_t n, int64_t m, bool det = false) {
  WsLayout L{};
  L.mpad = (m + 63) & ~int64_t(63);
  L.npad = (n + 63) & ~int64_t(63);
  size_t off = 0;
  L.ctl = off; off = align256(off + sizeof(Control));
  L.err = off; off = align256(off + 6 * sizeof(double));
  for (int k = 0; k < 3; ++k) { L.c[k] = off; off = align256(off + size_t(L.mpad) * 4); }
  L.r = off; off = align256(off + size_t(L.npad) * 4);
  L.f = off; off = align256(off + size_t(L.npad) * 4);
  L.g = off; off = align256(off + size_t(L.mpad) * 4);
  L.bws = off; off = align256(off + size_t(L.mpad) * 4);
  L.ctr = off; off = align256(off + 9 * sizeof(int32_t));
  L.beta = off; off = align256(off + size_t(L.mpad) * 4);
  L.log2k = off; off = align256(off + sizeof(double));
  L.u = off; off = align256(off + size_t(L.npad) * 4);
  L.crep = off;
  if (L.mpad <= PERSIST_REP_MAX_M) off = align256(off + size_t(3 * PERSIST_REPS) * size_t(L.mpad) * 4);
  L.part = off;
  if (det) off = align256(off + size_t(DET_SLOTS) * size_t(L.mpad) * 4);
  L.err_part = off;
  if (det) off = align256(off + size_t(DET_SLOTS) * 2 * sizeof(double));
  L.total = off;
  return L;
}

// Arguments of one fused iteration pass.
struct FusedArgs {
  void* plan;
  int64_t ldp;
  int n, m;
  const float* a;
  const float* b;
  float fi;
  int t;               // 1-based iteration index of this pass
  int first;           // 1: no pending column factor (beta = 1)
  int track;           // 1: record row sums and the stopping-error sums
  int check_prev;      // 1: test the stopping rule on iteration t-1 first
  double tol;
  const float* c_prev; // column sums of iteration t-1 (pending beta)
  float* c_next;       // column sums of iteration t (accumulated, pre-zeroed)
  float* c_clear;      // buffer to clear for iteration t+1
  int mpad;
  float* r_prev;       // row sums of iteration t-1 -> overwritten with r_t
  const double* err_prev;
  double* err_next;
  double* err_clear;
  Control* ctl;
  int stages;          // ring depth
  const float* b_ws;   // b, zero-padded to mpad (16-byte aligned)
  int* row_ctr;        // rows taken so far in this pass (dynamic schedule)
  int* ctr_clear;      // counter to clear for iteration t+1
  int dynamic;         // 1: dynamic row schedule (single-CTA rows, bulk copies)
  int* arrive;         // CTAs that finished this pass
  int* arrive_clear;   // arrival counter to clear for iteration t+1
  int* slice_ctr;      // column slices of the end-of-pass job taken so far
  int* slice_clear;    // slice counter to clear for iteration t+1
  float* U;            // kernel form: row scalings (read and updated per row)
  const double* log2k; // kernel form: log2 k for the power-of-two gauge
  const float* beta;   // beta_{t-1}, zero-padded to mpad (read unless first)
  float* beta_out;     // beta_t, written by the last CTAs of this pass
  float* save_r;       // kernel form, optional: r_t (n) of this iteration
  float* save_U;       // U_t (n)
  float* save_c;       // c_t (m)
  float* save_V;       // V_t (m)
  int pot;             // kernel form: scaling-vector rule (uot_rule POT)
  float kscale;        // kernel form: storage scale of K (2^s; FP16 K is stored x 2^15)
  int det;             // 1: deterministic mode (static rows, partials to slots)
  int no_factors;      // 1: leave the column sums in c_next, skip the end-of-pass job
                       //    (row-sharded passes: the sums are reduced across processes)
  float* part;         // deterministic: column partials, slot g at part + g * mpad
  double* err_part;    // deterministic: stopping-error partials, slot g at 2 * g
};

// History of a kernel-form solve kept for the adjoint: a header, then for
// t = 0..iters the scalings U_t (npad floats), V_t (mpad), row sums r_t (npad)
// and column sums c_t (mpad); entries t = 0 of r and c are unused.
struct HistHeader {
  double log2k;
  int32_t n, m, iters;
  float k_scale_inv;
};
struct HistLayout {
  size_t U, V, r, c, total;  // offsets of the t = 0 arrays
  size_t strideU, strideV;   // bytes per iteration
};
inline HistLayout hist_layout(int64_t n, int64_t m, int iters) {
  HistLayout L{};
  const int64_t npad = (n + 63) & ~int64_t(63), mpad = (m + 63) & ~int64_t(63);
  const size_t T1 = size_t(iters) + 1;
  L.strideU = size_t(npad) * 4;
  L.strideV = size_t(mpad) * 4;
  size_t off = align256(sizeof(HistHeader));
  L.U = off; off += T1 * L.strideU;
  L.V = off; off += T1 * L.strideV;
  L.r = off; off += T1 * L.strideU;
  L.c = off; off += T1 * L.strideV;
  L.total = align256(off);
  return L;
}

struct FusedConfig {
  int dtype;
  int threads;
  int vecs;     // 16-byte vectors per thread per row
  int cols;     // columns per CTA
  int max_regs_ok;
};

int fused_num_configs();
bool fused_config_info(int k, FusedConfig* out);
// Picks a configuration for dtype/m (tile = 0: automatic; else k+1).
int fused_pick(int dtype, int64_t m, int tile);
// Launch geometry for config k (in place, or kernel form when kf) at cluster
// size cs: grid (CTAs), ring depth and dynamic shared memory.
cudaError_t fused_geometry(bool kf, int k, int cs, int n, int* grid, int* stages, size_t* smem);
cudaError_t fused_launch(bool kf, int k, int cs, int grid, size_t smem, bool tma,
                         const FusedArgs& args, cudaStream_t s);
// Deterministic mode: after a pass over `groups` row groups, adds the column
// partial slots in slot order into the column sums of iteration t, forms the
// next column factors (kernel form: the new V), and adds the stopping-error
// slots in order.
cudaError_t det_reduce_launch(bool kf, int groups, const FusedArgs& args, cudaStream_t s);

// Simple kernels (simple.cu).
cudaError_t launch_init(const float* C, int64_t ldc, void* P, int64_t ldp, int n, int m,
                        float reg, int dtype, float scale, cudaStream_t s);
cudaError_t launch_kform_reset(float* U, int n, float u0, float* V_ws, int m, int mpad,
                               const float* a, const float* b, float fi, bool pot, double* log2k,
                               cudaStream_t s);
cudaError_t launch_kform_finish(float* V, int m, int iters, const uint8_t* ws, WsLayout L,
                                double tol, cudaStream_t s);
cudaError_t launch_kform_plan(const void* K, int64_t ldk, int k_dtype, const float* U,
                              const float* V, int n, int m, void* P, int64_t ldp, int p_dtype,
                              cudaStream_t s);
cudaError_t launch_kform_materialize(void* P, int64_t ldp, int dtype, const float* U,
                                     const float* V, int n, int m, cudaStream_t s);
cudaError_t launch_kform_cost(const void* K, int64_t ldk, int k_dtype, const float* U,
                              const float* V, const float* C, int64_t ldc, int n, int m,
                              double* out, cudaStream_t s);
cudaError_t launch_finish(void* P, int64_t ldp, int n, int m, int dtype, const float* b,
                          float fi, int iters, const uint8_t* ws, WsLayout L, double tol,
                          int check_every, bool beta_ready, cudaStream_t s);
cudaError_t launch_cost(const void* P, int64_t ldp, const float* C, int64_t ldc, int n, int m,
                        int dtype, double* out, cudaStream_t s);
// Row-sharded passes: workspace set-up of one pass (beta_in copied into the
// zero-padded factor buffer, or ones when NULL; column sums and counters
// cleared), the column factors from reduced sums, and the last column scale.
cudaError_t launch_shard_prep(uint8_t* ws, WsLayout L, const float* beta_in, int m, cudaStream_t s);
cudaError_t launch_shard_factors(const float* c, const float* b, int m, float fi, float* beta,
                                 uint32_t* status, cudaStream_t s);
cudaError_t launch_scale_cols(void* P, int64_t ldp, int n, int m, int dtype, const float* beta,
                              cudaStream_t s);
cudaError_t launch_reset(uint8_t* ws, WsLayout L, const float* b, int m, cudaStream_t s);
cudaError_t launch_factor_selftest(const float* target, const float* total, int64_t count,
                                   float fi, float* out, uint32_t* status, cudaStream_t s);
cudaError_t launch_wait_selftest(const int* counter, int target, int complete, uint64_t limit_ns,
                                 uint32_t* status, cudaStream_t s);
cudaError_t launch_multipass_iter(void* P, int64_t ldp, int n, int m, int dtype, const float* a,
                                  const float* b, float fi, int t, double tol, int check_every,
                                  uint8_t* ws, WsLayout L, cudaStream_t s, int* launches);

cudaError_t launch_hist_init(uint8_t* hist, int n, int m, int iters, float u0, const double* log2k,
                             cudaStream_t s);

// Kernel-form pass with two rows per step (kform_pair.cu): the configuration
// for rows of m columns of `dtype` and its cluster size (-1 if none), its
// launch geometry for n rows, and one launch.
int kform_pair_pick(int dtype, int64_t m, int* cs);
cudaError_t kform_pair_geometry(int pair, int cs, int n, int* grid, int* stages, size_t* smem);
cudaError_t kform_pair_launch(int pair, int cs, int grid, size_t smem, const FusedArgs& args,
                              cudaStream_t s);

// Persistent iteration (persistent.cu): every iteration in one cooperative
// launch with each CTA's rows held in shared memory.  persistent_plan sets
// ok = false when the plan does not fit (or cooperative launches are not
// available).
struct PersistPlan {
  bool ok;
  int grid, rows, ldm;
  size_t smem;
};
cudaError_t persistent_plan(int dtype, bool kf, int n, int m, int max_ctas, PersistPlan* out);
cudaError_t persistent_launch(int dtype, bool kf, const PersistPlan& pl, void* plan, int64_t ldp,
                              int n, int m, const float* a, const float* b, float fi, int iters,
                              double tol, int check_every, uint8_t* ws, const WsLayout& L,
                              float* U, float* V, int pot, float kscale, bool write_plan,
                              cudaStream_t s);

void count_launch(int k = 1);

}  // namespace uot
