/*
 * uot.h -- C ABI of libuot, the GB300 (sm_103a) Sinkhorn iteration for
 * entropy-regularised unbalanced optimal transport (MAP-UOT).
 *
 * The method (Section 2.1): given a non-negative N x M matrix P and targets
 * a (length N, row target) and b (length M, column target), each iteration
 * rescales every row i by alpha_i = (a_i / sum_j P_ij)^fi and then every
 * column j by beta_j = (b_j / sum_i P_ij)^fi, with fi = reg_m / (reg_m + reg).
 * MAP-UOT (Section 4, Algorithm 1) performs one iteration as a single sweep
 * over the matrix: the pending column factor of the previous iteration and the
 * row rescaling of the current one are applied to a row while it is on chip,
 * and the column sums for the next factor are accumulated in the same pass.
 *
 * Conventions for every entry point
 *  - Matrices are dense and row-major with a leading dimension (elements
 *    between row starts) >= the number of columns.  All array pointers are
 *    DEVICE pointers owned by the caller unless stated otherwise.
 *  - Sizes: 1 <= n, m <= 2^30 (row and column indices and the per-pass row
 *    counters stay in 32-bit range); other sizes are UOT_ERR_INVALID_ARG.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Work is enqueued asynchronously; nothing synchronises unless stated.
 *  - Nothing is allocated or freed on the device by the library; scratch
 *    memory is a caller-owned workspace sized by uot_workspace_size().
 *  - Errors are return codes; nothing is thrown across the ABI.  Argument
 *    errors are detected on the host before anything is enqueued.  Conditions
 *    found on the device (zero or non-finite sums) are OR-ed into a status
 *    word in the workspace and reported through uot_result.
 *  - The plan dtype is FP32, BF16 or FP16 (uot_dtype); row/column sums and
 *    factors are always FP32; the transport cost and the stopping error are
 *    accumulated in FP64.
 */
#ifndef UOT_H
#define UOT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum uot_status {
  UOT_OK = 0,
  UOT_ERR_INVALID_ARG = 1,  /* bad size, pointer, parameter or alignment      */
  UOT_ERR_CUDA = 2,         /* a CUDA runtime call failed                      */
  UOT_ERR_NONFINITE = 3,    /* device saw a non-finite sum or factor           */
  UOT_ERR_ZERO_SUM = 4,     /* device saw a zero sum with a positive target    */
  UOT_ERR_TIMEOUT = 5,      /* a bounded device wait gave up                    */
  UOT_ERR_UNSUPPORTED = 6,  /* valid request this build does not implement     */
  UOT_ERR_WORKSPACE = 7     /* workspace NULL, too small or misaligned         */
} uot_status;

typedef enum uot_dtype { UOT_F32 = 0, UOT_BF16 = 1, UOT_F16 = 2 } uot_dtype;

/* How uot_sinkhorn sweeps the plan.
 * FUSED:     one read and one write of the plan per iteration (Algorithm 1's
 *            single double loop, Section 4.1.1), the default.
 * MULTIPASS: the separate row-sum, row-scale, column-sum and column-scale
 *            sweeps of the baseline form of Section 2.1 (three reads and two
 *            writes of the plan per iteration plus one more read), kept as the
 *            plain GPU reference the fused path is compared against. */
typedef enum uot_algo { UOT_ALGO_FUSED = 0, UOT_ALGO_MULTIPASS = 1 } uot_algo;

/* Which update the iteration applies.
 * PAPER: the rule of Section 2.1 as printed: each row of the plan is
 *        rescaled by (a_i / rowsum_i)^fi, then each column by
 *        (b_j / colsum_j)^fi.  Its limit is a balanced entropic OT plan
 *        between rescaled marginals (the masses meet in between).
 * POT:   the scaling-vector form of unbalanced Sinkhorn (the update of POT's
 *        sinkhorn_unbalanced): with the plan diag(u) K diag(v),
 *        u <- (a / (K v))^fi, then v <- (b / (K^T u))^fi.  As a plan rescale
 *        this is the PAPER factor times u_i^(fi - 1).  Its limit minimises
 *        <P,C> + reg sum P (log P - 1) + reg_m KL(P 1 | a) + reg_m KL(P^T 1 | b).
 *        Only the kernel form keeps u and v, so only the kernel-form entry
 *        points, uot_sinkhorn with UOT_STORAGE_KFORM and the batched engines
 *        accept it; the two rules agree when fi = 1.  The adjoint
 *        (uot_sinkhorn_backward) is for PAPER only. */
typedef enum uot_rule { UOT_RULE_PAPER = 0, UOT_RULE_POT = 1 } uot_rule;

/* How uot_sinkhorn keeps the plan during the iterations (both give the plan
 * after the column step of the last iteration in `plan` on return).
 * INPLACE: every fused pass reads the plan and writes it back rescaled, one
 *          read and one write per iteration (Section 3.1's minimum for a
 *          rewritten plan).  Each pass rounds every entry (twice), and near
 *          the fixed point the factors change little from pass to pass, so
 *          an entry can be rounded the same way many times: in FP32 the
 *          worst entry's error grows about linearly with the iteration count
 *          (measured on the GPU against the FP64 rule: 2.6e-6 after 100,
 *          8e-6 after 500 iterations of a 2048 x 16384 plan).
 * KFORM:   the plan of Section 2.1 is always diag(U) K diag(V) with K the
 *          initial plan, so the buffer is kept as K, read-only, while FP32
 *          scalings U (in the workspace) and V are updated; one read per
 *          iteration, and a last sweep writes U_i K_ij V_j over the buffer.
 *          Every entry is rounded once at the end (1.1e-6 after 500
 *          iterations of the same plan).  Fused algorithm only. */
typedef enum uot_storage { UOT_STORAGE_INPLACE = 0, UOT_STORAGE_KFORM = 1 } uot_storage;

/* How uot_sinkhorn and uot_sinkhorn_kform launch the iterations.
 * AUTO:       PERSISTENT when its conditions hold, else PASSES.
 * PASSES:     one fused-pass launch per iteration (Algorithm 1's sweep with
 *             the plan streamed from memory each time).
 * PERSISTENT: one cooperative launch runs every iteration: each CTA (one per
 *             SM) keeps a block of rows in shared memory for the whole solve,
 *             adds its column partial sums into the workspace, and meets the
 *             other CTAs at a bounded grid barrier once per iteration; the
 *             rows go back to memory once, at the end.  For plans that fit in
 *             the shared memory of the GPU's CTAs (about 220 KB per CTA: up to
 *             about 30 MB of FP32 plan, e.g. N = M = 2048) where the per-pass
 *             launch would dominate.  Needs the fused algorithm, no forced
 *             tile or cluster, and no deterministic mode or adjoint history;
 *             otherwise (or if the plan does not fit) UOT_ERR_UNSUPPORTED. */
typedef enum uot_schedule {
  UOT_SCHED_AUTO = 0,
  UOT_SCHED_PASSES = 1,
  UOT_SCHED_PERSISTENT = 2
} uot_schedule;

/* Bits of uot_result.dev_status. */
#define UOT_DEV_ZERO_SUM 1u
#define UOT_DEV_NONFINITE 2u
#define UOT_DEV_TIMEOUT 4u

typedef struct uot_options {
  int32_t dtype;        /* uot_dtype of the plan storage (default UOT_F32)    */
  int32_t algo;         /* uot_algo (default UOT_ALGO_FUSED)                  */
  int32_t check_every;  /* stopping-rule period in iterations, >= 1           */
  int32_t tile;         /* 0 = automatic; k > 0 forces fused config k-1 of
                           uot_fused_config() (for tuning and tests)          */
  int32_t cluster;      /* 0 = automatic; else CTAs per row (1..8), fused only */
  int32_t max_ctas;     /* 0 = as many CTAs as fit; else at most this many per
                           launch (to run several solves side by side, e.g.
                           as parallel branches of one CUDA graph)          */
  int32_t rule;         /* uot_rule (default UOT_RULE_PAPER)                  */
  int32_t storage;      /* uot_storage of uot_sinkhorn (default INPLACE)      */
  int32_t deterministic;/* 1: bit-identical results from run to run with the
                           same inputs, options and device: every CTA keeps a
                           fixed set of rows, writes its column partial sums
                           to its own slot of the workspace, and a reduction
                           launch after each pass adds the slots in a fixed
                           order (instead of floating-point atomics and a
                           dynamic row schedule).  Slower (static rows, one
                           more launch per iteration); one row per step.
                           uot_sinkhorn and uot_sinkhorn_kform only.        */
  int32_t schedule;     /* uot_schedule (default UOT_SCHED_AUTO)              */
  int32_t reserved[1];  /* must be 0                                          */
  void* pass_events[2]; /* optional cudaEvent_t pair: uot_sinkhorn records
                           [0] on `stream` just before its first iteration
                           pass and [1] just after its last (NULL = none);
                           used to time the passes alone                     */
} uot_options;

typedef struct uot_result {
  int32_t iters_done;   /* iterations completed (< iters if tol stopped it)   */
  uint32_t dev_status;  /* UOT_DEV_* bits seen on the device                  */
  double err;           /* last stopping error computed, or +inf if none      */
} uot_result;

/* Fills *opt with the defaults above. */
void uot_default_options(uot_options* opt);

/* Human-readable name of a status code (static string). */
const char* uot_status_string(uot_status s);

/* Bytes of device workspace uot_sinkhorn needs for an n x m plan (a multiple
 * of 256).  The workspace must be 256-byte aligned.  Returns 0 on bad sizes. */
size_t uot_workspace_size(int64_t n, int64_t m, const uot_options* opt);

/* Number of kernels this library has launched in the calling process (a
 * monotone counter, for accounting in benchmarks). */
uint64_t uot_launch_count(void);

/*
 * uot_selftest_wait -- shows on the device that the library's bounded waits
 * give up instead of hanging (failure detection without a GPU fault).  One
 * thread waits on an mbarrier phase with the same helper the bulk-copy rings
 * use, then spins with acquire loads on the device int *counter_dev until it
 * reaches `target`, as the inter-CTA barriers do; each wait gives up after
 * limit_s seconds (0 < limit_s <= 10).  With complete == 0 nothing arrives
 * on the barrier.  status_dev (two device uint32) receives UOT_DEV_TIMEOUT
 * or 0 for the barrier and for the counter.  The kernel returns either way
 * and the context stays usable.  Asynchronous.  Errors: UOT_ERR_INVALID_ARG
 * (NULL or misaligned pointers, limit out of range), UOT_ERR_CUDA.
 */
uot_status uot_selftest_wait(const int32_t* counter_dev, int32_t target, int32_t complete,
                             double limit_s, uint32_t* status_dev, void* stream);

/*
 * uot_selftest_factor -- evaluates the rescaling factor of Section 2.1,
 * (target / total)^fi, exactly as every pass of the library does (FP32
 * division, then the fast power intrinsic; degenerate readings: target 0
 * gives 0, a zero total with a positive target gives 1 and UOT_DEV_ZERO_SUM,
 * a non-finite total or factor sets UOT_DEV_NONFINITE), for `count` pairs:
 * out[k] from target[k] and total[k] (device FP32 arrays, 4-byte aligned),
 * with the status bits OR-ed into *status_dev (one device uint32, which the
 * caller clears).  For checking the factor's accuracy against a reference
 * power.  Asynchronous.  Errors: UOT_ERR_INVALID_ARG (NULL or misaligned
 * pointers, count < 1 or > 2^30, fi outside (0, 1]), UOT_ERR_CUDA.
 */
uot_status uot_selftest_factor(const float* target, const float* total, int64_t count, float fi,
                               float* out, uint32_t* status_dev, void* stream);

/*
 * uot_init_kernel -- initial plan P0_ij = exp(-C_ij / reg).
 * Section 2.1 starts from a "given matrix"; the Gibbs kernel of the cost is
 * the usual one for entropic transport.  C: n x m FP32, leading dimension ldc.
 * plan: n x m of opt->dtype (FP32 if opt is NULL), leading dimension ldp,
 * written with round-to-nearest-even.  FP32 expf, no fast-math.
 * Errors: UOT_ERR_INVALID_ARG (n, m < 1; ld < m; reg not > 0 or not finite;
 * NULL pointers), UOT_ERR_CUDA.
 */
uot_status uot_init_kernel(const float* C, int64_t ldc, void* plan, int64_t ldp,
                           int64_t n, int64_t m, float reg,
                           const uot_options* opt, void* stream);

/*
 * uot_sinkhorn -- `iters` iterations of the Section 2.1 rule on `plan`, in place.
 * Each iteration: row step (alpha_i = (a_i/r_i)^fi) then column step
 * (beta_j = (b_j/c_j)^fi); fi = reg_m/(reg_m+reg), reg_m = +INFINITY gives
 * fi = 1 (balanced Sinkhorn).  The fused algorithm runs one plan sweep per
 * iteration plus one final sweep that applies the last column factor, so on
 * return `plan` holds the plan after the column step of the last iteration.
 * opt->storage chooses how the plan is kept during the iterations
 * (uot_storage: rewritten in place by every pass, or kept as K with FP32
 * scalings and written once at the end); opt->deterministic makes the result
 * bit-identical from run to run.
 * Degenerate factors: target 0 gives factor 0; a zero sum with a positive
 * target gives factor 1 and UOT_DEV_ZERO_SUM.
 * Stopping (the paper leaves the error undefined): when tol > 0, after every
 * check_every-th iteration t >= 2, err_t = sum_i |r_t,i - r_{t-1},i| /
 * sum_i r_t,i (FP64) is compared with tol and the remaining iterations are
 * skipped on the device once err_t <= tol (no host synchronisation).
 *   plan      n x m, dtype opt->dtype, leading dimension ldp, in/out.
 *   a, b      FP32 targets of length n and m, read-only, >= 0.
 *   workspace device scratch of >= uot_workspace_size(n, m, opt) bytes,
 *             256-byte aligned, owned by the caller; ws_bytes is its size.
 *             It also holds the result (iterations done, error, status) until
 *             the next call with the same workspace.
 *   out       host pointer: if non-NULL the call synchronises `stream` and
 *             fills *out, returning UOT_ERR_NONFINITE / UOT_ERR_ZERO_SUM /
 *             UOT_ERR_TIMEOUT if the device flagged one.  If NULL the call is
 *             fully asynchronous (and may be captured in a CUDA graph); read
 *             the result later with uot_read_result().
 * Errors: UOT_ERR_INVALID_ARG, UOT_ERR_WORKSPACE, UOT_ERR_CUDA, device codes.
 */
uot_status uot_sinkhorn(void* plan, int64_t ldp, const float* a, const float* b,
                        int64_t n, int64_t m, float reg, float reg_m,
                        int32_t iters, double tol, void* workspace, size_t ws_bytes,
                        const uot_options* opt, void* stream, uot_result* out);

/*
 * Kernel form.  The plan of Section 2.1 is always diag(U) K diag(V), with K
 * the initial plan and U, V the products of the row and column factors so
 * far; the same iteration can therefore keep K read-only and update only the
 * FP32 vectors U (length n) and V (length m).  One fused pass per iteration
 * (Algorithm 1's single sweep) reads K once -- sizeof(K element) bytes per
 * element instead of a read and a write of the plan -- and K is rounded only
 * once, which is what makes 16-bit storage accurate enough.  In real
 * arithmetic the iterates equal uot_sinkhorn's.
 *
 * uot_init_kernel_scaled -- K = exp(-C/reg) * 2^log2_scale in opt->dtype
 * (log2_scale an integer in [-100, 100]; FP16 needs a positive scale to keep
 * small entries out of its subnormal range, e.g. 15 when max K = 1).
 * Errors as uot_init_kernel.
 */
uot_status uot_init_kernel_scaled(const float* C, int64_t ldc, void* K, int64_t ldk, int64_t n,
                                  int64_t m, float reg, float log2_scale,
                                  const uot_options* opt, void* stream);

/*
 * uot_sinkhorn_kform -- `iters` iterations of the Section 2.1 rule in kernel
 * form.  K: n x m of opt->dtype (FP32/BF16/FP16), leading dimension ldk,
 * read-only, stored scaled by 2^k_log2_scale (integer; 0 if unscaled).  On
 * return U (n floats) and V (m floats), device arrays owned by the caller,
 * hold the scalings with the storage scale folded into U, so the plan is
 * P_ij = U_i K_ij V_j for K as stored.  U and V are determined up to a common
 * power of two (U 2^e, V 2^-e): at the fixed point the row factors tend to
 * k = (sum a / sum b)^(fi/(2-fi)) and the column factors to 1/k, so each pass
 * moves an exact power of two between them to keep both in FP32 range.  U
 * and V are overwritten (the call starts from U = 2^-k_log2_scale, V = 1).  Row/column sums, factors and
 * scalings are FP32; the stopping error is FP64 (same rule as uot_sinkhorn).
 * Only the fused algorithm exists in this form.  Other arguments, the
 * workspace and errors are those of uot_sinkhorn.
 */
uot_status uot_sinkhorn_kform(const void* K, int64_t ldk, const float* a, const float* b,
                              int64_t n, int64_t m, float reg, float reg_m, int32_t iters,
                              double tol, float k_log2_scale, float* U, float* V,
                              void* workspace, size_t ws_bytes, const uot_options* opt,
                              void* stream, uot_result* out);

/* uot_kform_plan -- materialises P_ij = (U_i K_ij) V_j (FP32 products) into
 * `plan` (n x m, plan_dtype, leading dimension ldp).  K of k_dtype.  Async. */
uot_status uot_kform_plan(const void* K, int64_t ldk, int32_t k_dtype, const float* U,
                          const float* V, int64_t n, int64_t m, void* plan, int64_t ldp,
                          int32_t plan_dtype, void* stream);

/* uot_kform_cost -- <diag(U) K diag(V), C> without materialising the plan;
 * each term (U_i K_ij) V_j C_ij is accumulated in an error-free FP32 pair and
 * the partial sums in FP64.  out_dev: one device double, overwritten.  Async. */
uot_status uot_kform_cost(const void* K, int64_t ldk, int32_t k_dtype, const float* U,
                          const float* V, const float* C, int64_t ldc, int64_t n, int64_t m,
                          double* out_dev, void* stream);

/*
 * Differentiation of the unrolled iteration (the paper has no adjoint; this
 * is reverse mode through the Section 2.1 rule in log space).
 *
 * uot_grad_hist_size -- bytes of the history a solve of `iters` iterations
 * keeps for its adjoint: the scalings U_t, V_t and the row/column sums r_t,
 * c_t for every t (about (iters + 1) * 8 * (n + m) bytes).
 *
 * uot_sinkhorn_kform_save -- uot_sinkhorn_kform (fixed `iters`, no stopping
 * rule) that also fills `hist` (device, caller-owned, 256-byte aligned,
 * >= uot_grad_hist_size bytes).
 */
size_t uot_grad_hist_size(int64_t n, int64_t m, int32_t iters);
uot_status uot_sinkhorn_kform_save(const void* K, int64_t ldk, const float* a, const float* b,
                                   int64_t n, int64_t m, float reg, float reg_m, int32_t iters,
                                   float k_log2_scale, float* U, float* V, void* hist,
                                   size_t hist_bytes, void* workspace, size_t ws_bytes,
                                   const uot_options* opt, void* stream, uot_result* out);

/*
 * uot_sinkhorn_backward -- gradients of L = <P_T, C> times grad_out with
 * respect to C (dC, n x m FP32, leading dimension lddc), a (da, n) and b
 * (db, m), for the solve recorded in `hist` by uot_sinkhorn_kform_save with
 * FP32 K = exp(-C/reg) (k_log2_scale 0) and the same iters, reg, reg_m.
 * Reverse steps t = T..1, one read-only sweep of K each: Q_t =
 * diag(U_t) K diag(V_{t-1}) and R_t = diag(U_{t-1}) K diag(V_{t-1}) are
 * recomputed per row, the row adjoint F and column adjoint G follow
 *   w = -fi G / c_t,  db += fi G / b,  F += Q_t w,  G = (1 - fi) G,
 *   z = -fi F / r_t,  da += fi F / a,  G += R_t^T z, F = (1 - fi) F,
 * and dl = P_T * C + sum_t (Q_t * w + R_t * z) is formed once at the end
 * from vectors each step records (the sum is K times a rank-2T matrix; one
 * FP32 contraction of depth 2T), giving dC = g (P_T - dl / reg) and da, db
 * times g, where g = grad_out, times *grad_out_dev when grad_out_dev (one
 * device double, 8-byte aligned, read by the last launches) is not NULL --
 * so a caller whose incoming gradient lives on the device need not
 * synchronise.  K and dC must be 16-byte aligned with ldk and lddc multiples
 * of 4; m <= 8192.  The workspace (uot_backward_workspace_size(n, m, iters)
 * bytes, about (iters + 3) * 4 (2n + m) bytes, 256-byte aligned) is
 * caller-owned.  opt may be NULL; only opt->max_ctas is used.  Asynchronous.
 */
size_t uot_backward_workspace_size(int64_t n, int64_t m, int32_t iters);
uot_status uot_sinkhorn_backward(const float* K, int64_t ldk, const float* C, int64_t ldc,
                                 const float* a, const float* b, int64_t n, int64_t m, float reg,
                                 float reg_m, int32_t iters, const void* hist, size_t hist_bytes,
                                 double grad_out, const double* grad_out_dev, float* dC,
                                 int64_t lddc, float* da, float* db, void* workspace,
                                 size_t ws_bytes, const uot_options* opt, void* stream);

/*
 * uot_sinkhorn_backward_batch -- uot_sinkhorn_backward for `batch` problems
 * of one shape (n x m, iters, reg, reg_m) in one set of launches: each
 * reverse step is a single launch over a grid of problems x row blocks,
 * instead of one launch per problem and step.  Problem k's K, C and dC
 * start stride_k, stride_c and stride_dc elements after problem 0's (same
 * leading dimensions; stride_k and stride_dc multiples of 4; no overlap),
 * its history hist_stride bytes after problem 0's (>= uot_grad_hist_size,
 * a multiple of 256; hist 256-byte aligned), and a, b, da, db are packed
 * [batch][n] / [batch][m].  grad_out multiplies every problem's gradients;
 * grad_out_dev, when not NULL, holds `batch` device doubles (problem k's
 * factor).  The workspace is uot_backward_batch_workspace_size(batch, n, m,
 * iters) bytes, 256-byte aligned, caller-owned.  opt->max_ctas caps the
 * CTAs of a reverse launch over the whole batch.  1 <= batch <= 65535.
 * Otherwise as uot_sinkhorn_backward (which is this call with batch 1).
 */
size_t uot_backward_batch_workspace_size(int32_t batch, int64_t n, int64_t m, int32_t iters);
uot_status uot_sinkhorn_backward_batch(int32_t batch, const float* K, int64_t ldk,
                                       int64_t stride_k, const float* C, int64_t ldc,
                                       int64_t stride_c, const float* a, const float* b,
                                       int64_t n, int64_t m, float reg, float reg_m,
                                       int32_t iters, const void* hist, size_t hist_stride,
                                       double grad_out, const double* grad_out_dev, float* dC,
                                       int64_t lddc, int64_t stride_dc, float* da, float* db,
                                       void* workspace, size_t ws_bytes, const uot_options* opt,
                                       void* stream);

/* Synchronises `stream` and reads the result of the last uot_sinkhorn call
 * that used `workspace` (same n, m, opt).  Returns the device status as a
 * uot_status as uot_sinkhorn does with a non-NULL `out`. */
uot_status uot_read_result(const void* workspace, int64_t n, int64_t m,
                           const uot_options* opt, void* stream, uot_result* out);

/*
 * uot_cost -- transport cost <P, C> = sum_ij P_ij C_ij; each product is
 * accumulated exactly in an error-free FP32 pair (Dekker / Knuth), and the
 * partial sums in FP64.
 * plan: n x m of `dtype` (uot_dtype), leading dimension ldp; C: n x m FP32,
 * leading dimension ldc; out_dev: one device double, OVERWRITTEN with the cost
 * (the call zeroes it first on `stream`).  Asynchronous.
 * Errors: UOT_ERR_INVALID_ARG, UOT_ERR_CUDA.
 */
uot_status uot_cost(const void* plan, int64_t ldp, const float* C, int64_t ldc,
                    int64_t n, int64_t m, int32_t dtype, double* out_dev, void* stream);

/*
 * uot_sinkhorn_noalloc -- uot_sinkhorn for callers that cannot allocate.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot hand the library a device buffer -- for example a plugin inside a
 * host application that owns all device memory and offers its plugins no
 * allocation hook, or code on a latency-critical path that must not call
 * cudaMalloc (which can synchronise the device) and has no pool to draw from.
 * It runs exactly uot_sinkhorn, but its scratch memory is a fixed array of
 * UOT_STATIC_SCRATCH_BYTES bytes compiled into the library: every GPU that
 * loads the library holds that array until the process exits, and the call
 * allocates nothing (no cudaMalloc, cudaFree or allocating library routine).
 * The caller still passes the plan and targets.
 *  - Size limit: problems whose uot_workspace_size(n, m, opt) exceeds
 *    UOT_STATIC_SCRATCH_BYTES (2 MiB) are rejected with UOT_ERR_WORKSPACE
 *    before anything is enqueued; N = M = 32768 needs about 1 MiB.
 *  - Set-up: the array's device address belongs to the CUDA context that
 *    loaded the library's module, so the first call in each context -- on
 *    each device, again after cudaDeviceReset, and in any context the caller
 *    creates and makes current -- looks it up once (keyed by the driver's
 *    context id) with that context current; make that first call before any
 *    stream capture in that context.
 *  - Sharing: every call on a device uses the same array, and the array keeps
 *    the last call's contents (each call re-initialises what must start at
 *    zero).  Calls whose work overlaps on the GPU -- on different streams, or
 *    from different host threads -- race on the array and must be serialised
 *    by the caller.
 *  - Result: the iteration count, last error and device status live in the
 *    shared array, so pass `out` (the call then synchronises `stream`) to get
 *    them; with out == NULL the call is asynchronous and they are not
 *    retrievable.
 * Arguments and errors are those of uot_sinkhorn without the workspace.
 */
#define UOT_STATIC_SCRATCH_BYTES ((size_t)2 << 20)
uot_status uot_sinkhorn_noalloc(void* plan, int64_t ldp, const float* a, const float* b,
                                int64_t n, int64_t m, float reg, float reg_m, int32_t iters,
                                double tol, const uot_options* opt, void* stream,
                                uot_result* out);

/*
 * Row-sharded iteration (Section 5.5: the rows are split over processes, and
 * the one exchange per iteration is an all-reduce of the column-sum vector,
 * which replaces the final reduction of Algorithm 1).  A process holds the
 * rows [lo, hi) of the plan (n = hi - lo rows here, all m columns), their
 * targets a[lo..hi), and all of b.  One iteration t = 1, 2, ...:
 *   uot_shard_pass     the fused pass over the block: applies the column
 *                      factors of iteration t-1 (beta_in, m device floats;
 *                      NULL at t = 1: none pending), forms and applies the
 *                      row factors (a_i / r_i)^fi, and writes the block's
 *                      column sums of iteration t to colsum (m device floats,
 *                      overwritten);
 *   (caller)           all-reduces colsum (sum) over the processes;
 *   uot_shard_factors  beta_j = (b_j / c_j)^fi from the reduced sums into
 *                      beta (m device floats); degenerate-case bits are OR-ed
 *                      into *status_dev when it is not NULL.
 * After the last iteration uot_shard_finish multiplies column j of the block
 * by beta_j, so the block holds its rows of the plan after the column step
 * of the last iteration, as uot_sinkhorn would leave them.  With one process
 * the sequence equals uot_sinkhorn's (in-place storage, fused passes).
 * uot_shard_pass takes the workspace of uot_sinkhorn for an n x m problem; t
 * only sets the direction in which the pass visits the rows.  Options: FP32,
 * BF16 or FP16 plans, the rule of Section 2.1, in-place storage and fused
 * passes only (UOT_ERR_UNSUPPORTED otherwise); no stopping rule (the caller
 * decides after the reduction).  The row factors' degenerate-case bits
 * accumulate in the workspace from the first pass (beta_in NULL) on:
 * uot_read_result reports them.  All three are asynchronous.
 */
uot_status uot_shard_pass(void* plan, int64_t ldp, const float* a, int64_t n, int64_t m,
                          float reg, float reg_m, int32_t t, const float* beta_in, float* colsum,
                          void* workspace, size_t ws_bytes, const uot_options* opt,
                          void* stream);
uot_status uot_shard_factors(const float* colsum, const float* b, int64_t m, float reg,
                             float reg_m, float* beta, uint32_t* status_dev, void* stream);
uot_status uot_shard_finish(void* plan, int64_t ldp, int64_t n, int64_t m, int32_t dtype,
                            const float* beta, void* stream);

/*
 * Three-way form.  The paper notes that the method applies to higher-
 * dimensional tensors; this is the rule of Section 2.1 on a plan of
 * n1 x n2 x n3 entries with mode targets a (n1), b (n2), c (n3): every
 * iteration rescales along mode 1, then mode 2, then mode 3 by
 * (target / marginal sum)^fi (degenerate readings as in uot_sinkhorn).  One
 * sweep of the plan per iteration, as Algorithm 1 does for the matrix: a
 * slice P[i, :, :] is a row of the mode-1 unfolding (n1 x n2 n3), so the
 * fused pass applies the pending mode-2 and mode-3 factors, forms the slice
 * factor and accumulates M_jk = sum_i of the rescaled slices; the mode-2
 * factors come from the sums over k of M, the mode-3 factors from the sums
 * over j of M weighted by the new mode-2 factors.
 *   P          device, contiguous n1 x n2 x n3 (k fastest), FP32/BF16/FP16
 *              (opt->dtype), in/out: P0 in, the plan after the mode-3 step
 *              of the last iteration out.
 *   a, b, c    device FP32 targets, read-only.
 *   workspace  >= uot_tensor3_workspace_size(n1, n2, n3) bytes, 256-byte
 *              aligned, caller-owned (0 on bad sizes: each >= 1, n2 n3 <= 2^30).
 *   out        as in uot_sinkhorn (NULL: asynchronous).
 * A slice is one row of the fused pass, split over at most a cluster of 8
 * CTAs: n2 n3 <= 8 x 16384 = 131072 (wider slices: UOT_ERR_UNSUPPORTED).
 * Options: fused passes, in-place storage, the rule of Section 2.1, no
 * deterministic mode, no persistent schedule (UOT_ERR_UNSUPPORTED
 * otherwise); no stopping rule.  Errors as uot_sinkhorn.
 */
size_t uot_tensor3_workspace_size(int64_t n1, int64_t n2, int64_t n3);
uot_status uot_sinkhorn_tensor3(void* P, int64_t n1, int64_t n2, int64_t n3, const float* a,
                                const float* b, const float* c, float reg, float reg_m,
                                int32_t iters, void* workspace, size_t ws_bytes,
                                const uot_options* opt, void* stream, uot_result* out);

/*
 * Batched iteration: many independent problems of uneven size (Section 2.1
 * rule, one sweep per iteration as in Algorithm 1; FP32 plans, overwritten
 * by the result).  Two engines share a batch:
 *   on chip    a problem whose initial plan fits in the shared memory of one
 *              CTA or of a cluster of up to 16 CTAs keeps it there for all
 *              its iterations (one launch per cluster size, each cluster
 *              taking problems from a queue; cluster barriers and
 *              distributed shared memory for the column sums);
 *   streaming  the others are grouped into size classes served by teams of
 *              CTAs (a power of two, more CTAs for larger problems) in one
 *              persistent cooperative launch; inside a team each CTA owns a
 *              contiguous block of rows for all iterations (its row
 *              scalings stay in shared memory), and the team meets at a
 *              bounded software barrier once per iteration.  Both engines
 *              keep the plan in kernel form during the iterations (K read,
 *              FP32 scalings updated) and write diag(U) K diag(V) at the end.
 */
typedef struct uot_problem {
  void* plan;        /* device, n x m FP32, row-major; 16-byte aligned, ldp % 4 == 0 */
  int64_t ldp;       /* leading dimension (elements) */
  int64_t n, m;      /* 1 <= m <= 4096 */
  const float* a;    /* device, length n */
  const float* b;    /* device, length m */
  float reg, reg_m;  /* fi = reg_m / (reg_m + reg); reg_m = +INFINITY gives fi = 1 */
  int32_t iters;     /* iterations for this problem (>= 0) */
  int32_t rule;      /* uot_rule of this problem */
} uot_problem;

/* Schedule knobs (uot_batch_default_tuning fills the defaults):
 *   stages        ring depth per streaming CTA (2..6 slots of 32 KB);
 *   max_team      largest streaming team size (a power of two);
 *   target_elems  element-iterations per CTA used to size the teams: a
 *                 problem of N*M*(iters+1) element-iterations gets the
 *                 smallest power-of-two team with team * target >= work;
 *   resident_max_cluster
 *                 largest cluster for on-chip solves (0, 1, 2, 4, 8 or 16;
 *                 0 sends every problem to the streaming engine).  A problem
 *                 goes on chip with the smallest cluster that holds it;
 *   reserved      must be 0. */
typedef struct uot_batch_tuning {
  int32_t stages;
  int32_t max_team;
  double target_elems;
  int32_t resident_max_cluster;
  int32_t reserved[3];
} uot_batch_tuning;

void uot_batch_default_tuning(uot_batch_tuning* t);

/* Workspace bytes for a batch (0 on bad sizes). */
size_t uot_batched_workspace_size(const uot_problem* probs, int32_t nprob,
                                  const uot_options* opt);

/* Validates the host array `probs`, builds the schedule and uploads it, with
 * the per-problem descriptors, into the caller-owned device workspace
 * (synchronises `stream` once).  Call again whenever a problem changes. */
uot_status uot_batched_prepare(const uot_problem* probs, int32_t nprob, const uot_options* opt,
                               const uot_batch_tuning* tuning, void* workspace,
                               size_t ws_bytes, void* stream);

/* Runs every prepared problem: one reset launch, one launch per on-chip
 * cluster size in use and one persistent streaming launch (when any problem
 * streams), fully asynchronous (capturable in a CUDA graph once prepared). */
uot_status uot_sinkhorn_batched(void* workspace, void* stream);

/* Where prepare put each problem, for i < min(nprob, prepared count):
 * cluster[i] = the on-chip cluster size (1..16) or 0 for the streaming
 * engine; team[i] = the size of the streaming team class the problem was
 * assigned to (a power of two; its team may later split into smaller teams
 * when the class's queue runs dry) or 0 for an on-chip problem.  Host only;
 * returns the prepared count, or -1 for a workspace that was never prepared.
 * `cluster` and `team` may be NULL. */
int32_t uot_batched_placement(const void* workspace, int32_t nprob, int32_t* cluster,
                              int32_t* team);

/* Synchronises `stream` and copies each problem's result to out[0..nprob). */
uot_status uot_batched_results(const void* workspace, int32_t nprob, uot_result* out,
                               void* stream);

/* Description of fused-pass configuration k (0-based), for tuning tools:
 * writes dtype, threads per CTA, 16-byte vectors per thread per row and the
 * columns one CTA covers.  Returns the number of configurations when k < 0 or
 * k is out of range (then nothing is written). */
int32_t uot_fused_config(int32_t k, int32_t* dtype, int32_t* threads,
                         int32_t* vecs, int32_t* cols_per_cta);

#ifdef __cplusplus
}
#endif
#endif /* UOT_H */
