// Shared between the two batched engines: the per-problem descriptor and the
// on-chip (shared-memory resident) solver's host interface.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "uot_internal.h"

namespace uot {

struct BatchProblem {
  float* plan;
  int64_t ldp;
  int n, m;
  const float* a;
  const float* b;
  float fi;
  int iters;
  int mpad;
  float* c;       // 3 x mpad column sums of U K (ring)
  int* ctr;       // 3 row counters (ring)
  float* U;       // n row scalings
  double* log2k;  // log2 of the fixed-point row factor (gauge; 0 for the POT rule)
  Control* ctl;
  int pot;        // scaling-vector rule: u <- (a / K v)^fi, v <- (b / K^T u)^fi
};

// Resident solver: a problem whose initial plan fits in the shared memory of
// a cluster of `cs` CTAs (cs a power of two up to 16) is solved entirely on
// chip, each CTA holding a block of rows.
constexpr int RESIDENT_MAX_CLUSTER = 16;

// Dynamic shared memory one CTA needs for an n x m problem split over cs CTAs.
size_t resident_smem_need(int64_t n, int64_t m, int cs);
// Largest dynamic shared memory a resident CTA may use on this device.
cudaError_t resident_smem_cap(size_t* cap);
// Clusters of `cs` CTAs with `smem` bytes each that fit on the device at once
// (0 if none).
cudaError_t resident_max_clusters(int cs, size_t smem, int* clusters);
// One launch of `grid` CTAs (clusters of `cs`) that takes the `count`
// problems listed in `order` from the queue `cursor` until it runs dry.
cudaError_t resident_launch(const BatchProblem* probs, const int* order, int count, int* cursor,
                            int cs, int grid, size_t smem, cudaStream_t s);

}  // namespace uot
