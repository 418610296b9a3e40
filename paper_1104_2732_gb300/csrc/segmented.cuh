// Segmented batched selection: kernel arguments and host-side launch helpers.
#pragma once

#include <cstdint>

#include "common.cuh"

namespace gbs {

struct SegArgs {
  const float* x;
  const long long* off;   // [S+1]
  int S;
  const long long* kk;    // [S] ranks or nullptr (medians)
  float* out;             // [S]
  const int* order;       // [S] processing order (largest segments first)
  Ctrl* ctrl;             // w_count: queue head; status
  int maxit;
  float sigma_stats;
  int* seg_passes;        // [S] passes over each segment, or nullptr
};

struct SegLaunch {
  const float* x;
  const long long* off;
  int S;
  const long long* kk;
  float* out;
  int* order;
  Ctrl* ctrl;
  int* seg_passes;
};

int seg_num_variants();
int seg_variant_threads(int v);
int seg_variant_cap(int v);
// Enqueues the schedule kernel and the persistent segmented kernel of `variant`.
gbs_status seg_launch(gbs_ctx* c, const SegLaunch& L, int variant, cudaStream_t stream);

}  // namespace gbs
