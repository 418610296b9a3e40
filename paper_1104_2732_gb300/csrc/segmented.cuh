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
  // trimmed-sum mode (LTS): kk holds h; the kernel also writes
  //   outsum[s] = sum of the h smallest elements and out2[s] = the kk2[s]-th smallest
  //   when that rank lies in the compacted bracket, else flags[s] = 1
  const long long* kk2;
  float* out2;
  double* outsum;
  int* flags;
  long long k_const, k2_const;   // ranks used for every segment when kk / kk2 are null (0: median)
  // per-CTA compaction regions in device memory (CTA g owns zg[g * zg_cap, (g + 1) * zg_cap)) for
  // brackets too large for shared memory; nullptr: shared memory only
  float* zg;
  int zg_cap;
  // bracket-proposal network (float32 parameters) for learned starts of the medians, or nullptr
  const float* W;
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
  const int* mask;        // [S]: only segments with mask[s] != 0 are selected (nullptr: all)
  const long long* kk2;   // trimmed-sum mode (see SegArgs); nullptr otherwise
  float* out2;
  double* outsum;
  int* flags;
  long long k_const, k2_const;
  float* zg = nullptr;            // compaction area shared out among the CTAs (see SegArgs)
  long long zg_elems = 0;
};

// Bytes of the segmented workspace for S segments: the processing order, the pass
// counts and the compaction area.
size_t seg_workspace_bytes(int S);
// Ensures the workspace for S segments and points L.order, L.seg_passes and L.zg into it.
gbs_status seg_attach_workspace(gbs_ctx* c, int S, SegLaunch* L);

int seg_num_variants();
int seg_variant_threads(int v);
int seg_variant_cap(int v);
// Enqueues the schedule kernel and the persistent segmented kernel of `variant`
// (trimmed-sum mode when L.outsum is set).
gbs_status seg_launch(gbs_ctx* c, const SegLaunch& L, int variant, cudaStream_t stream);

}  // namespace gbs
