// Internal layout of a context (not part of the C-ABI).
#pragma once

#include <cstddef>
#include <cuda_runtime.h>

#include "gbselect.h"

namespace gbs {
struct Ctrl;
struct PassPartial;
struct StatsPartial;
}  // namespace gbs

struct gbs_ctx {
  int device = 0;
  int num_sms = 0;
  gbs_config cfg{};
  // one device allocation, carved into the pieces below
  void* ws = nullptr;
  size_t ws_bytes = 0;
  gbs::Ctrl* ctrl = nullptr;
  gbs::PassPartial* part = nullptr;
  gbs::StatsPartial* spart = nullptr;
  unsigned long long* ghist = nullptr;
  gbs_run_stats* rs = nullptr;
  void* aux = nullptr;          // fixed-size area for the other subsystems
  size_t aux_bytes = 1 << 20;
  void* z = nullptr;            // compaction regions (grows with n)
  size_t z_bytes = 0;
  cudaStream_t last_stream = nullptr;
  int last_grid = 0;
  int seg_variant = 0;          // launch variant of the segmented select (autotuned; 0 was fastest on the
                                // 4096-array benchmark batch in every run)
  int last_segments = 0;
  // LMS / LTS: residual matrix and per-candidate arrays
  void* lms_buf = nullptr;
  size_t lms_bytes = 0;
  int lms_off_C = 0;
  long long lms_off_n = 0;
  // fused LMS / LTS: split X and theta, per-candidate state, compaction buffers
  void* fused_buf = nullptr;
  size_t fused_bytes = 0;
  // kNN: padded rows and queries, brackets, compaction buffers, partial sums
  void* knn_buf = nullptr;
  size_t knn_bytes = 0;
  cudaEvent_t knn_ev[2] = {nullptr, nullptr};   // around the fused pass launches
  gbs_knn_stats knn_last{};
  cudaEvent_t lms_ev[4] = {nullptr, nullptr, nullptr, nullptr};   // around the fused LMS passes
  gbs_lms_stats lms_last{};
  // LMS / LTS search: squares of a batch of candidates, C-step state; search arrays
  void* search_buf = nullptr;
  size_t search_bytes = 0;
  void* search_aux = nullptr;
  size_t search_aux_bytes = 0;
  // bracket-proposal network: weights | Adam m | Adam v | gradient | scalars (device)
  float* model = nullptr;
  int model_loaded = 0;
  long long adam_t = 0;
};

// Grows the workspace so that its z area holds at least z_bytes.  Synchronous.
gbs_status gbs_internal_ensure(gbs_ctx* c, size_t z_bytes);
// Frees the resources other subsystems attached to the context.
void gbs_internal_release(gbs_ctx* c);
void gbs_internal_release_lms(gbs_ctx* c);
void gbs_internal_release_fused(gbs_ctx* c);
void gbs_internal_release_model(gbs_ctx* c);
void gbs_internal_release_knn(gbs_ctx* c);
void gbs_internal_release_search(gbs_ctx* c);
