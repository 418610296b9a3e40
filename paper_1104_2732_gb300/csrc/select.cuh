// Arguments and per-CTA partial records of the persistent selection kernel.
#pragma once

#include <cstdint>

#include "common.cuh"
#include "layout.cuh"

namespace gbs {

enum { kModeSelect = 0, kModeStats = 1, kModeEval = 2 };

// One CTA's share of a fused pass (Algorithm 1, step 1.2).
struct __align__(16) PassPartial {
  unsigned long long c_lt;   // #(x < t)
  unsigned long long c_le;   // #(x <= t)
  unsigned long long c_aux;  // #(x <= a): eval mode and the first cutting-plane pass
  unsigned long long c_aux2; // #(x < b): the first cutting-plane pass
  unsigned long long c_reg;  // elements this CTA compacted
  double S;                  // sum over a < x < t of (t - x), float64 total of float32 partials
};

// One CTA's share of pass 0 (Sec. 3, step 0).
struct __align__(16) StatsPartial {
  unsigned long long n_nan, n_neginf, n_posinf, n_negzero, n_finite;
  unsigned long long c_mn, c_mx;   // multiplicities of the finite min / max (IEEE equality)
  double mn, mx;                   // finite min / max (+inf / -inf if none)
  double sum;                      // sum of the finite elements
  // a proposed bracket (a, b] checked in pass 0
  unsigned long long c_le_a, c_lt_b, c_le_b;   // #(x <= a), #(x < b), #(x <= b)
  unsigned long long c_reg;                    // elements of (a, b] this CTA compacted
  double s_ab;                                 // sum over a < x < b of (b - x)
};

template <typename T>
struct SelArgs {
  const T* x;
  long long n;
  long long k;
  T* out;
  int mode;
  int maxit;
  long long cap;
  double a_eval, t_eval;           // kModeEval
  float sigma_stats;               // power-of-two scale of the pass-0 float32 sums
  Ctrl* ctrl;
  PassPartial* part;               // [2][grid]
  StatsPartial* spart;             // [grid]
  unsigned long long* ghist;       // [kMaxRounds][kBins]
  T* z;                            // compaction area, regions at region_start(g)
  long long z_elems;               // its size in elements
  T* z2;                           // the finish's second-level buffer (16-byte aligned), or nullptr
  long long z2_cap;                // its size in elements
  gbs_run_stats* rs;               // device record of this call
  const double* proposal;          // learned bracket {a, b, valid} for pass 0, or nullptr
  gbs_array_stats* stats_out;      // kModeStats
  gbs_cost_eval* eval_out;         // kModeEval
};

// Launches the persistent kernel (mode: kModeSelect / kModeStats / kModeEval).
gbs_status run_select(gbs_ctx* c, const float* x, long long n, long long k, float* out, int mode, double a,
                      double t, gbs_array_stats* sout, gbs_cost_eval* eout, cudaStream_t stream);
gbs_status run_select(gbs_ctx* c, const double* x, long long n, long long k, double* out, int mode, double a,
                      double t, gbs_array_stats* sout, gbs_cost_eval* eout, cudaStream_t stream);
// Grows the workspace for selections of up to n elements of elem_bytes.
gbs_status reserve_select(gbs_ctx* c, long long n, int elem_bytes);

// Pieces of the float32 launch for callers that bring their own scratch: the size of the
// compaction area, the pass-0 sum scale, CTAs per SM that fit, and the cooperative launch.
long long select_z_elems_f32(long long n, int grid);
float select_stats_sigma_f32(long long n, int grid);
int select_occupancy_f32();
cudaError_t select_launch_f32(const SelArgs<float>& A, int grid, cudaStream_t stream);

}  // namespace gbs
