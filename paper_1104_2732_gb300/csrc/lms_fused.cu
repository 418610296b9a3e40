// LMS and LTS objectives (Sec. 5) for many candidates theta_c without writing the
// residual matrix: every pass of the cutting plane (Algorithm 1, Sec. 3) recomputes the
// squared residuals s_ic = (y_i - x_i . theta_c)^2 of all candidates from X and y, which
// stay in L2, and reduces them per candidate in the epilogue of the product.
//
// The product D = Theta X^T (candidates x rows, K = p) runs on the tensor cores as three
// TF32 products of a two-term split of each operand (hi*hi + hi*lo + lo*hi, float32
// accumulation), which recovers float32 accuracy.  A warp owns 16 candidates (its A
// fragments stay in registers for the whole launch) and walks row tiles of 8; each lane
// holds two candidates x two rows of every tile and accumulates that candidate pair's
// counts, cost and sums over all of its rows, so the only cross-lane reduction is one per
// launch.  A CTA (8 warps, 128 candidates) stages 128-row tiles of the split X (stored
// interleaved so that a lane's four B-fragment words are one 16-byte load) and of y in
// shared memory with cp.async, double-buffered.  Rows past the end get y = NaN, so their
// squared residuals satisfy no comparison and need no per-row test.
//
// Passes: statistics (min, max, sum of s per candidate; non-finite count), then one fused
// cost + count pass per iterate, then one pass that compacts each candidate's bracket
// (a_c, b_c] and sums s <= a_c.  Every cost pass also keeps each lane's count #(s <= t) in
// a ring, so the lanes' shares of (a, b] -- and from a prefix each lane's place in the
// candidate's buffer -- are known before the compaction pass: no atomics, deterministic
// order.  A one-thread-per-candidate step kernel between
// passes runs the cutting plane for the pair of ranks (k, h) of LMS and LTS: the bracket
// keeps #(s <= a) < min(k, h) and #(s <= b) >= max(k, h), so the compacted set holds both
// order statistics.  The finish is the segmented select in its trimmed-sum mode over the
// compacted sets; LTS adds the sum below the bracket.  A candidate whose residuals are not
// all finite, whose bracket outgrows its compaction buffer or whose counts disagree is
// recomputed by the materialising batched form.
//
// Sampled start (the default for n >= 65536): each candidate's squares on 8192 evenly
// spread rows give order statistics around both ranks, and the proposed bracket (a, b] is
// compacted straight away in one pass: every lane gets a region of the candidate's buffer
// sized from the sample's share of (a, b] (1.3 times it plus 6 standard deviations), and
// the pass counts #(s <= a), the kept elements and #(s > b) exactly (a NaN square is in none
// of them, so the three add up to n only without one).  When
// the bracket holds both ranks and no lane outgrew its region, the lanes' shares are
// gathered in lane order (each lane's count is kept in the ring) and finished; otherwise
// the candidate goes to the materialising form.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdint>
#include <new>
#include <vector>

#include "api_internal.h"
#include "common.cuh"
#include "elem.cuh"
#include "segmented.cuh"

namespace gbs {
namespace {

constexpr int kFW = 8;                 // warps per CTA
constexpr int kFT = kFW * 32;          // threads per CTA
constexpr int kFCand = 16 * kFW;       // candidates per CTA
constexpr int kFRows = 128;            // rows per staged tile
constexpr long long kFCap = 49152;     // compaction buffer per candidate (elements)
constexpr int kFVariant = 2;           // segmented variant of the finish (1024 threads, 49152 in smem)
constexpr int kRing = 16;              // cost passes whose per-lane counts are kept

enum { kFStats = 0, kFCost = 1, kFWrite = 3 };
enum { kPhIter = 0, kPhDone = 1, kPhCompact = 2, kPhFallback = 3, kPhFinish = 4, kPhDirect = 5 };
constexpr int kSampleRows = 8192;           // rows of the sampled start
constexpr long long kSampleMinN = 65536;    // smaller problems start from the extremes

struct FusedCand {
  float a, b, t;        // bracket (a, b] and the point of the next cost pass
  float sigma;          // cost scale of the next pass
  int fx;               // fraction bits of its fixed-point cost total
  int phase;
  int it, use_bisect, stalled, dfv;
  long long cle_a, clt_b, cle_b;
  double dF;            // Phi(b) - Phi(a) for the lower rank
  float mn;             // smallest s (the result when all s are equal)
  int pa_pass, pb_pass; // cost pass that set a / b (-1: the starting ends)
};

struct FusedTot {
  unsigned long long le, sfix;       // cost pass
  unsigned long long kept, le_a;     // compaction pass: #(a < s <= b), #(s <= a)
  unsigned long long nonfinite;      // statistics pass
  unsigned long long gt_b;           // compaction pass: #(s > b)
  unsigned long long overflow;       // direct compaction pass: lanes whose share outgrew their region
  unsigned int mn, mx;               // statistics pass: bits of min / max (s >= 0)
  double sum;                        // statistics: sum of s; compaction: sum of s <= a
};

struct FusedArgs {
  const float* xi;    // [n][16 KS]: per 8-column block and q = 0..3, (hi q, hi q+4, lo q, lo q+4)
  const float* y;     // [n], 16-byte aligned copy
  long long n;
  const float* th;    // [Cpad][8 KS] hi part of theta
  const float* tl;    // lo part
  int C, ncb, nrc;    // candidates, candidate blocks of kFCand, row chunks
  long long rows_per_item;
  FusedCand* cand;
  FusedTot* tot;
  float* zbuf;        // [C][zstride]
  long long zstride;   // elements of a candidate's compaction buffer
  unsigned int lane_room; // direct compaction: capacity of each lane's region (its offset in loff)
  unsigned int* lring; // [kRing][C][nrc][4]: each lane's #(s <= t) of the last kRing cost passes
  int ring_slot;       // slot this cost pass writes
  unsigned int* loff;  // [C][nrc][4]: where each lane writes its share of (a, b]
};

__device__ __forceinline__ uint32_t to_tf32(float v) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return r;
}
__device__ __forceinline__ void mma_tf32(float* d, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 "
      "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(s), "l"(gmem), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Stores v at addr when p holds, without a branch around the store.
__device__ __forceinline__ void st_global_if(bool p, float* addr, float v) {
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %0, 0;\n\t@q st.global.f32 [%1], %2;\n\t}" ::"r"((unsigned int)p),
               "l"(addr), "f"(v)
               : "memory");
}

// One element of a cost pass: le += [s <= t], S += [a < s <= t] * sigma * (t - s).
__device__ __forceinline__ void core_le(float s, float a, float t, float nsig, float tsig, unsigned& le, float& S) {
  asm("{\n\t"
      ".reg .pred q, r;\n\t"
      ".reg .f32 d;\n\t"
      "setp.le.f32 q, %2, %4;\n\t"
      "setp.gt.and.f32 r, %2, %3, q;\n\t"
      "fma.rn.f32 d, %2, %5, %6;\n\t"
      "@q add.u32 %0, %0, 1;\n\t"
      "@r add.f32 %1, %1, d;\n\t"
      "}"
      : "+r"(le), "+f"(S)
      : "f"(s), "f"(a), "f"(t), "f"(nsig), "f"(tsig));
}

// theta split into TF32 hi/lo (zero padded to 8 KS columns and to Cpad rows).
__global__ void split_rows_kernel(const float* __restrict__ src, long long rows, int p, int p8, float* __restrict__ hi,
                                  float* __restrict__ lo, long long src_rows) {
  const long long total = rows * p8;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long r = i / p8;
    const int j = (int)(i - r * p8);
    const float v = (r < src_rows && j < p) ? src[r * p + j] : 0.f;
    const uint32_t h = to_tf32(v);
    hi[i] = __uint_as_float(h);
    lo[i] = __uint_as_float(to_tf32(v - __uint_as_float(h)));
  }
}

// X split into TF32 hi/lo and interleaved: row r, block ks, lane column q ->
// xi[r][16 ks + 4 q + {0, 1, 2, 3}] = (hi(8ks+q), hi(8ks+q+4), lo(8ks+q), lo(8ks+q+4)).
__global__ void interleave_x_kernel(const float* __restrict__ X, long long n, int p, int KS,
                                    float* __restrict__ xi) {
  const long long total = n * 16 * KS;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long r = i / (16 * KS);
    const int w = (int)(i - r * 16 * KS);
    const int ks = w >> 4, qq = (w >> 2) & 3, e = w & 3;
    const int j = ks * 8 + qq + ((e & 1) ? 4 : 0);
    const float v = j < p ? X[r * p + j] : 0.f;
    const uint32_t h = to_tf32(v);
    xi[i] = (e < 2) ? __uint_as_float(h) : __uint_as_float(to_tf32(v - __uint_as_float(h)));
  }
}

// One work item of a pass: the CTA's 128 candidates over one chunk of rows.
template <int KS, int MODE>
__device__ __forceinline__ void fused_item(const FusedArgs& A, long long item, float (&xs)[2][kFRows * 16 * KS],
                                           float (&ys)[2][kFRows]) {
  constexpr int RW = 16 * KS;                     // floats of one interleaved row
  constexpr int RS = RW;                           // row stride (16-byte loads: conflict-free for KS = 1)

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, q = lane & 3;
  const int cb = (int)(item % A.ncb);
  const int rc = (int)(item / A.ncb);
  const long long r_begin = (long long)rc * A.rows_per_item;
  const long long r_end = min(A.n, r_begin + A.rows_per_item);
  const int c0 = cb * kFCand + warp * 16 + g, c1 = c0 + 8;

  // candidate parameters for this lane's two candidates
  bool act0 = false, act1 = false;
  float pa[2] = {0.f, 0.f}, pt[2] = {0.f, 0.f}, pb[2] = {0.f, 0.f}, nsig[2] = {0.f, 0.f}, tsig[2] = {0.f, 0.f};
  int fx[2] = {kSFixBits, kSFixBits};
  float* zp[2] = {nullptr, nullptr};   // write pass: this lane's slots in the candidate's buffer
  unsigned int room[2] = {0u, 0u};
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const int c = j ? c1 : c0;
    bool act = false;
    if (c < A.C) {
      const FusedCand& fc = A.cand[c];
      if (MODE == kFStats) act = true;
      if (MODE == kFCost) act = fc.phase == kPhIter;
      if (MODE == kFWrite) act = fc.phase == kPhCompact || fc.phase == kPhDirect;
      pa[j] = fc.a; pt[j] = fc.t; pb[j] = fc.b;
      nsig[j] = -fc.sigma; tsig[j] = fc.t * fc.sigma; fx[j] = fc.fx;
      if (MODE == kFWrite && act) {
        const unsigned int base = A.loff[((long long)c * A.nrc + rc) * 4 + q];
        zp[j] = A.zbuf + (long long)c * A.zstride + base;
        room[j] = fc.phase == kPhDirect ? A.lane_room : (unsigned int)(A.zstride - base);
      }
    }
    if (j) act1 = act; else act0 = act;
  }
  const bool warp_active = __any_sync(0xffffffffu, act0 || act1);

  // A fragments (Theta rows of the warp's 16 candidates), hi and lo
  uint32_t ah[KS][4], al[KS][4];
#pragma unroll
  for (int ks = 0; ks < KS; ++ks) {
    const long long r0 = (long long)(cb * kFCand + warp * 16 + g) * (8 * KS) + ks * 8 + q;
    const long long r1 = r0 + 8 * (8 * KS);
    ah[ks][0] = __float_as_uint(A.th[r0]); ah[ks][1] = __float_as_uint(A.th[r1]);
    ah[ks][2] = __float_as_uint(A.th[r0 + 4]); ah[ks][3] = __float_as_uint(A.th[r1 + 4]);
    al[ks][0] = __float_as_uint(A.tl[r0]); al[ks][1] = __float_as_uint(A.tl[r1]);
    al[ks][2] = __float_as_uint(A.tl[r0 + 4]); al[ks][3] = __float_as_uint(A.tl[r1 + 4]);
  }

  // per-lane accumulators for candidates (c0, c1)
  unsigned int le[2] = {0u, 0u}, kept[2] = {0u, 0u}, lea[2] = {0u, 0u}, nf[2] = {0u, 0u};
  float S[2] = {0.f, 0.f}, part[2] = {0.f, 0.f}, comp[2] = {0.f, 0.f};
  float mn[2] = {FLT_MAX, FLT_MAX}, mx[2] = {0.f, 0.f};

  auto stage = [&](int buf, long long r0) {
    constexpr int kChunksRow = RW / 4;
    for (int i = tid; i < kFRows * kChunksRow; i += kFT) {
      const int r = i / kChunksRow, ch = i - r * kChunksRow;
      const long long gr = r0 + r;
      cp_async16(xs[buf] + r * RS + ch * 4, A.xi + (gr < r_end ? gr : r_begin) * RW + ch * 4, gr < r_end ? 16 : 0);
    }
    for (int i = tid; i < kFRows / 4; i += kFT) {
      const long long gr = r0 + 4 * i;
      const long long left = r_end - gr;
      const int bytes = left >= 4 ? 16 : (left > 0 ? (int)left * 4 : 0);
      cp_async16(&ys[buf][4 * i], A.y + (bytes ? gr : r_begin), bytes);
    }
    cp_async_commit();
  };

  const long long ntiles = (r_end - r_begin + kFRows - 1) / kFRows;
  if (ntiles > 0) stage(0, r_begin);
  for (long long it = 0; it < ntiles; ++it) {
    const int buf = (int)(it & 1);
    const long long r0 = r_begin + it * kFRows;
    if (it + 1 < ntiles) {
      stage(buf ^ 1, r0 + kFRows);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    if (tid < kFRows / 4) {   // rows past the end: y = NaN (same thread as the copy of that chunk)
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (r0 + 4 * tid + e >= r_end) ys[buf][4 * tid + e] = __int_as_float(0x7fc00000);
    }
    __syncthreads();
    if (warp_active) {
      const float* xb = xs[buf];
      const bool full = r0 + kFRows <= r_end;     // no row of this stage past the end
      float stage_sum[2] = {0.f, 0.f};            // write pass: at most 32 terms per lane and candidate
      (void)full;
#pragma unroll 2
      for (int rt = 0; rt < kFRows / 8; ++rt) {
        float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int ks = 0; ks < KS; ++ks) {
          const float4 f = *reinterpret_cast<const float4*>(xb + (rt * 8 + g) * RS + ks * 16 + 4 * q);
          const uint32_t bh[2] = {__float_as_uint(f.x), __float_as_uint(f.y)};
          const uint32_t bl[2] = {__float_as_uint(f.z), __float_as_uint(f.w)};
          mma_tf32(d, al[ks], bh);     // small products first
          mma_tf32(d, ah[ks], bl);
          mma_tf32(d, ah[ks], bh);
        }
        const int lr = rt * 8 + 2 * q;
        const float2 yy = *reinterpret_cast<const float2*>(&ys[buf][lr]);
        // d[0] = (c0, row lr), d[1] = (c0, lr + 1), d[2] = (c1, lr), d[3] = (c1, lr + 1)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int j = e >> 1;
          const float r = ((e & 1) ? yy.y : yy.x) - d[e];
          const float s = r * r;            // NaN for rows past the end
          if (MODE == kFStats) {
            const bool valid = full || (r0 + lr + (e & 1)) < r_end;
            const bool ok = valid && (s <= FLT_MAX);   // finite (s >= 0; NaN fails)
            mn[j] = ok ? fminf(mn[j], s) : mn[j];
            mx[j] = ok ? fmaxf(mx[j], s) : mx[j];
            part[j] += ok ? s : 0.f;
            nf[j] += (valid && !ok) ? 1u : 0u;
          } else if (MODE == kFCost) {
            core_le(s, pa[j], pt[j], nsig[j], tsig[j], le[j], S[j]);
          } else {
            // below the bracket: the stage's partial sum; inside: the lane's next slot; above:
            // counted (a NaN square, or a row past the end, fails all three tests)
            const bool above = s > pb[j];
            const bool below = s <= pa[j];
            const bool keep = (s > pa[j]) & !above;
            nf[j] += above ? 1u : 0u;
            stage_sum[j] += below ? s : 0.f;
            lea[j] += below ? 1u : 0u;
            // a predicated store, no branch (room is 0 for inactive lanes)
            st_global_if(keep & (kept[j] < room[j]), zp[j] + kept[j], s);
            kept[j] += keep ? 1u : 0u;
          }
        }
      }
      if (MODE == kFWrite) {   // compensated sum of the stage partials
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const float yk = stage_sum[j] - comp[j];
          const float tk = part[j] + yk;
          comp[j] = (tk - part[j]) - yk;
          part[j] = tk;
        }
      }
    }
    __syncthreads();
  }

  unsigned int ovf = 0;
  if (MODE == kFWrite) {   // each lane's share of (a, b] (the direct route gathers by it)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int c = j ? c1 : c0;
      if (c < A.C && (j ? act1 : act0)) {
        A.lring[(((long long)A.ring_slot * A.C + c) * A.nrc + rc) * 4 + q] = kept[j];
        ovf |= (kept[j] > room[j] ? 1u : 0u) << j;
      }
    }
  }
  if (MODE == kFCost) {           // each lane's own #(s <= t), for the compaction offsets
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int c = j ? c1 : c0;
      if (c < A.C && (j ? act1 : act0))
        A.lring[(((long long)A.ring_slot * A.C + c) * A.nrc + rc) * 4 + q] = le[j];
    }
  }
  double dsum[2];
#pragma unroll
  for (int j = 0; j < 2; ++j) dsum[j] = (double)part[j] - (double)comp[j];
  // the four lanes of a candidate pair (same g) combine, then one lane adds to the totals
#pragma unroll
  for (int o = 1; o <= 2; o <<= 1) {
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      le[j] += __shfl_xor_sync(0xffffffffu, le[j], o);
      lea[j] += __shfl_xor_sync(0xffffffffu, lea[j], o);
      kept[j] += __shfl_xor_sync(0xffffffffu, kept[j], o);
      nf[j] += __shfl_xor_sync(0xffffffffu, nf[j], o);
      if (MODE == kFWrite && j == 0) ovf |= __shfl_xor_sync(0xffffffffu, ovf, o);
      S[j] += __shfl_xor_sync(0xffffffffu, S[j], o);
      mn[j] = fminf(mn[j], __shfl_xor_sync(0xffffffffu, mn[j], o));
      mx[j] = fmaxf(mx[j], __shfl_xor_sync(0xffffffffu, mx[j], o));
      dsum[j] += __shfl_xor_sync(0xffffffffu, dsum[j], o);
    }
  }
  if (q == 0) {
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int c = j ? c1 : c0;
      const bool act = j ? act1 : act0;
      if (c >= A.C || !act) continue;
      FusedTot& T = A.tot[c];
      if (MODE == kFStats) {
        if (nf[j]) atomicAdd(&T.nonfinite, (unsigned long long)nf[j]);
        if (mn[j] <= mx[j]) {
          atomicMin(&T.mn, __float_as_uint(mn[j]));
          atomicMax(&T.mx, __float_as_uint(mx[j]));
        }
        atomicAdd(&T.sum, dsum[j]);
      } else if (MODE == kFCost) {
        if (le[j]) atomicAdd(&T.le, (unsigned long long)le[j]);
        const unsigned long long sf = __double2ull_rn(ldexp((double)S[j], fx[j]));
        if (sf) atomicAdd(&T.sfix, sf);
      } else {
        if (lea[j]) atomicAdd(&T.le_a, (unsigned long long)lea[j]);
        if (kept[j]) atomicAdd(&T.kept, (unsigned long long)kept[j]);
        if (nf[j]) atomicAdd(&T.gt_b, (unsigned long long)nf[j]);
        if ((ovf >> j) & 1u) atomicAdd(&T.overflow, 1ull);
        atomicAdd(&T.sum, dsum[j]);
      }
    }
  }
}

// One pass: a persistent grid walks the work items (candidate block x row chunk).
template <int KS, int MODE>
__global__ void __launch_bounds__(kFT, (MODE == kFWrite && KS == 1) ? 3 : 2) fused_pass_kernel(FusedArgs A) {
  __shared__ __align__(16) float xs[2][kFRows * 16 * KS];
  __shared__ __align__(16) float ys[2][kFRows];
  const long long items = (long long)A.ncb * A.nrc;
  for (long long it = blockIdx.x; it < items; it += gridDim.x) fused_item<KS, MODE>(A, it, xs, ys);
}

struct StepArgs {
  FusedCand* cand;
  FusedTot* tot;
  int C;
  long long n, k_lo, k_hi, cap;
  int maxit;
  long long per_lane;
  int nrc;                  // row chunks
  long long rows_per_item;
  int pass;                 // index of the cost pass just finished (its ring slot: pass % kRing)
  const unsigned int* lring;// [kRing][C][nrc][4] each lane's #(s <= t) of recent cost passes
  unsigned int* loff;       // [C][nrc][4] where each lane writes its share of (a, b]
  unsigned int* counters;   // [0] candidates still iterating, [1] candidates needing the fallback
  // finish preparation
  long long* seg_len;       // [C] compacted elements (0 unless the candidate finishes by the select)
  long long* kk;            // [C] rank of LTS inside the compacted set
  long long* kk2;           // [C] rank of LMS inside the compacted set
  int* mask;                // [C] 1: finished by the segmented select
  double* below;            // [C] sum of s <= a
  long long k_lms, h_lts;
  float* lms_out;
  double* lts_out;
};

__device__ __forceinline__ float inside_f(float v, float a, float b) {
  float t = v;
  if (!(t > a)) t = nextafterf(a, INFINITY);
  if (!(t < b)) t = nextafterf(b, -INFINITY);
  return t;
}

// Next point of an iterating candidate (Algorithm 1, step 1.1 with the safeguards of the
// single-array kernel), or the move to compaction.
__device__ void fused_next(FusedCand& s, const StepArgs& P) {
  const long long pop = s.cle_b - s.cle_a;
  if (pop <= P.cap || s.it >= P.maxit || s.stalled >= 2) {
    s.phase = kPhCompact;
    return;
  }
  float t;
  if (s.use_bisect || !s.dfv) {
    const uint32_t ka = ukey(s.a), kb = ukey(s.b);
    t = inside_f(ukey_value(ka + (kb - ka) / 2, 0.f), s.a, s.b);
  } else {
    const double gL = (double)(s.cle_a - P.k_lo) + 0.5, gR = (double)(s.clt_b - P.k_lo) + 0.5;
    const double w = (double)s.b - (double)s.a;
    t = inside_f((float)((double)s.a + (gR * w - s.dF) / (gR - gL)), s.a, s.b);
  }
  s.t = t;
  const double width = (double)t - (double)s.a;
  s.sigma = cost_scale(width, P.per_lane);
  s.fx = cost_fix_bits(width, P.per_lane, s.sigma);
}

template <int MODE>
__global__ void fused_step_kernel(StepArgs P) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= P.C) return;
  FusedCand s = P.cand[c];
  FusedTot& T = P.tot[c];
  if (MODE == kFStats) {
    // starting bracket (a0, M] with a0 the float below min s (Sec. 3, step 0; exact counts)
    s.it = 0; s.use_bisect = 0; s.stalled = 0; s.dfv = 1;
    const float m = __uint_as_float(T.mn), M = __uint_as_float(T.mx);
    s.mn = m;
    s.a = s.b = s.t = 0.f; s.sigma = 1.f; s.fx = kSFixBits;
    s.cle_a = s.clt_b = s.cle_b = 0; s.dF = 0.0; s.pa_pass = s.pb_pass = -1;
    if (T.nonfinite > 0 || !(m <= M)) {
      s.phase = kPhFallback;
    } else if (!(m < M)) {
      s.phase = kPhDone;    // every residual equal
    } else {
      s.phase = kPhIter;
      s.a = nextafterf(m, -INFINITY);
      s.b = M;
      s.cle_a = 0; s.cle_b = P.n; s.clt_b = P.n - 1;
      const double gL = (double)(0 - P.k_lo) + 0.5;
      s.dF = gL * ((double)M - (double)s.a) + (double)P.n * (double)M - T.sum;
      fused_next(s, P);
    }
  } else if (MODE == kFCost) {
    if (s.phase == kPhIter) {
      const long long cle = (long long)T.le;   // #(s < t) is not counted: #(s <= t) stands for it
      const double S = ldexp((double)T.sfix, -s.fx) / (double)s.sigma;
      const double gL = (double)(s.cle_a - P.k_lo) + 0.5;
      const double dphi = gL * ((double)s.t - (double)s.a) + S;
      const long long pop = s.cle_b - s.cle_a;
      s.it++;
      if (cle < P.k_lo) {                 // step 1.4: both ranks above t
        s.a = s.t; s.cle_a = cle; s.dF = s.dF - dphi; s.pa_pass = P.pass;
      } else if (cle >= P.k_hi) {         // both ranks at or below t
        s.b = s.t; s.clt_b = cle; s.cle_b = cle; s.dF = dphi; s.dfv = 1; s.pb_pass = P.pass;
      } else {                            // t separates the ranks: (a, b] holds both
        s.phase = kPhCompact;
      }
      if (s.phase == kPhIter) {
        const long long npop = s.cle_b - s.cle_a;
        const int prev = s.use_bisect;
        s.use_bisect = (!prev) && ((double)npop > 0.75 * (double)pop);
        s.stalled = ((double)npop > 0.875 * (double)pop) ? s.stalled + 1 : 0;
        fused_next(s, P);
      }
    }
  } else {   // after the write pass: check, and prepare the segmented finish
    int fin = 0;
    if (s.phase == kPhDirect) {
      // one pass counted #(s <= a), #(s > b), compacted (a, b] into the lanes' regions and
      // summed s <= a: the bracket holds both ranks, no square is NaN (each row fell in one
      // of the three ranges; an infinite square above b affects neither objective), no
      // lane's share outgrew its region and the set fits the finish's shared memory (kFCap,
      // as for the start from the extremes), or the candidate goes to the fallback
      const long long la = (long long)T.le_a, kept = (long long)T.kept;
      const bool all_rows = la + kept + (long long)T.gt_b == P.n;
      if (all_rows && T.overflow == 0 && la < P.k_lo && P.k_hi <= la + kept && kept <= kFCap) {
        s.phase = kPhFinish;
        s.cle_a = la; s.cle_b = la + kept; s.clt_b = s.cle_b;
        fin = 1;
        P.seg_len[c] = kept;
        P.kk[c] = P.h_lts - la;
        P.kk2[c] = P.k_lms - la;
        P.below[c] = T.sum;
      } else {
        s.phase = kPhFallback;
      }
    } else if (s.phase == kPhCompact) {
      const long long kept = (long long)T.kept;
      if ((long long)T.le_a != s.cle_a || kept != s.cle_b - s.cle_a) {
        s.phase = kPhFallback;
      } else {
        s.phase = kPhFinish;
        fin = 1;
        P.seg_len[c] = kept;
        P.kk[c] = P.h_lts - s.cle_a;
        P.kk2[c] = P.k_lms - s.cle_a;
        P.below[c] = T.sum;
      }
    }
    if (!fin) P.seg_len[c] = 0;
    P.mask[c] = fin;
    if (s.phase == kPhDone) {
      P.lms_out[c] = s.mn;
      P.lts_out[c] = (double)P.h_lts * (double)s.mn;
    }
    if (s.phase == kPhFallback) atomicAdd(&P.counters[1], 1u);
  }
  if (s.phase == kPhIter) atomicAdd(&P.counters[0], 1u);
  P.cand[c] = s;
  // totals start from zero for the next pass (min starts at +inf bits)
  T.le = T.sfix = T.kept = T.le_a = T.nonfinite = T.gt_b = T.overflow = 0ull;
  T.mn = 0x7F7FFFFFu; T.mx = 0u; T.sum = 0.0;
}

// Each compacting candidate's lanes: their share of (a, b] from the ring counts of the
// passes that set a and b (#(s <= a0) = 0; #(s <= M) = all of the lane's rows), and from
// an exclusive prefix (row-chunk major) each lane's place.  One warp per candidate.  A
// candidate whose ends were set too long ago, or whose shares do not add up to its
// bracket population, moves to the fallback.
__global__ void fused_offsets_ring_kernel(StepArgs P) {
  const int warp = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (warp >= P.C) return;
  FusedCand& s = P.cand[warp];
  if (s.phase != kPhCompact) return;
  const bool stale = (s.pa_pass >= 0 && P.pass - s.pa_pass >= kRing) || (s.pb_pass >= 0 && P.pass - s.pb_pass >= kRing);
  if (stale) {
    if (lane == 0) s.phase = kPhFallback;
    return;
  }
  const long long entries = (long long)P.nrc * 4;
  const unsigned int* ra = s.pa_pass >= 0 ? P.lring + ((long long)(s.pa_pass % kRing) * P.C + warp) * entries : nullptr;
  const unsigned int* rb = s.pb_pass >= 0 ? P.lring + ((long long)(s.pb_pass % kRing) * P.C + warp) * entries : nullptr;
  unsigned int* off = P.loff + (long long)warp * entries;
  unsigned long long run = 0;
  for (long long i0 = 0; i0 < entries; i0 += 32) {
    const long long i = i0 + lane;
    unsigned int v = 0;
    if (i < entries) {
      const long long rc = i >> 2;
      const int q = (int)(i & 3);
      unsigned int lb;
      if (rb) {
        lb = rb[i];
      } else {                       // b = M: every row of the lane
        const long long r0 = rc * P.rows_per_item;
        const long long len = min(P.n, r0 + P.rows_per_item) - r0;
        const long long rem = len & 7;
        lb = (unsigned int)(2 * (len >> 3) + min(2ll, max(0ll, rem - 2 * q)));
      }
      const unsigned int la = ra ? ra[i] : 0u;
      v = lb - la;
    }
    unsigned int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (i < entries) off[i] = (unsigned int)min(run + incl - v, (unsigned long long)kFCap);
    run += __shfl_sync(0xffffffffu, incl, 31);
  }
  if (lane == 0 && ((long long)run != s.cle_b - s.cle_a || (long long)run > kFCap || run < 1ull ||
                    P.k_lo - s.cle_a < 1 || P.k_hi - s.cle_a > (long long)run))
    s.phase = kPhFallback;
}

__global__ void fused_init_kernel(FusedTot* tot, int C, unsigned int* counters) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < C) {
    FusedTot& T = tot[c];
    T.le = T.sfix = T.kept = T.le_a = T.nonfinite = T.gt_b = T.overflow = 0ull;
    T.mn = 0x7F7FFFFFu; T.mx = 0u; T.sum = 0.0;
  }
  if (c == 0) counters[0] = counters[1] = 0u;
}

// Exclusive prefix of the compacted lengths into segment offsets (one CTA).
__global__ void __launch_bounds__(1024) fused_offsets_kernel(const long long* len, int C, long long* off) {
  __shared__ long long part[1024];
  const int tid = threadIdx.x;
  const int per = (C + 1023) / 1024;
  long long s = 0;
  for (int i = 0; i < per; ++i) {
    const int c = tid * per + i;
    if (c < C) s += len[c];
  }
  part[tid] = s;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const long long v = tid >= o ? part[tid - o] : 0;
    __syncthreads();
    part[tid] += v;
    __syncthreads();
  }
  long long base = tid ? part[tid - 1] : 0;
  for (int i = 0; i < per; ++i) {
    const int c = tid * per + i;
    if (c < C) {
      off[c] = base;
      base += len[c];
    }
  }
  if (tid == 1023) off[C] = part[1023];
}

// Copies each finishing candidate's compacted elements to its segment.
__global__ void fused_gather_kernel(const float* __restrict__ zbuf, long long zstride, const long long* __restrict__ off,
                                    int C, float* __restrict__ zcat) {
  const int c = blockIdx.x;
  if (c >= C) return;
  const long long o = off[c], len = off[c + 1] - o;
  const float* src = zbuf + (long long)c * zstride;
  for (long long i = threadIdx.x; i < len; i += blockDim.x) zcat[o + i] = src[i];
}

// The direct route's gather: candidate c's share of lane l (count cnt[l], from the ring
// slot of the direct pass) sits at zbuf[c * zstride + l * room]; the shares go to zcat
// from off[c] in lane order.  One CTA of 8 warps per candidate: warp w takes a contiguous
// range of lanes, starts after the earlier warps' totals, and walks its lanes 32 at a time
// (a warp scan gives each share's place), copying each share with consecutive accesses.
__global__ void __launch_bounds__(256) fused_gather_lanes_kernel(const float* __restrict__ zbuf, long long zstride,
                                                                 const unsigned int* __restrict__ cnt_all, int nl,
                                                                 unsigned int room, const long long* __restrict__ off,
                                                                 int C, float* __restrict__ zcat) {
  __shared__ unsigned int s_w[8];
  const int c = blockIdx.x;
  if (c >= C) return;
  const long long o = off[c], len = off[c + 1] - o;
  if (len == 0) return;
  const unsigned int* cnt = cnt_all + (long long)c * nl;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int wper = (nl + 7) / 8;
  const int wl0 = min(nl, warp * wper), wl1 = min(nl, wl0 + wper);
  unsigned int t = 0;
  for (int l = wl0 + lane; l < wl1; l += 32) t += min(cnt[l], room);
  t = __reduce_add_sync(0xffffffffu, t);
  if (lane == 0) s_w[warp] = t;
  __syncthreads();
  unsigned long long base = (unsigned long long)o;
  for (int w = 0; w < warp; ++w) base += s_w[w];
  const float* src = zbuf + (long long)c * zstride;
  for (int g0 = wl0; g0 < wl1; g0 += 32) {
    const int l = g0 + lane;
    const unsigned int m = l < wl1 ? min(cnt[l], room) : 0u;
    unsigned int incl = m;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const unsigned int v = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += v;
    }
    const unsigned int excl = incl - m;
    const int nj = min(32, wl1 - g0);
    for (int j = 0; j < nj; ++j) {
      const unsigned int mj = __shfl_sync(0xffffffffu, m, j), ej = __shfl_sync(0xffffffffu, excl, j);
      const float* sl = src + (long long)(g0 + j) * room;
      for (unsigned int i = lane; i < mj; i += 32) zcat[base + ej + i] = sl[i];
    }
    base += __shfl_sync(0xffffffffu, incl, 31);
  }
}

// Lane regions of the direct route: lane (rc, q) of candidate c writes from (rc * 4 + q) * room.
__global__ void fused_direct_offsets_kernel(unsigned int* loff, int C, int nl, unsigned int room) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < (long long)C * nl) loff[i] = (unsigned int)(i % nl) * room;
}

// LTS of finishing candidates: the trimmed sum inside the bracket plus the sum below it.
__global__ void fused_combine_kernel(const int* mask, const double* below, int C, double* lts_out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < C && mask[c]) lts_out[c] += below[c];
}

__global__ void fused_fallback_list_kernel(const FusedCand* cand, int C, int* list, unsigned int* count) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < C && cand[c].phase == kPhFallback) list[atomicAdd(count, 1u)] = c;
}
__global__ void fused_gather_theta_kernel(const float* theta, int p, const int* list, int m, float* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m * p) out[i] = theta[(long long)list[i / p] * p + (i % p)];
}
__global__ void fused_scatter_kernel(const int* list, int m, const float* lms, const double* lts, float* lms_out,
                                     double* lts_out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) {
    lms_out[list[i]] = lms[i];
    lts_out[list[i]] = lts[i];
  }
}

// Persistent grid of one pass: every CTA of that pass's kernel that fits at once.
template <int KS, int MODE>
gbs_status launch_mode(const FusedArgs& A, int num_sms, cudaStream_t s) {
  static int occ[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  int& o = occ[dev & 63];
  if (o == 0) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, fused_pass_kernel<KS, MODE>, kFT, 0) != cudaSuccess ||
        o < 1) {
      cudaGetLastError();
      o = 1;
    }
  }
  const long long items = (long long)A.ncb * A.nrc;
  const unsigned int grid = (unsigned int)std::min<long long>(items, (long long)num_sms * o);
  fused_pass_kernel<KS, MODE><<<grid, kFT, 0, s>>>(A);
  return cudaGetLastError() == cudaSuccess ? GBS_OK : GBS_ECUDA;
}

template <int KS>
gbs_status launch_pass(int mode, const FusedArgs& A, int num_sms, cudaStream_t s) {
  if (mode == kFStats) return launch_mode<KS, kFStats>(A, num_sms, s);
  if (mode == kFCost) return launch_mode<KS, kFCost>(A, num_sms, s);
  return launch_mode<KS, kFWrite>(A, num_sms, s);
}

// The ns sampled rows (row (j * n) / ns of X and y), gathered into xs [ns][p] and ys [ns].
__global__ void lms_sample_rows_kernel(const float* __restrict__ X, const float* __restrict__ y, long long n, int p,
                                       int ns, float* __restrict__ xs, float* __restrict__ ys) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)ns * (p + 1)) return;
  const int j = (int)(idx / (p + 1)), q = (int)(idx - (long long)j * (p + 1));
  const long long i = (long long)j * n / ns;
  if (q < p) xs[(long long)j * p + q] = X[i * p + q];
  else ys[j] = y[i];
}

// Squared residuals of every candidate on the sampled rows, candidate-major; a non-finite
// square is stored as +inf.  float32 FMAs: the sample only proposes brackets, which the
// check pass then counts on the fused pass's own residuals.
__global__ void lms_sample_kernel(const float* __restrict__ xs, const float* __restrict__ ys, int p,
                                  const float* __restrict__ theta, int C, int ns, float* __restrict__ out) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)C * ns) return;
  const int c = (int)(idx / ns), j = (int)(idx - (long long)c * ns);
  float d = 0.f;
  for (int q = 0; q < p; ++q) d = fmaf(xs[(long long)j * p + q], theta[(long long)c * p + q], d);
  const float r = ys[j] - d;
  const float sq = r * r;
  out[idx] = sq <= FLT_MAX ? sq : INFINITY;
}

__global__ void lms_sample_offsets_kernel(long long* off, int C, int ns) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c <= C) off[c] = (long long)c * ns;
}

// The proposed brackets (lo[c], hi[c]] from the sample's order statistics (a rank below
// the sample: -1, below every square; above it: FLT_MAX); a bracket that is not a finite
// a < b sends its candidate to the fallback.
__global__ void lms_propose_kernel(FusedCand* cand, int C, const float* lo, const float* hi, int lo_in, int hi_in) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  FusedCand s;
  s.a = lo_in ? lo[c] : -1.f;
  s.b = hi_in ? hi[c] : FLT_MAX;
  s.t = 0.f; s.sigma = 1.f; s.fx = kSFixBits;
  s.it = 0; s.use_bisect = 0; s.stalled = 0; s.dfv = 0;
  s.cle_a = s.clt_b = s.cle_b = 0; s.dF = 0.0; s.mn = 0.f; s.pa_pass = s.pb_pass = -1;
  s.phase = (s.a < s.b && s.b <= FLT_MAX) ? kPhDirect : kPhFallback;
  cand[c] = s;
}

size_t up256f(size_t v) { return (v + 255) / 256 * 256; }

}  // namespace
}  // namespace gbs

void gbs_internal_release_fused(gbs_ctx* c) {
  if (c->fused_buf) {
    cudaDeviceSynchronize();
    cudaFree(c->fused_buf);
    c->fused_buf = nullptr;
    c->fused_bytes = 0;
  }
}

extern "C" gbs_status gbs_lms_lts_fused_f32(gbs_ctx* c, const float* X, const float* y, int64_t n, int32_t p,
                                           const float* theta, int32_t C, int64_t k_lms, int64_t h_lts,
                                           float* lms_out, double* lts_out, int32_t* passes, void* stream) {
  using namespace gbs;
  if (!c || !X || !y || !theta || !lms_out || !lts_out) return GBS_EINVAL;
  if (n < 1 || n > (1ll << 31) || p < 1 || p > 16 || C < 1) return GBS_EINVAL;
  if (k_lms < 1 || k_lms > n || h_lts < 1 || h_lts > n) return GBS_EINVAL;
  DeviceGuard g(c->device);
  if (!g.ok) return GBS_ECUDA;
  cudaStream_t strm = static_cast<cudaStream_t>(stream);
  const int KS = p <= 8 ? 1 : 2, P8 = 8 * KS;
  const int ncb = (C + kFCand - 1) / kFCand, Cpad = ncb * kFCand;
  // persistent grid: every resident CTA; work items (candidate blocks x row chunks) about
  // eight per CTA, so that the last round of items is a small share of the pass
  int occ = 0;
  if ((KS == 1 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fused_pass_kernel<1, kFCost>, kFT, 0)
               : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fused_pass_kernel<2, kFCost>, kFT, 0)) !=
          cudaSuccess ||
      occ < 1) {
    cudaGetLastError();
    occ = 1;
  }
  const long long resident = (long long)c->num_sms * occ;
  const long long target = resident * 8;
  long long nrc = std::max<long long>(1, (target + ncb - 1) / ncb);
  long long rpi = (n + nrc - 1) / nrc;
  rpi = (rpi + kFRows - 1) / kFRows * kFRows;
  nrc = (n + rpi - 1) / rpi;
  // sampled start: the sample's ranks around k and h (3.5 binomial standard deviations and
  // 2 ranks of margin on each side: at the medians of 1e6 rows the bracket holds about
  // 3.9 % of them and a side misses with probability ~2e-4), and the direct route's lane
  // regions: each lane (2 of every 8 rows of its items) gets room for 1.3 times the
  // sample's share of its rows plus 6 standard deviations
  const int ns = kSampleRows;
  bool sampled = false;
  long long jl = 0, jh = 0, zstride = kFCap;
  unsigned int lane_room = 0;
  const long long nl = nrc * 4;
  if (c->cfg.lms_start == 0 && n >= kSampleMinN) {
    const double pl = (double)std::min(k_lms, h_lts) / (double)n, ph = (double)std::max(k_lms, h_lts) / (double)n;
    jl = (long long)std::floor(ns * pl - 3.5 * std::sqrt(ns * pl * (1.0 - pl))) - 2;
    jh = (long long)std::ceil(ns * ph + 3.5 * std::sqrt(ns * ph * (1.0 - ph))) + 2;
    const double f = (double)(std::min<long long>(jh, ns) - std::max<long long>(jl, 1) + 1) / ns;
    // the expected bracket must fit the finish's shared memory (ranks far apart take the
    // start from the extremes, which sends such candidates to the materialising form)
    const bool fits = f * (double)n <= 0.9 * (double)kFCap;
    const double lane_rows = (double)rpi / 4.0;
    const double mean = lane_rows * std::min(1.0, f * 1.3);
    long long R = (long long)std::ceil(mean + 6.0 * std::sqrt(mean) + 8.0);
    R = std::min<long long>((R + 3) / 4 * 4, (long long)lane_rows);
    const long long zs = std::max<long long>(kFCap, nl * R);
    if (fits && (double)C * (double)zs * 8.0 <= 4.0 * 1073741824.0) {   // zbuf + zcat within 4 GiB
      sampled = true;
      zstride = zs;
      lane_room = (unsigned int)R;
    }
  }
  // workspace: xi | th | tl | cand | tot | counters | seg_len | kk | kk2 | mask | below | off |
  //            list | zbuf | zcat
  size_t o = 0;
  const size_t o_xi = o; o = up256f(o + sizeof(float) * (size_t)n * 2 * P8);
  const size_t o_th = o; o = up256f(o + sizeof(float) * (size_t)Cpad * P8);
  const size_t o_tl = o; o = up256f(o + sizeof(float) * (size_t)Cpad * P8);
  const size_t o_cand = o; o = up256f(o + sizeof(FusedCand) * (size_t)C);
  const size_t o_tot = o; o = up256f(o + sizeof(FusedTot) * (size_t)C);
  const size_t o_cnt = o; o = up256f(o + sizeof(unsigned int) * 4);
  const size_t o_len = o; o = up256f(o + sizeof(long long) * (size_t)C);
  const size_t o_kk = o; o = up256f(o + sizeof(long long) * (size_t)C);
  const size_t o_kk2 = o; o = up256f(o + sizeof(long long) * (size_t)C);
  const size_t o_mask = o; o = up256f(o + sizeof(int) * (size_t)C);
  const size_t o_below = o; o = up256f(o + sizeof(double) * (size_t)C);
  const size_t o_off = o; o = up256f(o + sizeof(long long) * (size_t)(C + 1));
  const size_t o_list = o; o = up256f(o + sizeof(int) * (size_t)C);
  const size_t o_q = o; o = up256f(o + sizeof(float) * (size_t)C);
  const size_t o_flags = o; o = up256f(o + sizeof(int) * (size_t)C);
  const size_t o_plo = o; o = up256f(o + sizeof(float) * (size_t)C);   // sampled start: proposed ends
  const size_t o_phi = o; o = up256f(o + sizeof(float) * (size_t)C);
  const size_t o_srow = o; o = up256f(o + sizeof(float) * (size_t)kSampleRows * (p + 1));   // sampled rows
  const size_t o_z = o; o = up256f(o + sizeof(float) * (size_t)C * zstride);
  const size_t o_zc = o; o = up256f(o + sizeof(float) * (size_t)C * zstride);
  const size_t o_y = o; o = up256f(o + sizeof(float) * (size_t)n);
  const size_t o_ring = o; o = up256f(o + sizeof(unsigned int) * (size_t)kRing * C * nrc * 4);
  const size_t o_loff = o; o = up256f(o + sizeof(unsigned int) * (size_t)C * nrc * 4);
  const size_t bytes = o;
  if (!c->fused_buf || c->fused_bytes < bytes) {
    gbs_internal_release_fused(c);
    void* ptr = nullptr;
    if (cudaMalloc(&ptr, bytes) != cudaSuccess) {
      cudaGetLastError();
      return GBS_ENOMEM;
    }
    c->fused_buf = ptr;
    c->fused_bytes = bytes;
  }
  gbs_status st = gbs_internal_ensure(c, seg_workspace_bytes(C));
  if (st != GBS_OK) return st;
  char* b = static_cast<char*>(c->fused_buf);
  FusedArgs A;
  A.xi = reinterpret_cast<float*>(b + o_xi);
  A.y = reinterpret_cast<float*>(b + o_y);   // 16-byte aligned copy for cp.async
  A.n = n;
  A.th = reinterpret_cast<float*>(b + o_th);
  A.tl = reinterpret_cast<float*>(b + o_tl);
  A.C = C;
  A.ncb = ncb;
  A.cand = reinterpret_cast<FusedCand*>(b + o_cand);
  A.tot = reinterpret_cast<FusedTot*>(b + o_tot);
  A.zbuf = reinterpret_cast<float*>(b + o_z);
  A.zstride = zstride;
  A.lane_room = 0;
  A.rows_per_item = rpi;
  A.nrc = (int)nrc;
  A.lring = reinterpret_cast<unsigned int*>(b + o_ring);
  A.ring_slot = 0;
  A.loff = reinterpret_cast<unsigned int*>(b + o_loff);
  if (nrc < 1 || nrc * ncb > 0x7fffffffll) return GBS_EINVAL;

  StepArgs P;
  P.cand = A.cand; P.tot = A.tot; P.C = C; P.n = n;
  P.k_lo = std::min(k_lms, h_lts); P.k_hi = std::max(k_lms, h_lts);
  P.cap = std::min<long long>(kFCap, std::max<long long>(n / 16, 4096));
  P.maxit = 64;
  P.per_lane = rpi;
  P.nrc = (int)nrc;
  P.lring = A.lring;
  P.rows_per_item = rpi;
  P.pass = -1;
  P.loff = A.loff;
  P.counters = reinterpret_cast<unsigned int*>(b + o_cnt);
  P.seg_len = reinterpret_cast<long long*>(b + o_len);
  P.kk = reinterpret_cast<long long*>(b + o_kk);
  P.kk2 = reinterpret_cast<long long*>(b + o_kk2);
  P.mask = reinterpret_cast<int*>(b + o_mask);
  P.below = reinterpret_cast<double*>(b + o_below);
  P.k_lms = k_lms; P.h_lts = h_lts;
  P.lms_out = lms_out; P.lts_out = lts_out;
  long long* off = reinterpret_cast<long long*>(b + o_off);
  int* list = reinterpret_cast<int*>(b + o_list);
  float* qbuf = reinterpret_cast<float*>(b + o_q);
  int* flags = reinterpret_cast<int*>(b + o_flags);
  float* zcat = reinterpret_cast<float*>(b + o_zc);

  const unsigned int sgrid = (unsigned int)((C + 255) / 256);
  auto check = [&]() { return cudaGetLastError() == cudaSuccess ? GBS_OK : GBS_ECUDA; };
  if (cudaMemcpyAsync(const_cast<float*>(A.y), y, sizeof(float) * (size_t)n, cudaMemcpyDeviceToDevice, strm) !=
      cudaSuccess)
    return GBS_ECUDA;
  // split X and theta
  interleave_x_kernel<<<std::min<long long>((n * 2 * P8 + 255) / 256, (long long)c->num_sms * 16), 256, 0, strm>>>(
      X, n, p, KS, const_cast<float*>(A.xi));
  split_rows_kernel<<<std::max(1, std::min((Cpad * P8 + 255) / 256, c->num_sms * 16)), 256, 0, strm>>>(
      theta, Cpad, p, P8, const_cast<float*>(A.th), const_cast<float*>(A.tl), C);
  fused_init_kernel<<<sgrid, 256, 0, strm>>>(A.tot, C, P.counters);
  if ((st = check()) != GBS_OK) return st;
  // the passes' device time: events 0/1 around a statistics or cost pass (read after the
  // synchronisation that follows it), 2/3 around the compaction pass (read at the end)
  for (int e = 0; e < 4; ++e)
    if (!c->lms_ev[e] && cudaEventCreate(&c->lms_ev[e]) != cudaSuccess) return GBS_ECUDA;
  c->lms_last = gbs_lms_stats{};
  bool timed_open = false;
  auto read_timed = [&]() {
    float ms = 0.f;
    if (timed_open && cudaEventElapsedTime(&ms, c->lms_ev[0], c->lms_ev[1]) == cudaSuccess) c->lms_last.pass_ms += ms;
    timed_open = false;
  };
  auto pass = [&](int mode) {
    const int w = mode == kFWrite ? 2 : 0;
    if (cudaEventRecord(c->lms_ev[w], strm) != cudaSuccess) return GBS_ECUDA;
    const gbs_status r =
        KS == 1 ? launch_pass<1>(mode, A, c->num_sms, strm) : launch_pass<2>(mode, A, c->num_sms, strm);
    if (r != GBS_OK) return r;
    if (cudaEventRecord(c->lms_ev[w + 1], strm) != cudaSuccess) return GBS_ECUDA;
    if (mode != kFWrite) timed_open = true;
    c->lms_last.pass_launches += 1;
    return GBS_OK;
  };
  int npass = 0;
  unsigned int h_cnt[2] = {0u, 0u};
  if (sampled) {
    // sampled start: order statistics of the candidates' squares on ns sampled rows
    // propose (a, b] around both ranks; one direct pass counts #(s <= a) and the elements
    // of (a, b] exactly while compacting them into the lanes' regions and summing s <= a
    const int lo_in = jl >= 1, hi_in = jh <= ns;
    float* plo = reinterpret_cast<float*>(b + o_plo);
    float* phi = reinterpret_cast<float*>(b + o_phi);
    float* rs = zcat;   // C x ns squares (the finish's buffer, free until the gather)
    float* sx = reinterpret_cast<float*>(b + o_srow);
    float* sy = sx + (size_t)ns * p;
    lms_sample_rows_kernel<<<(unsigned int)(((long long)ns * (p + 1) + 255) / 256), 256, 0, strm>>>(X, y, n, p, ns,
                                                                                                  sx, sy);
    lms_sample_kernel<<<(unsigned int)(((long long)C * ns + 255) / 256), 256, 0, strm>>>(sx, sy, p, theta, C, ns, rs);
    lms_sample_offsets_kernel<<<(unsigned int)((C + 1 + 255) / 256), 256, 0, strm>>>(off, C, ns);
    if ((st = check()) != GBS_OK) return st;
    // both order statistics from one load of each candidate's sample: the segmented
    // select's two-rank mode (its trimmed sums and flags land in buffers the finish fills
    // later)
    SegLaunch Ls;
    if ((st = seg_attach_workspace(c, C, &Ls)) != GBS_OK) return st;
    Ls.x = rs; Ls.off = off; Ls.S = C; Ls.kk = nullptr; Ls.ctrl = c->ctrl; Ls.mask = nullptr; Ls.kk2 = nullptr;
    Ls.k_const = std::max<long long>(jl, 1); Ls.out = plo;
    Ls.k2_const = std::min<long long>(jh, ns); Ls.out2 = phi;
    Ls.outsum = P.below; Ls.flags = flags;
    if ((st = seg_launch(c, Ls, 0, strm)) != GBS_OK) return st;
    lms_propose_kernel<<<sgrid, 256, 0, strm>>>(A.cand, C, plo, phi, lo_in, hi_in);
    fused_direct_offsets_kernel<<<(unsigned int)(((long long)C * nl + 255) / 256), 256, 0, strm>>>(A.loff, C, (int)nl,
                                                                                                 lane_room);
    if (cudaMemsetAsync(P.counters, 0, sizeof(unsigned int) * 2, strm) != cudaSuccess) return GBS_ECUDA;
    A.lane_room = lane_room;
    A.ring_slot = 0;   // each lane's share of (a, b], for the gather
    if ((st = pass(kFWrite)) != GBS_OK) return st;
    ++npass;
    fused_step_kernel<kFWrite><<<sgrid, 256, 0, strm>>>(P);
    fused_offsets_kernel<<<1, 1024, 0, strm>>>(P.seg_len, C, off);
    fused_gather_lanes_kernel<<<C, 256, 0, strm>>>(A.zbuf, zstride, A.lring, (int)nl, lane_room, off, C, zcat);
    if ((st = check()) != GBS_OK) return st;
  } else {
    // statistics pass and the starting brackets
    if ((st = pass(kFStats)) != GBS_OK) return st;
    ++npass;
    fused_step_kernel<kFStats><<<sgrid, 256, 0, strm>>>(P);
    if ((st = check()) != GBS_OK) return st;
    // cutting-plane passes until every candidate is ready to compact
    for (int it = 0; it <= P.maxit + 1; ++it) {
      if (cudaMemcpyAsync(h_cnt, P.counters, sizeof(h_cnt), cudaMemcpyDeviceToHost, strm) != cudaSuccess ||
          cudaStreamSynchronize(strm) != cudaSuccess)
        return GBS_ECUDA;
      read_timed();
      if (h_cnt[0] == 0) break;
      if (cudaMemsetAsync(P.counters, 0, sizeof(unsigned int), strm) != cudaSuccess) return GBS_ECUDA;
      A.ring_slot = it % kRing;
      P.pass = it;
      if ((st = pass(kFCost)) != GBS_OK) return st;
      ++npass;
      fused_step_kernel<kFCost><<<sgrid, 256, 0, strm>>>(P);
      if ((st = check()) != GBS_OK) return st;
    }
    // compaction, finish preparation
    if (cudaMemsetAsync(P.counters, 0, sizeof(unsigned int) * 2, strm) != cudaSuccess) return GBS_ECUDA;
    fused_offsets_ring_kernel<<<(unsigned int)((C * 32ll + 255) / 256), 256, 0, strm>>>(P);
    if ((st = pass(kFWrite)) != GBS_OK) return st;
    npass += 1;
    fused_step_kernel<kFWrite><<<sgrid, 256, 0, strm>>>(P);
    fused_offsets_kernel<<<1, 1024, 0, strm>>>(P.seg_len, C, off);
    fused_gather_kernel<<<C, 256, 0, strm>>>(A.zbuf, zstride, off, C, zcat);
    if ((st = check()) != GBS_OK) return st;
  }
  SegLaunch L;
  if ((st = seg_attach_workspace(c, C, &L)) != GBS_OK) return st;   // already large enough: no reallocation
  L.x = zcat; L.off = off; L.S = C; L.kk = P.kk; L.out = qbuf;
  L.ctrl = c->ctrl;
  L.mask = P.mask; L.kk2 = P.kk2; L.out2 = lms_out; L.outsum = lts_out; L.flags = flags;
  L.k_const = 0; L.k2_const = 0;
  if ((st = seg_launch(c, L, kFVariant, strm)) != GBS_OK) return st;
  fused_combine_kernel<<<sgrid, 256, 0, strm>>>(P.mask, P.below, C, lts_out);
  if ((st = check()) != GBS_OK) return st;
  // candidates the fused passes could not finish: the materialising batched form
  if (cudaMemcpyAsync(h_cnt, P.counters, sizeof(h_cnt), cudaMemcpyDeviceToHost, strm) != cudaSuccess ||
      cudaStreamSynchronize(strm) != cudaSuccess)
    return GBS_ECUDA;
  if (passes) *passes = npass;
  c->lms_last.passes = npass;
  read_timed();
  {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->lms_ev[2], c->lms_ev[3]) == cudaSuccess) {
      c->lms_last.write_ms = ms;
      c->lms_last.pass_ms += ms;
    }
  }
  const int m = (int)h_cnt[1];
  if (m > 0) {
    unsigned int* cnt2 = P.counters + 2;
    if (cudaMemsetAsync(cnt2, 0, sizeof(unsigned int), strm) != cudaSuccess) return GBS_ECUDA;
    fused_fallback_list_kernel<<<sgrid, 256, 0, strm>>>(A.cand, C, list, cnt2);
    // the fallback reuses the buffers of the finish: theta subset, then its outputs
    float* th_sub = zcat;
    float* lms_sub = zcat + (size_t)m * p;
    double* lts_sub = reinterpret_cast<double*>(A.zbuf);
    fused_gather_theta_kernel<<<(m * p + 255) / 256, 256, 0, strm>>>(theta, p, list, m, th_sub);
    if ((st = check()) != GBS_OK) return st;
    st = gbs_lms_lts_f32(c, X, y, n, p, th_sub, m, k_lms, h_lts, lms_sub, lts_sub, 1, 1, stream);
    if (st != GBS_OK) return st;
    fused_scatter_kernel<<<(m + 255) / 256, 256, 0, strm>>>(list, m, lms_sub, lts_sub, lms_out, lts_out);
    if ((st = check()) != GBS_OK) return st;
  }
  c->last_segments = C;
  return GBS_OK;
}

extern "C" gbs_status gbs_lms_last_stats(gbs_ctx* c, gbs_lms_stats* out) {
  if (!c || !out) return GBS_EINVAL;
  *out = c->lms_last;
  return GBS_OK;
}
