// k-nearest-neighbour regression and classification through the k-th order statistic of
// the distances (Sec. 5, last application).  Instead of sorting each query's distances,
// the k nearest points are marked by an indicator against d_(k): 1 below it, 0 above it,
// and the share (k - #(d < d_(k))) / #(d = d_(k)) for the points exactly at d_(k), as the
// a/b weight at the order statistic of Eq. (med_reg).  One reduction of the indicator
// times the weights gives the prediction; per-class indicator sums give the vote.
//
// Distances.  Which points are the k nearest is an integer decision taken on float
// values, so every kernel here forms d^2 in one stated order: for t = 0 .. p-1,
// e = q_t - x_t, then acc = acc + e * e, each difference, product and sum rounded to
// float32 on its own (no fused multiply-add).  Coordinates are padded with zeros to a
// multiple of 4; a padded term adds an exact +0.  d^2 >= +0 always, so the float bits
// order distances like unsigned integers.
//
// Sampled start (n >= 65536).  Each query's distances to 8192 evenly spread rows give
// two sample order statistics around rank k (3.5 binomial standard deviations and two
// ranks of margin), the proposed bracket a < d_(k) <= b.  One fused pass over all rows
// then forms every distance once and sorts it into three classes, all exact counts:
//   d <= a      counted, weighted sums and class votes accumulated (indicator 1);
//   a < d < b   compacted as (d^2, row) into the query's buffer;
//   d == b      counted, sums and votes accumulated separately (the ties at b).
// A finish kernel per query checks #(d <= a) < k <= #(d <= b) and that the compacted set
// fit its buffer; it then finds d_(k) by a radix select of the compacted keys (or takes b
// when the rank falls on the ties at b) and adds the compacted points' shares.
//
// Plain form (the fallback of a query whose check fails, and gbs_config.knn_start = 1
// for all): the query's whole distance row is written out, the segmented select finds
// d_(k) exactly (Algorithm 1 per row), and the fused pass runs again with the bracket
// (largest float below d_(k), d_(k)]: nothing is compacted, the points below d_(k) and the
// ties at it are reduced directly.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdint>

#include "api_internal.h"
#include "common.cuh"
#include "segmented.cuh"

namespace gbs {
namespace {

constexpr int kKT = 256;              // threads of the pass and finish kernels
constexpr int kKW = kKT / 32;
constexpr int kKTile = 128;           // rows per shared-memory tile of the pass
constexpr int kKSample = 8192;        // sampled rows per query (sampled start)
constexpr long long kKMinN = 65536;   // smaller problems take the plain form
constexpr int kKMaxClasses = 1024;
constexpr int kKGroup = 16384;        // queries handled per round of kernels
constexpr long long kKRowsBytes = 1ll << 30;   // distance rows of the plain form per batch

// ------------------------------------------------------------------ distances
template <int PM>
__device__ __forceinline__ float sqdist(const float (&q)[PM], const float* __restrict__ x) {
  float e = __fsub_rn(q[0], x[0]);
  float d = __fmul_rn(e, e);
#pragma unroll
  for (int t = 1; t < PM; ++t) {
    e = __fsub_rn(q[t], x[t]);
    d = __fadd_rn(d, __fmul_rn(e, e));
  }
  return d;
}

__device__ __forceinline__ double knn_weight(float d2, int weight, double eps) {
  return weight ? 1.0 / (sqrt((double)d2) + eps) : 1.0;
}

// Deterministic sum over a CTA of kKT threads (fixed tree); valid in every thread.
template <typename V>
__device__ __forceinline__ V cta_sum(V v, V* scratch /* kKW */) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) scratch[threadIdx.x >> 5] = v;
  __syncthreads();
  V r = V(0);
#pragma unroll
  for (int i = 0; i < kKW; ++i) r += scratch[i];
  __syncthreads();
  return r;
}

// ------------------------------------------------------------------ preparation
// Copies rows of width p into rows of width PM (zero padded) and flags a non-finite
// coordinate in *status (GBS_ENAN).
__global__ void knn_pad_kernel(const float* __restrict__ src, long long rows, int p, int PM, float* __restrict__ dst,
                               int* status) {
  const long long total = rows * PM;
  bool bad = false;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long r = i / PM;
    const int t = (int)(i - r * PM);
    float v = 0.f;
    if (t < p) {
      v = src[r * p + t];
      bad |= !(fabsf(v) <= FLT_MAX);
    }
    dst[i] = v;
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicCAS(status, 0, (int)GBS_ENAN);
}

// A label outside [0, C) is an argument error found on the device.
__global__ void knn_labels_kernel(const int* __restrict__ labels, long long n, int C, int* status) {
  bool bad = false;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    bad |= (unsigned)labels[i] >= (unsigned)C;
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicCAS(status, 0, (int)GBS_EINVAL);
}

__global__ void knn_iota_kernel(int* list, int m, int base) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) list[i] = base + i;
}

// Per-query counters and vote tables of the queries in `list` set to zero.
__global__ void knn_zero_kernel(const int* list, int mq, int qbase, unsigned int* cnt, unsigned int* zc,
                                unsigned int* vb, unsigned int* vt, int C) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long per = 3 + 2ll * C;
  if (idx >= (long long)mq * per) return;
  const int j = (int)(idx / per);
  const long long w = idx - (long long)j * per;
  const int q = list[j] - qbase;
  if (w < 2) cnt[2ll * q + w] = 0u;
  else if (w == 2) zc[q] = 0u;
  else if (w < 3 + C) { if (vb) vb[(long long)q * C + (w - 3)] = 0u; }
  else if (vt) vt[(long long)q * C + (w - 3 - C)] = 0u;
}

// ------------------------------------------------------------------ distance rows
// out[j][i] = d^2(query list[j], row rows_of(i)) for j < mq, i < nr; row rows_of(i) is i
// (stride 0) or (i * n) / nr (the evenly spread sample).  A CTA takes 32 queries (their
// coordinates in shared memory) and kKT consecutive rows, one row a thread.
template <int PM>
__global__ void __launch_bounds__(kKT) knn_rows_kernel(const float* __restrict__ xp, long long n, long long nr,
                                                       bool spread, const float* __restrict__ qp,
                                                       const int* __restrict__ list, int qbase, int mq,
                                                       float* __restrict__ out) {
  __shared__ float s_q[32][PM];
  const int j0 = blockIdx.y * 32;
  for (int i = threadIdx.x; i < 32 * PM; i += kKT) {
    const int jj = i / PM, t = i - jj * PM;
    s_q[jj][t] = (j0 + jj < mq) ? qp[(long long)(list[j0 + jj] - qbase) * PM + t] : 0.f;
  }
  __syncthreads();
  const long long i = (long long)blockIdx.x * kKT + threadIdx.x;
  if (i >= nr) return;
  const long long row = spread ? (long long)((unsigned long long)i * (unsigned long long)n / (unsigned long long)nr) : i;
  float x[PM];
#pragma unroll
  for (int t = 0; t < PM; t += 4) {
    const float4 v = *reinterpret_cast<const float4*>(xp + row * PM + t);
    x[t] = v.x; x[t + 1] = v.y; x[t + 2] = v.z; x[t + 3] = v.w;
  }
  const int jn = min(32, mq - j0);
  for (int jj = 0; jj < jn; ++jj) {
    float e = __fsub_rn(s_q[jj][0], x[0]);
    float d = __fmul_rn(e, e);
#pragma unroll
    for (int t = 1; t < PM; ++t) {
      e = __fsub_rn(s_q[jj][t], x[t]);
      d = __fadd_rn(d, __fmul_rn(e, e));
    }
    out[(long long)(j0 + jj) * nr + i] = d;
  }
}

__global__ void knn_offsets_kernel(long long* off, int S, long long len) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s <= S) off[s] = (long long)s * len;
}

// Brackets of the sampled start: a = the lower sample order statistic (or -1, below
// every distance, when its rank falls below the sample), b = the upper one (+inf above
// the sample); a >= b (ties in the sample) moves a just below b.
__global__ void knn_sample_bracket_kernel(int mq, const float* lo, const float* hi, bool lo_in, bool hi_in, float* qa,
                                          float* qb) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= mq) return;
  float a = lo_in ? lo[q] : -1.f;
  const float b = hi_in ? hi[q] : INFINITY;
  if (!(a < b)) a = b > 0.f ? nextafterf(b, -INFINITY) : -1.f;
  qa[q] = a;
  qb[q] = b;
}

// Brackets of the plain form: (largest float below d_(k), d_(k)], nothing strictly inside.
__global__ void knn_known_bracket_kernel(const int* list, int mq, int qbase, const float* kth, float* qa, float* qb) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= mq) return;
  const int q = list[j] - qbase;
  const float v = kth[j];
  qa[q] = v > 0.f ? nextafterf(v, -INFINITY) : -1.f;
  qb[q] = v;
}

// ------------------------------------------------------------------ the fused pass
struct KnnPass {
  const float* xp;        // n x PM padded rows
  long long n;
  long long rows_per_chunk;
  const float* qp;        // group's queries, PM padded
  const int* list;        // queries of this pass (group-relative after subtracting qbase)
  int qbase, mq, mg;      // list offset, list length, queries in the group
  const float* qa;        // [mg] brackets
  const float* qb;
  const float* f;         // [n] ordinates or nullptr
  const int* labels;      // [n] labels or nullptr
  int C;
  int weight;
  double eps;
  unsigned int* cnt;      // [mg][2]: #(d <= a), #(d == b)
  unsigned int* zc;       // [mg]: #(a < d < b)
  float* zd;              // [mg][cap] compacted distances
  int* zi;                // [mg][cap] their rows
  long long cap;
  double* part;           // [chunks][mg][4]: sums w f and w over d <= a, then over d == b
  unsigned int* vb;       // [mg][C] votes of d <= a
  unsigned int* vt;       // [mg][C] votes of d == b
};

// CTA (chunk, query block): kKT threads, each owning QPT queries (slots tid + j*kKT)
// with their coordinates in registers; the CTA's rows are staged tile by tile in shared
// memory and read by every thread (broadcast).  The three classes of a distance are rare
// next to "above b", so they take a branch; their counts and sums go to per-thread-owned
// shared slots (no atomics, row order), written out once per CTA.
template <int PM, int QPT>
__global__ void __launch_bounds__(kKT, 2) knn_pass_kernel(KnnPass A) {
  __shared__ __align__(16) float s_x[kKTile * PM];
  __shared__ unsigned int s_cnt[2][kKT * QPT];
  __shared__ double s_sum[4][kKT * QPT];
  const int tid = threadIdx.x;
  const long long r0 = (long long)blockIdx.x * A.rows_per_chunk;
  const long long r1 = min(A.n, r0 + A.rows_per_chunk);
  float q[QPT][PM];
  float qa[QPT], qb[QPT];
  int qid[QPT];
#pragma unroll
  for (int j = 0; j < QPT; ++j) {
    const int slot = tid + j * kKT;
    const int li = blockIdx.y * (kKT * QPT) + slot;
    qid[j] = -1;
    qa[j] = 0.f;
    qb[j] = -INFINITY;   // no distance is <= -inf: an empty slot takes no branch
#pragma unroll
    for (int t = 0; t < PM; ++t) q[j][t] = 0.f;
    if (li < A.mq) {
      const int g = A.list[li] - A.qbase;
      qid[j] = g;
      qa[j] = A.qa[g];
      qb[j] = A.qb[g];
#pragma unroll
      for (int t = 0; t < PM; t += 4) {
        const float4 v = *reinterpret_cast<const float4*>(A.qp + (long long)g * PM + t);
        q[j][t] = v.x; q[j][t + 1] = v.y; q[j][t + 2] = v.z; q[j][t + 3] = v.w;
      }
    }
    s_cnt[0][slot] = 0u; s_cnt[1][slot] = 0u;
    s_sum[0][slot] = 0.0; s_sum[1][slot] = 0.0; s_sum[2][slot] = 0.0; s_sum[3][slot] = 0.0;
  }
  for (long long rt = r0; rt < r1; rt += kKTile) {
    const int rows = (int)min((long long)kKTile, r1 - rt);
    __syncthreads();
    for (int i = tid; i < rows * (PM / 4); i += kKT)
      reinterpret_cast<float4*>(s_x)[i] = __ldg(reinterpret_cast<const float4*>(A.xp + rt * PM) + i);
    __syncthreads();
    for (int r = 0; r < rows; ++r) {
      float x[PM];
#pragma unroll
      for (int t = 0; t < PM; t += 4) {
        const float4 v = reinterpret_cast<const float4*>(s_x + r * PM)[t / 4];
        x[t] = v.x; x[t + 1] = v.y; x[t + 2] = v.z; x[t + 3] = v.w;
      }
#pragma unroll
      for (int j = 0; j < QPT; ++j) {
        const float d = sqdist<PM>(q[j], x);
        if (d <= qb[j]) {
          const int slot = tid + j * kKT;
          const long long row = rt + r;
          const int g = qid[j];
          if (d <= qa[j] || d == qb[j]) {
            const int cls = d <= qa[j] ? 0 : 1;
            s_cnt[cls][slot] += 1u;
            if (A.f) {
              const double w = knn_weight(d, A.weight, A.eps);
              s_sum[2 * cls][slot] += w * (double)A.f[row];
              s_sum[2 * cls + 1][slot] += w;
            }
            if (A.labels) {
              const int lab = A.labels[row];
              if ((unsigned)lab < (unsigned)A.C)
                atomicAdd((cls == 0 ? A.vb : A.vt) + (long long)g * A.C + lab, 1u);
            }
          } else {
            const unsigned int pos = atomicAdd(A.zc + g, 1u);
            if (pos < (unsigned long long)A.cap) {
              A.zd[(long long)g * A.cap + pos] = d;
              A.zi[(long long)g * A.cap + pos] = (int)row;
            }
          }
        }
      }
    }
  }
#pragma unroll
  for (int j = 0; j < QPT; ++j) {
    const int slot = tid + j * kKT;
    const int g = qid[j];
    if (g < 0) continue;
    if (s_cnt[0][slot]) atomicAdd(A.cnt + 2ll * g, s_cnt[0][slot]);
    if (s_cnt[1][slot]) atomicAdd(A.cnt + 2ll * g + 1, s_cnt[1][slot]);
    double* pp = A.part + ((long long)blockIdx.x * A.mg + g) * 4;
    pp[0] = s_sum[0][slot]; pp[1] = s_sum[1][slot]; pp[2] = s_sum[2][slot]; pp[3] = s_sum[3][slot];
  }
}

// ------------------------------------------------------------------ the finish
struct KnnFin {
  const int* list;
  int qbase, mq, mg;
  long long k;
  int nchunks;
  const float* qb;
  const unsigned int* cnt;
  const unsigned int* zc;
  const float* zd;
  const int* zi;
  long long cap;
  const double* part;
  const unsigned int* vb;
  const unsigned int* vt;
  const float* f;
  const int* labels;
  int C, weight;
  double eps;
  const int* status;      // non-finite coordinates / bad labels: outputs are NaN
  int* fail_list;         // queries whose check failed (group-relative), and their count
  unsigned int* fail_count;
  int final_round;        // 1: a failed check is an internal error (the plain form cannot fail)
  int* err;               // GBS_EINTERNAL recorded here
  // outputs, indexed by the global query (qbase_out + group-relative index)
  long long out_base;
  float* kth;
  double* pred;
  int* cls;
  double* votes;
};

// One CTA per query: checks the bracket, finds d_(k) in the compacted set (8-bit radix
// select on the float bits of d^2 >= +0, keys in dynamic shared memory) or at b, and
// combines the pass's sums and votes with the compacted points' shares.
__global__ void __launch_bounds__(kKT) knn_finish_kernel(KnnFin F) {
  extern __shared__ unsigned int s_key[];   // [cap]
  __shared__ unsigned int s_hist[256];
  __shared__ unsigned int s_vb[kKMaxClasses], s_vt[kKMaxClasses];
  __shared__ double s_red[kKW];
  __shared__ unsigned long long s_red_u[kKW];
  __shared__ unsigned int s_prefix, s_rank;
  __shared__ int s_fail;
  const int tid = threadIdx.x;
  const int g = F.list[blockIdx.x] - F.qbase;
  const long long out_i = F.out_base + g;
  const long long k = F.k;
  const long long below = F.cnt[2ll * g], tieb = F.cnt[2ll * g + 1];
  const long long P = F.zc[g];
  const float b = F.qb[g];
  const bool bad_input = *F.status != 0;
  if (tid == 0) {
    s_fail = bad_input ? 2 : ((below >= k || below + P + tieb < k || P > F.cap) ? 1 : 0);
  }
  __syncthreads();
  if (s_fail) {
    if (tid == 0) {
      if (s_fail == 1 && !F.final_round) {
        F.fail_list[atomicAdd(F.fail_count, 1u)] = g + F.qbase;
      } else {
        if (s_fail == 1) atomicCAS(F.err, 0, (int)GBS_EINTERNAL);
        if (F.kth) F.kth[out_i] = NAN;
        if (F.pred) F.pred[out_i] = NAN;
        if (F.cls) F.cls[out_i] = -1;
      }
    }
    if (F.votes && (s_fail == 2 || F.final_round))
      for (int c = tid; c < F.C; c += kKT) F.votes[out_i * F.C + c] = NAN;
    return;
  }
  const bool at_b = below + P < k;   // d_(k) is b: every compacted point is below it
  const float* zd = F.zd + (long long)g * F.cap;
  const int* zi = F.zi + (long long)g * F.cap;
  // d_(k): rank k - below among the compacted keys, or b
  unsigned int qbits;
  if (at_b) {
    qbits = __float_as_uint(b);
  } else {
    for (long long i = tid; i < P; i += kKT) s_key[i] = __float_as_uint(zd[i]);
    if (tid == 0) { s_prefix = 0u; s_rank = (unsigned int)(k - below); }
    for (int round = 0; round < 4; ++round) {
      const int sh = 24 - 8 * round;
      for (int i = tid; i < 256; i += kKT) s_hist[i] = 0u;
      __syncthreads();
      const unsigned int pre = s_prefix;
      for (long long i = tid; i < P; i += kKT) {
        const unsigned int key = s_key[i];
        if (round == 0 || (key >> (sh + 8)) == (pre >> (sh + 8))) atomicAdd(&s_hist[(key >> sh) & 255u], 1u);
      }
      __syncthreads();
      if (tid == 0) {
        unsigned int want = s_rank, c = 0u;
        int d = 255;
        for (int i = 0; i < 256; ++i) {
          if (c + s_hist[i] >= want) { d = i; break; }
          c += s_hist[i];
        }
        s_rank = want - c;
        s_prefix = pre | ((unsigned int)d << sh);
      }
      __syncthreads();
    }
    qbits = s_prefix;
  }
  const float qv = __uint_as_float(qbits);
  // the compacted points: below d_(k) (indicator 1) and at it (the tie share)
  const bool regress = F.f != nullptr, classify = F.labels != nullptr;
  if (classify)
    for (int c = tid; c < F.C; c += kKT) { s_vb[c] = 0u; s_vt[c] = 0u; }
  __syncthreads();
  double swf_lo = 0.0, sw_lo = 0.0, swf_eq = 0.0, sw_eq = 0.0;
  unsigned long long n_lo = 0, n_eq = 0;
  for (long long i = tid; i < P; i += kKT) {
    const float d = zd[i];
    const int lt = d < qv, eq = d == qv;
    if (!(lt | eq)) continue;
    n_lo += lt; n_eq += eq;
    const int row = zi[i];
    if (regress) {
      const double w = knn_weight(d, F.weight, F.eps);
      const double wf = w * (double)F.f[row];
      if (lt) { swf_lo += wf; sw_lo += w; } else { swf_eq += wf; sw_eq += w; }
    }
    if (classify) {
      const int lab = F.labels[row];
      if ((unsigned)lab < (unsigned)F.C) atomicAdd(lt ? &s_vb[lab] : &s_vt[lab], 1u);
    }
  }
  n_lo = cta_sum<unsigned long long>(n_lo, s_red_u);
  n_eq = cta_sum<unsigned long long>(n_eq, s_red_u);
  if (regress) {
    swf_lo = cta_sum<double>(swf_lo, s_red);
    sw_lo = cta_sum<double>(sw_lo, s_red);
    swf_eq = cta_sum<double>(swf_eq, s_red);
    sw_eq = cta_sum<double>(sw_eq, s_red);
  }
  // the pass's sums over d <= a and d == b, over its row chunks in a fixed order
  double pa0 = 0.0, pa1 = 0.0, pb0 = 0.0, pb1 = 0.0;
  if (regress) {
    for (int ch = tid; ch < F.nchunks; ch += kKT) {
      const double* pp = F.part + ((long long)ch * F.mg + g) * 4;
      pa0 += pp[0]; pa1 += pp[1]; pb0 += pp[2]; pb1 += pp[3];
    }
    pa0 = cta_sum<double>(pa0, s_red);
    pa1 = cta_sum<double>(pa1, s_red);
    pb0 = cta_sum<double>(pb0, s_red);
    pb1 = cta_sum<double>(pb1, s_red);
  }
  // the tie share a_t / b_t at d_(k)
  long long ta, tb;
  if (at_b) { ta = k - below - P; tb = tieb; }
  else { ta = k - below - (long long)n_lo; tb = (long long)n_eq; }
  if (tid == 0) {
    if (F.kth) F.kth[out_i] = qv;
    if (regress) {
      const double share = (double)ta / (double)tb;
      double num, den;
      if (at_b) {
        num = pa0 + swf_lo + share * pb0;
        den = pa1 + sw_lo + share * pb1;
      } else {
        num = pa0 + swf_lo + share * swf_eq;
        den = pa1 + sw_lo + share * sw_eq;
      }
      F.pred[out_i] = num / den;
    }
  }
  if (classify) {
    __syncthreads();
    // exact scores below_c * tb + tie_c * ta; the vote is their ratio to tb, rounded once
    long long best_s = -1;
    int best_c = 0x7fffffff;
    for (int c = tid; c < F.C; c += kKT) {
      // below d_(k): the pass's points d <= a and the compacted points below it (all of
      // them when d_(k) is b); at d_(k): the ties at b, or the compacted ties
      const long long lo = (long long)F.vb[(long long)g * F.C + c] + s_vb[c];
      const long long eq = at_b ? (long long)F.vt[(long long)g * F.C + c] : (long long)s_vt[c];
      const long long score = lo * tb + eq * ta;
      if (F.votes) F.votes[out_i * F.C + c] = (double)score / (double)tb;
      if (score > best_s || (score == best_s && c < best_c)) { best_s = score; best_c = c; }
    }
    // arg max over the CTA, smallest class on ties
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const long long os = __shfl_xor_sync(0xffffffffu, best_s, o);
      const int oc = __shfl_xor_sync(0xffffffffu, best_c, o);
      if (os > best_s || (os == best_s && oc < best_c)) { best_s = os; best_c = oc; }
    }
    __shared__ long long s_bs[kKW];
    __shared__ int s_bc[kKW];
    if ((tid & 31) == 0) { s_bs[tid >> 5] = best_s; s_bc[tid >> 5] = best_c; }
    __syncthreads();
    if (tid == 0) {
      for (int w = 1; w < kKW; ++w)
        if (s_bs[w] > best_s || (s_bs[w] == best_s && s_bc[w] < best_c)) { best_s = s_bs[w]; best_c = s_bc[w]; }
      if (F.cls) F.cls[out_i] = best_c;
    }
  }
}

// The call's device status: an input error found by the preparation kernels takes
// precedence over what a segmented select recorded on the same control block.
__global__ void knn_status_kernel(const int* knn_status, const int* err, Ctrl* ctrl) {
  if (threadIdx.x == 0) {
    if (*knn_status) atomicExch(&ctrl->status, *knn_status);
    else if (*err) atomicCAS(&ctrl->status, 0, *err);
  }
}

size_t up256k(size_t v) { return (v + 255) / 256 * 256; }

// Queries per thread of the pass: registers hold QPT * PM coordinates.
template <int PM> constexpr int qpt_of() { return PM <= 8 ? 4 : (PM == 16 ? 2 : 1); }
int qpt_for(int PM) { return PM <= 8 ? 4 : (PM == 16 ? 2 : 1); }

template <int PM>
gbs_status launch_pass_pm(const KnnPass& A, int nchunks, cudaStream_t s) {
  constexpr int QPT = qpt_of<PM>();
  constexpr int per = kKT * QPT;
  const dim3 grid((unsigned)nchunks, (unsigned)((A.mq + per - 1) / per));
  knn_pass_kernel<PM, QPT><<<grid, kKT, 0, s>>>(A);
  return cudaGetLastError() == cudaSuccess ? GBS_OK : GBS_ECUDA;
}

gbs_status launch_pass(int PM, const KnnPass& A, int nchunks, cudaStream_t s) {
  switch (PM) {
    case 4: return launch_pass_pm<4>(A, nchunks, s);
    case 8: return launch_pass_pm<8>(A, nchunks, s);
    case 16: return launch_pass_pm<16>(A, nchunks, s);
    default: return launch_pass_pm<32>(A, nchunks, s);
  }
}

gbs_status launch_rows(int PM, const float* xp, long long n, long long nr, bool spread, const float* qp,
                       const int* list, int qbase, int mq, float* out, cudaStream_t s) {
  const dim3 grid((unsigned)((nr + kKT - 1) / kKT), (unsigned)((mq + 31) / 32));
  switch (PM) {
    case 4: knn_rows_kernel<4><<<grid, kKT, 0, s>>>(xp, n, nr, spread, qp, list, qbase, mq, out); break;
    case 8: knn_rows_kernel<8><<<grid, kKT, 0, s>>>(xp, n, nr, spread, qp, list, qbase, mq, out); break;
    case 16: knn_rows_kernel<16><<<grid, kKT, 0, s>>>(xp, n, nr, spread, qp, list, qbase, mq, out); break;
    default: knn_rows_kernel<32><<<grid, kKT, 0, s>>>(xp, n, nr, spread, qp, list, qbase, mq, out); break;
  }
  return cudaGetLastError() == cudaSuccess ? GBS_OK : GBS_ECUDA;
}

}  // namespace

// ------------------------------------------------------------------ host driver
gbs_status knn_run(gbs_ctx* c, const float* X, long long n, int p, const float* Q, int m, long long k,
                   const float* f, int weight, double eps, const int* labels, int C, float* kth, double* pred,
                   int* cls, double* votes, int* passes_out, cudaStream_t strm) {
  const int PM = p <= 4 ? 4 : (p <= 8 ? 8 : (p <= 16 ? 16 : 32));
  const int qpt = qpt_for(PM);
  const int G = std::min(m, kKGroup);   // queries per group
  // sampled start: sample ranks around k, and the compaction buffer sized from the
  // expected bracket population (2.5 times it plus 6 standard deviations)
  const int ns = kKSample;
  bool sampled = c->cfg.knn_start == 0 && n >= kKMinN;
  long long jl = 0, jh = 0, cap = 256;
  if (sampled) {
    const double pk = (double)k / (double)n;
    const double sd = std::sqrt(ns * pk * (1.0 - pk));
    jl = (long long)std::floor(ns * pk - 3.5 * sd) - 2;
    jh = (long long)std::ceil(ns * pk + 3.5 * sd) + 2;
    const double frac = (double)(std::min<long long>(jh, ns + 1) - std::max<long long>(jl, 0)) / ns;
    const double mean = frac * (double)n;
    cap = (long long)std::ceil(2.5 * mean + 6.0 * std::sqrt(mean) + 256.0);
    cap = std::max<long long>(4096, (cap + 255) / 256 * 256);
    // the finish keeps the keys in shared memory (at most 48K keys = 192 KiB)
    if (cap > 49152) sampled = false;
  }
  if (!sampled) cap = 256;
  // row chunks of the pass: about four CTAs per resident slot (two per SM)
  const int nqb_full = (G + kKT * qpt - 1) / (kKT * qpt);
  long long nch = std::max<long long>(1, ((long long)c->num_sms * 2 * 4 + nqb_full - 1) / nqb_full);
  long long rpc = (n + nch - 1) / nch;
  rpc = (rpc + kKTile - 1) / kKTile * kKTile;
  nch = (n + rpc - 1) / rpc;
  const long long batch_rows = std::max<long long>(1, std::min<long long>(G, kKRowsBytes / (4 * n)));
  // workspace: xp | qp | qa | qb | cnt | zc | zd | zi | part | vb | vt | rows | off | lo | hi |
  //            osum | flags | list | fail | kthb | status
  size_t o = 0;
  const size_t o_xp = o; o = up256k(o + sizeof(float) * (size_t)n * PM);
  const size_t o_qp = o; o = up256k(o + sizeof(float) * (size_t)G * PM);
  const size_t o_qa = o; o = up256k(o + sizeof(float) * (size_t)G);
  const size_t o_qb = o; o = up256k(o + sizeof(float) * (size_t)G);
  const size_t o_cnt = o; o = up256k(o + sizeof(unsigned int) * 2 * (size_t)G);
  const size_t o_zc = o; o = up256k(o + sizeof(unsigned int) * (size_t)G);
  const size_t o_zd = o; o = up256k(o + sizeof(float) * (size_t)G * cap);
  const size_t o_zi = o; o = up256k(o + sizeof(int) * (size_t)G * cap);
  const size_t o_part = o; o = up256k(o + sizeof(double) * 4 * (size_t)nch * G);
  const size_t o_vb = o; o = up256k(o + sizeof(unsigned int) * (size_t)G * (labels ? C : 0));
  const size_t o_vt = o; o = up256k(o + sizeof(unsigned int) * (size_t)G * (labels ? C : 0));
  const size_t rows_elems = std::max<size_t>(sampled ? (size_t)G * ns : 0, (size_t)batch_rows * n);
  const size_t o_rows = o; o = up256k(o + sizeof(float) * rows_elems);
  const size_t o_off = o; o = up256k(o + sizeof(long long) * ((size_t)G + 1));
  const size_t o_lo = o; o = up256k(o + sizeof(float) * (size_t)G);
  const size_t o_hi = o; o = up256k(o + sizeof(float) * (size_t)G);
  const size_t o_osum = o; o = up256k(o + sizeof(double) * (size_t)G);
  const size_t o_flags = o; o = up256k(o + sizeof(int) * (size_t)G);
  const size_t o_list = o; o = up256k(o + sizeof(int) * (size_t)G);
  const size_t o_fail = o; o = up256k(o + sizeof(int) * (size_t)G);
  const size_t o_st = o; o = up256k(o + sizeof(int) * 8);
  const size_t bytes = o;
  if (!c->knn_buf || c->knn_bytes < bytes) {
    gbs_internal_release_knn(c);
    void* ptr = nullptr;
    if (cudaMalloc(&ptr, bytes) != cudaSuccess) {
      cudaGetLastError();
      return GBS_ENOMEM;
    }
    c->knn_buf = ptr;
    c->knn_bytes = bytes;
  }
  gbs_status st = gbs_internal_ensure(c, seg_workspace_bytes(std::max<int>(G, (int)batch_rows)));
  if (st != GBS_OK) return st;
  char* B = static_cast<char*>(c->knn_buf);
  float* xp = reinterpret_cast<float*>(B + o_xp);
  float* qp = reinterpret_cast<float*>(B + o_qp);
  float* qa = reinterpret_cast<float*>(B + o_qa);
  float* qb = reinterpret_cast<float*>(B + o_qb);
  unsigned int* cnt = reinterpret_cast<unsigned int*>(B + o_cnt);
  unsigned int* zc = reinterpret_cast<unsigned int*>(B + o_zc);
  float* zd = reinterpret_cast<float*>(B + o_zd);
  int* zi = reinterpret_cast<int*>(B + o_zi);
  double* part = reinterpret_cast<double*>(B + o_part);
  unsigned int* vb = labels ? reinterpret_cast<unsigned int*>(B + o_vb) : nullptr;
  unsigned int* vt = labels ? reinterpret_cast<unsigned int*>(B + o_vt) : nullptr;
  float* rows = reinterpret_cast<float*>(B + o_rows);
  long long* off = reinterpret_cast<long long*>(B + o_off);
  float* lo = reinterpret_cast<float*>(B + o_lo);
  float* hi = reinterpret_cast<float*>(B + o_hi);
  double* osum = reinterpret_cast<double*>(B + o_osum);
  int* flags = reinterpret_cast<int*>(B + o_flags);
  int* list = reinterpret_cast<int*>(B + o_list);
  int* fail = reinterpret_cast<int*>(B + o_fail);
  int* status = reinterpret_cast<int*>(B + o_st);          // [0] input status, [1] internal error,
  unsigned int* fcount = reinterpret_cast<unsigned int*>(status + 2);   // [2] failed queries
  auto check = [&]() { return cudaGetLastError() == cudaSuccess ? GBS_OK : GBS_ECUDA; };

  if (cudaMemsetAsync(status, 0, sizeof(int) * 8, strm) != cudaSuccess ||
      cudaMemsetAsync(c->rs, 0, sizeof(gbs_run_stats), strm) != cudaSuccess)
    return GBS_ECUDA;
  knn_pad_kernel<<<(unsigned)std::min<long long>((n * PM + 255) / 256, (long long)c->num_sms * 16), 256, 0, strm>>>(
      X, n, p, PM, xp, status);
  if (labels)
    knn_labels_kernel<<<(unsigned)std::min<long long>((n + 255) / 256, (long long)c->num_sms * 8), 256, 0, strm>>>(
        labels, n, C, status);
  if ((st = check()) != GBS_OK) return st;

  KnnPass A;
  A.xp = xp; A.n = n; A.rows_per_chunk = rpc; A.qp = qp;
  A.qa = qa; A.qb = qb; A.f = f; A.labels = labels; A.C = C; A.weight = weight; A.eps = eps;
  A.cnt = cnt; A.zc = zc; A.zd = zd; A.zi = zi; A.cap = cap; A.part = part; A.vb = vb; A.vt = vt;
  KnnFin F;
  F.k = k; F.nchunks = (int)nch; F.qb = qb; F.cnt = cnt; F.zc = zc; F.zd = zd; F.zi = zi; F.cap = cap;
  F.part = part; F.vb = vb; F.vt = vt; F.f = f; F.labels = labels; F.C = C; F.weight = weight; F.eps = eps;
  F.status = status; F.fail_list = fail; F.fail_count = fcount; F.err = status + 1;
  F.kth = kth; F.pred = pred; F.cls = cls; F.votes = votes;
  const size_t fin_smem_sampled = sizeof(unsigned int) * (size_t)cap;
  if (cudaFuncSetAttribute(knn_finish_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)std::max<size_t>(fin_smem_sampled, 1024)) != cudaSuccess) {
    cudaGetLastError();
    return GBS_ECUDA;
  }
  int npass = 0;
  for (int q0 = 0; q0 < m; q0 += G) {
    const int mg = std::min(G, m - q0);
    knn_pad_kernel<<<(unsigned)std::min<long long>(((long long)mg * PM + 255) / 256, (long long)c->num_sms * 16), 256,
                     0, strm>>>(Q + (long long)q0 * p, mg, p, PM, qp, status);
    knn_iota_kernel<<<(mg + 255) / 256, 256, 0, strm>>>(list, mg, q0);
    if ((st = check()) != GBS_OK) return st;
    A.qbase = q0; A.mg = mg; F.qbase = q0; F.mg = mg; F.out_base = q0;
    int nfail = mg;
    const int* flist = list;
    if (sampled) {
      // sample order statistics: the distances to ns evenly spread rows, then both ranks
      // from one load of each query's sample (the segmented select's two-rank mode)
      if ((st = launch_rows(PM, xp, n, ns, true, qp, list, q0, mg, rows, strm)) != GBS_OK) return st;
      knn_offsets_kernel<<<(mg + 1 + 255) / 256, 256, 0, strm>>>(off, mg, ns);
      if ((st = check()) != GBS_OK) return st;
      const bool lo_in = jl >= 1, hi_in = jh <= ns;
      SegLaunch Ls;
      if ((st = seg_attach_workspace(c, mg, &Ls)) != GBS_OK) return st;
      Ls.x = rows; Ls.off = off; Ls.S = mg; Ls.kk = nullptr; Ls.ctrl = c->ctrl; Ls.mask = nullptr; Ls.kk2 = nullptr;
      Ls.k_const = std::max<long long>(jl, 1); Ls.out = lo;
      Ls.k2_const = std::min<long long>(jh, ns); Ls.out2 = hi;
      Ls.outsum = osum; Ls.flags = flags;
      if ((st = seg_launch(c, Ls, 0, strm)) != GBS_OK) return st;
      knn_sample_bracket_kernel<<<(mg + 255) / 256, 256, 0, strm>>>(mg, lo, hi, lo_in, hi_in, qa, qb);
      knn_zero_kernel<<<(unsigned)(((long long)mg * (3 + 2 * (labels ? C : 0)) + 255) / 256), 256, 0, strm>>>(
          list, mg, q0, cnt, zc, vb, vt, labels ? C : 0);
      if ((st = check()) != GBS_OK) return st;
      A.list = list; A.mq = mg;
      if ((st = launch_pass(PM, A, (int)nch, strm)) != GBS_OK) return st;
      if (q0 == 0) ++npass;
      if (cudaMemsetAsync(fcount, 0, sizeof(unsigned int), strm) != cudaSuccess) return GBS_ECUDA;
      F.list = list; F.mq = mg; F.final_round = 0;
      knn_finish_kernel<<<mg, kKT, fin_smem_sampled, strm>>>(F);
      if ((st = check()) != GBS_OK) return st;
      unsigned int h_fail = 0;
      if (cudaMemcpyAsync(&h_fail, fcount, sizeof(h_fail), cudaMemcpyDeviceToHost, strm) != cudaSuccess ||
          cudaStreamSynchronize(strm) != cudaSuccess)
        return GBS_ECUDA;
      nfail = (int)h_fail;
      flist = fail;
    }
    // the plain form for the rest: whole distance rows, d_(k) by the segmented select,
    // then the pass with the bracket (just below d_(k), d_(k)]
    for (int j0 = 0; j0 < nfail; j0 += (int)batch_rows) {
      const int mb = std::min<int>((int)batch_rows, nfail - j0);
      const int* bl = flist + j0;
      if ((st = launch_rows(PM, xp, n, n, false, qp, bl, q0, mb, rows, strm)) != GBS_OK) return st;
      knn_offsets_kernel<<<(mb + 1 + 255) / 256, 256, 0, strm>>>(off, mb, n);
      if ((st = check()) != GBS_OK) return st;
      SegLaunch L;
      if ((st = seg_attach_workspace(c, mb, &L)) != GBS_OK) return st;
      L.x = rows; L.off = off; L.S = mb; L.kk = nullptr; L.ctrl = c->ctrl; L.mask = nullptr; L.kk2 = nullptr;
      L.k_const = k; L.k2_const = 0; L.out = lo; L.out2 = nullptr; L.outsum = nullptr; L.flags = nullptr;
      if ((st = seg_launch(c, L, c->seg_variant, strm)) != GBS_OK) return st;
      knn_known_bracket_kernel<<<(mb + 255) / 256, 256, 0, strm>>>(bl, mb, q0, lo, qa, qb);
      knn_zero_kernel<<<(unsigned)(((long long)mb * (3 + 2 * (labels ? C : 0)) + 255) / 256), 256, 0, strm>>>(
          bl, mb, q0, cnt, zc, vb, vt, labels ? C : 0);
      if ((st = check()) != GBS_OK) return st;
      A.list = bl; A.mq = mb;
      if ((st = launch_pass(PM, A, (int)nch, strm)) != GBS_OK) return st;
      F.list = bl; F.mq = mb; F.final_round = 1;
      knn_finish_kernel<<<mb, kKT, fin_smem_sampled, strm>>>(F);
      if ((st = check()) != GBS_OK) return st;
    }
    if (q0 == 0 && nfail > 0) npass += 2;   // the distance rows and the second pass
  }
  knn_status_kernel<<<1, 32, 0, strm>>>(status, status + 1, c->ctrl);
  if ((st = check()) != GBS_OK) return st;
  if (passes_out) *passes_out = npass;
  c->last_stream = strm;
  return GBS_OK;
}

}  // namespace gbs

void gbs_internal_release_knn(gbs_ctx* c) {
  if (c->knn_buf) {
    cudaDeviceSynchronize();
    cudaFree(c->knn_buf);
    c->knn_buf = nullptr;
    c->knn_bytes = 0;
  }
}

namespace {
gbs_status knn_check(gbs_ctx* c, const float* X, int64_t n, int32_t p, const float* Q, int32_t m, int64_t k) {
  if (!c || !X || !Q) return GBS_EINVAL;
  if (n < 1 || n > 0x7fffffffll || p < 1 || p > 32 || m < 1 || k < 1 || k > n) return GBS_EINVAL;
  return GBS_OK;
}
}  // namespace

extern "C" gbs_status gbs_knn_regress_f32(gbs_ctx* c, const float* X, int64_t n, int32_t p, const float* f,
                                          const float* Q, int32_t m, int64_t k, int32_t weight, double eps,
                                          double* pred, float* kth_d2, void* stream) {
  gbs_status st = knn_check(c, X, n, p, Q, m, k);
  if (st != GBS_OK) return st;
  if (!f || !pred || (weight != 0 && weight != 1)) return GBS_EINVAL;
  if (weight == 1 && !(eps > 0.0 && std::isfinite(eps))) return GBS_EINVAL;
  gbs::DeviceGuard g(c->device);
  if (!g.ok) return GBS_ECUDA;
  return gbs::knn_run(c, X, n, p, Q, m, k, f, weight, eps, nullptr, 0, kth_d2, pred, nullptr, nullptr, nullptr,
                      static_cast<cudaStream_t>(stream));
}

extern "C" gbs_status gbs_knn_classify_f32(gbs_ctx* c, const float* X, int64_t n, int32_t p, const int32_t* labels,
                                           int32_t n_classes, const float* Q, int32_t m, int64_t k, int32_t* cls,
                                           double* votes, float* kth_d2, void* stream) {
  gbs_status st = knn_check(c, X, n, p, Q, m, k);
  if (st != GBS_OK) return st;
  if (!labels || !cls || n_classes < 1 || n_classes > gbs::kKMaxClasses) return GBS_EINVAL;
  gbs::DeviceGuard g(c->device);
  if (!g.ok) return GBS_ECUDA;
  return gbs::knn_run(c, X, n, p, Q, m, k, nullptr, 0, 0.0, labels, n_classes, kth_d2, nullptr, cls, votes, nullptr,
                      static_cast<cudaStream_t>(stream));
}
