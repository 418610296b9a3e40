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
// Sampled start (n >= 65536).  One CTA per query forms its distances to 8192 evenly
// spread rows in shared memory and selects two of their order statistics around rank k
// (4.5 binomial standard deviations and four ranks of margin on each side): the proposed
// bracket a < d_(k) <= b.  One fused pass over all rows then forms every distance once
// and sorts it into three classes, all exact counts:
//   d <= a      counted, weighted sums and class votes accumulated (indicator 1);
//   a < d < b   compacted as (d^2, row) into the query's buffer;
//   d == b      counted, sums and votes accumulated separately (the ties at b).
// A finish kernel per query checks #(d <= a) < k <= #(d <= b) and that the compacted set
// fit its buffer; it then finds d_(k) by a radix select of the compacted keys (or takes b
// when the rank falls on the ties at b) and adds the compacted points' shares.
//
// Plain form (a query whose check fails, and every query with gbs_config.knn_start = 1):
// the query's whole distance row is written out, d_(k) is selected exactly from it --
// by the single-array select kernel for a few rows, by the segmented select (Algorithm 1
// per row) for many -- and one CTA per row reduces the indicator against d_(k) from the
// written row.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdint>

#include "api_internal.h"
#include "common.cuh"
#include "segmented.cuh"
#include "select.cuh"

namespace gbs {
namespace {

constexpr int kKT = 256;              // threads of the pass and finish kernels
constexpr int kKW = kKT / 32;
constexpr int kKTile = 128;           // rows per shared-memory tile of the pass
constexpr int kKSampleMinLog2 = 10;   // sampled rows per query: 2^10 .. 2^15 (sampled start)
constexpr int kKSampleMaxLog2 = 15;
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

// ------------------------------------------------------------------ CTA radix select
// The rank-th smallest (1-based) of the P keys in shared memory.  The keys' common
// leading bits (from their minimum and maximum) are known at once; the rest is taken in
// digits of up to 8 bits, each from a histogram whose adds are aggregated over the lanes
// of a warp that share a digit (distances crowd into few bins).  The digit holding the
// rank is found by warp 0 (eight bins a lane, a shuffle scan).  Every thread returns the
// key.  rank must lie in [1, P]; blockDim.x is a multiple of 32 and at most kKT.
__device__ unsigned int cta_select(const unsigned int* s_keys, int P, unsigned int rank, unsigned int* s_hist,
                                   unsigned int* s_state /* [3]: prefix, rank, known bits */) {
  __shared__ unsigned int s_mn[kKW], s_mx[kKW];
  const int tid = threadIdx.x, lane = tid & 31;
  unsigned int mn = 0xffffffffu, mx = 0u;
  for (int i = tid; i < P; i += blockDim.x) {
    const unsigned int key = s_keys[i];
    mn = min(mn, key);
    mx = max(mx, key);
  }
  mn = __reduce_min_sync(0xffffffffu, mn);
  mx = __reduce_max_sync(0xffffffffu, mx);
  if (lane == 0) { s_mn[tid >> 5] = mn; s_mx[tid >> 5] = mx; }
  __syncthreads();
  if (tid == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) { mn = min(mn, s_mn[w]); mx = max(mx, s_mx[w]); }
    const unsigned int diff = mn ^ mx;
    const int known = diff ? __clz(diff) : 32;
    s_state[0] = known == 32 ? mx : (known == 0 ? 0u : (mx >> (32 - known)) << (32 - known));
    s_state[1] = rank;
    s_state[2] = (unsigned int)known;
  }
  __syncthreads();
  bool first = true;   // the first histogram after the common bits is the crowded one
  while (s_state[2] < 32u) {
    const int known = (int)s_state[2];
    const unsigned int pre = s_state[0];
    const int nbits = min(8, 32 - known);
    const int sh = 32 - known - nbits;
    for (int i = tid; i < 256; i += blockDim.x) s_hist[i] = 0u;
    __syncthreads();
    if (first) {
      for (int base = 0; base < P; base += blockDim.x) {
        const int i = base + tid;
        unsigned int d = 0xffffffffu;
        if (i < P) d = (s_keys[i] >> sh) & ((1u << nbits) - 1u);   // every key shares the known bits
        const unsigned int grp = __match_any_sync(0xffffffffu, d);
        if (d != 0xffffffffu && (int)(__ffs(grp) - 1) == lane) atomicAdd(&s_hist[d], (unsigned int)__popc(grp));
      }
    } else {
      for (int i = tid; i < P; i += blockDim.x) {
        const unsigned int key = s_keys[i];
        if ((key >> (32 - known)) == (pre >> (32 - known))) atomicAdd(&s_hist[(key >> sh) & ((1u << nbits) - 1u)], 1u);
      }
    }
    first = false;
    __syncthreads();
    if (tid < 32) {
      unsigned int h[8], local = 0u;
#pragma unroll
      for (int j = 0; j < 8; ++j) { h[j] = s_hist[tid * 8 + j]; local += h[j]; }
      unsigned int incl = local;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (tid >= o) incl += y;
      }
      const unsigned int want = s_state[1];
      const unsigned int excl = incl - local;
      const bool mine = excl < want && want <= incl;
      if (mine) {
        unsigned int c = excl;
        int d = tid * 8 + 7;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          if (c + h[j] >= want) { d = tid * 8 + j; break; }
          c += h[j];
        }
        s_state[1] = want - c;
        s_state[0] = pre | ((unsigned int)d << sh);
      }
      if (__ballot_sync(0xffffffffu, mine) == 0u && tid == 0) s_state[1] = 1u;   // inconsistent counts: stop
      __syncwarp();
      if (tid == 0) s_state[2] = (unsigned int)(known + nbits);
    }
    __syncthreads();
  }
  const unsigned int r = s_state[0];
  __syncthreads();   // every thread has read the result before s_state is reused
  return r;
}

// ------------------------------------------------------------------ the sampled bracket
// One CTA per query: its distances to the ns = 2^ns_log2 evenly spread rows (i * n) / ns, in shared
// memory, and their order statistics of ranks jl (if jl >= 1) and jh (if jh <= ns): the
// bracket a < b of the fused pass (a = -1, below every distance, and b = +inf for ranks
// off the sample; a >= b from ties in the sample moves a just below b).
template <int PM>
__global__ void __launch_bounds__(kKT) knn_sample_kernel(const float* __restrict__ xp, long long n, int ns_log2,
                                                         const float* __restrict__ qp, const int* __restrict__ list,
                                                         int qbase, long long jl, long long jh, float* qa, float* qb) {
  extern __shared__ unsigned int s_d[];   // [ns]
  __shared__ unsigned int s_hist[256], s_state[3];
  const int ns = 1 << ns_log2;
  const int g = list[blockIdx.x] - qbase;
  float q[PM];
#pragma unroll
  for (int t = 0; t < PM; t += 4) {
    const float4 v = *reinterpret_cast<const float4*>(qp + (long long)g * PM + t);
    q[t] = v.x; q[t + 1] = v.y; q[t + 2] = v.z; q[t + 3] = v.w;
  }
  for (int j = threadIdx.x; j < ns; j += kKT) {
    const long long row = (long long)(((unsigned long long)j * (unsigned long long)n) >> ns_log2);
    float x[PM];
#pragma unroll
    for (int t = 0; t < PM; t += 4) {
      const float4 v = __ldg(reinterpret_cast<const float4*>(xp + row * PM + t));
      x[t] = v.x; x[t + 1] = v.y; x[t + 2] = v.z; x[t + 3] = v.w;
    }
    s_d[j] = __float_as_uint(sqdist<PM>(q, x));
  }
  __syncthreads();
  float a = -1.f, b = INFINITY;
  if (jl >= 1) a = __uint_as_float(cta_select(s_d, ns, (unsigned int)jl, s_hist, s_state));
  if (jh <= ns) b = __uint_as_float(cta_select(s_d, ns, (unsigned int)jh, s_hist, s_state));
  if (threadIdx.x == 0) {
    if (!(a < b)) a = b > 0.f ? nextafterf(b, -INFINITY) : -1.f;
    qa[g] = a;
    qb[g] = b;
  }
}

// ------------------------------------------------------------------ distance rows
// out[j][i] = d^2(query list[j], row i) for j < mq, i < n.  A CTA takes 32 queries (their
// coordinates in shared memory) and kKT consecutive rows, one row a thread.
template <int PM>
__global__ void __launch_bounds__(kKT) knn_rows_kernel(const float* __restrict__ xp, long long n,
                                                       const float* __restrict__ qp, const int* __restrict__ list,
                                                       int qbase, int mq, float* __restrict__ out) {
  __shared__ float s_q[32][PM];
  const int j0 = blockIdx.y * 32;
  for (int i = threadIdx.x; i < 32 * PM; i += kKT) {
    const int jj = i / PM, t = i - jj * PM;
    s_q[jj][t] = (j0 + jj < mq) ? qp[(long long)(list[j0 + jj] - qbase) * PM + t] : 0.f;
  }
  __syncthreads();
  const long long i = (long long)blockIdx.x * kKT + threadIdx.x;
  if (i >= n) return;
  float x[PM];
#pragma unroll
  for (int t = 0; t < PM; t += 4) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(xp + i * PM + t));
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
    out[(long long)(j0 + jj) * n + i] = d;
  }
}

__global__ void knn_offsets_kernel(long long* off, int S, long long len) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s <= S) off[s] = (long long)s * len;
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
  float negzero;          // -0.0f (the addend of the packed squares)
};

// Packed pairs of float32 (Blackwell's f32x2 arithmetic): two queries' differences,
// squares and sums in one instruction, each half rounded exactly as its scalar
// operation (round to nearest, no fused multiply-add).
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 pack2(float lo, float hi) {
  f32x2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void unpack2(f32x2 v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f32x2 sub2(f32x2 a, f32x2 b) {
  f32x2 r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
// The square e*e rounded on its own: an fma whose addend is -0 (e*e + -0 = e*e exactly,
// +0 included) taken from a kernel argument.  A plain packed multiply followed by the
// packed add is contracted into one fused operation by the code generator, which would
// round the sum once instead of twice.
__device__ __forceinline__ f32x2 sq2(f32x2 e, f32x2 negzero) {
  f32x2 r;
  asm("fma.rn.f32x2 %0, %1, %1, %2;" : "=l"(r) : "l"(e), "l"(negzero));
  return r;
}
__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b) {
  f32x2 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}

// Per-warp queue of compaction events in shared memory: a lane appends (d, row, query)
// with a shared-memory atomic and goes on; the warp flushes the queue to the queries'
// buffers (one global atomic a lane, all lanes at once) when it may not hold another row's
// events, and at the end.  So no lane waits on a global atomic inside the row loop.
constexpr int kQCap = 256;   // entries per warp
struct EventQueue {
  float* d;          // [kKW][kQCap]
  int* row;
  int* g;
  unsigned int* n;   // [kKW]
};

// The rare branch of the pass: distance d of query slot `slot` (query g) to `row` is <= b.
template <int QPT>
__device__ __forceinline__ void knn_event(const KnnPass& A, float d, float qa, float qb, int g, int slot,
                                          long long row, unsigned int (*s_cnt)[kKT * QPT],
                                          double (*s_sum)[kKT * QPT], const EventQueue& Qe, int warp) {
  if (d <= qa || d == qb) {
    const int cls = d <= qa ? 0 : 1;
    s_cnt[cls][slot] += 1u;
    if (A.f) {
      const double w = knn_weight(d, A.weight, A.eps);
      s_sum[2 * cls][slot] += w * (double)A.f[row];
      s_sum[2 * cls + 1][slot] += w;
    }
    if (A.labels) {
      const int lab = A.labels[row];
      if ((unsigned)lab < (unsigned)A.C) atomicAdd((cls == 0 ? A.vb : A.vt) + (long long)g * A.C + lab, 1u);
    }
  } else {
    const unsigned int e = atomicAdd(Qe.n + warp, 1u);
    Qe.d[warp * kQCap + e] = d;
    Qe.row[warp * kQCap + e] = (int)row;
    Qe.g[warp * kQCap + e] = g;
  }
}

// Flushes warp `warp`'s queue (called by all its lanes).
__device__ __forceinline__ void knn_flush(const KnnPass& A, const EventQueue& Qe, int warp, int lane) {
  __syncwarp();
  const unsigned int ne = Qe.n[warp];
  for (unsigned int e = lane; e < ne; e += 32) {
    const int g = Qe.g[warp * kQCap + e];
    const unsigned int pos = atomicAdd(A.zc + g, 1u);
    if (pos < (unsigned long long)A.cap) {
      A.zd[(long long)g * A.cap + pos] = Qe.d[warp * kQCap + e];
      A.zi[(long long)g * A.cap + pos] = Qe.row[warp * kQCap + e];
    }
  }
  __syncwarp();
  if (lane == 0) Qe.n[warp] = 0u;
  __syncwarp();
}

// Shared memory of the pass: two tiles of duplicated coordinates, the per-thread sums and
// counts.
constexpr int kTileF = 1024;   // floats of X per tile
template <int QPT>
constexpr size_t pass_smem_bytes() {
  return 2 * kTileF * sizeof(float2) + 4 * kKT * QPT * sizeof(double) + 2 * kKT * QPT * sizeof(unsigned int) +
         kKW * kQCap * (sizeof(float) + 2 * sizeof(int)) + kKW * sizeof(unsigned int);
}

template <int PM, int QPT>
__global__ void __launch_bounds__(kKT, 2) knn_pass_kernel(KnnPass A) {
  static_assert(QPT % 2 == 0 && QPT <= 4, "queries are processed in packed pairs");
  constexpr int kRowsTile = kTileF / PM;
  extern __shared__ __align__(16) unsigned char s_raw[];
  float2* s_x = reinterpret_cast<float2*>(s_raw);   // [2][kTileF], double-buffered
  double(*s_sum)[kKT * QPT] = reinterpret_cast<double(*)[kKT * QPT]>(s_raw + 2 * kTileF * sizeof(float2));
  unsigned char* s_after = s_raw + 2 * kTileF * sizeof(float2) + 4 * kKT * QPT * sizeof(double);
  unsigned int(*s_cnt)[kKT * QPT] = reinterpret_cast<unsigned int(*)[kKT * QPT]>(s_after);
  s_after += 2 * kKT * QPT * sizeof(unsigned int);
  EventQueue Qe;
  Qe.d = reinterpret_cast<float*>(s_after);
  Qe.row = reinterpret_cast<int*>(s_after + kKW * kQCap * sizeof(float));
  Qe.g = reinterpret_cast<int*>(s_after + kKW * kQCap * (sizeof(float) + sizeof(int)));
  Qe.n = reinterpret_cast<unsigned int*>(s_after + kKW * kQCap * (sizeof(float) + 2 * sizeof(int)));
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  if (lane == 0) Qe.n[warp] = 0u;
  const long long r0 = (long long)blockIdx.x * A.rows_per_chunk;
  const long long r1 = min(A.n, r0 + A.rows_per_chunk);
  const f32x2 nz2 = pack2(A.negzero, A.negzero);
  f32x2 q2[QPT / 2][PM];
  float qa[QPT], qb[QPT];
  int qid[QPT];
#pragma unroll
  for (int jp = 0; jp < QPT / 2; ++jp) {
    float q[2][PM];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int j = 2 * jp + h;
      const int slot = tid + j * kKT;
      const int li = blockIdx.y * (kKT * QPT) + slot;
      qid[j] = -1;
      qa[j] = 0.f;
      qb[j] = -INFINITY;   // no distance is <= -inf: an empty slot takes no branch
#pragma unroll
      for (int t = 0; t < PM; ++t) q[h][t] = 0.f;
      if (li < A.mq) {
        const int g = A.list[li] - A.qbase;
        qid[j] = g;
        qa[j] = A.qa[g];
        qb[j] = A.qb[g];
#pragma unroll
        for (int t = 0; t < PM; t += 4) {
          const float4 v = *reinterpret_cast<const float4*>(A.qp + (long long)g * PM + t);
          q[h][t] = v.x; q[h][t + 1] = v.y; q[h][t + 2] = v.z; q[h][t + 3] = v.w;
        }
      }
      s_cnt[0][slot] = 0u; s_cnt[1][slot] = 0u;
      s_sum[0][slot] = 0.0; s_sum[1][slot] = 0.0; s_sum[2][slot] = 0.0; s_sum[3][slot] = 0.0;
    }
#pragma unroll
    for (int t = 0; t < PM; ++t) q2[jp][t] = pack2(q[0][t], q[1][t]);
  }
  // the next tile's four floats a thread are loaded before the current tile is used and
  // stored (duplicated into both halves of a pair) after it
  const int ntiles = (int)((r1 - r0 + kRowsTile - 1) / kRowsTile);
  float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
  auto load_tile = [&](int t) {
    const long long rt = r0 + (long long)t * kRowsTile;
    const int nf = (int)min((long long)kRowsTile, r1 - rt) * PM;
    if (tid * 4 < nf) v = __ldg(reinterpret_cast<const float4*>(A.xp + rt * PM) + tid);
  };
  auto store_tile = [&](int t) {
    const long long rt = r0 + (long long)t * kRowsTile;
    const int nf = (int)min((long long)kRowsTile, r1 - rt) * PM;
    if (tid * 4 < nf) {
      float4* d = reinterpret_cast<float4*>(s_x + (t & 1) * kTileF + tid * 4);
      d[0] = make_float4(v.x, v.x, v.y, v.y);
      d[1] = make_float4(v.z, v.z, v.w, v.w);
    }
  };
  load_tile(0);
  store_tile(0);
  __syncthreads();
  for (int tile = 0; tile < ntiles; ++tile) {
    if (tile + 1 < ntiles) load_tile(tile + 1);
    const long long rt = r0 + (long long)tile * kRowsTile;
    const int rows = (int)min((long long)kRowsTile, r1 - rt);
    const float2* sx = s_x + (tile & 1) * kTileF;
#pragma unroll 2
    for (int r = 0; r < rows; ++r) {
      f32x2 x2[PM];
#pragma unroll
      for (int t = 0; t < PM; t += 2) {
        const ulonglong2 xv = reinterpret_cast<const ulonglong2*>(sx + r * PM)[t / 2];
        x2[t] = xv.x; x2[t + 1] = xv.y;
      }
      float d[QPT];
#pragma unroll
      for (int jp = 0; jp < QPT / 2; ++jp) {
        f32x2 e = sub2(q2[jp][0], x2[0]);
        f32x2 acc = sq2(e, nz2);
#pragma unroll
        for (int t = 1; t < PM; ++t) {
          e = sub2(q2[jp][t], x2[t]);
          acc = add2(acc, sq2(e, nz2));
        }
        unpack2(acc, d[2 * jp], d[2 * jp + 1]);
      }
      bool any = false;
#pragma unroll
      for (int j = 0; j < QPT; ++j) any |= d[j] <= qb[j];
      if (any) {
#pragma unroll
        for (int j = 0; j < QPT; ++j)
          if (d[j] <= qb[j])
            knn_event<QPT>(A, d[j], qa[j], qb[j], qid[j], tid + j * kKT, rt + r, s_cnt, s_sum, Qe, warp);
      }
      // room for one more row's events (at most 32 QPT) in the warp's queue
      __syncwarp();
      if (Qe.n[warp] > (unsigned int)(kQCap - 32 * QPT)) knn_flush(A, Qe, warp, lane);
    }
    if (tile + 1 < ntiles) store_tile(tile + 1);
    __syncthreads();
  }
  knn_flush(A, Qe, warp, lane);
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

// ------------------------------------------------------------------ outputs
struct KnnOut {
  const float* f;
  const int* labels;
  int C, weight;
  double eps;
  long long k;
  float* kth;
  double* pred;
  int* cls;
  double* votes;
};

// Writes the outputs of one query from its indicator's pieces: d_(k) (qv), the sums of
// w f and w below d_(k) and at it, the tie share ta / tb, and per class the points below
// d_(k) (lo_g[c] + s_lo[c]) and at it (eq_g[c] if eq_g, else s_eq[c]).  The class vote is
// (lo tb + eq ta) / tb: an exact integer ratio rounded once; the class, its arg max on
// the exact integers (the smallest class among equal votes).  Called by every thread.
__device__ void knn_emit(const KnnOut& O, long long out_i, float qv, double swf_lo, double sw_lo, double swf_eq,
                         double sw_eq, long long ta, long long tb, const unsigned int* lo_g, const unsigned int* eq_g,
                         const unsigned int* s_lo, const unsigned int* s_eq) {
  const int tid = threadIdx.x;
  if (tid == 0) {
    if (O.kth) O.kth[out_i] = qv;
    if (O.f) {
      const double share = (double)ta / (double)tb;
      O.pred[out_i] = (swf_lo + share * swf_eq) / (sw_lo + share * sw_eq);
    }
  }
  if (!O.labels) return;
  __shared__ long long s_bs[kKW];
  __shared__ int s_bc[kKW];
  long long best_s = -1;
  int best_c = 0x7fffffff;
  for (int c = tid; c < O.C; c += kKT) {
    const long long lo = (lo_g ? (long long)lo_g[c] : 0ll) + (long long)s_lo[c];
    const long long eq = eq_g ? (long long)eq_g[c] : (long long)s_eq[c];
    const long long score = lo * tb + eq * ta;
    if (O.votes) O.votes[out_i * O.C + c] = (double)score / (double)tb;
    if (score > best_s || (score == best_s && c < best_c)) { best_s = score; best_c = c; }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long os = __shfl_xor_sync(0xffffffffu, best_s, o);
    const int oc = __shfl_xor_sync(0xffffffffu, best_c, o);
    if (os > best_s || (os == best_s && oc < best_c)) { best_s = os; best_c = oc; }
  }
  if ((tid & 31) == 0) { s_bs[tid >> 5] = best_s; s_bc[tid >> 5] = best_c; }
  __syncthreads();
  if (tid == 0) {
    for (int w = 1; w < kKW; ++w)
      if (s_bs[w] > best_s || (s_bs[w] == best_s && s_bc[w] < best_c)) { best_s = s_bs[w]; best_c = s_bc[w]; }
    if (O.cls) O.cls[out_i] = best_c;
  }
}

__device__ void knn_emit_nan(const KnnOut& O, long long out_i) {
  if (threadIdx.x == 0) {
    if (O.kth) O.kth[out_i] = NAN;
    if (O.pred) O.pred[out_i] = NAN;
    if (O.cls) O.cls[out_i] = -1;
  }
  if (O.votes)
    for (int c = threadIdx.x; c < O.C; c += kKT) O.votes[out_i * O.C + c] = NAN;
}

// ------------------------------------------------------------------ the finish
struct KnnFin {
  const int* list;
  int qbase, mg;
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
  const int* status;      // non-finite coordinates / bad labels: outputs are NaN
  int* fail_list;         // queries whose check failed (group-relative + qbase), and their count
  unsigned int* fail_count;
  int final_round;        // 1: the plain form's bracket, which cannot fail: a failure is an internal error
  int* err;               // GBS_EINTERNAL recorded here
  KnnOut O;
};

// One CTA per query: checks the bracket, finds d_(k) in the compacted set (8-bit radix
// select on the float bits of d^2 >= +0, keys in dynamic shared memory) or at b, and
// combines the pass's sums and votes with the compacted points' shares.
__global__ void __launch_bounds__(kKT) knn_finish_kernel(KnnFin F) {
  extern __shared__ unsigned int s_key[];   // [cap]
  __shared__ unsigned int s_hist[256], s_state[3];
  __shared__ unsigned int s_vb[kKMaxClasses], s_vt[kKMaxClasses];
  __shared__ unsigned long long s_red_u[kKW];
  const int tid = threadIdx.x;
  const int g = F.list[blockIdx.x] - F.qbase;
  const long long out_i = F.qbase + g;
  const long long k = F.O.k;
  const long long below = F.cnt[2ll * g], tieb = F.cnt[2ll * g + 1];
  const long long P = F.zc[g];
  const float b = F.qb[g];
  if (*F.status != 0) {
    knn_emit_nan(F.O, out_i);
    return;
  }
  if (below >= k || below + P + tieb < k || P > F.cap) {   // the bracket failed its check
    if (F.final_round) {
      if (tid == 0) atomicCAS(F.err, 0, (int)GBS_EINTERNAL);
      knn_emit_nan(F.O, out_i);
    } else if (tid == 0) {
      F.fail_list[atomicAdd(F.fail_count, 1u)] = g + F.qbase;
    }
    return;
  }
  const bool at_b = below + P < k;   // d_(k) is b: every compacted point is below it
  const float* zd = F.zd + (long long)g * F.cap;
  const int* zi = F.zi + (long long)g * F.cap;
  unsigned int qbits;
  if (at_b) {
    qbits = __float_as_uint(b);
  } else {
    for (long long i = tid; i < P; i += kKT) s_key[i] = __float_as_uint(zd[i]);
    __syncthreads();
    qbits = cta_select(s_key, (int)P, (unsigned int)(k - below), s_hist, s_state);
  }
  const float qv = __uint_as_float(qbits);
  // the compacted points: below d_(k) (indicator 1) and at it (the tie share).  Their
  // positions are gathered densely first (into s_key, free after the select), so that the
  // float64 weights run on full warps: float64 arithmetic is narrow on this GPU and costs
  // per warp instruction, whatever the number of active lanes.
  const bool regress = F.O.f != nullptr, classify = F.O.labels != nullptr;
  __shared__ unsigned int s_n;
  __shared__ double s_red6[4][6];
  if (tid == 0) s_n = 0u;
  if (classify)
    for (int c = tid; c < F.O.C; c += kKT) { s_vb[c] = 0u; s_vt[c] = 0u; }
  __syncthreads();
  unsigned long long n_lo = 0, n_eq = 0;
  for (long long i = tid; i < P; i += kKT) {
    const float d = zd[i];
    const int lt = d < qv, eq = d == qv;
    if (!(lt | eq)) continue;
    n_lo += lt; n_eq += eq;
    if (regress) s_key[atomicAdd(&s_n, 1u)] = (unsigned int)i;
    if (classify) {
      const int lab = F.O.labels[zi[i]];
      if ((unsigned)lab < (unsigned)F.O.C) atomicAdd(lt ? &s_vb[lab] : &s_vt[lab], 1u);
    }
  }
  n_lo = cta_sum<unsigned long long>(n_lo, s_red_u);   // its barriers also publish s_n
  n_eq = cta_sum<unsigned long long>(n_eq, s_red_u);
  // sums (valid in thread 0): w f and w below d_(k) -- the compacted points and the pass's
  // points d <= a over its row chunks -- and at d_(k) among the compacted points, and the
  // pass's sums at b; four warps (one per SM sub-partition) share the float64 work
  double swf_lo = 0.0, sw_lo = 0.0, swf_eq = 0.0, sw_eq = 0.0, pb0 = 0.0, pb1 = 0.0;
  if (regress) {
    if (tid < 128) {
      double v[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
      const int cnt = (int)s_n;
      for (int t = tid; t < cnt; t += 128) {
        const unsigned int i = s_key[t];
        const float d = zd[i];
        const double w = knn_weight(d, F.O.weight, F.O.eps);
        const double wf = w * (double)F.O.f[zi[i]];
        if (d < qv) { v[0] += wf; v[1] += w; } else { v[2] += wf; v[3] += w; }
      }
      for (int ch = tid; ch < F.nchunks; ch += 128) {
        const double* pp = F.part + ((long long)ch * F.mg + g) * 4;
        v[0] += pp[0]; v[1] += pp[1]; v[4] += pp[2]; v[5] += pp[3];
      }
#pragma unroll
      for (int q = 0; q < 6; ++q) v[q] = warp_sum_f64(v[q]);
      if ((tid & 31) == 0)
#pragma unroll
        for (int q = 0; q < 6; ++q) s_red6[tid >> 5][q] = v[q];
    }
    __syncthreads();
    if (tid == 0) {
      double t6[6];
#pragma unroll
      for (int q = 0; q < 6; ++q) t6[q] = ((s_red6[0][q] + s_red6[1][q]) + s_red6[2][q]) + s_red6[3][q];
      swf_lo = t6[0]; sw_lo = t6[1]; swf_eq = t6[2]; sw_eq = t6[3]; pb0 = t6[4]; pb1 = t6[5];
    }
  }
  if (at_b) {   // every compacted point is below b; the ties are the pass's points at b
    knn_emit(F.O, out_i, qv, swf_lo, sw_lo, pb0, pb1, k - below - P, tieb, F.vb ? F.vb + (long long)g * F.O.C : nullptr,
             F.vt ? F.vt + (long long)g * F.O.C : nullptr, s_vb, s_vt);
  } else {
    knn_emit(F.O, out_i, qv, swf_lo, sw_lo, swf_eq, sw_eq, k - below - (long long)n_lo, (long long)n_eq,
             F.vb ? F.vb + (long long)g * F.O.C : nullptr, nullptr, s_vb, s_vt);
  }
}

// ------------------------------------------------------------------ the plain form's reduction
// CTA (chunk, row j) over the written distance row D[j] of query list[j], whose bracket
// is (just below d_(k), d_(k)]: the points below d_(k) and at it, counted and summed into
// the same per-chunk records the fused pass writes (its chunks of rows), so that the
// finish kernel completes the query by its "d_(k) is b" branch.
__global__ void __launch_bounds__(kKT) knn_reduce_rows_kernel(const float* __restrict__ D, const int* list, int qbase,
                                                              KnnPass A) {
  __shared__ double s_red[kKW];
  __shared__ unsigned long long s_red_u[kKW];
  const int tid = threadIdx.x;
  const int j = blockIdx.y;
  const int g = list[j] - qbase;
  const float qa = A.qa[g], qb = A.qb[g];
  const long long r0 = (long long)blockIdx.x * A.rows_per_chunk;
  const long long r1 = min(A.n, r0 + A.rows_per_chunk);
  const float* row = D + (long long)j * A.n;
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  unsigned long long n_lo = 0, n_eq = 0;
  for (long long i = r0 + tid; i < r1; i += kKT) {
    const float d = row[i];
    if (!(d <= qb)) continue;
    const int cls = d <= qa ? 0 : 1;
    n_lo += cls == 0; n_eq += cls == 1;
    if (A.f) {
      const double w = knn_weight(d, A.weight, A.eps);
      v[2 * cls] += w * (double)A.f[i];
      v[2 * cls + 1] += w;
    }
    if (A.labels) {
      const int lab = A.labels[i];
      if ((unsigned)lab < (unsigned)A.C) atomicAdd((cls == 0 ? A.vb : A.vt) + (long long)g * A.C + lab, 1u);
    }
  }
  n_lo = cta_sum<unsigned long long>(n_lo, s_red_u);
  n_eq = cta_sum<unsigned long long>(n_eq, s_red_u);
  if (A.f)
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] = cta_sum<double>(v[q], s_red);
  if (tid == 0) {
    if (n_lo) atomicAdd(A.cnt + 2ll * g, (unsigned int)n_lo);
    if (n_eq) atomicAdd(A.cnt + 2ll * g + 1, (unsigned int)n_eq);
    double* pp = A.part + ((long long)blockIdx.x * A.mg + g) * 4;
    pp[0] = v[0]; pp[1] = v[1]; pp[2] = v[2]; pp[3] = v[3];
  }
}

// The call's device status: an input error found by the preparation kernels takes
// precedence over what a select recorded on the same control block.
__global__ void knn_status_kernel(const int* knn_status, const int* err, Ctrl* ctrl) {
  if (threadIdx.x == 0) {
    if (*knn_status) atomicExch(&ctrl->status, *knn_status);
    else if (*err) atomicCAS(&ctrl->status, 0, *err);
  }
}

size_t up256k(size_t v) { return (v + 255) / 256 * 256; }

// Queries per thread of the pass: registers hold QPT * PM coordinates.
template <int PM> constexpr int qpt_of() { return PM <= 8 ? 4 : 2; }
int qpt_for(int PM) { return PM <= 8 ? 4 : 2; }

template <int PM>
gbs_status launch_pass_pm(const KnnPass& A, int nchunks, cudaStream_t s) {
  constexpr int QPT = qpt_of<PM>();
  constexpr int per = kKT * QPT;
  constexpr size_t smem = pass_smem_bytes<QPT>();
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(knn_pass_kernel<PM, QPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess) {
      cudaGetLastError();
      return GBS_ECUDA;
    }
    attr = true;
  }
  const dim3 grid((unsigned)nchunks, (unsigned)((A.mq + per - 1) / per));
  knn_pass_kernel<PM, QPT><<<grid, kKT, smem, s>>>(A);
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

gbs_status launch_rows(int PM, const float* xp, long long n, const float* qp, const int* list, int qbase, int mq,
                       float* out, cudaStream_t s) {
  const dim3 grid((unsigned)((n + kKT - 1) / kKT), (unsigned)((mq + 31) / 32));
  switch (PM) {
    case 4: knn_rows_kernel<4><<<grid, kKT, 0, s>>>(xp, n, qp, list, qbase, mq, out); break;
    case 8: knn_rows_kernel<8><<<grid, kKT, 0, s>>>(xp, n, qp, list, qbase, mq, out); break;
    case 16: knn_rows_kernel<16><<<grid, kKT, 0, s>>>(xp, n, qp, list, qbase, mq, out); break;
    default: knn_rows_kernel<32><<<grid, kKT, 0, s>>>(xp, n, qp, list, qbase, mq, out); break;
  }
  return cudaGetLastError() == cudaSuccess ? GBS_OK : GBS_ECUDA;
}

template <int PM>
gbs_status launch_sample_pm(const float* xp, long long n, int ns_log2, const float* qp, const int* list, int qbase,
                            int mq, long long jl, long long jh, float* qa, float* qb, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(knn_sample_kernel<PM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(unsigned int) << kKSampleMaxLog2)) != cudaSuccess) {
      cudaGetLastError();
      return GBS_ECUDA;
    }
    attr = true;
  }
  const size_t smem = sizeof(unsigned int) << ns_log2;
  knn_sample_kernel<PM><<<mq, kKT, smem, s>>>(xp, n, ns_log2, qp, list, qbase, jl, jh, qa, qb);
  return cudaGetLastError() == cudaSuccess ? GBS_OK : GBS_ECUDA;
}

gbs_status launch_sample(int PM, const float* xp, long long n, int ns_log2, const float* qp, const int* list,
                         int qbase, int mq, long long jl, long long jh, float* qa, float* qb, cudaStream_t s) {
  switch (PM) {
    case 4: return launch_sample_pm<4>(xp, n, ns_log2, qp, list, qbase, mq, jl, jh, qa, qb, s);
    case 8: return launch_sample_pm<8>(xp, n, ns_log2, qp, list, qbase, mq, jl, jh, qa, qb, s);
    case 16: return launch_sample_pm<16>(xp, n, ns_log2, qp, list, qbase, mq, jl, jh, qa, qb, s);
    default: return launch_sample_pm<32>(xp, n, ns_log2, qp, list, qbase, mq, jl, jh, qa, qb, s);
  }
}

}  // namespace

// ------------------------------------------------------------------ host driver
gbs_status knn_run(gbs_ctx* c, const float* X, long long n, int p, const float* Q, int m, long long k,
                   const float* f, int weight, double eps, const int* labels, int C, float* kth, double* pred,
                   int* cls, double* votes, cudaStream_t strm) {
  const int PM = p <= 4 ? 4 : (p <= 8 ? 8 : (p <= 16 ? 16 : 32));
  const int qpt = qpt_for(PM);
  const int G = std::min(m, kKGroup);   // queries per group
  // sampled start: sample ranks around k (4.5 binomial standard deviations and four ranks
  // of margin), the compaction buffer sized from the bracket's population (n/ns times a
  // Gamma(h - l) spacing: its mean plus 6 standard deviations and 12), and the sample size
  // 2^10 .. 2^15 (at most half the rows) with the least work per query: the sample plus
  // the bracket
  int ns_log2 = 0;
  long long jl = 0, jh = 0, cap = 256;
  if (c->cfg.knn_start == 0 && n >= kKMinN) {
    double best = 0.0;
    for (int lg = kKSampleMinLog2; lg <= kKSampleMaxLog2 && (2ll << lg) <= n; ++lg) {
      const long long ns = 1ll << lg;
      const double pk = (double)k / (double)n;
      const double sd = std::sqrt(ns * pk * (1.0 - pk));
      const long long l = (long long)std::floor(ns * pk - 4.5 * sd) - 4;
      const long long h = (long long)std::ceil(ns * pk + 4.5 * sd) + 4;
      // the bracket holds about n/ns times a Gamma(h - l) spacing of the sample
      const double span = (double)(std::min<long long>(h, ns + 1) - std::max<long long>(l, 0));
      const double mean = span / ns * (double)n;
      long long cp = (long long)std::ceil((span + 6.0 * std::sqrt(span) + 12.0) / ns * (double)n + 256.0);
      cp = std::max<long long>(4096, (cp + 255) / 256 * 256);
      if (cp > 49152) continue;   // the finish keeps the keys in shared memory (192 KiB)
      // per element, the bracket costs the fused pass and the finish about 1.5 times what a
      // sampled distance costs (measured on GB300 at n = 2^20, p = 8)
      const double cost = (double)ns + 1.5 * mean;
      if (ns_log2 == 0 || cost < best) {
        best = cost; ns_log2 = lg; jl = l; jh = h; cap = cp;
      }
    }
  }
  const bool sampled = ns_log2 > 0;
  if (!sampled) cap = 256;
  // row chunks of the pass: about four CTAs per resident slot (two per SM)
  const int nqb_full = (G + kKT * qpt - 1) / (kKT * qpt);
  long long nch = std::max<long long>(1, ((long long)c->num_sms * 2 * 4 + nqb_full - 1) / nqb_full);
  long long rpc = (n + nch - 1) / nch;
  rpc = (rpc + kKTile - 1) / kKTile * kKTile;
  nch = (n + rpc - 1) / rpc;
  // distance rows of the plain form: at most 1 GiB, at most a group, per batch
  const long long batch_rows = std::max<long long>(1, std::min<long long>(G, kKRowsBytes / (4 * n)));
  // workspace: xp | qp | qa | qb | cnt | zc | zd | zi | part | vb | vt | rows | off | kthb | list | fail | status
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
  const size_t o_rows = o; o = up256k(o + sizeof(float) * (size_t)batch_rows * n);
  const size_t o_off = o; o = up256k(o + sizeof(long long) * ((size_t)batch_rows + 1));
  const size_t o_kthb = o; o = up256k(o + sizeof(float) * (size_t)batch_rows);
  const size_t o_list = o; o = up256k(o + sizeof(int) * (size_t)G);
  const size_t o_fail = o; o = up256k(o + sizeof(int) * (size_t)G);
  const size_t o_st = o; o = up256k(o + sizeof(int) * 8);
  const size_t bytes = o;
  if (!c->knn_buf || c->knn_bytes < bytes) {
    if (c->knn_buf) {
      cudaDeviceSynchronize();
      cudaFree(c->knn_buf);
      c->knn_buf = nullptr;
      c->knn_bytes = 0;
    }
    void* ptr = nullptr;
    if (cudaMalloc(&ptr, bytes) != cudaSuccess) {
      cudaGetLastError();
      return GBS_ENOMEM;
    }
    c->knn_buf = ptr;
    c->knn_bytes = bytes;
  }
  gbs_status st = gbs_internal_ensure(c, seg_workspace_bytes((int)batch_rows));
  if (st != GBS_OK) return st;
  st = reserve_select(c, n, 4);   // a few failed queries take the single-array select
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
  float* kthb = reinterpret_cast<float*>(B + o_kthb);
  int* list = reinterpret_cast<int*>(B + o_list);
  int* fail = reinterpret_cast<int*>(B + o_fail);
  int* status = reinterpret_cast<int*>(B + o_st);                       // [0] input status, [1] internal error
  unsigned int* fcount = reinterpret_cast<unsigned int*>(status + 2);   // [2] failed queries
  auto check = [&]() { return cudaGetLastError() == cudaSuccess ? GBS_OK : GBS_ECUDA; };
  for (int e = 0; e < 2; ++e)
    if (!c->knn_ev[e] && cudaEventCreate(&c->knn_ev[e]) != cudaSuccess) return GBS_ECUDA;
  c->knn_last = gbs_knn_stats{};
  c->knn_last.queries = m;

  if (cudaMemsetAsync(status, 0, sizeof(int) * 8, strm) != cudaSuccess ||
      cudaMemsetAsync(c->rs, 0, sizeof(gbs_run_stats), strm) != cudaSuccess)
    return GBS_ECUDA;
  knn_pad_kernel<<<(unsigned)std::min<long long>((n * PM + 255) / 256, (long long)c->num_sms * 16), 256, 0, strm>>>(
      X, n, p, PM, xp, status);
  if (labels)
    knn_labels_kernel<<<(unsigned)std::min<long long>((n + 255) / 256, (long long)c->num_sms * 8), 256, 0, strm>>>(
        labels, n, C, status);
  if ((st = check()) != GBS_OK) return st;

  KnnOut O;
  O.f = f; O.labels = labels; O.C = C; O.weight = weight; O.eps = eps; O.k = k;
  O.kth = kth; O.pred = pred; O.cls = cls; O.votes = votes;
  KnnPass A;
  A.xp = xp; A.n = n; A.rows_per_chunk = rpc; A.qp = qp;
  A.qa = qa; A.qb = qb; A.f = f; A.labels = labels; A.C = C; A.weight = weight; A.eps = eps;
  A.cnt = cnt; A.zc = zc; A.zd = zd; A.zi = zi; A.cap = cap; A.part = part; A.vb = vb; A.vt = vt;
  A.negzero = -0.0f;
  KnnFin F;
  F.nchunks = (int)nch; F.qb = qb; F.cnt = cnt; F.zc = zc; F.zd = zd; F.zi = zi; F.cap = cap;
  F.part = part; F.vb = vb; F.vt = vt; F.status = status; F.fail_list = fail; F.fail_count = fcount; F.O = O;
  F.err = status + 1; F.final_round = 0;
  const size_t fin_smem = sizeof(unsigned int) * (size_t)cap;
  if (cudaFuncSetAttribute(knn_finish_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)std::max<size_t>(fin_smem, 1024)) != cudaSuccess) {
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
    A.qbase = q0; A.mg = mg; F.qbase = q0; F.mg = mg;
    int nfail = mg;
    const int* flist = list;
    if (sampled) {
      if ((st = launch_sample(PM, xp, n, ns_log2, qp, list, q0, mg, jl, jh, qa, qb, strm)) != GBS_OK) return st;
      knn_zero_kernel<<<(unsigned)(((long long)mg * (3 + 2 * (labels ? C : 0)) + 255) / 256), 256, 0, strm>>>(
          list, mg, q0, cnt, zc, vb, vt, labels ? C : 0);
      if ((st = check()) != GBS_OK) return st;
      A.list = list; A.mq = mg;
      if (cudaEventRecord(c->knn_ev[0], strm) != cudaSuccess) return GBS_ECUDA;
      if ((st = launch_pass(PM, A, (int)nch, strm)) != GBS_OK) return st;
      if (cudaEventRecord(c->knn_ev[1], strm) != cudaSuccess) return GBS_ECUDA;
      if (q0 == 0) ++npass;
      if (cudaMemsetAsync(fcount, 0, sizeof(unsigned int), strm) != cudaSuccess) return GBS_ECUDA;
      F.list = list; F.final_round = 0;
      knn_finish_kernel<<<mg, kKT, fin_smem, strm>>>(F);
      if ((st = check()) != GBS_OK) return st;
      unsigned int h_fail = 0;
      if (cudaMemcpyAsync(&h_fail, fcount, sizeof(h_fail), cudaMemcpyDeviceToHost, strm) != cudaSuccess ||
          cudaStreamSynchronize(strm) != cudaSuccess)
        return GBS_ECUDA;
      nfail = (int)h_fail;
      flist = fail;
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, c->knn_ev[0], c->knn_ev[1]) == cudaSuccess) {
        c->knn_last.pass_ms += ms;
        c->knn_last.pass_launches += 1;
      }
    }
    // the plain form for the rest: whole distance rows, d_(k) selected from each, then
    // the indicator reduced from the written rows
    for (int j0 = 0; j0 < nfail; j0 += (int)batch_rows) {
      const int mb = std::min<int>((int)batch_rows, nfail - j0);
      const int* bl = flist + j0;
      if ((st = launch_rows(PM, xp, n, qp, bl, q0, mb, rows, strm)) != GBS_OK) return st;
      if (mb <= 8) {
        for (int j = 0; j < mb; ++j)
          if ((st = run_select(c, rows + (size_t)j * n, n, k, kthb + j, kModeSelect, 0.0, 0.0, nullptr, nullptr,
                               strm)) != GBS_OK)
            return st;
      } else {
        knn_offsets_kernel<<<(mb + 1 + 255) / 256, 256, 0, strm>>>(off, mb, n);
        if ((st = check()) != GBS_OK) return st;
        SegLaunch L;
        if ((st = seg_attach_workspace(c, mb, &L)) != GBS_OK) return st;
        L.x = rows; L.off = off; L.S = mb; L.kk = nullptr; L.ctrl = c->ctrl; L.mask = nullptr; L.kk2 = nullptr;
        L.k_const = k; L.k2_const = 0; L.out = kthb; L.out2 = nullptr; L.outsum = nullptr; L.flags = nullptr;
        if ((st = seg_launch(c, L, c->seg_variant, strm)) != GBS_OK) return st;
      }
      knn_known_bracket_kernel<<<(mb + 255) / 256, 256, 0, strm>>>(bl, mb, q0, kthb, qa, qb);
      knn_zero_kernel<<<(unsigned)(((long long)mb * (3 + 2 * (labels ? C : 0)) + 255) / 256), 256, 0, strm>>>(
          bl, mb, q0, cnt, zc, vb, vt, labels ? C : 0);
      knn_reduce_rows_kernel<<<dim3((unsigned)nch, (unsigned)mb), kKT, 0, strm>>>(rows, bl, q0, A);
      F.list = bl; F.final_round = 1;
      knn_finish_kernel<<<mb, kKT, fin_smem, strm>>>(F);
      if ((st = check()) != GBS_OK) return st;
    }
    if (q0 == 0 && nfail > 0) npass += 2;   // the distance rows written and read back
    c->knn_last.plain_queries += nfail;
  }
  knn_status_kernel<<<1, 32, 0, strm>>>(status, status + 1, c->ctrl);
  if ((st = check()) != GBS_OK) return st;
  c->knn_last.passes = npass;
  c->last_stream = strm;
  return GBS_OK;
}

}  // namespace gbs

void gbs_internal_release_knn(gbs_ctx* c) {
  for (int e = 0; e < 2; ++e)
    if (c->knn_ev[e]) {
      cudaEventDestroy(c->knn_ev[e]);
      c->knn_ev[e] = nullptr;
    }
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
  return gbs::knn_run(c, X, n, p, Q, m, k, f, weight, eps, nullptr, 0, kth_d2, pred, nullptr, nullptr,
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
  return gbs::knn_run(c, X, n, p, Q, m, k, nullptr, 0, 0.0, labels, n_classes, kth_d2, nullptr, cls, votes,
                      static_cast<cudaStream_t>(stream));
}

extern "C" gbs_status gbs_knn_last_stats(gbs_ctx* c, gbs_knn_stats* out) {
  if (!c || !out) return GBS_EINVAL;
  gbs::DeviceGuard g(c->device);
  if (!g.ok) return GBS_ECUDA;
  if (c->knn_buf && cudaStreamSynchronize(c->last_stream) != cudaSuccess) {
    cudaGetLastError();
    return GBS_ECUDA;
  }
  *out = c->knn_last;
  return GBS_OK;
}
