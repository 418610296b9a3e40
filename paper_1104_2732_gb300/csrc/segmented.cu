// Segmented batched selection: out[s] = x_(k_s) of x[off[s], off[s+1]) for thousands of
// arrays of uneven sizes in one persistent launch.
//
// Each CTA takes whole segments from a work queue ordered largest first (a small
// schedule kernel buckets the segments by size).  A segment that fits in shared memory
// is loaded once and radix-selected there.  A larger one runs the cutting plane of
// Algorithm 1 (Sec. 3) with CTA-wide reductions: pass 0 (extremes, sum), then one fused
// cost + count pass per iterate; the pass that sees a bracket small enough for shared
// memory compacts it there, or one of at most n/2 elements into the CTA's own
// device-memory region, and the answer is radix-selected inside it (the hybrid of
// Sec. 3; from device memory the rounds move to shared memory once the chosen digit's
// elements fit there).  No CTA waits on another, so the launch needs no grid-wide barrier and the
// whole call (schedule + kernel) can be captured in a CUDA graph.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdint>

#include "api_internal.h"
#include "bracket.cuh"
#include "common.cuh"
#include "elem.cuh"
#include "segmented.cuh"

namespace gbs {

namespace {

// Segments are queued largest first: by 8 buckets per octave of the size (the exponent of
// the float32 image of n and its top three mantissa bits, a monotone key), so the largest
// segments start first even within one power of two.
constexpr int kSchedBuckets = 64 * 8;
__device__ __forceinline__ int sched_bucket(long long n) {
  if (n <= 1) return 0;
  const unsigned int u = __float_as_uint((float)n);   // (float)n is monotone in n, so is the key
  return (int)((u >> 20) - (127u << 3));              // 8 * exponent + top 3 mantissa bits
}
constexpr long long kSegGlobalDiv = 2;   // device-memory compaction once pop <= n / 2
// smallest segment whose median starts from a learned bracket: every segment too large for
// shared memory (in a sweep of 2^13..2^16 on 4096 normal arrays, all gave identical results
// and 2^13 the shortest batch)
constexpr long long kSegLearnMinN = 1ll << 13;

// Buckets segment ids by size, largest bucket first; also checks offsets.
__global__ void seg_schedule_kernel(const long long* __restrict__ off, int S, int* __restrict__ order,
                                    const int* __restrict__ mask, Ctrl* ctrl) {
  __shared__ unsigned int hist[kSchedBuckets];
  __shared__ unsigned int base[kSchedBuckets];
  for (int i = threadIdx.x; i < kSchedBuckets; i += blockDim.x) hist[i] = 0;
  __syncthreads();
  for (int s = threadIdx.x; s < S; s += blockDim.x) {
    if (mask && !mask[s]) continue;
    const long long n = off[s + 1] - off[s];
    if (n < 0) atomicCAS(&ctrl->status, 0, (int)GBS_EINVAL);
    atomicAdd(&hist[kSchedBuckets - 1 - sched_bucket(n)], 1u);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int acc = 0;
    for (int i = 0; i < kSchedBuckets; ++i) {
      base[i] = acc;
      acc += hist[i];
    }
    ctrl->w_len = acc;
  }
  __syncthreads();
  for (int s = threadIdx.x; s < S; s += blockDim.x) {
    if (mask && !mask[s]) continue;
    const long long n = off[s + 1] - off[s];
    order[atomicAdd(&base[kSchedBuckets - 1 - sched_bucket(n)], 1u)] = s;
  }
}

// CTA-wide sum of six values for a CTA of B threads (fixed order).
template <int B>
__device__ __forceinline__ Sum6 cta_sum6(Sum6 v, Sum6* scratch /* [B/32 + 1] */) {
  constexpr int NW = B / 32;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int i = 0; i < 5; ++i) v.u[i] += __shfl_xor_sync(0xffffffffu, v.u[i], o);
    v.d += __shfl_xor_sync(0xffffffffu, v.d, o);
  }
  __syncthreads();
  if (lane == 0) scratch[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    Sum6 r = scratch[0];
    for (int i = 1; i < NW; ++i) {
#pragma unroll
      for (int q = 0; q < 5; ++q) r.u[q] += scratch[i].u[q];
      r.d += scratch[i].d;
    }
    scratch[NW] = r;
  }
  __syncthreads();
  return scratch[NW];
}

// Calls f(element) on every element of xs[0, n) handled by this thread of the CTA.
template <int B, typename Fn>
__device__ __forceinline__ void cta_stream(const float* __restrict__ xs, const Geometry<float>& g, Fn& f) {
  const int tid = threadIdx.x;
  if (tid < g.head) f(xs[tid]);
  if (tid < g.n - g.tail0) f(xs[g.tail0 + tid]);
  const float4* xv = reinterpret_cast<const float4*>(xs + g.head);
  long long v = tid;
  for (; v + 3 * B < g.nv; v += 4 * B) {
    float4 r[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) r[u] = __ldcs(xv + v + u * B);
#pragma unroll
    for (int u = 0; u < 4; ++u) Ops<float>::each(r[u], f);
  }
  for (; v < g.nv; v += B) {
    const float4 r = __ldcs(xv + v);
    Ops<float>::each(r, f);
  }
}

// As cta_stream, and appends every element with keep(element) to zb (shared memory or
// this CTA's device-memory region, counter *cnt; appends past zcap are counted, not
// written, so the caller's count check catches them).  Per warp iteration (16 elements a
// lane) one atomic reserves the warp's kept elements and a prefix sum over the lanes'
// counts gives each lane its place: a lane writes its own kept elements one after
// another (no dependent chain of ballots over the element slots).
template <int B, typename Fn, typename Keep>
__device__ __forceinline__ void cta_stream_compact(const float* __restrict__ xs, const Geometry<float>& g, Fn& f,
                                                   Keep& keep, float* zb, unsigned int zcap, unsigned int* cnt) {
  const int tid = threadIdx.x, lane = tid & 31;
  if (tid < g.head) {
    const float e = xs[tid];
    f(e);
    if (keep(e)) {
      const unsigned int q = atomicAdd(cnt, 1u);
      if (q < zcap) zb[q] = e;
    }
  }
  if (tid < g.n - g.tail0) {
    const float e = xs[g.tail0 + tid];
    f(e);
    if (keep(e)) {
      const unsigned int q = atomicAdd(cnt, 1u);
      if (q < zcap) zb[q] = e;
    }
  }
  const float4* xv = reinterpret_cast<const float4*>(xs + g.head);
  for (long long w0 = tid - lane; w0 < g.nv; w0 += 4 * B) {
    float4 r[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const long long i = w0 + lane + (long long)u * B;
      if (i < g.nv) r[u] = __ldcs(xv + i);
    }
    unsigned int kmask = 0;   // bit 4u + e: this lane keeps element e of vector u
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const long long i = w0 + lane + (long long)u * B;
      if (i < g.nv) {
        Ops<float>::each(r[u], f);
#pragma unroll
        for (int e = 0; e < 4; ++e) kmask |= (keep(Ops<float>::get(r[u], e)) ? 1u : 0u) << (u * 4 + e);
      }
    }
    // each lane writes its kept elements at its place after those of the lower lanes
    const unsigned int kc = (unsigned int)__popc(kmask);
    unsigned int incl = kc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const unsigned int total = __shfl_sync(0xffffffffu, incl, 31);
    if (total) {
      unsigned int pos = 0;
      if (lane == 31) pos = atomicAdd(cnt, total);
      pos = __shfl_sync(0xffffffffu, pos, 31) + (incl - kc);
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const bool kk = (kmask >> (u * 4 + e)) & 1u;
          if (kk && pos < zcap) zb[pos] = Ops<float>::get(r[u], e);
          pos += kk ? 1u : 0u;
        }
    }
  }
}

// As cta_stream_compact for the elements of (a, b], staged through shared memory (`slots`,
// 16 floats per thread): a lane stores its kept elements in its own column of its warp's
// 512 slots (slot q of lane L at 32 q + L), the warp issues the loads of its next
// iteration, and only then reserves room for its kept elements with one atomic and has
// each lane copy its column out after those of the lower lanes, four slots at a time.
// The next vectors are in flight during the reservation and the copy-out; a column is
// written and read by its own lane only.
template <int B, typename Fn>
__device__ __forceinline__ void cta_stream_compact_staged(const float* __restrict__ xs, const Geometry<float>& g,
                                                          Fn& f, float a, float b, float* slots, float* zb,
                                                          unsigned int zcap, unsigned int* cnt) {
  const int tid = threadIdx.x, lane = tid & 31;
  auto scalar = [&](float e) {
    f(e);
    if ((e > a) & (e <= b)) {
      const unsigned int q = atomicAdd(cnt, 1u);
      if (q < zcap) zb[q] = e;
    }
  };
  if (tid < g.head) scalar(xs[tid]);
  if (tid < g.n - g.tail0) scalar(xs[g.tail0 + tid]);
  const float4* xv = reinterpret_cast<const float4*>(xs + g.head);
  const unsigned int col = smem_u32(slots + (tid >> 5) * 512 + lane);
  long long w0 = tid - lane;
  float4 r[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const long long i = w0 + lane + (long long)u * B;
    if (i < g.nv) r[u] = __ldcs(xv + i);
  }
  for (; w0 < g.nv; w0 += 4 * B) {
    unsigned int off = col;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const long long i = w0 + lane + (long long)u * B;
      if (i < g.nv) {
        Ops<float>::each(r[u], f);
#pragma unroll
        for (int e = 0; e < 4; ++e) keep_only(Ops<float>::get(r[u], e), a, b, off);
      }
    }
    const unsigned int kc = (off - col) >> 7;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const long long i = w0 + 4 * B + lane + (long long)u * B;
      if (i < g.nv) r[u] = __ldcs(xv + i);
    }
    unsigned int incl = kc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const unsigned int total = __shfl_sync(0xffffffffu, incl, 31);
    if (total) {
      unsigned int pos = 0;
      if (lane == 31) pos = atomicAdd(cnt, total);
      pos = __shfl_sync(0xffffffffu, pos, 31) + (incl - kc);
      const unsigned int maxk = __reduce_max_sync(0xffffffffu, kc);
      for (unsigned int q = 0; q < maxk; q += 4) {
        float v[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) ld_shared(col + min(q + j, 15u) * 128u, v[j]);   // the column's 16 slots
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (q + j < kc && pos + q + j < zcap) zb[pos + q + j] = v[j];
      }
    }
  }
}

// State of an in-CTA radix select (shared memory).
struct RadixState {
  unsigned int hist[256];
  uint32_t prefix;          // the key's known leading bits
  int known;                // how many
  unsigned long long rank;  // rank among the elements with that prefix (0 flags an inconsistency)
  unsigned int bucket;      // elements in the digit chosen last
  unsigned int cnt;         // append counter of the gather
  // a second rank selected with the same histograms while both share a prefix
  uint32_t prefix2;
  unsigned long long rank2;
  unsigned int bucket2;
  int split;                // 1: the two ranks' digits differed in the last round
  // without a filter: the leading key bits every element shares (set by the caller)
  int known0;
  uint32_t prefix0;
};

constexpr int kRadixV = 2;   // 16-byte loads in flight per thread in the radix sweeps

// Whether an element (value v, key) takes part in a round: in (a, b] when filtering, and
// its key starts with the known prefix.
__device__ __forceinline__ bool radix_takes(float v, uint32_t key, bool filter, float a, float b, int known,
                                            uint32_t prefix) {
  return (!filter || ((v > a) && (v <= b))) && (known == 0 || (key >> (32 - known)) == prefix);
}

// Calls fn(valid, value) on every element of buf[0, m) (16-byte aligned) for this warp's
// share, kRadixV 16-byte loads in flight per lane; the warp loop is uniform (fn may use
// warp collectives), and the last m mod 4 elements go to warp 0.
template <int B, typename Fn>
__device__ __forceinline__ void radix_sweep(const float* buf, int m, Fn& fn) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float4* b4 = reinterpret_cast<const float4*>(buf);
  const int m4 = m >> 2;
  for (int base = warp * 32; base < m4; base += B * kRadixV) {
    float4 v[kRadixV];
#pragma unroll
    for (int u = 0; u < kRadixV; ++u) {
      const int i = base + u * B + lane;
      v[u] = i < m4 ? b4[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < kRadixV; ++u) {
      const bool ok = base + u * B + lane < m4;
      fn(ok, v[u].x);
      fn(ok, v[u].y);
      fn(ok, v[u].z);
      fn(ok, v[u].w);
    }
  }
  if (warp == 0 && (m & 3)) {
    const bool ok = lane < (m & 3);
    fn(ok, ok ? buf[4 * m4 + lane] : 0.f);
  }
}

// Histogram of the next digit (bits [sh, sh + 8) of the key) over the elements of buf that
// take part.
// A lane adds its elements' digits one by one to the shared histogram, except the digit
// it met twice in a row most recently, which it counts in a register (runs of tied values
// would serialise on one counter); no warp-wide votes, so no dependent chain of them.
template <int B>
__device__ __forceinline__ void radix_hist(const float* buf, int m, bool filter, float a, float b, int known,
                                           uint32_t prefix, int sh, unsigned int dmask, unsigned int* hist) {
  unsigned int hot = 0xffffffffu, last = 0xffffffffu, hcnt = 0;
  auto fn = [&](bool ok, float v) {
    const uint32_t key = ukey(v);
    const bool in = ok && radix_takes(v, key, filter, a, b, known, prefix);
    const unsigned int d = (key >> sh) & dmask;
    const bool hh = in && d == hot;
    const bool at = in && !hh;
    const bool sw = at && d == last;
    hcnt += hh ? 1u : 0u;
    if (at) atomicAdd(&hist[d], 1u);
    if (sw && hcnt) atomicAdd(&hist[hot], hcnt);
    hot = sw ? d : hot;
    hcnt = sw ? 0u : hcnt;
    last = at ? d : last;
  };
  radix_sweep<B>(buf, m, fn);
  if (hcnt) atomicAdd(&hist[hot], hcnt);
}

// Appends the elements of buf that take part to zs (counter *cnt; any order; at most cap
// are written).
template <int B>
__device__ __forceinline__ void radix_gather(const float* buf, int m, bool filter, float a, float b, int known,
                                             uint32_t prefix, float* zs, unsigned int cap, unsigned int* cnt) {
  const int lane = threadIdx.x & 31;
  auto fn = [&](bool ok, float v) {
    const bool t = ok && radix_takes(v, ukey(v), filter, a, b, known, prefix);
    const unsigned int bal = __ballot_sync(0xffffffffu, t);
    if (bal) {
      unsigned int b0 = 0;
      if (lane == 0) b0 = atomicAdd(cnt, (unsigned int)__popc(bal));
      b0 = __shfl_sync(0xffffffffu, b0, 0);
      const unsigned int pos = b0 + __popc(bal & ((1u << lane) - 1u));
      if (t && pos < cap) zs[pos] = v;
    }
  };
  radix_sweep<B>(buf, m, fn);
}

// Known leading key bits of (a, b] (all 32 when a single key lies in it); without a filter
// the bits every element shares (known0, prefix0).  (a, b] under IEEE comparison on keys: a
// zero end takes the key of +0 (x > -0 and x > +0 both exclude the zeros, x <= -0 and
// x <= +0 both include them).
__device__ __forceinline__ void radix_known(bool filter, float a, float b, int known0, uint32_t prefix0, int* known,
                                            uint32_t* prefix) {
  *known = known0;
  *prefix = prefix0;
  if (filter) {
    const uint32_t lo = ukey(a == 0.f ? 0.f : a) + 1, hi = ukey(b == 0.f ? 0.f : b);
    const uint32_t diff = lo ^ hi;
    *known = diff == 0 ? 32 : __clz(diff);
    *prefix = *known == 0 ? 0u : (*known == 32 ? hi : (hi >> (32 - *known)));
  }
}

// One round's digit for a rank by warp 0 from the histogram h[] (lane L holds bins
// 8L..8L+7 and the inclusive count incl of bins up to its last): the lane holding the
// rank writes the new prefix, the rank within the digit and the digit's count.
__device__ __forceinline__ void radix_pick(const unsigned int (&h)[8], unsigned long long incl, unsigned int local,
                                           unsigned long long want, uint32_t prefix, int nbits, uint32_t* o_prefix,
                                           unsigned long long* o_rank, unsigned int* o_bucket, bool* found) {
  const int lane = threadIdx.x & 31;
  const unsigned long long excl = incl - local;
  const bool mine = excl < want && want <= incl;
  *found = __ballot_sync(0xffffffffu, mine) != 0;
  if (mine) {
    unsigned long long c = excl;
    int d = 0;
    unsigned int bk = 0;
    for (int j = 0; j < 8; ++j) {
      if (c + h[j] >= want) { d = lane * 8 + j; bk = h[j]; break; }
      c += h[j];
    }
    *o_rank = want - c;
    *o_prefix = (prefix << nbits) | (uint32_t)d;
    *o_bucket = bk;
  }
}

// The radix rounds from the state in st (known bits, prefix, rank) over cur[0, mc), which is
// buf[0, m) or, once gathered, zs: 8-bit digits of the elements that lie in (a, b] (all when
// !filter) and start with the prefix.  When cur is buf in device memory, zs (shared memory,
// cap elements, else nullptr) takes the elements of the chosen digit once they fit, and
// the later rounds run there.  The selected key ends in st.prefix.
template <int B>
__device__ void radix_rounds(const float* buf, int m, const float* cur, int mc, bool filter, float a, float b,
                             float* zs, int cap, RadixState& st) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  while (st.known < 32) {
    const int known = st.known;
    const uint32_t prefix = st.prefix;
    const int nbits = (32 - known) < 8 ? (32 - known) : 8;
    const int sh = 32 - known - nbits;
    const unsigned int dmask = (1u << nbits) - 1u;
    for (int i = tid; i < 256; i += B) st.hist[i] = 0;
    __syncthreads();
    radix_hist<B>(cur, mc, filter, a, b, known, prefix, sh, dmask, st.hist);
    __syncthreads();
    if (warp == 0) {
      unsigned int h[8];
      unsigned int local = 0;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        h[j] = st.hist[lane * 8 + j];
        local += h[j];
      }
      unsigned long long incl = local;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      bool found;
      radix_pick(h, incl, local, st.rank, prefix, nbits, &st.prefix, &st.rank, &st.bucket, &found);
      if (lane == 0) {
        st.known = known + nbits;
        st.cnt = 0;
        if (!found) {   // no bin holds the rank: inconsistent counts, flagged by rank 0
          st.known = 32;
          st.prefix = 0;
          st.rank = 0;
          st.bucket = 0xffffffffu;
        }
      }
    }
    __syncthreads();
    if (zs != nullptr && cur == buf && st.known < 32 && st.bucket <= (unsigned int)cap) {
      radix_gather<B>(buf, m, filter, a, b, st.known, st.prefix, zs, (unsigned int)cap, &st.cnt);
      __syncthreads();
      cur = zs;
      mc = (int)min(st.cnt, (unsigned int)cap);   // equal to the bucket's count
    }
  }
}

// Radix select inside the CTA: the rank-th (1-based) smallest, in totalOrder, of the
// elements of buf[0, m) that lie in (a, b] (all of them when !filter).  Returns the
// element's key (st.rank == 0 afterwards flags inconsistent counts).  8-bit digits from
// the highest bit where the bracket's keys differ; zs and cap as for radix_rounds.
template <int B>
__device__ __noinline__ uint32_t radix_select(const float* buf, int m, unsigned long long rank, bool filter, float a,
                                              float b, float* zs, int cap, RadixState& st) {
  if (threadIdx.x == 0) {
    radix_known(filter, a, b, st.known0, st.prefix0, &st.known, &st.prefix);
    st.rank = rank;
  }
  __syncthreads();
  radix_rounds<B>(buf, m, buf, m, filter, a, b, zs, cap, st);
  return st.prefix;
}

// Two ranks at once (as radix_select for each): the rounds share their histograms while
// both ranks fall in the same digit, then each continues alone from where they parted.
// The keys land in *key1 and *key2 (shared memory); st.rank == 0 afterwards flags
// inconsistent counts for either.
template <int B>
__device__ __noinline__ void radix_select2(const float* buf, int m, unsigned long long rank1,
                                           unsigned long long rank2, bool filter, float a, float b, float* zs,
                                           int cap, RadixState& st, uint32_t* key1, uint32_t* key2) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    radix_known(filter, a, b, st.known0, st.prefix0, &st.known, &st.prefix);
    st.prefix2 = st.prefix;
    st.rank = rank1;
    st.rank2 = rank2;
    st.split = 0;
  }
  __syncthreads();
  const float* cur = buf;
  int mc = m;
  while (st.known < 32 && !st.split) {
    const int known = st.known;
    const uint32_t prefix = st.prefix;
    const int nbits = (32 - known) < 8 ? (32 - known) : 8;
    const int sh = 32 - known - nbits;
    const unsigned int dmask = (1u << nbits) - 1u;
    for (int i = tid; i < 256; i += B) st.hist[i] = 0;
    __syncthreads();
    radix_hist<B>(cur, mc, filter, a, b, known, prefix, sh, dmask, st.hist);
    __syncthreads();
    if (warp == 0) {
      unsigned int h[8];
      unsigned int local = 0;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        h[j] = st.hist[lane * 8 + j];
        local += h[j];
      }
      unsigned long long incl = local;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      const unsigned long long w1 = st.rank, w2 = st.rank2;
      bool f1, f2;
      radix_pick(h, incl, local, w1, prefix, nbits, &st.prefix, &st.rank, &st.bucket, &f1);
      radix_pick(h, incl, local, w2, prefix, nbits, &st.prefix2, &st.rank2, &st.bucket2, &f2);
      __syncwarp();
      if (lane == 0) {
        st.known = known + nbits;
        st.cnt = 0;
        st.split = st.prefix != st.prefix2;
        if (!f1 || !f2) {
          st.known = 32;
          st.prefix = st.prefix2 = 0;
          st.rank = 0;
          st.split = 0;
        }
      }
    }
    __syncthreads();
    if (!st.split && zs != nullptr && cur == buf && st.known < 32 && st.bucket <= (unsigned int)cap) {
      radix_gather<B>(buf, m, filter, a, b, st.known, st.prefix, zs, (unsigned int)cap, &st.cnt);
      __syncthreads();
      cur = zs;
      mc = (int)min(st.cnt, (unsigned int)cap);
    }
  }
  if (!st.split) {
    if (tid == 0) { *key1 = st.prefix; *key2 = st.prefix; }
    __syncthreads();
    return;
  }
  // parted: the first rank's rounds, then the second's from the same point
  const int known_at = st.known;
  const uint32_t p2 = st.prefix2;
  const unsigned long long r2 = st.rank2;
  radix_rounds<B>(buf, m, cur, mc, filter, a, b, zs, cap, st);
  const uint32_t k1 = st.prefix;
  const bool bad1 = st.rank == 0;
  __syncthreads();
  if (tid == 0) {
    *key1 = k1;
    st.known = known_at;
    st.prefix = p2;
    st.rank = r2;
    st.cnt = 0;
  }
  __syncthreads();
  // when cur was gathered into zs before the split it still holds both ranks' elements
  // (the first rank's rounds read it without gathering again)
  radix_rounds<B>(buf, m, cur, mc, filter, a, b, zs, cap, st);
  if (tid == 0) {
    *key2 = st.prefix;
    if (bad1) st.rank = 0;
  }
  __syncthreads();
}

struct SegShared {
  Sum6 sum6[33];
  float mn[32], mx[32];
  uint32_t kmn[32], kmx[32];   // per warp: smallest and largest key of a small segment
  RadixState rx;
  uint32_t key1, key2;   // keys of a two-rank select
  unsigned int zcnt;
  int seg;
  // bracket state (thread 0 writes, all read)
  float a, b, t, m, M, sig, result;
  long long cle_a, clt_b, cle_b, nneg, npos, nnz, n_nan, clt_res, cle_res;
  long long cle_a0;   // #(x <= a) of the bracket that was compacted
  float a0, b0;       // that bracket
  double dF, sum;
  int it, use_bisect, stalled, compact, first, phase, how, passes;
  int zglob;          // 1: the compacted bracket is in this CTA's device-memory region
  int lean;           // 1: a learned start ran its lean pass on this segment
  float pa, pb;       // its proposed bracket
};

// Sum of the elements below q and their number, over this thread's share of buf[0, m)
// (16-byte aligned; the whole CTA: reduced into sh.sum6 by the caller).
template <int B>
__device__ __noinline__ void below_sums(const float* buf, int m, float q, float& sum, unsigned int& cnt) {
  auto fn = [&](bool ok, float v) {
    if (ok && v < q) { sum += v; ++cnt; }
  };
  radix_sweep<B>(buf, m, fn);
}

// The streaming passes of a large segment, kept out of line so that their registers are
// allocated apart from the kernel's control (the whole kernel runs at 64 registers).
struct SegStatsAcc {
  float mn, mx, sum;
  unsigned int nnan, nneg, npos, nnz, seen;
};
template <int B>
__device__ __noinline__ void seg_stats_pass(const float* __restrict__ xs, const Geometry<float>& g, float sig0,
                                            float x0s, SegStatsAcc& out) {
  float mn = INFINITY, mx = -INFINITY, sum = 0.f;
  unsigned int nnan = 0, nneg = 0, npos = 0, nnz = 0, seen = 0;
  auto f = [&](float v) {
    ++seen;
    if (fabsf(v) <= FLT_MAX) {
      mn = fminf(mn, v);
      mx = fmaxf(mx, v);
      sum += fmaf(v, sig0, -x0s);
      nnz += (__float_as_uint(v) == 0x80000000u);
    } else {
      nnan += (v != v);
      nneg += (v == -INFINITY);
      npos += (v == INFINITY);
    }
  };
  cta_stream<B>(xs, g, f);
  out.mn = mn; out.mx = mx; out.sum = sum;
  out.nnan = nnan; out.nneg = nneg; out.npos = npos; out.nnz = nnz; out.seen = seen;
}

struct SegPassAcc {
  unsigned int lt, le, xa, xb;
  float S, sle;
};
// One cutting-plane pass over a segment at t (Algorithm 1, step 1.2); FIRST also counts at
// the extremes, COMPACT appends (a, b] to zb (capacity zcap; with STAGE through the shared
// memory `slots`, 16 floats a thread), SUMLE sums the elements at or below a.
template <int B, bool FIRST, bool COMPACT, bool SUMLE, bool STAGE>
__device__ __noinline__ void seg_cut_pass(const float* __restrict__ xs, const Geometry<float>& g, float ca, float ct,
                                          float cb, float nsig, float tsig, float* zb, unsigned int zcap,
                                          unsigned int* cnt, float* slots, SegPassAcc& acc) {
  unsigned int lt = 0, le = 0, xa = 0, xb = 0;
  float S = 0.f, sle = 0.f;
  auto f = [&](float v) {
    core(v, ca, ct, nsig, tsig, lt, le, S);
    if (FIRST) {
      xa += (v <= ca);
      xb += (v < cb);
    }
    if (SUMLE) {
      if (v <= ca) sle += v;
    }
  };
  if (COMPACT && STAGE) {
    cta_stream_compact_staged<B>(xs, g, f, ca, cb, slots, zb, zcap, cnt);
  } else if (COMPACT) {
    auto keep = [&](float v) { return (v > ca) & (v <= cb); };
    cta_stream_compact<B>(xs, g, f, keep, zb, zcap, cnt);
  } else {
    cta_stream<B>(xs, g, f);
  }
  acc.lt = lt; acc.le = le; acc.xa = xa; acc.xb = xb; acc.S = S; acc.sle = sle;
}

// Learned starting bracket for the median of a large segment (the proposal of the
// single-array select, computed by this CTA): 1024 strided samples sorted on their keys by
// a shared-memory bitonic network, the sketch features, the network forward, and the
// bracket (*pa, *pb].  `scratch` is shared memory of at least 3.5 * kSample floats.
// Returns false (in every thread) when a sample is not finite or the bracket is not a
// finite a < b.
template <int B>
__device__ __noinline__ bool seg_propose(const float* __restrict__ xs, long long n, const float* __restrict__ W,
                                         float* scratch, float* pa, float* pb) {
  __shared__ double s_mu, s_sd;
  __shared__ int s_ok;
  uint32_t* kb = reinterpret_cast<uint32_t*>(scratch);
  double* sv = reinterpret_cast<double*>(scratch + kSample);
  float* f = scratch + 3 * kSample;
  float* h1 = f + 64;
  float* h2 = h1 + kHid;
  float* o = h2 + kHid;
  // thread t holds the E consecutive sample keys from position E * t (ascending bitonic
  // network over the 1024 positions): a stage of distance j < E compares within the
  // thread, j < 32 E with the lane t ^ (j / E) by a shuffle, longer ones through shared
  // memory (kb)
  constexpr int E = kSample / B;
  static_assert(E >= 1 && E * B == kSample, "the sample is spread evenly over the CTA");
  const int t = threadIdx.x;
  const long long stride = n / kSample;
  bool bad = false;
  uint32_t key[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const float v = xs[(long long)(E * t + e) * stride];
    bad |= !(fabsf(v) <= FLT_MAX);
    key[e] = ukey(v);
  }
  if (__syncthreads_or(bad)) return false;
  for (int k = 2; k <= kSample; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      if (j < E) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int e2 = e ^ j;
          if (e2 > e) {
            const bool up = (((E * t + e) & k) == 0);
            const uint32_t u = key[e], v = key[e2];
            if ((u > v) == up) { key[e] = v; key[e2] = u; }
          }
        }
      } else if (j < 32 * E) {
        const int lanes = j / E;
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int i = E * t + e;
          const uint32_t w = __shfl_xor_sync(0xffffffffu, key[e], lanes);
          const bool up = ((i & k) == 0), lower = ((i & j) == 0);
          key[e] = (up == lower) ? min(key[e], w) : max(key[e], w);
        }
      } else {
#pragma unroll
        for (int e = 0; e < E; ++e) kb[E * t + e] = key[e];
        __syncthreads();
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int i = E * t + e;
          const uint32_t w = kb[i ^ j];
          const bool up = ((i & k) == 0), lower = ((i & j) == 0);
          key[e] = (up == lower) ? min(key[e], w) : max(key[e], w);
        }
        __syncthreads();
      }
    }
#pragma unroll
  for (int e = 0; e < E; ++e) sv[E * t + e] = (double)ukey_value(key[e], 0.f);
  __syncthreads();
  if (threadIdx.x < 32) sketch_features_warp(sv, f, &s_mu, &s_sd);
  __syncthreads();
  mlp_forward_rows<B / 32>(W, f, h1, h2, o);
  if (threadIdx.x == 0) {
    double a, b;
    const bool valid = proposal_from_outputs(o, s_mu, s_sd, &a, &b);
    const float fa = (float)a, fb = (float)b;
    s_ok = valid && fa < fb && fabsf(fa) <= FLT_MAX && fabsf(fb) <= FLT_MAX;
    *pa = fa;
    *pb = fb;
  }
  __syncthreads();
  return s_ok != 0;
}

// The lean first pass of a learned start: NaN count, #(x <= a), and (a, b] compacted into
// zb in device memory (capacity zcap, counter *cnt, which also gives #(a < x <= b)),
// staged through the shared memory `slots`.
struct SegLeanAcc {
  unsigned int nnan, le_a;
};
template <int B>
__device__ __noinline__ void seg_lean_pass(const float* __restrict__ xs, const Geometry<float>& g, float a, float b,
                                           float* zb, unsigned int zcap, unsigned int* cnt, float* slots,
                                           SegLeanAcc& acc) {
  unsigned int nnan = 0, le_a = 0;
  auto f = [&](float v) {
    nnan += (v != v);
    le_a += (v <= a);
  };
  cta_stream_compact_staged<B>(xs, g, f, a, b, slots, zb, zcap, cnt);
  acc.nnan = nnan;
  acc.le_a = le_a;
}

// STAGE: the dynamic shared memory holds 16 B staging floats past the CAP of the buffer,
// and every compacting pass goes through them (cta_stream_compact_staged).
template <int B, int CAP, bool LTS, bool STAGE>
__global__ void __launch_bounds__(B, 1024 / B) seg_kernel(SegArgs A) {
  static_assert(CAP >= 16 * B, "the lean pass stages through 16 floats of the buffer a thread");
  extern __shared__ __align__(16) float zb[];   // CAP floats (+ 16 B staging floats with STAGE)
  __shared__ SegShared sh;
  const int tid = threadIdx.x, lane = tid & 31;
  constexpr int NW = B / 32;
  for (;;) {
    if (tid == 0) {
      const unsigned long long q = atomicAdd(&A.ctrl->w_count, 1ull);
      sh.seg = q < A.ctrl->w_len ? A.order[q] : -1;
    }
    __syncthreads();
    const int s = sh.seg;
    if (s < 0) break;
    const long long o0 = A.off[s];
    const long long n = A.off[s + 1] - o0;
    const long long k = A.kk ? A.kk[s] : (A.k_const > 0 ? A.k_const : (n + 1) / 2);
    const long long k2 = LTS ? (A.kk2 ? A.kk2[s] : (A.k2_const > 0 ? A.k2_const : (n + 1) / 2)) : 0;
    if (n < 1 || k < 1 || k > n || (LTS && (k2 < 1 || k2 > n))) {
      if (tid == 0) {
        A.out[s] = NAN;
        if (LTS) { A.out2[s] = NAN; A.outsum[s] = NAN; A.flags[s] = 0; }
        atomicCAS(&A.ctrl->status, 0, (int)GBS_EINVAL);
        if (A.seg_passes) A.seg_passes[s] = 0;
      }
      __syncthreads();
      continue;
    }
    const float* xs = A.x + o0;
    const Geometry<float> g(xs, n);

    if (n <= CAP) {
      // ---- small segment: load once, radix select in shared memory ----
      // load: the scalar head and tail, and the 16-byte body four vectors per thread in flight;
      // the smallest and largest keys give the leading bits every element shares, where
      // the radix rounds start
      unsigned int nan_here = 0;
      uint32_t kmn = 0xffffffffu, kmx = 0u;
      auto see = [&](float v) {
        nan_here += (v != v);
        const uint32_t kv = ukey(v);
        kmn = min(kmn, kv);
        kmx = max(kmx, kv);
      };
      if (tid < g.head) {
        const float v = xs[tid];
        see(v);
        zb[tid] = v;
      }
      if (tid < n - g.tail0) {
        const float v = xs[g.tail0 + tid];
        see(v);
        zb[g.tail0 + tid] = v;
      }
      {
        const float4* xv = reinterpret_cast<const float4*>(xs + g.head);
        float* zh = zb + g.head;
        auto put = [&](long long q, const float4 r) {
          see(r.x); see(r.y); see(r.z); see(r.w);
          zh[4 * q] = r.x; zh[4 * q + 1] = r.y; zh[4 * q + 2] = r.z; zh[4 * q + 3] = r.w;
        };
        long long q = tid;
        for (; q + 3 * B < g.nv; q += 4 * B) {
          float4 r[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) r[u] = __ldcs(xv + q + u * B);
#pragma unroll
          for (int u = 0; u < 4; ++u) put(q + u * B, r[u]);
        }
        for (; q < g.nv; q += B) put(q, __ldcs(xv + q));
      }
      kmn = __reduce_min_sync(0xffffffffu, kmn);
      kmx = __reduce_max_sync(0xffffffffu, kmx);
      if (lane == 0) { sh.kmn[tid >> 5] = kmn; sh.kmx[tid >> 5] = kmx; }
      Sum6 v6;
      v6.u[0] = nan_here; v6.u[1] = v6.u[2] = v6.u[3] = v6.u[4] = 0; v6.d = 0.0;
      const Sum6 r6 = cta_sum6<B>(v6, sh.sum6);   // its barriers also publish sh.kmn / sh.kmx
      if (r6.u[0] > 0) {
        if (tid == 0) {
          A.out[s] = NAN;
          if (LTS) { A.out2[s] = NAN; A.outsum[s] = NAN; A.flags[s] = 0; }
          atomicCAS(&A.ctrl->status, 0, (int)GBS_ENAN);
          if (A.seg_passes) A.seg_passes[s] = 1;
        }
        __syncthreads();
        continue;
      }
      if (tid == 0) {
        uint32_t lo = sh.kmn[0], hi = sh.kmx[0];
        for (int w = 1; w < NW; ++w) { lo = min(lo, sh.kmn[w]); hi = max(hi, sh.kmx[w]); }
        const uint32_t diff = lo ^ hi;
        const int known = diff == 0 ? 32 : __clz(diff);
        sh.rx.known0 = known;
        sh.rx.prefix0 = known == 0 ? 0u : (known == 32 ? hi : (hi >> (32 - known)));
      }
      // the free part of the buffer past the segment (16-byte aligned) takes the elements
      // of the chosen digit once they fit, so that the later rounds sweep only those
      const int zoff = (int)((n + 3) & ~3ll);
      float* const zsp = zoff + 256 <= CAP ? zb + zoff : nullptr;
      const int zscap = zsp != nullptr ? CAP - zoff : 0;
      // trimmed-sum mode: both ranks from shared rounds
      if (LTS) radix_select2<B>(zb, (int)n, (unsigned long long)k, (unsigned long long)k2, false, 0.f, 0.f, zsp, zscap,
                                sh.rx, &sh.key1, &sh.key2);
      const uint32_t key =
          LTS ? sh.key1 : radix_select<B>(zb, (int)n, (unsigned long long)k, false, 0.f, 0.f, zsp, zscap, sh.rx);
      const float q = ukey_value(key, 0.f);
      if (tid == 0) {
        if (sh.rx.rank == 0) atomicCAS(&A.ctrl->status, 0, (int)GBS_EINTERNAL);
        A.out[s] = q;
        if (A.seg_passes) A.seg_passes[s] = 1;
      }
      if (LTS) {
        // trimmed sum: the k smallest = everything below q plus (k - #below) copies of q
        float bs = 0.f;
        unsigned int bc = 0;
        below_sums<B>(zb, (int)n, q, bs, bc);
        Sum6 w6;
        w6.u[0] = bc; w6.u[1] = w6.u[2] = w6.u[3] = w6.u[4] = 0; w6.d = (double)bs;
        const Sum6 t6 = cta_sum6<B>(w6, sh.sum6);
        const uint32_t key2 = sh.key2;
        if (tid == 0) {
          A.outsum[s] = t6.d + (double)(k - (long long)t6.u[0]) * (double)q;
          A.out2[s] = ukey_value(key2, 0.f);
          A.flags[s] = 0;
        }
      }
      __syncthreads();
      continue;
    }

    // ---- large segment, learned start (medians, with a model): proposal and lean pass ----
    if (tid == 0) { sh.phase = 0; sh.lean = 0; sh.zcnt = 0; }
    __syncthreads();
    if (!LTS && A.W != nullptr && A.zg != nullptr && n >= kSegLearnMinN && k == (n + 1) / 2 &&
        seg_propose<B>(xs, n, A.W, zb, &sh.pa, &sh.pb)) {
      SegLeanAcc la;
      seg_lean_pass<B>(xs, g, sh.pa, sh.pb, A.zg + (long long)blockIdx.x * A.zg_cap, (unsigned int)A.zg_cap,
                       &sh.zcnt, zb, la);
      Sum6 v6;
      v6.u[0] = la.nnan; v6.u[1] = la.le_a; v6.u[2] = v6.u[3] = v6.u[4] = 0; v6.d = 0.0;
      const Sum6 r6 = cta_sum6<B>(v6, sh.sum6);   // also orders the appends before the finish
      if (tid == 0) {
        const long long le_a = (long long)r6.u[1], zc = (long long)sh.zcnt;
        sh.lean = 1;
        sh.passes = 1;
        sh.how = GBS_HOW_NONE;
        if (r6.u[0] > 0) {
          sh.phase = 3;
          sh.result = NAN;
        } else if (le_a < k && k <= le_a + zc && zc <= (long long)A.zg_cap) {
          // the proposal holds the median and all of (a, b] is compacted: the finish
          sh.phase = 2;
          sh.a0 = sh.pa; sh.b0 = sh.pb; sh.cle_a0 = le_a; sh.zglob = 1; sh.sum = 0.0;
        }
      }
      __syncthreads();
    }

    // ---- large segment: pass 0 (extremes, sum, non-finite and -0 counts) ----
    if (sh.phase == 0) {
      const float sig0 = A.sigma_stats;
      float x0 = 0.f;
      if (tid < n && Ops<float>::is_finite(xs[tid])) x0 = xs[tid];
      const float x0s = x0 * sig0;
      SegStatsAcc sa;
      seg_stats_pass<B>(xs, g, sig0, x0s, sa);
      float mn = sa.mn, mx = sa.mx;
      const float sum = sa.sum;
      const unsigned int nnan = sa.nnan, nneg = sa.nneg, npos = sa.npos, nnz = sa.nnz, seen = sa.seen;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      }
      if (lane == 0) { sh.mn[tid >> 5] = mn; sh.mx[tid >> 5] = mx; }
      const unsigned int nfin = seen - nnan - nneg - npos;
      Sum6 v6;
      v6.u[0] = nnan; v6.u[1] = nneg; v6.u[2] = npos; v6.u[3] = nnz; v6.u[4] = nfin;
      v6.d = (double)sum / (double)sig0 + (double)nfin * (double)x0;
      const Sum6 r6 = cta_sum6<B>(v6, sh.sum6);
      if (tid == 0) {
        float bm = sh.mn[0], bM = sh.mx[0];
        for (int w = 1; w < NW; ++w) { bm = fminf(bm, sh.mn[w]); bM = fmaxf(bM, sh.mx[w]); }
        sh.m = bm; sh.M = bM;
        sh.n_nan = (long long)r6.u[0]; sh.nneg = (long long)r6.u[1]; sh.npos = (long long)r6.u[2];
        sh.nnz = (long long)r6.u[3]; sh.sum = r6.d;
        sh.passes = 1 + sh.lean; sh.it = 0; sh.use_bisect = 0; sh.stalled = 0; sh.first = 0; sh.phase = 0;
        sh.how = GBS_HOW_NONE; sh.clt_res = -1; sh.cle_res = -1; sh.result = 0.f;
        if (sh.n_nan > 0) {
          sh.phase = 3; sh.result = NAN;
        } else if (k <= sh.nneg) {
          sh.phase = 1; sh.result = -INFINITY;
        } else if (k > n - sh.npos) {
          sh.phase = 1; sh.result = INFINITY;
        } else if (!(bm < bM)) {
          sh.phase = 1; sh.result = bm; sh.clt_res = sh.nneg;
        } else {
          sh.a = bm; sh.b = bM;
          sh.cle_a = sh.nneg + 1; sh.clt_b = n - sh.npos - 1; sh.cle_b = n - sh.npos; sh.first = 1;
          const double gL = (double)(sh.cle_a - k) + 0.5;
          const double inner = sh.sum - (double)bm - (double)bM;
          sh.dF = gL * ((double)bM - (double)bm) + (double)(sh.clt_b - sh.cle_a) * (double)bM - inner;
        }
      }
      __syncthreads();
    }

    // ---- cutting-plane passes ----
    const long long per_thread = ((g.nv + B - 1) / B) * 4 + 8;
    while (sh.phase == 0) {
      if (tid == 0) {   // step 1.1 (with the key-midpoint safeguard)
        // compaction of (a, b] in this pass: into shared memory when it fits there, else into
        // the CTA's device-memory region once the bracket holds at most n / 2 elements
        const long long pop = sh.cle_b - sh.cle_a;
        sh.compact = pop <= CAP ? 1
                     : (A.zg != nullptr && pop <= (long long)A.zg_cap && pop * kSegGlobalDiv <= n) ? 2 : 0;
        const uint32_t ka = ukey(sh.a), kb = ukey(sh.b);
        float t;
        if (kb - ka <= 1u) {
          // no float strictly inside: every element of (a, b] equals b
          sh.phase = 1; sh.result = sh.b; sh.clt_res = sh.cle_a;
        } else {
          const bool bis = sh.use_bisect || sh.stalled >= 2 || sh.it >= A.maxit;
          if (bis) {
            t = inside<float>(ukey_value(ka + (kb - ka) / 2, 0.f), sh.a, sh.b);
          } else {
            const double gL = (double)(sh.cle_a - k) + 0.5;
            const double gR = (double)(sh.clt_b - k) + 0.5;
            const double w = (double)sh.b - (double)sh.a;
            t = inside<float>((float)((double)sh.a + (gR * w - sh.dF) / (gR - gL)), sh.a, sh.b);
          }
          sh.t = t;
          sh.sig = cost_scale((double)t - (double)sh.a, per_thread);
          sh.zcnt = 0;
        }
      }
      __syncthreads();
      if (sh.phase != 0) break;
      const float ca = sh.a, ct = sh.t, cb = sh.b, nsig = -sh.sig, tsig = sh.t * sh.sig;
      const int first = sh.first, compact = sh.compact;
      float* const zdst = compact == 2 ? A.zg + (long long)blockIdx.x * A.zg_cap : zb;
      const unsigned int zcap = compact == 2 ? (unsigned int)A.zg_cap : (unsigned int)CAP;
      SegPassAcc pacc;
      float* const slots = zb + CAP;   // the staging slots past the buffer (STAGE variants)
#define GBS_SEG_PASS(F, C, SL) \
  seg_cut_pass<B, F, C, SL, STAGE>(xs, g, ca, ct, cb, nsig, tsig, zdst, zcap, &sh.zcnt, slots, pacc)
      if (first) {
        if (compact) {
          if (LTS) GBS_SEG_PASS(true, true, true); else GBS_SEG_PASS(true, true, false);
        } else {
          GBS_SEG_PASS(true, false, false);
        }
      } else {
        if (compact) {
          if (LTS) GBS_SEG_PASS(false, true, true); else GBS_SEG_PASS(false, true, false);
        } else {
          GBS_SEG_PASS(false, false, false);
        }
      }
#undef GBS_SEG_PASS
      const unsigned int lt = pacc.lt, le = pacc.le, xa = pacc.xa, xb = pacc.xb;
      const float S = pacc.S, sle = pacc.sle;
      Sum6 v6;
      v6.u[0] = lt; v6.u[1] = le; v6.u[2] = xa; v6.u[3] = xb; v6.u[4] = 0; v6.d = (double)S;
      const Sum6 r6 = cta_sum6<B>(v6, sh.sum6);   // also orders every append before the reads below
      double sle_tot = 0.0;
      if (LTS && compact) {
        Sum6 w6;
        w6.u[0] = w6.u[1] = w6.u[2] = w6.u[3] = w6.u[4] = 0; w6.d = (double)sle;
        sle_tot = cta_sum6<B>(w6, sh.sum6).d;
      }
      if (tid == 0) {   // steps 1.3-1.4
        sh.passes++;
        const long long clt = (long long)r6.u[0], cle = (long long)r6.u[1];
        bool resolved = false;
        if (sh.first) {
          const long long cle_m = (long long)r6.u[2], clt_M = (long long)r6.u[3];
          sh.first = 0;
          if (cle_m >= k) {
            sh.phase = 1; sh.result = sh.a; sh.clt_res = sh.nneg; sh.cle_res = cle_m; resolved = true;
          } else if (clt_M < k) {
            sh.phase = 1; sh.result = sh.b; sh.clt_res = clt_M; sh.cle_res = n - sh.npos; resolved = true;
          } else {
            const double cmn = (double)(cle_m - sh.nneg), cmx = (double)(n - sh.npos - clt_M);
            const double gL = (double)(cle_m - k) + 0.5;
            const double inner = sh.sum - cmn * (double)sh.a - cmx * (double)sh.b;
            sh.cle_a = cle_m; sh.clt_b = clt_M;
            sh.dF = gL * ((double)sh.b - (double)sh.a) + (double)(clt_M - cle_m) * (double)sh.b - inner;
          }
        }
        if (!resolved) {
          const long long pop = sh.cle_b - sh.cle_a;
          if (compact) {   // the bracket just compacted and the sum below it
            sh.cle_a0 = sh.cle_a; sh.a0 = sh.a; sh.b0 = sh.b; sh.sum = sle_tot; sh.zglob = compact == 2;
          }
          if (clt < k && k <= cle) {
            sh.phase = 1; sh.result = sh.t; sh.clt_res = clt; sh.cle_res = cle;
          } else {
            const double gL = (double)(sh.cle_a - k) + 0.5;
            const double dphi = gL * ((double)sh.t - (double)sh.a) + r6.d / (double)sh.sig;
            if (cle < k) {
              sh.a = sh.t; sh.cle_a = cle; sh.dF -= dphi;
            } else {
              sh.b = sh.t; sh.clt_b = clt; sh.cle_b = cle; sh.dF = dphi;
            }
            const long long npop = sh.cle_b - sh.cle_a;
            sh.use_bisect = (!sh.use_bisect) && ((double)npop > 0.75 * (double)pop);
            sh.stalled = ((double)npop > 0.875 * (double)pop) ? sh.stalled + 1 : 0;
            sh.it++;
            if (compact) sh.phase = ((long long)sh.zcnt == pop) ? 2 : 4;
          }
        }
      }
      __syncthreads();
    }

    float result = sh.result;
    if (sh.phase == 2) {
      // the compacted bracket (a0, b0] holds ranks cle_a0 + 1 .. cle_a0 + zcnt
      const int m = (int)sh.zcnt;
      const float* zf = sh.zglob ? A.zg + (long long)blockIdx.x * A.zg_cap : zb;
      float* const zs = sh.zglob ? zb : nullptr;   // gathers the last digits into shared memory
      // trimmed-sum mode with the second rank inside the bracket: both from shared rounds
      const bool inside2 = LTS && sh.cle_a0 < k2 && k2 <= sh.cle_a0 + m;
      uint32_t key;
      if (inside2) {
        radix_select2<B>(zf, m, (unsigned long long)(k - sh.cle_a0), (unsigned long long)(k2 - sh.cle_a0), true,
                         sh.a0, sh.b0, zs, CAP, sh.rx, &sh.key1, &sh.key2);
        key = sh.key1;
      } else {
        key = radix_select<B>(zf, m, (unsigned long long)(k - sh.cle_a0), true, sh.a0, sh.b0, zs, CAP, sh.rx);
      }
      if (tid == 0 && sh.rx.rank == 0) atomicCAS(&A.ctrl->status, 0, (int)GBS_EINTERNAL);
      result = ukey_value(key, 0.f);
      if (LTS) {
        float bs = 0.f;
        unsigned int bc = 0;
        below_sums<B>(zf, m, result, bs, bc);
        Sum6 w6;
        w6.u[0] = bc; w6.u[1] = w6.u[2] = w6.u[3] = w6.u[4] = 0; w6.d = (double)bs;
        const Sum6 t6 = cta_sum6<B>(w6, sh.sum6);
        const long long below = sh.cle_a0 + (long long)t6.u[0];
        const float r2 = inside2 ? ukey_value(sh.key2, 0.f) : NAN;
        if (tid == 0) {
          A.outsum[s] = sh.sum + t6.d + (double)(k - below) * (double)result;
          A.out2[s] = r2;
          A.flags[s] = inside2 ? 0 : 1;
        }
      }
    } else if (sh.phase == 1) {
      if (result == 0.f && sh.clt_res >= 0) result = (k - sh.clt_res) <= sh.nnz ? -0.f : 0.f;
      if (LTS) {
        // resolved by counts: one more pass for the sum below the result
        const float q = result;
        float bs = 0.f;
        unsigned int bc = 0;
        auto fb = [&](float v) { if (v < q) { bs += v; ++bc; } };
        cta_stream<B>(xs, g, fb);
        Sum6 w6;
        w6.u[0] = bc; w6.u[1] = w6.u[2] = w6.u[3] = w6.u[4] = 0; w6.d = (double)bs;
        const Sum6 t6 = cta_sum6<B>(w6, sh.sum6);
        if (tid == 0) {
          sh.passes++;
          A.outsum[s] = t6.d + (double)(k - (long long)t6.u[0]) * (double)q;
          const bool same = sh.clt_res >= 0 && sh.clt_res < k2 && k2 <= sh.cle_res;
          A.out2[s] = same ? q : NAN;
          A.flags[s] = same ? 0 : 1;
        }
      }
    } else if (LTS && tid == 0) {
      A.out2[s] = NAN;
      A.outsum[s] = NAN;
      A.flags[s] = 0;
    }
    if (tid == 0) {
      if (sh.phase == 3) atomicCAS(&A.ctrl->status, 0, (int)GBS_ENAN);
      if (sh.phase == 4) atomicCAS(&A.ctrl->status, 0, (int)GBS_EINTERNAL);
      A.out[s] = result;
      if (A.seg_passes) A.seg_passes[s] = sh.passes;
    }
    __syncthreads();
  }
}

// The launch variants the autotuner chooses from: CTA size and shared-memory capacity
// for the direct / finishing select.
// `stage` staging floats follow the buffer where they fit at the variant's occupancy.
struct Variant {
  int threads, cap, stage;
  void (*kernel)(SegArgs);
  void (*kernel_lts)(SegArgs);
};
const Variant kVariants[] = {
    {512, 12288, 16 * 512, seg_kernel<512, 12288, false, true>, seg_kernel<512, 12288, true, true>},
    {512, 24576, 0, seg_kernel<512, 24576, false, false>, seg_kernel<512, 24576, true, false>},
    {1024, 49152, 0, seg_kernel<1024, 49152, false, false>, seg_kernel<1024, 49152, true, false>},
    {256, 12288, 0, seg_kernel<256, 12288, false, false>, seg_kernel<256, 12288, true, false>},
};
constexpr int kNumVariants = sizeof(kVariants) / sizeof(kVariants[0]);

}  // namespace

int seg_num_variants() { return kNumVariants; }

gbs_status seg_launch(gbs_ctx* c, const SegLaunch& L, int variant, cudaStream_t stream) {
  if (variant < 0 || variant >= kNumVariants) return GBS_EINVAL;
  const Variant& v = kVariants[variant];
  const bool lts = L.outsum != nullptr;
  void (*kern)(SegArgs) = lts ? v.kernel_lts : v.kernel;
  const size_t smem = (size_t)(v.cap + v.stage) * sizeof(float);
  static bool attr_done[2][kNumVariants] = {};
  if (!attr_done[lts][variant]) {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
      cudaGetLastError();
      return GBS_ECUDA;
    }
    attr_done[lts][variant] = true;
  }
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, v.threads, smem) != cudaSuccess || occ < 1) {
    cudaGetLastError();
    return GBS_ECUDA;
  }
  const int grid = c->num_sms * occ;
  if (cudaMemsetAsync(L.ctrl, 0, sizeof(Ctrl), stream) != cudaSuccess) return GBS_ECUDA;
  seg_schedule_kernel<<<1, 1024, 0, stream>>>(L.off, L.S, L.order, L.mask, L.ctrl);
  SegArgs A;
  A.x = L.x; A.off = L.off; A.S = L.S; A.kk = L.kk; A.out = L.out; A.order = L.order; A.ctrl = L.ctrl;
  A.maxit = 48;
  // the compaction area shared out among the CTAs (multiples of 32 elements each)
  A.zg = nullptr;
  A.zg_cap = 0;
  if (L.zg != nullptr) {
    const long long per = (L.zg_elems / grid) / 32 * 32;
    if (per >= 32) {
      A.zg = L.zg;
      A.zg_cap = (int)std::min<long long>(per, 1ll << 30);
    }
  }
  A.seg_passes = L.seg_passes;
  A.k_const = L.k_const; A.k2_const = L.k2_const;
  A.kk2 = L.kk2; A.out2 = L.out2; A.outsum = L.outsum; A.flags = L.flags;
  // learned starting brackets for the medians (gbs_config.use_learned with a model loaded)
  A.W = (!lts && c->cfg.use_learned && c->model_loaded) ? c->model : nullptr;
  // pass-0 sums: a thread adds at most ceil(1e6 / threads) * ... terms of a segment; the
  // scale keeps any float32 partial finite for segments up to 2^31 elements
  A.sigma_stats = std::ldexp(1.0f, -24);
  kern<<<grid, v.threads, smem, stream>>>(A);
  if (cudaGetLastError() != cudaSuccess) return GBS_ECUDA;
  return GBS_OK;
}

int seg_variant_threads(int v) { return (v >= 0 && v < kNumVariants) ? kVariants[v].threads : 0; }

// Device-memory compaction area of a segmented launch, shared out among its CTAs (1 GiB:
// about 880,000 elements a CTA at two CTAs on each of 152 SMs, so that a bracket of half
// of a 10^6-element segment fits).
constexpr size_t kSegZgBytes = size_t(1024) << 20;

size_t seg_workspace_bytes(int S) {
  const size_t head = ((size_t)S * 2 * sizeof(int) + 255) / 256 * 256;
  return head + kSegZgBytes;
}

gbs_status seg_attach_workspace(gbs_ctx* c, int S, SegLaunch* L) {
  const gbs_status st = gbs_internal_ensure(c, seg_workspace_bytes(S));
  if (st != GBS_OK) return st;
  L->order = static_cast<int*>(c->z);
  L->seg_passes = static_cast<int*>(c->z) + S;
  L->zg = reinterpret_cast<float*>(static_cast<char*>(c->z) + ((size_t)S * 2 * sizeof(int) + 255) / 256 * 256);
  L->zg_elems = (long long)(kSegZgBytes / sizeof(float));
  return GBS_OK;
}
int seg_variant_cap(int v) { return (v >= 0 && v < kNumVariants) ? kVariants[v].cap : 0; }

}  // namespace gbs

// ---------------------------------------------------------------------------------
// C-ABI.
// ---------------------------------------------------------------------------------
namespace {
gbs_status seg_prepare(gbs_ctx* c, const float* x, const int64_t* off, int32_t S, float* out,
                       gbs::SegLaunch* L, const int64_t* k) {
  if (!c || !x || !off || !out || S < 1) return GBS_EINVAL;
  gbs_status st = gbs::seg_attach_workspace(c, S, L);
  if (st != GBS_OK) return st;
  L->x = x; L->off = reinterpret_cast<const long long*>(off); L->S = S;
  L->kk = reinterpret_cast<const long long*>(k); L->out = out;
  L->ctrl = c->ctrl;
  L->mask = nullptr; L->kk2 = nullptr; L->out2 = nullptr; L->outsum = nullptr; L->flags = nullptr;
  L->k_const = 0; L->k2_const = 0;
  return GBS_OK;
}
}  // namespace

extern "C" {

gbs_status gbs_select_segmented_f32(gbs_ctx* c, const float* x, const int64_t* offsets, int32_t S,
                                    const int64_t* k, float* out, void* stream) {
  gbs::SegLaunch L;
  gbs_status st = seg_prepare(c, x, offsets, S, out, &L, k);
  if (st != GBS_OK) return st;
  gbs::DeviceGuard g(c->device);
  if (!g.ok) return GBS_ECUDA;
  st = gbs::seg_launch(c, L, c->seg_variant, static_cast<cudaStream_t>(stream));
  if (st == GBS_OK) {
    c->last_stream = static_cast<cudaStream_t>(stream);
    c->last_segments = S;
  }
  return st;
}

gbs_status gbs_segmented_autotune_f32(gbs_ctx* c, const float* x, const int64_t* offsets, int32_t S,
                                      const int64_t* k, float* out, void* stream, int32_t* chosen,
                                      float* ms_per_variant, int32_t n_variants) {
  gbs::SegLaunch L;
  gbs_status st = seg_prepare(c, x, offsets, S, out, &L, k);
  if (st != GBS_OK) return st;
  gbs::DeviceGuard g(c->device);
  if (!g.ok) return GBS_ECUDA;
  cudaStream_t strm = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return GBS_ECUDA;
  int best = -1;
  float best_ms = 0.f;
  for (int v = 0; v < gbs::seg_num_variants(); ++v) {
    float ms = -1.f;
    if (gbs::seg_launch(c, L, v, strm) == GBS_OK) {   // warm-up
      cudaEventRecord(e0, strm);
      gbs_status s2 = GBS_OK;
      for (int r = 0; r < 2 && s2 == GBS_OK; ++r) s2 = gbs::seg_launch(c, L, v, strm);
      cudaEventRecord(e1, strm);
      if (s2 == GBS_OK && cudaEventSynchronize(e1) == cudaSuccess) {
        cudaEventElapsedTime(&ms, e0, e1);
        ms *= 0.5f;
      }
    }
    cudaGetLastError();
    if (ms_per_variant && v < n_variants) ms_per_variant[v] = ms;
    if (ms > 0.f && (best < 0 || ms < best_ms)) {
      best = v;
      best_ms = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (best < 0) return GBS_ECUDA;
  c->seg_variant = best;
  if (chosen) *chosen = best;
  c->last_stream = strm;
  c->last_segments = S;
  return gbs::seg_launch(c, L, best, strm);   // leaves `out` from the chosen variant
}

gbs_status gbs_segmented_set_variant(gbs_ctx* c, int32_t variant) {
  if (!c || variant < 0 || variant >= gbs::seg_num_variants()) return GBS_EINVAL;
  c->seg_variant = variant;
  return GBS_OK;
}

gbs_status gbs_segmented_get_variant(gbs_ctx* c, int32_t* variant, int32_t* threads, int32_t* smem_cap,
                                     int32_t* n_variants) {
  if (!c) return GBS_EINVAL;
  if (variant) *variant = c->seg_variant;
  if (threads) *threads = gbs::seg_variant_threads(c->seg_variant);
  if (smem_cap) *smem_cap = gbs::seg_variant_cap(c->seg_variant);
  if (n_variants) *n_variants = gbs::seg_num_variants();
  return GBS_OK;
}

gbs_status gbs_segmented_passes(gbs_ctx* c, int32_t* passes, int32_t S) {
  if (!c || !passes || S < 1 || S > c->last_segments || !c->z) return GBS_EINVAL;
  gbs::DeviceGuard g(c->device);
  if (!g.ok) return GBS_ECUDA;
  if (cudaStreamSynchronize(c->last_stream) != cudaSuccess ||
      cudaMemcpy(passes, static_cast<int*>(c->z) + c->last_segments, (size_t)S * sizeof(int),
                 cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return GBS_ECUDA;
  }
  return GBS_OK;
}

}  // extern "C"
