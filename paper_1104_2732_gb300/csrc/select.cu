// Persistent cutting-plane selection kernel (float32 and float64).
//
// One cooperative launch runs the whole of Algorithm 1 (Sec. 3) plus the hybrid finish:
//   pass 0      min / max / counts / sum over x (Sec. 3, step 0)
//   pass j>=1   the fused cost + count pass at the iterate t (step 1.2; the figure's
//               Objective()), then, redundantly in every CTA, the bracket update
//               (steps 1.3-1.4) and the next tangent intersection (step 1.1)
//   compaction  the pass that sees a bracket of <= cap elements also writes them out
//   finish      8-bit radix select on totalOrder keys inside the final bracket
// Every pass ends in one grid-wide barrier; each CTA then sums the per-CTA partials in
// the same fixed order, so all CTAs take identical decisions without a second barrier.
#include <cfloat>
#include <cmath>
#include <cstdint>

#include "common.cuh"
#include "elem.cuh"
#include "layout.cuh"
#include "select.cuh"
#include "api_internal.h"
#include "bracket.cuh"

namespace gbs {

template <typename T, typename Fn>
__device__ __forceinline__ void stream_edges(const T* __restrict__ x, const Geometry<T>& g, Fn& f) {
  const long long gtid = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (gtid < g.head) f(x[gtid]);
  if (gtid < g.n - g.tail0) f(x[g.tail0 + gtid]);
}

// Streaming over this CTA's chunks of the 16-byte-vector body: chunk c = bid + j*grid
// (reverse order when `rev`), thread t loads vectors t + u*kThreads (u < kVPT) of each,
// with 128-bit streaming loads, all kVPT of them in flight before any is used.
constexpr int kVPT = (int)(kChunkVecs / kThreads);

// Calls f on this thread's elements of chunk c (vectors threadIdx.x + u*kThreads); only
// the last chunk of the body (c == last) can be partial.  32-bit chunk indices keep the
// loop's registers low (no spills in the passes at 64 registers a thread).
template <typename T, typename Fn>
__device__ __forceinline__ void stream_chunk(const typename Ops<T>::V* __restrict__ xv, unsigned int c,
                                             unsigned int last, long long nv, Fn& f) {
  using V = typename Ops<T>::V;
  const V* p = xv + (long long)c * kChunkVecs + threadIdx.x;
  if (c != last) {
    V r[kVPT];
#pragma unroll
    for (int u = 0; u < kVPT; ++u) r[u] = load_stream(p + u * kThreads);
#pragma unroll
    for (int u = 0; u < kVPT; ++u) Ops<T>::each(r[u], f);
  } else {
    const long long lim = nv - (long long)c * kChunkVecs - threadIdx.x;   // vectors left from p on
    for (int u = 0; u < kVPT; ++u)
      if ((long long)u * kThreads < lim) {
        const V r = load_stream(p + u * kThreads);
        Ops<T>::each(r, f);
      }
  }
}

template <typename T, typename Fn>
__device__ __forceinline__ void stream_chunks(const T* __restrict__ x, const Geometry<T>& g, bool rev, Fn& f) {
  using V = typename Ops<T>::V;
  const V* xv = reinterpret_cast<const V*>(x + g.head);
  const unsigned int G = gridDim.x, bid = blockIdx.x;
  const unsigned int nch = (unsigned int)chunk_count(g.nv);
  const unsigned int my = bid < nch ? (nch - 1 - bid) / G + 1 : 0;
  for (unsigned int j = 0; j < my; ++j) stream_chunk<T>(xv, bid + (rev ? my - 1 - j : j) * G, nch - 1, g.nv, f);
}

// As stream_chunks, and the elements the pass keeps are appended to `zr` (counter *cnt
// in shared memory).  fk(v, off) counts v and, when it keeps v, stores it at the shared
// address off and advances off by one slot: slot j of lane L is wb[L + 32 j] (no bank
// conflicts), so the loaded vectors are dead before the warp's prefix sum; each lane then
// copies its kept elements of the chunk to their places after those of the lower lanes.
// on_kept(v, act) follows each copy in every lane of the warp (act: the lane copied v).
template <typename T, typename FK, typename OnKept>
__device__ __forceinline__ void stream_chunks_compact(const T* __restrict__ x, const Geometry<T>& g, bool rev,
                                                      FK& fk, T* __restrict__ zr, unsigned int* cnt, T* wb,
                                                      OnKept& on_kept) {
  using V = typename Ops<T>::V;
  constexpr int kVec = Ops<T>::kVec;
  constexpr unsigned int kSlot = 32u * sizeof(T);
  const int lane = threadIdx.x & 31;
  const unsigned int off0 = smem_u32(wb + lane);
  const V* xv = reinterpret_cast<const V*>(x + g.head);
  const unsigned int G = gridDim.x, bid = blockIdx.x;
  const unsigned int nch = (unsigned int)chunk_count(g.nv);
  const unsigned int my = bid < nch ? (nch - 1 - bid) / G + 1 : 0;
  // the loads of chunk j + 1 are issued before chunk j's prefix sum and copy-out, so that
  // they are in flight during that serial part
  V r[kVPT];
  auto load = [&](unsigned int j) {
    const unsigned int c = bid + (rev ? my - 1 - j : j) * G;
    const V* p = xv + (long long)c * kChunkVecs + threadIdx.x;
    const long long lim = g.nv - (long long)c * kChunkVecs - threadIdx.x;
#pragma unroll
    for (int u = 0; u < kVPT; ++u)
      if ((long long)u * kThreads < lim) r[u] = load_stream(p + u * kThreads);
  };
  if (my) load(0);
  for (unsigned int j = 0; j < my; ++j) {
    const unsigned int c = bid + (rev ? my - 1 - j : j) * G;
    const long long lim = g.nv - (long long)c * kChunkVecs - threadIdx.x;
    unsigned int off = off0;
#pragma unroll
    for (int u = 0; u < kVPT; ++u) {
      if ((long long)u * kThreads < lim) {
#pragma unroll
        for (int e = 0; e < kVec; ++e) fk(Ops<T>::get(r[u], e), off);
      }
    }
    if (j + 1 < my) load(j + 1);
    const unsigned int k = (off - off0) / kSlot;
    unsigned int incl = k;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const unsigned int total = __shfl_sync(0xffffffffu, incl, 31);
    if (total) {
      unsigned int b0 = 0;
      if (lane == 31) b0 = atomicAdd(cnt, total);
      b0 = __shfl_sync(0xffffffffu, b0, 31);
      // each lane copies its own slots (so no lane reads another's): its q-th kept element
      // goes to b0 + (kept by lower lanes) + q
      T* dst = zr + b0 + (incl - k);
      const unsigned int maxk = __reduce_max_sync(0xffffffffu, k);
      for (unsigned int q = 0; q < maxk; ++q) {
        const bool act = q < k;
        T v = T(0);
        if (act) {
          ld_shared(off0 + q * kSlot, v);
          dst[q] = v;
        }
        on_kept(v, act);
      }
    }
  }
}

// Sums up to 6 per-thread values over the CTA in one exchange (fixed order, so every
// CTA that sums the same data gets the same bits).  Result valid in every thread.
// ---------------------------------------------------------------------------------
// The kernel.
// ---------------------------------------------------------------------------------
template <typename T>
struct BracketState {
  T a, b, t;
  long long cle_a, clt_b, cle_b;
  double dF;
  float sigma;
  int fx;           // fraction bits of the fixed-point cost total of this pass
  int it, use_bisect, stalled, compact;
  int first;        // 1: the multiplicities of the extremes are still estimates
  int dfv;          // 1: dF = Phi(b) - Phi(a) is known (else the next iterate bisects)
  int plain_start;  // 1: the bracket started at the data's extremes
  int learned;      // proposal: 0 none, 1 used, 2 failed its count check on a side
  int phase;        // 0 run, 1 done, 2 finish, 3 NaN, 4 internal error
  int how;          // GBS_HOW_* of a resolved result
  long long clt_res;// #(x < result) for the sign of a zero result
  T result;
};

// Grid totals of the pass partials in `slot` (identical in every CTA: fixed order).
struct Totals {
  unsigned long long c_lt, c_le, c_aux, c_aux2, c_reg;
  double S;
};
__device__ __forceinline__ Totals grid_totals(const PassPartial* part, unsigned int G, Sum6* scratch) {
  Sum6 v;
  v.u[0] = v.u[1] = v.u[2] = v.u[3] = v.u[4] = 0;
  v.d = 0.0;
  for (unsigned int i = threadIdx.x; i < G; i += kThreads) {
    const PassPartial* p = &part[i];
    v.u[0] += __ldcg(&p->c_lt); v.u[1] += __ldcg(&p->c_le); v.u[2] += __ldcg(&p->c_aux);
    v.u[3] += __ldcg(&p->c_aux2); v.u[4] += __ldcg(&p->c_reg); v.d += __ldcg(&p->S);
  }
  const Sum6 r = block_sum6(v, scratch);
  Totals t;
  t.c_lt = r.u[0]; t.c_le = r.u[1]; t.c_aux = r.u[2]; t.c_aux2 = r.u[3]; t.c_reg = r.u[4]; t.S = r.d;
  return t;
}

// Per-thread accumulators of one cutting-plane pass.
struct PassAcc {
  unsigned int lt, le, xa, xb;
  float S;
};

// Comparison thresholds of one pass (CmpOf images): a, t and b as needed by "<" and "<=".
template <typename T>
struct Thr {
  typename Ops<T>::C a_le, t_lt, t_le, b_lt, b_le;
};
template <typename T>
__device__ __forceinline__ Thr<T> thresholds(T a, T t, T b) {
  Thr<T> h;
  h.a_le = CmpOf<T>::le(a);
  h.t_lt = CmpOf<T>::lt(t);
  h.t_le = CmpOf<T>::le(t);
  h.b_lt = CmpOf<T>::lt(b);
  h.b_le = CmpOf<T>::le(b);
  return h;
}

// The first radix round of the finish over the elements of (a, b]: their keys lie above
// k_lo and at most k_hi (a zero end takes the key of +0, which makes the key test the IEEE
// one), the leading `known` bits where ukey(a) + 1 and ukey(b) agree form the prefix, and
// the digit is the next kDigitBits (fewer at the end of the key).
template <typename T>
struct FinDigit {
  using U = typename KeyOf<T>::U;
  U k_lo, k_hi, prefix;
  int known, sh;
  unsigned int dmask;
  bool exact;   // no zero end: every element of (a, b] passes the key and prefix tests
};
template <typename T>
__device__ __forceinline__ FinDigit<T> fin_digit0(T a, T b) {
  using U = typename KeyOf<T>::U;
  constexpr int W = KeyOf<T>::kBitsW;
  FinDigit<T> f;
  const U lo = ukey(a) + 1, hi = ukey(b);
  const U diff = lo ^ hi;
  const int known = diff == 0 ? W : (W == 32 ? __clz((unsigned int)diff) : __clzll((unsigned long long)diff));
  f.known = known;
  f.prefix = known == 0 ? U(0) : (known == W ? hi : (U)(hi >> (W - known)));
  f.k_lo = ukey(a == T(0) ? T(0) : a);
  f.k_hi = ukey(b == T(0) ? T(0) : b);
  const int nbits = (W - known) < kDigitBits ? (W - known) : kDigitBits;
  f.sh = W - known - nbits;
  f.dmask = (1u << nbits) - 1u;
  f.exact = a != T(0) && b != T(0);
  return f;
}

// One streaming pass over x at the iterate t (Algorithm 1, step 1.2).  FIRST also counts
// #(x <= a) and #(x < b); COMPACT also appends the elements of (a, b] to region `zr`, and
// a compacting pass after the first only does that (no cut at t: the finish ranks the
// compacted elements of (a, b] exactly, so a last cut would only have shrunk the range
// whose elements it has to read anyway).
// Kept out of line so that its registers are allocated apart from the kernel's control.
// A compacting pass after the first also forms the finish's first-round histogram of the
// elements it keeps (digits by dg, counts in hist), so that the finish starts at its digit
// search.
template <typename T, bool FIRST, bool COMPACT>
__device__ __noinline__ bool cut_pass(const T* __restrict__ x, const Geometry<T>& geo, bool rev, Thr<T> h,
                                      float nsig, float tsig, T* __restrict__ zr, unsigned int* s_cnt,
                                      T* wb, unsigned int* hist, const FinDigit<T>* dgp, PassAcc& acc) {
  using U = typename KeyOf<T>::U;
  constexpr int W = KeyOf<T>::kBitsW;
  using C = typename Ops<T>::C;
  using V = typename Ops<T>::V;
  unsigned int lt = 0, le = 0, xa = 0, xb = 0;
  float S = 0.f;
  auto f = [&](T v) {
    core(v, h.a_le, h.t_lt, h.t_le, nsig, tsig, lt, le, S);
    if (FIRST) {
      const C cv = CmpOf<T>::of(v);
      xa += (cv <= h.a_le);
      xb += (cv < h.b_lt);
    }
  };
  if (COMPACT) {
    auto fk = [&](T v, unsigned int& off) {
      if (FIRST) {
        core_keep(v, h.a_le, h.t_lt, h.t_le, h.b_le, nsig, tsig, lt, le, S, off);
        const C cv = CmpOf<T>::of(v);
        xa += (cv <= h.a_le);
        xb += (cv < h.b_lt);
      } else {
        keep_only(v, h.a_le, h.b_le, off);
      }
    };
    // the histogram of the kept elements (act: the lane holds one).  Per-lane shared-memory
    // adds: warp-wide aggregation (ballots over the lanes' digits) costs more here than
    // the conflicts of tied values it would save.
    auto on_kept = [&](T v, bool act) {
      if (!FIRST && act) {
        const U key = ukey(v);
        const FinDigit<T>& dg = *dgp;   // shared memory: read per kept element, not held
        if (dg.exact || (key > dg.k_lo && key <= dg.k_hi &&
                         (dg.known == 0 || (U)(key >> (W - dg.known)) == dg.prefix)))
          atomicAdd(&hist[(unsigned int)(key >> dg.sh) & dg.dmask], 1u);
      }
    };
    auto hist_one = [&](T v) {   // one element outside the warp-wide copy-out
      if (!FIRST) {
        const U key = ukey(v);
        const FinDigit<T>& dg = *dgp;
        if (key > dg.k_lo && key <= dg.k_hi && (dg.known == 0 || (U)(key >> (W - dg.known)) == dg.prefix))
          atomicAdd(&hist[(unsigned int)(key >> dg.sh) & dg.dmask], 1u);
      }
    };
    if ((long long)blockIdx.x * kThreads + threadIdx.x < geo.head + (geo.n - geo.tail0)) {
      const unsigned int o0 = smem_u32(wb + (threadIdx.x & 31));
      auto fe = [&](T v) {   // the scalar head and tail: kept elements go straight to zr
        unsigned int o = o0;
        fk(v, o);
        if (o != o0) {
          zr[atomicAdd(s_cnt, 1u)] = v;
          hist_one(v);
        }
      };
      stream_edges(x, geo, fe);
    }
    stream_chunks_compact(x, geo, rev, fk, zr, s_cnt, wb, on_kept);
  } else if (Ops<T>::kVec == 2 && !FIRST && core64_fast_ok((unsigned long long)h.a_le, (unsigned long long)h.t_lt,
                                                               (unsigned long long)h.t_le)) {
    // float64: decisions on the keys' high words (elem.cuh)
    const unsigned long long ka = (unsigned long long)h.a_le, kt = (unsigned long long)h.t_lt;
    const uint32_t a_hi = (uint32_t)(ka >> 32), t_hi = (uint32_t)(kt >> 32);
    auto f64 = [&](T v) { core64_fast((double)v, ka, kt, a_hi, t_hi, nsig, tsig, lt, le, S); };
    stream_edges(x, geo, f64);
    stream_chunks(x, geo, rev, f64);
  } else {
    stream_edges(x, geo, f);
    stream_chunks(x, geo, rev, f);
  }
  acc.lt = lt; acc.le = le; acc.xa = xa; acc.xb = xb; acc.S = S;
  return true;
}

// Per-thread accumulators of pass 0.
template <typename T>
struct StatsAcc {
  typename Ops<T>::C mn, mx;
  unsigned int nnan, nneg, npos, seen;
  float sum;   // sum over finite x of (x - x0) * sigma
};

// Pass 0 (Sec. 3, step 0): finite extremes and sum; NaN and infinities take a rare branch.
template <typename T>
__device__ __noinline__ bool stats_pass(const T* __restrict__ x, const Geometry<T>& geo, float sig,
                                        float x0s, StatsAcc<T>& out) {
  using C = typename Ops<T>::C;
  using V = typename Ops<T>::V;
  C mn = cmp_pos_inf<T>(), mx = cmp_neg_inf<T>();
  unsigned int nnan = 0, nneg = 0, npos = 0, seen = 0;
  float sum = 0.f;
  auto f = [&](T v) {
    ++seen;
    if (Ops<T>::is_finite(v)) {
      const C cv = CmpOf<T>::of(v);
      mn = cv < mn ? cv : mn;
      mx = cv > mx ? cv : mx;
      sum += fmaf(Ops<T>::img(v), sig, -x0s);
    } else {
      nnan += Ops<T>::is_nan(v);
      nneg += Ops<T>::is_neginf(v);
      npos += Ops<T>::is_posinf(v);
    }
  };
  stream_edges(x, geo, f);
  stream_chunks(x, geo, false, f);
  out.mn = mn; out.mx = mx; out.nnan = nnan; out.nneg = nneg; out.npos = npos; out.seen = seen; out.sum = sum;
  return true;
}

// Per-thread accumulators of the checks of a proposed bracket (a, b] in pass 0.
struct ProposalAcc {
  unsigned int la, lblt;   // #(x <= a), #(x < b); #(x <= b) = #(x <= a) + #compacted
};

// Pass 0 with a proposed bracket, the lean form: the NaN count, #(x <= a), #(x < b) and the
// elements of (a, b] compacted into this CTA's region.  The extremes, the infinities and
// the sum are needed only when an end of the proposal fails its check; the plain pass 0
// then follows.
template <typename T>
__device__ __noinline__ bool stats_pass_learned(const T* __restrict__ x, const Geometry<T>& geo,
                                                typename Ops<T>::C ca, typename Ops<T>::C cb_lt,
                                                typename Ops<T>::C cb_le, T* __restrict__ zr, unsigned int* s_cnt,
                                                T* wb, StatsAcc<T>& out, ProposalAcc& pa) {
  using C = typename Ops<T>::C;
  unsigned int nnan = 0, la = 0, lblt = 0;
  auto f = [&](T v) {
    nnan += Ops<T>::is_nan(v);
    const C cv = CmpOf<T>::of(v);
    la += (cv <= ca);
    lblt += (cv < cb_lt);
  };
  auto keep = [&](T v) { const C cv = CmpOf<T>::of(v); return !Ops<T>::is_nan(v) & (cv > ca) & (cv <= cb_le); };
  if ((long long)blockIdx.x * kThreads + threadIdx.x < geo.head + (geo.n - geo.tail0)) {
    auto fe = [&](T v) {
      f(v);
      if (keep(v)) zr[atomicAdd(s_cnt, 1u)] = v;
    };
    stream_edges(x, geo, fe);
  }
  auto fk = [&](T v, unsigned int& off) {
    f(v);
    const bool w = keep(v);
    if (w) st_shared(off, v);
    off += w ? 32u * (unsigned int)sizeof(T) : 0u;
  };
  auto no_hist = [](T, bool) {};
  stream_chunks_compact(x, geo, false, fk, zr, s_cnt, wb, no_hist);
  out.mn = cmp_pos_inf<T>(); out.mx = cmp_neg_inf<T>();
  out.nnan = nnan; out.nneg = 0; out.npos = 0; out.seen = nnan; out.sum = 0.f;
  pa.la = la; pa.lblt = lblt;
  return true;
}

// The finish's digit histogram: dynamic shared memory of kHistBytes (apart from the
// compaction staging buffers, since the compacting pass fills it).
constexpr int kHistBytes = 4 * kBins;
extern __shared__ __align__(16) unsigned int g_hist_smem[];

template <typename T>
__global__ void __launch_bounds__(kThreads, 2) select_kernel(SelArgs<T> A) {
  using C = typename Ops<T>::C;
  using U = typename KeyOf<T>::U;
  using V = typename Ops<T>::V;
  constexpr int W = KeyOf<T>::kBitsW;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int bid = blockIdx.x;
  const unsigned int G = gridDim.x;
  const long long n = A.n, k = A.k;

  __shared__ unsigned long long s_u64[kWarps];
  __shared__ double s_f64[kWarps];
  __shared__ BracketState<T> s_br;
  __shared__ unsigned int s_zcnt;
  __shared__ unsigned int s_z2n;   // elements this CTA copied to its segment of z2
  __shared__ int s_found;
  __shared__ unsigned long long s_tns[72];
  __shared__ int s_ntns;
  __shared__ long long s_pops[kMaxIt];
  __shared__ unsigned long long s_tstream[kMaxIt];
  __shared__ double s_iter[kMaxIt];
  __shared__ int s_nk, s_nb;
  __shared__ U s_prefix;
  __shared__ int s_known;
  __shared__ unsigned long long s_rank;
  __shared__ StatsPartial s_st;
  __shared__ Sum6 s_sum6[kWarps + 1];

  // the finish's region offsets and digit histogram, and before them the warps'
  // compaction staging buffers
  constexpr int kOffBytes = 8 * (kMaxGrid + 1);
  __shared__ __align__(16) unsigned char s_big[kChunkBytes > kOffBytes ? kChunkBytes : kOffBytes];
  unsigned long long* s_off = reinterpret_cast<unsigned long long*>(s_big);
  unsigned int* const s_hist = g_hist_smem;   // the finish's digit histogram (dynamic, kHistBytes)
  T* const s_wb = reinterpret_cast<T*>(s_big) + (tid >> 5) * (kChunkBytes / sizeof(T) / kWarps);

  const Geometry<T> geo(A.x, n);
  const long long nch = chunk_count(geo.nv);
  const long long per_thread = per_thread_bound(nch, G, Ops<T>::kVec);

  if (tid == 0) { s_ntns = 0; s_nk = 0; s_nb = 0; }
  // a selection that ends early (a wait that gave up, an internal inconsistency) leaves a
  // quiet NaN in *out; the normal exit overwrites it with the result
  if (A.mode == kModeSelect && bid == 0 && tid == 0) *A.out = T(NAN);
  if (bid == 0) {   // zero the radix histograms (visible after the first barrier)
    for (int i = tid; i < kMaxRounds * kBins; i += kThreads) A.ghist[i] = 0ull;
  }
  auto stamp = [&]() {
    if (bid == 0 && tid == 0 && s_ntns < 72) s_tns[s_ntns++] = globaltimer();
  };
  stamp();

  // Counting pass over x for three predicates: [x <= lo], [x < hi], [x is -0].  Used for
  // the multiplicities of the extremes (array statistics) and the sign of a zero result.
  auto aux_pass = [&](T lo, T hi, unsigned long long* o_le, unsigned long long* o_lt,
                      unsigned long long* o_nz) -> bool {
    const C cl = CmpOf<T>::le(lo), ch = CmpOf<T>::lt(hi);
    unsigned int a0 = 0, a1 = 0, a2 = 0;
    auto f = [&](T v) {
      const C cv = CmpOf<T>::of(v);
      a0 += (cv <= cl);
      a1 += (cv < ch);
      a2 += is_neg_zero_bits<T>(v);
    };
    stream_edges(A.x, geo, f);
    stream_chunks(A.x, geo, false, f);
    PassPartial pp;
    pp.c_lt = block_sum<unsigned long long>(a0, s_u64);
    pp.c_le = block_sum<unsigned long long>(a1, s_u64);
    pp.c_aux = block_sum<unsigned long long>(a2, s_u64);
    pp.c_aux2 = 0; pp.c_reg = 0; pp.S = 0.0;
    if (tid == 0) A.part[bid] = pp;
    if (!grid_sync(A.ctrl, G)) return false;
    stamp();
    Totals t = grid_totals(A.part, G, s_sum6);
    *o_le = t.c_lt; *o_lt = t.c_le; *o_nz = t.c_aux;
    return true;
  };

  if (A.mode == kModeEval) {
    // ---------------- one fused pass at (a, t) ----------------
    const T a = Ops<T>::from_double(A.a_eval), t = Ops<T>::from_double(A.t_eval);
    const C ca = CmpOf<T>::le(a), ct_lt = CmpOf<T>::lt(t), ct_le = CmpOf<T>::le(t);
    const float sig = cost_scale((double)Ops<T>::img(t) - (double)Ops<T>::img(a), per_thread);
    const float tsig = Ops<T>::img(t) * sig;
    unsigned int lt = 0, le = 0, lea = 0;
    float S = 0.f;
    auto f = [&](T v) {
      core(v, ca, ct_lt, ct_le, -sig, tsig, lt, le, S);
      lea += (CmpOf<T>::of(v) <= ca);
    };
    stream_edges(A.x, geo, f);
    stream_chunks(A.x, geo, false, f);
    PassPartial pp;
    pp.c_lt = block_sum<unsigned long long>(lt, s_u64);
    pp.c_le = block_sum<unsigned long long>(le, s_u64);
    pp.c_aux = block_sum<unsigned long long>(lea, s_u64);
    pp.c_aux2 = 0; pp.c_reg = 0;
    pp.S = block_sum<double>((double)S, s_f64);
    if (tid == 0) A.part[bid] = pp;
    if (!grid_sync(A.ctrl, G)) return;
    Totals tt = grid_totals(A.part, G, s_sum6);
    if (bid == 0 && tid == 0) {
      gbs_cost_eval e;
      e.c_lt_t = (long long)tt.c_lt; e.c_le_t = (long long)tt.c_le; e.c_le_a = (long long)tt.c_aux; e.pad = 0;
      e.S = tt.S / (double)sig;
      e.dphi = ((double)e.c_le_a - (double)k + 0.5) * ((double)t - (double)a) + e.S;
      *A.eval_out = e;
    }
    return;
  }

  // learned bracket proposal (the same decision in every CTA)
  T prop_a = T(0), prop_b = T(0);
  bool prop_ok = false;
  if (A.proposal != nullptr && A.mode == kModeSelect) {
    const double pa0 = __ldcg(&A.proposal[0]), pb0 = __ldcg(&A.proposal[1]), pv = __ldcg(&A.proposal[2]);
    prop_a = Ops<T>::from_double(pa0);
    prop_b = Ops<T>::from_double(pb0);
    prop_ok = pv > 0.5 && Ops<T>::is_finite(prop_a) && Ops<T>::is_finite(prop_b) && prop_a < prop_b;
  }

  // ---------------- pass 0: finite extremes, sum, non-finite counts (Sec. 3, step 0) ----------------
  // With a proposed bracket, pass 0 is first the lean check of the proposal; the plain
  // pass 0 follows only when an end fails its check (the same decision in every CTA).
  bool lean = prop_ok;
  bool hist0 = false;   // the compacting pass formed the finish's first-round histogram
  __shared__ unsigned long long s_prop[4];   // #(x <= a), #(x < b), #(x <= b), #compacted
  for (;;) {
    {
      const float sig = A.sigma_stats;
      float x0 = 0.f;   // per-thread shift of the float32 sum
      {
        const long long gtid = (long long)bid * kThreads + tid;
        const long long i0 = gtid < geo.head ? gtid : geo.head + gtid * Ops<T>::kVec;
        if (i0 < n) {
          const T e = A.x[i0];
          if (Ops<T>::is_finite(e)) x0 = Ops<T>::img(e);
        }
      }
      const float x0s = x0 * sig;
      StatsAcc<T> sa;
      ProposalAcc pa;
      pa.la = pa.lblt = 0;
      if (lean) {
        if (tid == 0) s_zcnt = 0;
        __syncthreads();
        if (!stats_pass_learned<T>(A.x, geo, CmpOf<T>::le(prop_a), CmpOf<T>::lt(prop_b), CmpOf<T>::le(prop_b),
                                   A.z + region_start(bid, nch, G, Ops<T>::kVec), &s_zcnt, s_wb, sa, pa))
          return;
      } else {
        if (!stats_pass<T>(A.x, geo, sig, x0s, sa)) return;
      }
      C mn = sa.mn, mx = sa.mx;
      const unsigned int nnan = sa.nnan, nneg = sa.nneg, npos = sa.npos, seen = sa.seen;
      const float sum = sa.sum;
      __shared__ C s_m[kWarps], s_M[kWarps];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const C omn = __shfl_xor_sync(0xffffffffu, mn, o);
        const C omx = __shfl_xor_sync(0xffffffffu, mx, o);
        mn = omn < mn ? omn : mn;
        mx = omx > mx ? omx : mx;
      }
      if (lane == 0) { s_m[tid >> 5] = mn; s_M[tid >> 5] = mx; }
      const unsigned int nfin = seen - nnan - nneg - npos;
      const unsigned long long b_nan = block_sum<unsigned long long>(nnan, s_u64);
      const unsigned long long b_neg = block_sum<unsigned long long>(nneg, s_u64);
      const unsigned long long b_pos = block_sum<unsigned long long>(npos, s_u64);
      const unsigned long long b_fin = block_sum<unsigned long long>(nfin, s_u64);
      const double own = (double)sum / (double)sig + (double)nfin * (double)x0;
      const double b_sum = block_sum<double>(own, s_f64);
      Sum6 p6;
      p6.u[0] = pa.la; p6.u[1] = pa.lblt; p6.u[2] = 0; p6.u[3] = 0; p6.u[4] = 0; p6.d = 0.0;
      if (lean) {
        __syncthreads();
        p6.u[3] = tid == 0 ? s_zcnt : 0u;
      }
      const Sum6 b6 = lean ? block_sum6(p6, s_sum6) : p6;
      if (tid == 0) {
        C bm = s_m[0], bM = s_M[0];
        for (int w = 1; w < kWarps; ++w) {
          bm = s_m[w] < bm ? s_m[w] : bm;
          bM = s_M[w] > bM ? s_M[w] : bM;
        }
        StatsPartial sp;
        sp.n_nan = b_nan; sp.n_neginf = b_neg; sp.n_posinf = b_pos; sp.n_negzero = 0; sp.n_finite = b_fin;
        sp.mn = (double)cmp_value(bm, T()); sp.mx = (double)cmp_value(bM, T());
        sp.c_mn = 0; sp.c_mx = 0; sp.sum = b_sum;
        sp.c_le_a = b6.u[0]; sp.c_lt_b = b6.u[1]; sp.c_le_b = b6.u[0] + b6.u[3]; sp.c_reg = b6.u[3];
        sp.s_ab = 0.0;
        A.spart[bid] = sp;
      }
    }
    if (!grid_sync(A.ctrl, G)) return;
    stamp();

    // every CTA: reduce the G pass-0 partials in the same order (thread i takes partials
    // i, i + kThreads, ...; then a fixed warp / block tree)
    {
      Sum6 v;
      v.u[0] = v.u[1] = v.u[2] = v.u[3] = v.u[4] = 0;
      v.d = 0.0;
      double m = INFINITY, M = -INFINITY;
      for (unsigned int i = tid; i < G; i += kThreads) {
        const StatsPartial* p = &A.spart[i];
        v.u[0] += __ldcg(&p->n_nan); v.u[1] += __ldcg(&p->n_neginf);
        v.u[2] += __ldcg(&p->n_posinf); v.u[3] += __ldcg(&p->n_finite);
        const double pm = __ldcg(&p->mn), pM = __ldcg(&p->mx);
        m = pm < m ? pm : m;
        M = pM > M ? pM : M;
        v.d += __ldcg(&p->sum);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double om = __shfl_xor_sync(0xffffffffu, m, o), oM = __shfl_xor_sync(0xffffffffu, M, o);
        m = om < m ? om : m;
        M = oM > M ? oM : M;
      }
      __shared__ double s_mm[kWarps], s_MM[kWarps];
      if (lane == 0) { s_mm[tid >> 5] = m; s_MM[tid >> 5] = M; }
      const Sum6 r = block_sum6(v, s_sum6);   // its barriers also publish s_mm / s_MM
      Sum6 w;
      w.u[0] = w.u[1] = w.u[2] = w.u[3] = w.u[4] = 0;
      w.d = 0.0;
      if (lean) {
        for (unsigned int i = tid; i < G; i += kThreads) {
          const StatsPartial* p = &A.spart[i];
          w.u[0] += __ldcg(&p->c_le_a); w.u[1] += __ldcg(&p->c_lt_b); w.u[2] += __ldcg(&p->c_le_b);
          w.u[3] += __ldcg(&p->c_reg);
        }
        w = block_sum6(w, s_sum6);
      }
      if (tid == 0) {
        StatsPartial t;
        t.n_nan = r.u[0]; t.n_neginf = r.u[1]; t.n_posinf = r.u[2]; t.n_finite = r.u[3];
        t.n_negzero = 0; t.c_mn = t.c_mx = 0; t.sum = r.d;
        t.c_le_a = w.u[0]; t.c_lt_b = w.u[1]; t.c_le_b = w.u[2]; t.c_reg = w.u[3]; t.s_ab = 0.0;
        t.mn = s_mm[0]; t.mx = s_MM[0];
        for (int w = 1; w < kWarps; ++w) {
          t.mn = s_mm[w] < t.mn ? s_mm[w] : t.mn;
          t.mx = s_MM[w] > t.mx ? s_MM[w] : t.mx;
        }
        if (lean) {
          s_prop[0] = t.c_le_a; s_prop[1] = t.c_lt_b; s_prop[2] = t.c_le_b; s_prop[3] = t.c_reg;
        } else if (prop_ok) {   // the plain pass after a failed end: keep the proposal's counts
          t.c_le_a = s_prop[0]; t.c_lt_b = s_prop[1]; t.c_le_b = s_prop[2]; t.c_reg = s_prop[3];
        }
        s_st = t;
      }
    }
    __syncthreads();
    if (lean) {
      const bool ok_a = (long long)s_st.c_le_a < k, ok_b = k <= (long long)s_st.c_le_b;
      if (s_st.n_nan == 0 && !(ok_a && ok_b)) {   // an end failed: the plain pass 0
        lean = false;
        if (!grid_sync(A.ctrl, G)) return;       // every CTA has read the partials
        continue;
      }
    }
    break;
  }
  // both ends of a proposal checked (the lean pass 0 only): the extremes are not known
  const bool prop_both = prop_ok && lean && s_st.n_nan == 0;
  const StatsPartial& st = s_st;     // read from shared memory where needed
  const long long nneg = (long long)st.n_neginf, npos = (long long)st.n_posinf;

  if (A.mode == kModeStats) {
    // multiplicities of the extremes and the -0 count need one more pass
    const bool any = st.n_finite > 0;
    unsigned long long cle = 0, clt = 0, nz = 0;
    if (!aux_pass((T)(any ? st.mn : 0.0), (T)(any ? st.mx : 0.0), &cle, &clt, &nz)) return;
    if (bid == 0 && tid == 0) {
      gbs_array_stats o;
      o.n = n;
      o.n_nan = (long long)st.n_nan; o.n_neginf = nneg; o.n_posinf = npos;
      o.n_negzero = (long long)nz; o.n_finite = (long long)st.n_finite;
      o.min = any ? st.mn + 0.0 : 0.0; o.max = any ? st.mx + 0.0 : 0.0;   // + 0.0: a zero extreme as +0
      o.c_le_min = any ? (long long)cle : 0;
      o.c_lt_max = any ? (long long)clt - (long long)st.n_nan : 0;
      o.sum = st.sum;
      *A.stats_out = o;
    }
    return;
  }

  // ---------------- trivial resolution and the starting bracket ----------------
  if (tid == 0) {
    BracketState<T> br;
    br.it = 0; br.use_bisect = 0; br.stalled = 0; br.compact = 0; br.phase = 0; br.first = 0;
    br.dfv = 1; br.plain_start = 1; br.learned = 0;
    br.how = GBS_HOW_NONE; br.clt_res = -1;
    br.result = T(0); br.sigma = 1.f; br.fx = kSFixBits;
    br.a = T(0); br.b = T(0); br.t = T(0); br.cle_a = 0; br.clt_b = 0; br.cle_b = 0; br.dF = 0.0;
    if (st.n_nan > 0) {
      br.phase = 3;
      br.result = T(NAN);
    } else if (prop_both) {
      // the proposed bracket (a, b] passed its count check in the lean pass 0
      const long long pla = (long long)st.c_le_a, plb_lt = (long long)st.c_lt_b, plb = (long long)st.c_le_b;
      br.learned = 1;
      if (plb_lt < k) {                        // x_(k) is b itself
        br.phase = 1; br.result = prop_b; br.how = GBS_HOW_HIT; br.clt_res = plb_lt;
      } else {
        br.a = prop_a; br.b = prop_b; br.cle_a = pla; br.clt_b = plb_lt; br.cle_b = plb;
        br.first = 0; br.plain_start = 0; br.dfv = 0;   // Phi(b) - Phi(a) unknown: bisect first
        // already compacted in pass 0: straight to the finish when the bracket holds at
        // most max(cap, n/8) elements (cheaper than the cutting-plane passes it saves)
        if (plb - pla <= (A.cap > n / 8 ? A.cap : n / 8))
          br.phase = ((long long)st.c_reg == plb - pla) ? 2 : 4;
      }
    } else if (k <= nneg) {
      br.phase = 1; br.result = T(-INFINITY); br.how = GBS_HOW_NEGINF;
    } else if (k > n - npos) {
      br.phase = 1; br.result = T(INFINITY); br.how = GBS_HOW_POSINF;
    } else {
      const T m = (T)st.mn, M = (T)st.mx;
      const T a0 = Ops<T>::next_down(m);
      if (!(m < M)) {             // every finite element has the same value
        br.phase = 1; br.result = m; br.how = GBS_HOW_MIN; br.clt_res = nneg;
      } else if (k == nneg + 1) { // the smallest finite element, whatever its multiplicity
        br.phase = 1; br.result = m; br.how = GBS_HOW_MIN; br.clt_res = nneg;
      } else if (k == n - npos) { // the largest finite element
        br.phase = 1; br.result = M; br.how = GBS_HOW_MAX; br.clt_res = 0;
      } else {
        if (Ops<T>::is_finite(a0)) {
          // (a0, M] with a0 the float below m: #(x <= a0) = n_-inf and #(x <= M) =
          // n - n_+inf are exact, and so is Phi(M) - Phi(a0), from the sum of the finite
          // elements; #(x < M) takes the paper's unique-extreme closed form (Sec. 3,
          // step 0) until b first moves.
          br.a = a0; br.b = M;
          br.cle_a = nneg; br.clt_b = n - npos - 1; br.cle_b = n - npos; br.first = 0;
          const double gL = (double)(nneg - k) + 0.5;
          const double nfin = (double)(n - nneg - npos);
          br.dF = gL * ((double)M - (double)a0) + nfin * (double)M - st.sum;
        } else {
          // m is the lowest finite value: start at (m, M] from the unique-extreme closed
          // forms; the first pass counts #(x <= m) and #(x < M) and corrects the state.
          br.a = m; br.b = M;
          br.cle_a = nneg + 1; br.clt_b = n - npos - 1; br.cle_b = n - npos; br.first = 1;
          const double gL = (double)(br.cle_a - k) + 0.5;
          const double inner = st.sum - (double)m - (double)M;
          br.dF = gL * ((double)M - (double)m) + (double)(br.clt_b - br.cle_a) * (double)M - inner;
        }
        if (prop_ok) {
          // an end of the proposed bracket failed its check in the lean pass 0; the other
          // end still narrows the start
          const long long pla = (long long)st.c_le_a, plb_lt = (long long)st.c_lt_b, plb = (long long)st.c_le_b;
          const bool va = pla < k, vb = k <= plb;
          br.learned = 2;
          if (vb) {                              // (m, b]: a falls back to the minimum
            br.b = prop_b; br.clt_b = plb_lt; br.cle_b = plb; br.plain_start = 0; br.dfv = 0;
          } else if (va) {                       // (a, M]: b falls back to the maximum
            br.a = prop_a; br.cle_a = pla; br.plain_start = 0; br.dfv = 0;
          }
        }
      }
    }
    s_br = br;
  }
  __syncthreads();

  // ---------------- cutting-plane passes (Algorithm 1, steps 1.1-1.4) ----------------
  int pass = 0;
  while (s_br.phase == 0) {
    if (tid == 0) {   // step 1.1: next iterate (identical in every CTA)
      BracketState<T> br = s_br;
      const long long pop = br.cle_b - br.cle_a;
      br.compact = (pop <= A.cap) || (br.it >= A.maxit) || (br.stalled >= 2);
      const double gL = (double)(br.cle_a - k) + 0.5;
      const double gR = (double)(br.clt_b - k) + 0.5;
      T t;
      if (br.use_bisect || !br.dfv) {
        const U ka = ukey(br.a), kb = ukey(br.b);
        const U mid = ka + (kb - ka) / 2;
        t = inside<T>(ukey_value(mid, T()), br.a, br.b);
        if (bid == 0) s_nb++;
      } else {
        const double w = (double)br.b - (double)br.a;
        const double ts = (double)br.a + (gR * w - br.dF) / (gR - gL);
        t = inside<T>(Ops<T>::from_double(ts), br.a, br.b);
        if (bid == 0) s_nk++;
      }
      br.t = t;
      const double width = (double)Ops<T>::img(t) - (double)Ops<T>::img(br.a);
      br.sigma = cost_scale(width, per_thread);
      br.fx = cost_fix_bits(width, per_thread, br.sigma);
      s_br = br;
    }
    __syncthreads();
    const Thr<T> thr = thresholds<T>(s_br.a, s_br.t, s_br.b);
    const float nsig = -s_br.sigma;
    const float tsig = Ops<T>::img(s_br.t) * s_br.sigma;
    const int first = s_br.first, compact = s_br.compact;
    const bool rev = (pass & 1) == 0;   // pass 0 ran forward
    // a compacting pass after the first also forms the finish's first-round histogram
    __shared__ FinDigit<T> s_dg;
    if (tid == 0) s_dg = fin_digit0(s_br.a, s_br.b);
    const FinDigit<T> dg = fin_digit0(s_br.a, s_br.b);
    const bool fill = compact && !first;
    if (tid == 0) s_zcnt = 0;
    if (fill)
      for (int i = tid; i < kBins; i += kThreads) s_hist[i] = 0;
    __syncthreads();
    PassAcc acc;
    T* zr = A.z + region_start(bid, nch, G, Ops<T>::kVec);
    bool ok;
    if (first) {
      if (compact) ok = cut_pass<T, true, true>(A.x, geo, rev, thr, nsig, tsig, zr, &s_zcnt, s_wb, s_hist, &s_dg, acc);
      else ok = cut_pass<T, true, false>(A.x, geo, rev, thr, nsig, tsig, zr, &s_zcnt, s_wb, s_hist, &s_dg, acc);
    } else {
      if (compact) ok = cut_pass<T, false, true>(A.x, geo, rev, thr, nsig, tsig, zr, &s_zcnt, s_wb, s_hist, &s_dg, acc);
      else ok = cut_pass<T, false, false>(A.x, geo, rev, thr, nsig, tsig, zr, &s_zcnt, s_wb, s_hist, &s_dg, acc);
    }
    if (!ok) return;
    if (bid == 0 && tid == 0 && pass < kMaxIt) s_tstream[pass] = globaltimer();
    const unsigned int lt = acc.lt, le = acc.le, xa = acc.xa, xb = acc.xb;
    const float S = acc.S;
    __syncthreads();   // every append to this CTA's region is done
    if (fill && dg.known < W) {   // the histogram of round 0 (visible after the barrier)
      for (int i = tid; i < kBins; i += kThreads)
        if (s_hist[i]) atomicAdd(&A.ghist[i], (unsigned long long)s_hist[i]);
      hist0 = true;
    }
    Sum6 v6;
    v6.u[0] = lt; v6.u[1] = le; v6.u[2] = xa; v6.u[3] = xb;
    v6.u[4] = (compact && tid == 0) ? s_zcnt : 0u;   // the CTA's count, once
    v6.d = (double)S;
    const Sum6 b6 = block_sum6_t0(v6, s_sum6);
    const int slot = pass & 1;
    if (tid == 0) {
      // the CTA's partial (its compacted count locates its region in the finish) and its
      // share of the pass totals: integer adds, so the totals do not depend on the order
      // in which CTAs arrive; S goes in as a fixed-point integer
      PassPartial pp;
      pp.c_lt = b6.u[0]; pp.c_le = b6.u[1]; pp.c_aux = b6.u[2]; pp.c_aux2 = b6.u[3]; pp.c_reg = b6.u[4];
      pp.S = b6.d;
      A.part[slot * G + bid] = pp;
      unsigned long long* acc = A.ctrl->acc[pass % 3];
#pragma unroll
      for (int q = 0; q < 5; ++q)
        if (b6.u[q]) atomicAdd(&acc[q], b6.u[q]);
      const unsigned long long sfix = __double2ull_rn(ldexp(b6.d, s_br.fx));
      if (sfix) atomicAdd(&acc[5], sfix);
      if (bid == 0) {   // the slot of the next pass (last read before the previous barrier)
        unsigned long long* nxt = A.ctrl->acc[(pass + 1) % 3];
#pragma unroll
        for (int q = 0; q < 6; ++q) nxt[q] = 0ull;
      }
    }
    if (!grid_sync(A.ctrl, G)) return;
    stamp();
    if (tid == 0) {   // steps 1.3-1.4
      Totals tt;
      {
        const unsigned long long* acc = A.ctrl->acc[pass % 3];
        tt.c_lt = __ldcg(&acc[0]); tt.c_le = __ldcg(&acc[1]); tt.c_aux = __ldcg(&acc[2]);
        tt.c_aux2 = __ldcg(&acc[3]); tt.c_reg = __ldcg(&acc[4]);
        tt.S = ldexp((double)__ldcg(&acc[5]), -s_br.fx);
      }
      const BracketState<T> br = s_br;
      BracketState<T> nb = br;
      const long long clt = (long long)tt.c_lt, cle = (long long)tt.c_le;
      if (bid == 0 && br.it < kMaxIt) s_iter[br.it] = (double)br.t;
      nb.it = br.it + 1;
      bool resolved = false;
      if (br.first) {
        const long long cle_m = (long long)tt.c_aux, clt_M = (long long)tt.c_aux2;
        nb.first = 0;
        if (cle_m >= k) {
          nb.phase = 1; nb.result = br.a; nb.how = GBS_HOW_MIN; nb.clt_res = nneg; resolved = true;
        } else if (clt_M < k) {
          nb.phase = 1; nb.result = br.b; nb.how = GBS_HOW_MAX; nb.clt_res = clt_M; resolved = true;
        } else {
          nb.cle_a = cle_m; nb.clt_b = clt_M;
          if (br.plain_start) {
            const double cmn = (double)(cle_m - nneg), cmx = (double)(n - npos - clt_M);
            const double gL = (double)(cle_m - k) + 0.5;
            const double inner = st.sum - cmn * (double)br.a - cmx * (double)br.b;
            nb.dF = gL * ((double)br.b - (double)br.a) + (double)(clt_M - cle_m) * (double)br.b - inner;
          }
        }
        if (resolved && bid == 0 && br.it < kMaxIt) s_pops[br.it] = 0;
      }
      if (!resolved && br.compact && !br.first) {
        // the compaction pass alone: the bracket stays, the finish ranks its elements
        const long long pop = nb.cle_b - nb.cle_a;
        if (bid == 0 && br.it < kMaxIt) { s_pops[br.it] = pop; s_iter[br.it] = (double)NAN; }
        nb.phase = ((long long)tt.c_reg == pop) ? 2 : 4;
      } else if (!resolved) {
        const long long pop = nb.cle_b - nb.cle_a;
        if (clt < k && k <= cle) {
          nb.phase = 1; nb.result = br.t; nb.how = GBS_HOW_HIT; nb.clt_res = clt;
          if (bid == 0 && br.it < kMaxIt) s_pops[br.it] = 0;
        } else {
          const double gL = (double)(nb.cle_a - k) + 0.5;
          const double dphi = gL * ((double)br.t - (double)br.a) + tt.S / (double)br.sigma;
          if (cle < k) {
            nb.a = br.t; nb.cle_a = cle; nb.dF = nb.dF - dphi;
          } else {
            nb.b = br.t; nb.clt_b = clt; nb.cle_b = cle; nb.dF = dphi; nb.dfv = 1;
          }
          const long long npop = nb.cle_b - nb.cle_a;
          if (bid == 0 && br.it < kMaxIt) s_pops[br.it] = npop;
          nb.use_bisect = (!br.use_bisect) && ((double)npop > 0.75 * (double)pop);
          nb.stalled = ((double)npop > 0.875 * (double)pop) ? br.stalled + 1 : 0;
          if (br.compact) {
            nb.phase = ((long long)tt.c_reg == pop) ? 2 : 4;
          }
        }
      }
      s_br = nb;
    }
    __syncthreads();
    ++pass;
  }

  const BracketState<T> fin = s_br;
  if (fin.phase == 4) {
    if (bid == 0 && tid == 0) atomicCAS(&A.ctrl->status, 0, (int)GBS_EINTERNAL);
    return;
  }
  int rounds = 0;
  int extra = 0;
  T result = fin.result;
  long long fpop = 0;
  if (fin.phase == 2) {
    // ---------------- exact finish: radix select inside (a, b] ----------------
    const int slot = (pass - 1) & 1;
    // region offsets (exclusive prefix of the per-CTA compaction counts)
    {   // a thread sums kOffPer consecutive counts, then a scan over the CTA
      constexpr int kOffPer = (kMaxGrid + kThreads - 1) / kThreads;
      unsigned long long v[kOffPer];
      unsigned long long loc = 0;
#pragma unroll
      for (int j = 0; j < kOffPer; ++j) {
        const unsigned int i = tid * kOffPer + j;
        v[j] = i >= G ? 0ull : (pass == 0 ? __ldcg(&A.spart[i].c_reg) : __ldcg(&A.part[slot * G + i].c_reg));
        loc += v[j];
      }
      unsigned long long incl = loc;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
        if ((tid & 31) >= o) incl += y;
      }
      if ((tid & 31) == 31) s_u64[tid >> 5] = incl;
      __syncthreads();
      unsigned long long run = incl - loc;
      for (int w = 0; w < (tid >> 5); ++w) run += s_u64[w];
#pragma unroll
      for (int j = 0; j < kOffPer; ++j) {
        const unsigned int i = tid * kOffPer + j;
        run += v[j];
        if (i < G) s_off[i + 1] = run;
      }
      if (tid == 0) s_off[0] = 0;
    }
    __syncthreads();
    if (tid == 0) {
      s_rank = (unsigned long long)(k - fin.cle_a);
      const U lo = ukey(fin.a) + 1, hi = ukey(fin.b);
      const U diff = lo ^ hi;
      int known = 0;
      if (diff == 0) known = W;
      else known = (W == 32) ? __clz((unsigned int)diff) : __clzll((unsigned long long)diff);
      s_known = known;
      s_prefix = known == 0 ? U(0) : (known == W ? hi : (U)(hi >> (W - known)));
    }
    __syncthreads();
    const unsigned long long P = s_off[G];
    fpop = (long long)P;
    const unsigned long long lo_i = P * bid / G, hi_i = P * (bid + 1) / G;
    const T fa = fin.a, fb = fin.b;
    // (a, b] on keys: x > a <=> key(x) > key_le(a), x <= b <=> key(x) <= key_le(b), where a
    // zero end takes the key of +0 (no NaN reaches the compacted regions)
    const U k_lo = ukey(fa == T(0) ? T(0) : fa), k_hi = ukey(fb == T(0) ? T(0) : fb);
    const int warp = tid >> 5;
    // the second sweep also copies the elements of the digit the first one chose into
    // this CTA's segment of z2, and later sweeps read only those.  Segment g starts at
    // round_down(lo_i) + g kVec, which keeps segments apart and 16-byte aligned, so z2
    // needs P + G kVec elements.
    constexpr unsigned long long kZV = Ops<T>::kVec;
    const bool use_z2 = A.z2 != nullptr && (long long)(P + (unsigned long long)G * kZV) <= A.z2_cap &&
                        P / G < (1ull << 31);
    T* const z2seg = use_z2 ? A.z2 + (lo_i / kZV * kZV + (unsigned long long)bid * kZV) : nullptr;
    if (tid == 0) s_z2n = 0;
    while (s_known < W) {
      const int known = s_known;
      const U prefix = s_prefix;
      const int nbits = (W - known) < kDigitBits ? (W - known) : kDigitBits;
      const int sh = W - known - nbits;
      const unsigned int dmask = (1u << nbits) - 1u;
      const bool copy = use_z2 && rounds == 1 && known + nbits < W;   // a later round will read z2
      const bool from_z2 = use_z2 && rounds >= 2;
      const bool pre = hist0 && rounds == 0;   // the compacting pass formed this round's histogram
      if (!pre) {
      for (int i = tid; i < kBins; i += kThreads) s_hist[i] = 0;
      __syncthreads();
      // One element a lane: the digit of an element of (a, b] under the known prefix goes to
      // the histogram; returns whether it did.  A lane counts one "hot" digit in a register
      // (the digit it met twice in a row most recently, so a run of tied values does not
      // serialise on one shared-memory address).
      unsigned int hot = 0xffffffffu, last = 0xffffffffu, hcnt = 0;
      auto take = [&](T v, bool valid) -> bool {
        const U key = ukey(v);
        const bool ok = valid && (key > k_lo) && (key <= k_hi) && (known == 0 || (U)(key >> (W - known)) == prefix);
        const unsigned int d = (unsigned int)(key >> sh) & dmask;
        // branch-free (lanes of a warp that disagree would otherwise serialise both paths)
        const bool h = ok && d == hot;
        const bool at = ok && !h;
        const bool sw = at && d == last;
        hcnt += h ? 1u : 0u;
        if (at) atomicAdd(&s_hist[d], 1u);
        if (sw && hcnt) atomicAdd(&s_hist[hot], hcnt);
        hot = sw ? d : hot;
        hcnt = sw ? 0u : hcnt;
        last = at ? d : last;
        return ok;
      };
      // The copying sweep appends a warp's taken elements of one trip to this CTA's segment
      // of z2: a prefix over the lanes' counts and one shared atomic a warp and trip (a
      // reservation per element slot serialised the warps on the counter when most
      // elements fall in the chosen digit, as a run of ties does), then each lane stores
      // its own elements one after another: vals(km, dst) stores, from dst on, the trip's
      // elements whose bits are set in km (bit i: the lane's i-th element of the trip).
      auto append = [&](unsigned int km, auto&& vals) {
        const unsigned int kc = (unsigned int)__popc(km);
        unsigned int incl = kc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const unsigned int y = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += y;
        }
        const unsigned int total = __shfl_sync(0xffffffffu, incl, 31);
        if (total) {
          unsigned int base = 0;
          if (lane == 31) base = atomicAdd(&s_z2n, total);
          T* dst = z2seg + __shfl_sync(0xffffffffu, base, 31) + (incl - kc);
          vals(km, dst);
        }
      };
      // a contiguous range [j0, j1) of src (16-byte aligned): 16-byte vectors, kFinU in
      // flight per lane, warp-uniform trips; the scalar head and tail by warp 0
      auto sweep = [&](const T* __restrict__ src, unsigned int j0, unsigned int j1) {
        using V = typename Ops<T>::V;
        constexpr int kVec = Ops<T>::kVec;
        constexpr int kFinU = 2;
        const unsigned int jv0 = (j0 + kVec - 1) / kVec, jv1 = j1 / kVec;
        const V* sv = reinterpret_cast<const V*>(src);
        if (jv0 < jv1) {
          for (unsigned int b = jv0 + (unsigned int)warp * 32; b < jv1; b += (unsigned int)kThreads * kFinU) {
            V r[kFinU];
#pragma unroll
            for (int u = 0; u < kFinU; ++u) {
              const unsigned int iv = b + (unsigned int)u * kThreads + lane;
              if (iv < jv1) r[u] = __ldcg(sv + iv);
            }
            unsigned int km = 0;
#pragma unroll
            for (int u = 0; u < kFinU; ++u) {
              const bool ok = b + (unsigned int)u * kThreads + lane < jv1;
#pragma unroll
              for (int e = 0; e < kVec; ++e)
                km |= take(ok ? Ops<T>::get(r[u], e) : fa, ok) ? 1u << (u * kVec + e) : 0u;
            }
            if (copy)
              append(km, [&](unsigned int m, T* dst) {
                unsigned int q = 0;
#pragma unroll
                for (int u = 0; u < kFinU; ++u)
#pragma unroll
                  for (int e = 0; e < kVec; ++e)
                    if ((m >> (u * kVec + e)) & 1u) dst[q++] = Ops<T>::get(r[u], e);
              });
          }
        }
        if (warp == 0) {   // the elements outside whole vectors (fewer than 2 kVec)
          const unsigned int h1 = jv0 < jv1 ? jv0 * kVec : j1;
          const unsigned int t0 = jv0 < jv1 ? jv1 * kVec : j1;
          const unsigned int nh = h1 - j0, nt = j1 - t0;
          const bool ok = (unsigned int)lane < nh + nt;
          const unsigned int j = (unsigned int)lane < nh ? j0 + lane : t0 + (lane - nh);
          const T v = ok ? __ldcg(src + j) : fa;
          const bool tk = take(v, ok);
          if (copy) append(tk ? 1u : 0u, [&](unsigned int m, T* dst) { if (m) dst[0] = v; });
        }
      };
      if (from_z2) {
        sweep(z2seg, 0u, s_z2n);   // this CTA's own copies (written by its own threads)
      } else {
        unsigned int r = 0;
        {
          unsigned int lo_r = 0, hi_r = G;   // largest r with s_off[r] <= lo_i
          while (hi_r - lo_r > 1) {
            const unsigned int mid = (lo_r + hi_r) / 2;
            if (s_off[mid] <= lo_i) lo_r = mid; else hi_r = mid;
          }
          r = lo_r;
        }
        for (; r < G && s_off[r] < hi_i; ++r) {
          const unsigned long long s0 = s_off[r] > lo_i ? s_off[r] : lo_i;
          const unsigned long long s1 = s_off[r + 1] < hi_i ? s_off[r + 1] : hi_i;
          const T* zr = A.z + region_start(r, nch, G, Ops<T>::kVec);
          sweep(zr, (unsigned int)(s0 - s_off[r]), (unsigned int)(s1 - s_off[r]));
        }
      }
      if (hcnt) atomicAdd(&s_hist[hot], hcnt);
      __syncthreads();
      for (int i = tid; i < kBins; i += kThreads)
        if (s_hist[i]) atomicAdd(&A.ghist[rounds * kBins + i], (unsigned long long)s_hist[i]);
      if (!grid_sync(A.ctrl, G)) return;
      stamp();
      }
      {   // the CTA finds the digit holding rank s_rank: kBins / kThreads bins a thread
        constexpr int kPer = kBins / kThreads;
        unsigned long long h[kPer];
        unsigned long long local = 0;
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
          h[j] = __ldcg(&A.ghist[rounds * kBins + tid * kPer + j]);
          local += h[j];
        }
        unsigned long long incl = local;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += y;
        }
        if (lane == 31) s_u64[warp] = incl;
        if (tid == 0) s_found = 0;
        __syncthreads();
        unsigned long long wbase = 0;
        for (int w = 0; w < warp; ++w) wbase += s_u64[w];
        const unsigned long long want = s_rank;
        const unsigned long long excl = wbase + incl - local;
        __syncthreads();   // every thread has read s_rank
        if (excl < want && want <= excl + local) {
          unsigned long long c = excl;
          int d = 0;
          for (int j = 0; j < kPer; ++j) {
            if (c + h[j] >= want) { d = tid * kPer + j; break; }
            c += h[j];
          }
          s_rank = want - c;
          s_prefix = (U)((prefix << nbits) | (U)d);
          s_known = known + nbits;
          s_found = 1;
        }
        __syncthreads();
        if (tid == 0 && !s_found) {   // no bin holds the rank: inconsistent counts
          atomicCAS(&A.ctrl->status, 0, (int)GBS_EINTERNAL);
          s_known = W;
          s_prefix = 0;                 // ukey_value(0) is a NaN: the result is flagged
        }
      }
      ++rounds;
      __syncthreads();
    }
    result = ukey_value(s_prefix, T());
  } else if (fin.phase == 1 && fin.result == T(0) && fin.clt_res >= 0) {
    // a zero result found by counts: -0 sorts before +0, so count the -0 elements
    unsigned long long d0 = 0, d1 = 0, nz = 0;
    if (!aux_pass(T(0), T(0), &d0, &d1, &nz)) return;
    // x_(k) is a zero: it is -0 when k - #(x < 0) is at most the number of -0 elements
    result = (k - (long long)d1) <= (long long)nz ? T(-0.0) : T(0.0);
    extra = 1;
  }

  if (bid == 0 && tid == 0) {
    if (fin.phase == 3) atomicCAS(&A.ctrl->status, 0, (int)GBS_ENAN);
    *A.out = result;
    gbs_run_stats* rs = A.rs;
    rs->status = ld_relaxed_i32(&A.ctrl->status);
    rs->how = fin.phase == 3 ? GBS_HOW_NONE : fin.phase == 2 ? GBS_HOW_FINISH : fin.how;
    rs->passes = 1 + pass + extra;
    rs->kelley_steps = s_nk;
    rs->bisect_steps = s_nb;
    rs->finish_rounds = rounds;
    rs->grid = (int)G;
    rs->learned = fin.learned;
    rs->n = n; rs->k = k;
    rs->finish_pop = fpop;
    const int ni = pass < kMaxIt ? pass : kMaxIt;
    for (int i = 0; i < kMaxIt; ++i) {
      rs->pops[i] = i < ni ? s_pops[i] : 0;
      rs->iterates[i] = i < ni ? s_iter[i] : 0.0;
      rs->t_stream_ns[i] = i < ni ? s_tstream[i] : 0;
    }
    stamp();
    rs->n_t = s_ntns;
    for (int i = 0; i < 72; ++i) rs->t_ns[i] = i < s_ntns ? s_tns[i] : 0;
  }
}

// ---------------------------------------------------------------------------------
// Host side: grid shape, workspace bounds and the cooperative launch.
// ---------------------------------------------------------------------------------
template <typename T> constexpr int vec_of() { return 16 / (int)sizeof(T); }

// Persistent grid: every SM holds the same number of CTAs (co-residency is required by
// the grid-wide barrier; the launch is cooperative).
template <typename T>
int grid_for(gbs_ctx* c, long long n) {
  int occ = 0;
  if (cudaFuncSetAttribute(select_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, kHistBytes) !=
          cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, select_kernel<T>, kThreads, kHistBytes) != cudaSuccess) {
    cudaGetLastError();
    occ = 1;
  }
  // one CTA per SM below 32 MiB of input (the per-pass barrier and reductions dominate
  // there and cost more with more CTAs), two above (more loads in flight per SM)
  const int bps_auto = (double)n * sizeof(T) >= 32.0 * 1048576.0 ? 2 : 1;
  int bps = c->cfg.blocks_per_sm > 0 ? c->cfg.blocks_per_sm : bps_auto;
  bps = std::max(1, std::min(bps, occ));
  return std::min(kMaxGrid, c->num_sms * bps);
}

// Elements of the compaction area for inputs of up to n elements (any alignment).
template <typename T>
long long z_elems_for(long long n, int grid) {
  const int vec = vec_of<T>();
  return region_start(grid, chunk_count(n / vec + 1), grid, vec);
}
// Elements of the finish's second-level buffer: the brackets compacted once they hold at
// most cap elements (a compaction forced by the iteration limit may exceed it and then
// reads the regions in every round).
// The default cap: a quarter of a float32 array (the finish reads the compacted elements
// at about a tenth of a pass's cost per element, so one more pass saves less than
// finishing a quarter of the array costs), an eighth of a float64 one (whose compaction
// and 64-bit finish rounds cost more per element).
template <typename T>
long long default_cap(long long n) {
  return std::max<long long>(sizeof(T) == 4 ? n / 4 : n / 8, 4096);
}
template <typename T>
long long z2_elems_for(long long n, long long cap, int grid) {
  const long long m = std::min<long long>(n, std::max<long long>(cap, default_cap<T>(n)));
  return (m + 3) / 4 * 4 + (long long)grid * vec_of<T>();
}

template <typename T>
float stats_sigma(long long n, int grid) {
  const int vec = vec_of<T>();
  const long long per_thread = per_thread_bound(chunk_count(n / vec + 1), grid, vec);
  int e = 0;
  while ((1ll << e) < per_thread) ++e;
  return std::ldexp(1.0f, -(e + 2));
}

inline gbs_status launch_propose(gbs_ctx* c, const float* x, long long n, double* p, cudaStream_t s) {
  return launch_propose_f32(c, x, n, p, s);
}
inline gbs_status launch_propose(gbs_ctx* c, const double* x, long long n, double* p, cudaStream_t s) {
  return launch_propose_f64(c, x, n, p, s);
}

template <typename T>
gbs_status launch_select(gbs_ctx* c, const T* x, long long n, long long k, T* out, int mode,
                                double a, double t, gbs_array_stats* sout, gbs_cost_eval* eout,
                                cudaStream_t stream) {
  DeviceGuard g(c->device);
  if (!g.ok) return GBS_ECUDA;
  const int grid = grid_for<T>(c, n);
  const long long zel = z_elems_for<T>(n, grid);
  const long long cap = c->cfg.cap > 0 ? c->cfg.cap : default_cap<T>(n);
  const size_t zb = mode == kModeSelect ? (size_t)(zel + z2_elems_for<T>(n, cap, grid)) * sizeof(T) : 0;
  gbs_status s = gbs_internal_ensure(c, zb);
  if (s != GBS_OK) return s;
  SelArgs<T> A;
  A.x = x; A.n = n; A.k = k; A.out = out; A.mode = mode;
  A.maxit = c->cfg.maxit > 0 ? c->cfg.maxit : 64;
  if (A.maxit > kMaxIt) A.maxit = kMaxIt;
  A.cap = cap;
  A.a_eval = a; A.t_eval = t;
  A.sigma_stats = stats_sigma<T>(n, grid);
  A.ctrl = c->ctrl; A.part = c->part; A.spart = c->spart; A.ghist = c->ghist;
  A.z = reinterpret_cast<T*>(c->z); A.z_elems = zel;
  // the finish's second-level buffer after the compaction regions (16-byte aligned)
  A.z2 = mode == kModeSelect ? A.z + zel : nullptr;
  A.z2_cap = mode == kModeSelect ? z2_elems_for<T>(n, cap, grid) : 0;
  A.rs = c->rs; A.stats_out = sout; A.eval_out = eout;
  A.proposal = nullptr;
  if (cudaMemsetAsync(c->ctrl, 0, sizeof(Ctrl), stream) != cudaSuccess) return GBS_ECUDA;
  if (mode == kModeSelect && cudaMemsetAsync(c->rs, 0, sizeof(gbs_run_stats), stream) != cudaSuccess)
    return GBS_ECUDA;
  // learned starting bracket for a median of a large enough array
  if (mode == kModeSelect && c->cfg.use_learned && c->model_loaded && k == (n + 1) / 2 && n >= kLearnMinN) {
    double* prop = reinterpret_cast<double*>(c->aux);
    if (launch_propose(c, x, n, prop, stream) == GBS_OK) A.proposal = prop;
  }
  void* args[] = {&A};
  cudaError_t e = cudaLaunchCooperativeKernel((const void*)select_kernel<T>, dim3(grid), dim3(kThreads), args,
                                              kHistBytes, stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return GBS_ECUDA;
  }
  c->last_stream = stream;
  c->last_grid = grid;
  return GBS_OK;
}


gbs_status run_select(gbs_ctx* c, const float* x, long long n, long long k, float* out, int mode, double a,
                      double t, gbs_array_stats* sout, gbs_cost_eval* eout, cudaStream_t stream) {
  return launch_select<float>(c, x, n, k, out, mode, a, t, sout, eout, stream);
}
gbs_status run_select(gbs_ctx* c, const double* x, long long n, long long k, double* out, int mode, double a,
                      double t, gbs_array_stats* sout, gbs_cost_eval* eout, cudaStream_t stream) {
  return launch_select<double>(c, x, n, k, out, mode, a, t, sout, eout, stream);
}
// Pieces of the float32 launch for callers that bring their own scratch.
long long select_z_elems_f32(long long n, int grid) { return z_elems_for<float>(n, grid); }
float select_stats_sigma_f32(long long n, int grid) { return stats_sigma<float>(n, grid); }
int select_occupancy_f32() {
  int occ = 0;
  if (cudaFuncSetAttribute(select_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, kHistBytes) !=
          cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, select_kernel<float>, kThreads, kHistBytes) !=
          cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return occ;
}
cudaError_t select_launch_f32(const SelArgs<float>& A, int grid, cudaStream_t stream) {
  SelArgs<float> a = A;
  void* args[] = {&a};
  const cudaError_t e =
      cudaFuncSetAttribute(select_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, kHistBytes);
  if (e != cudaSuccess) return e;
  return cudaLaunchCooperativeKernel((const void*)select_kernel<float>, dim3(grid), dim3(kThreads), args,
                                     kHistBytes, stream);
}

gbs_status reserve_select(gbs_ctx* c, long long n, int elem_bytes) {
  DeviceGuard g(c->device);
  if (!g.ok) return GBS_ECUDA;
  if (elem_bytes == 4) {
    const long long cap = c->cfg.cap > 0 ? c->cfg.cap : default_cap<float>(n);
    const int grid = grid_for<float>(c, n);
    return gbs_internal_ensure(c, (size_t)(z_elems_for<float>(n, grid) + z2_elems_for<float>(n, cap, grid)) * 4);
  }
  const long long cap = c->cfg.cap > 0 ? c->cfg.cap : default_cap<double>(n);
  const int grid = grid_for<double>(c, n);
  return gbs_internal_ensure(c, (size_t)(z_elems_for<double>(n, grid) + z2_elems_for<double>(n, cap, grid)) * 8);
}

}  // namespace gbs
