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
#include "select.cuh"
#include "api_internal.h"

namespace gbs {

// ---------------------------------------------------------------------------------
// Per-type element operations.  cmp(): the value compared against the iterate
// (IEEE float for float32, the signed integer key for float64).  img(): float32 image
// used only for the cost partials.
// ---------------------------------------------------------------------------------
template <typename T> struct Ops;
template <> struct Ops<float> {
  using C = float;
  using V = float4;
  static constexpr int kVec = 4;
  static __device__ __forceinline__ C cmp(float x) { return x; }
  static __device__ __forceinline__ float img(float x) { return x; }
  static __device__ __forceinline__ bool is_nan(float x) { return x != x; }
  static __device__ __forceinline__ bool is_neginf(float x) { return x == -INFINITY; }
  static __device__ __forceinline__ bool is_posinf(float x) { return x == INFINITY; }
  static __device__ __forceinline__ bool is_negzero(float x) { return __float_as_uint(x) == 0x80000000u; }
  static __device__ __forceinline__ bool is_finite(float x) { return fabsf(x) < INFINITY; }
  static __device__ __forceinline__ float next_up(float v) { return nextafterf(v, INFINITY); }
  static __device__ __forceinline__ float next_down(float v) { return nextafterf(v, -INFINITY); }
  static __device__ __forceinline__ float from_double(double v) { return (float)v; }
  template <typename Fn>
  static __device__ __forceinline__ void each(const V& r, Fn& f) { f(r.x); f(r.y); f(r.z); f(r.w); }
  static __device__ __forceinline__ float get(const V& r, int i) {
    return i == 0 ? r.x : i == 1 ? r.y : i == 2 ? r.z : r.w;
  }
};
template <> struct Ops<double> {
  using C = long long;
  using V = double2;
  static constexpr int kVec = 2;
  static __device__ __forceinline__ C cmp(double x) { return (long long)skey(x); }
  static __device__ __forceinline__ float img(double x) {
    return f64_to_f32_trunc((uint64_t)__double_as_longlong(x));
  }
  static __device__ __forceinline__ uint64_t mag(double x) {
    return (uint64_t)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
  }
  static __device__ __forceinline__ bool is_nan(double x) { return mag(x) > 0x7FF0000000000000ull; }
  static __device__ __forceinline__ bool is_neginf(double x) {
    return (uint64_t)__double_as_longlong(x) == 0xFFF0000000000000ull;
  }
  static __device__ __forceinline__ bool is_posinf(double x) {
    return (uint64_t)__double_as_longlong(x) == 0x7FF0000000000000ull;
  }
  static __device__ __forceinline__ bool is_negzero(double x) {
    return (uint64_t)__double_as_longlong(x) == 0x8000000000000000ull;
  }
  static __device__ __forceinline__ bool is_finite(double x) { return mag(x) < 0x7FF0000000000000ull; }
  // neighbours on the float64 grid (finite v; -0 and +0 both step to +-denorm_min)
  static __device__ __forceinline__ double next_up(double v) {
    long long b = __double_as_longlong(v);
    if ((b & 0x7FFFFFFFFFFFFFFFll) == 0) return __longlong_as_double(1ll);
    return __longlong_as_double(b >= 0 ? b + 1 : b - 1);
  }
  static __device__ __forceinline__ double next_down(double v) {
    long long b = __double_as_longlong(v);
    if ((b & 0x7FFFFFFFFFFFFFFFll) == 0) return __longlong_as_double((long long)0x8000000000000001ull);
    return __longlong_as_double(b >= 0 ? b - 1 : b + 1);
  }
  static __device__ __forceinline__ double from_double(double v) { return v; }
  template <typename Fn>
  static __device__ __forceinline__ void each(const V& r, Fn& f) { f(r.x); f(r.y); }
  static __device__ __forceinline__ double get(const V& r, int i) { return i == 0 ? r.x : r.y; }
};

__device__ __forceinline__ float4 load_stream(const float4* p) { return __ldcs(p); }
__device__ __forceinline__ double2 load_stream(const double2* p) { return __ldcs(p); }

constexpr int kUnroll = 4;   // vectors in flight per thread in the streaming loops

// Geometry of the streaming loops over x: an unaligned scalar head, 16-byte vectors,
// a scalar tail.  Shared with the host's region-capacity bound.
template <typename T>
struct Geometry {
  long long head, nv, tail0, n;
  __device__ __forceinline__ Geometry(const T* x, long long n_) : n(n_) {
    constexpr int kVec = Ops<T>::kVec;
    const unsigned long long addr = (unsigned long long)x;
    head = (long long)(((16u - (addr & 15u)) & 15u) / sizeof(T));
    if (head > n) head = n;
    nv = (n - head) / kVec;
    tail0 = head + nv * kVec;
  }
};

// Calls f(element) for every element of x handled by this thread.  Direction
// alternates with `reverse` so that consecutive passes start where the previous one
// ended (the most recently read lines are still in L2).
template <typename T, typename Fn>
__device__ __forceinline__ void stream_x(const T* __restrict__ x, const Geometry<T>& g, bool reverse, Fn& f) {
  using V = typename Ops<T>::V;
  const long long gtid = (long long)blockIdx.x * kThreads + threadIdx.x;
  const long long stride = (long long)gridDim.x * kThreads;
  if (gtid < g.head) f(x[gtid]);
  if (gtid < g.n - g.tail0) f(x[g.tail0 + gtid]);
  const V* xv = reinterpret_cast<const V*>(x + g.head);
  const long long nv = g.nv;
  long long v = gtid;
  for (; v + (kUnroll - 1) * stride < nv; v += kUnroll * stride) {
    V r[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      long long i = v + u * stride;
      r[u] = load_stream(xv + (reverse ? nv - 1 - i : i));
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) Ops<T>::each(r[u], f);
  }
  for (; v < nv; v += stride) {
    V r = load_stream(xv + (reverse ? nv - 1 - v : v));
    Ops<T>::each(r, f);
  }
}

// Streaming loop of a compacting pass: f(element) as above, plus every element with
// keep(element) true is appended to this CTA's region `zr` (counter `*s_cnt` in shared
// memory).  Warp-uniform loop so that the per-warp scan is legal.
template <typename T, typename Fn, typename Keep>
__device__ __forceinline__ void stream_x_compact(const T* __restrict__ x, const Geometry<T>& g,
                                                 bool reverse, Fn& f, Keep& keep, T* __restrict__ zr,
                                                 unsigned int* s_cnt) {
  using V = typename Ops<T>::V;
  constexpr int kVec = Ops<T>::kVec;
  const int lane = threadIdx.x & 31;
  const long long gtid = (long long)blockIdx.x * kThreads + threadIdx.x;
  const long long stride = (long long)gridDim.x * kThreads;
  // scalar head and tail (at most 2*kVec elements, first threads of CTA 0)
  if (gtid < g.head) {
    T e = x[gtid];
    f(e);
    if (keep(e)) zr[atomicAdd(s_cnt, 1u)] = e;
  }
  if (gtid < g.n - g.tail0) {
    T e = x[g.tail0 + gtid];
    f(e);
    if (keep(e)) zr[atomicAdd(s_cnt, 1u)] = e;
  }
  const V* xv = reinterpret_cast<const V*>(x + g.head);
  const long long nv = g.nv;
  const long long wbase0 = gtid - lane;           // warp-uniform
  for (long long wb = wbase0; wb < nv; wb += kUnroll * stride) {
    V r[kUnroll];
    bool ok[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      long long i = wb + lane + u * stride;
      ok[u] = i < nv;
      if (ok[u]) r[u] = load_stream(xv + (reverse ? nv - 1 - i : i));
    }
    unsigned int mask = 0, cnt = 0;
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      if (ok[u]) {
        Ops<T>::each(r[u], f);
#pragma unroll
        for (int j = 0; j < kVec; ++j) {
          bool kk = keep(Ops<T>::get(r[u], j));
          mask |= (kk ? 1u : 0u) << (u * kVec + j);
          cnt += kk;
        }
      }
    }
    // warp exclusive scan of cnt
    unsigned int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      unsigned int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    unsigned int total = __shfl_sync(0xffffffffu, incl, 31);
    unsigned int base = 0;
    if (total) {
      if (lane == 31) base = atomicAdd(s_cnt, total);
      base = __shfl_sync(0xffffffffu, base, 31);
      unsigned int pos = base + incl - cnt;
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
        for (int j = 0; j < kVec; ++j) {
          if (mask & (1u << (u * kVec + j))) zr[pos++] = Ops<T>::get(r[u], j);
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------------
// Pass-0 accumulators.
// ---------------------------------------------------------------------------------
template <typename T>
struct StatsAcc {
  using C = typename Ops<T>::C;
  unsigned int nnan = 0, nneg = 0, npos = 0, nnz = 0, nfin = 0;
  C mn, mx;
  unsigned int cmn = 0, cmx = 0;
  float sum = 0.f;     // sum of (x - x0) * sigma over finite x
  float x0s = 0.f;     // x0 * sigma
  float x0 = 0.f;      // float image of the shift
  float sigma = 1.f;
};

template <typename T> __device__ __forceinline__ typename Ops<T>::C cmp_pos_inf();
template <> __device__ __forceinline__ float cmp_pos_inf<float>() { return INFINITY; }
template <> __device__ __forceinline__ long long cmp_pos_inf<double>() { return 0x7FF0000000000000ll; }

// value of a comparison key
__device__ __forceinline__ float cmp_value(float c, float) { return c; }
__device__ __forceinline__ double cmp_value(long long c, double) { return skey_value(c); }

// ---------------------------------------------------------------------------------
// The kernel.
// ---------------------------------------------------------------------------------
template <typename T>
struct BracketState {
  T a, b, t;
  long long cle_a, clt_b, cle_b;
  double dF;
  float sigma;
  int it, use_bisect, stalled, compact, phase;   // phase: 0 run, 1 done, 2 finish, 3 error
  T result;
};

template <typename T>
__device__ __forceinline__ T inside(T tt, T a, T b) {
  if (!(tt > a)) tt = Ops<T>::next_up(a);
  if (!(tt < b)) tt = Ops<T>::next_down(b);
  return tt;
}

// Power-of-two scale keeping per-thread float32 cost partials finite: a thread sums at
// most `per_thread` terms, each at most `width` in magnitude.
__device__ __forceinline__ float cost_scale(double width, long long per_thread) {
  double bound = (double)per_thread * width;
  if (!(bound > 0.0)) return 1.f;
  double lim = 8.0e37 / bound;
  if (lim >= 1.0) return 1.f;
  int e = ilogb(lim);
  if (e < -120) e = -120;
  return ldexpf(1.f, e);
}

template <typename T>
__device__ __forceinline__ T zero_signed(T v, long long k, long long clt_v, long long nnegzero) {
  if (v == T(0)) return (k - clt_v) <= nnegzero ? T(-0.0) : T(0.0);
  return v;
}

template <typename T>
__global__ void __launch_bounds__(kThreads, 2) select_kernel(SelArgs<T> A) {
  using C = typename Ops<T>::C;
  using U = typename KeyOf<T>::U;
  constexpr int W = KeyOf<T>::kBitsW;
  const int tid = threadIdx.x;
  const int bid = blockIdx.x;
  const unsigned int G = gridDim.x;
  const long long n = A.n, k = A.k;

  __shared__ unsigned long long s_u64[kWarps];
  __shared__ double s_f64[kWarps];
  __shared__ BracketState<T> s_br;
  __shared__ unsigned int s_zcnt;
  __shared__ unsigned int s_hist[kBins];
  __shared__ unsigned long long s_off[kMaxGrid + 1];
  __shared__ unsigned long long s_tot[8];
  __shared__ unsigned long long s_tns[72];
  __shared__ int s_ntns;
  __shared__ long long s_pops[kMaxIt];
  __shared__ double s_iter[kMaxIt];
  __shared__ int s_nk, s_nb;
  __shared__ U s_prefix;
  __shared__ int s_known;
  __shared__ unsigned long long s_rank;

  const Geometry<T> geo(A.x, n);
  const long long per_thread = (geo.nv + (long long)G * kThreads - 1) / ((long long)G * kThreads) * Ops<T>::kVec + 2 * Ops<T>::kVec;

  if (tid == 0) { s_ntns = 0; s_nk = 0; s_nb = 0; }
  if (bid == 0) {   // zero the radix histograms (visible after the first barrier)
    for (int i = tid; i < kMaxRounds * kBins; i += kThreads) A.ghist[i] = 0ull;
  }
  auto stamp = [&]() {
    if (bid == 0 && tid == 0 && s_ntns < 72) s_tns[s_ntns++] = globaltimer();
  };
  stamp();

  if (A.mode == kModeEval) {
    // ---------------- one fused pass at (a, t) ----------------
    const T a = Ops<T>::from_double(A.a_eval), t = Ops<T>::from_double(A.t_eval);
    const C ca = Ops<T>::cmp(a), ct = Ops<T>::cmp(t);
    const float sig = cost_scale((double)Ops<T>::img(t) - (double)Ops<T>::img(a), per_thread);
    const float tsig = Ops<T>::img(t) * sig;
    unsigned int lt = 0, le = 0, lea = 0;
    float S = 0.f;
    auto fn = [&](T xv) {
      C cx = Ops<T>::cmp(xv);
      lt += (cx < ct);
      le += (cx <= ct);
      lea += (cx <= ca);
      bool in = (cx > ca) & (cx < ct);
      float d = fmaf(Ops<T>::img(xv), -sig, tsig);
      S += in ? d : 0.f;
    };
    stream_x(A.x, geo, false, fn);
    unsigned long long blt = block_sum<unsigned long long>(lt, s_u64);
    unsigned long long ble = block_sum<unsigned long long>(le, s_u64);
    unsigned long long blea = block_sum<unsigned long long>(lea, s_u64);
    double bS = block_sum<double>((double)S, s_f64);
    if (tid == 0) {
      PassPartial p;
      p.c_lt = blt; p.c_le = ble; p.c_aux = blea; p.S = bS;
      A.part[bid] = p;
    }
    if (!grid_sync(A.ctrl, G)) return;
    if (bid == 0) {
      unsigned long long l0 = 0, l1 = 0, l2 = 0;
      double dS = 0.0;
      for (unsigned int i = tid; i < G; i += kThreads) {
        l0 += __ldcg(&A.part[i].c_lt); l1 += __ldcg(&A.part[i].c_le); l2 += __ldcg(&A.part[i].c_aux);
        dS += __ldcg(&A.part[i].S);
      }
      l0 = block_sum<unsigned long long>(l0, s_u64);
      l1 = block_sum<unsigned long long>(l1, s_u64);
      l2 = block_sum<unsigned long long>(l2, s_u64);
      dS = block_sum<double>(dS, s_f64);
      if (tid == 0) {
        gbs_cost_eval e;
        e.c_lt_t = (long long)l0; e.c_le_t = (long long)l1; e.c_le_a = (long long)l2; e.pad = 0;
        e.S = dS / (double)sig;
        e.dphi = ((double)e.c_le_a - (double)k + 0.5) * ((double)t - (double)a) + e.S;
        *A.eval_out = e;
      }
    }
    return;
  }

  // ---------------- pass 0: extremes, counts, sum (Sec. 3, step 0) ----------------
  {
    StatsAcc<T> acc;
    acc.mn = cmp_pos_inf<T>();
    acc.mx = -cmp_pos_inf<T>();
    acc.sigma = A.sigma_stats;
    {
      const long long gtid = (long long)bid * kThreads + tid;
      long long i0 = gtid < geo.head ? gtid : geo.head + gtid * Ops<T>::kVec;
      if (i0 < n) {
        T e = A.x[i0];
        if (Ops<T>::is_finite(e)) acc.x0 = Ops<T>::img(e);
      }
      acc.x0s = acc.x0 * acc.sigma;
    }
    auto fn = [&](T xv) {
      acc.nnan += Ops<T>::is_nan(xv);
      acc.nneg += Ops<T>::is_neginf(xv);
      acc.npos += Ops<T>::is_posinf(xv);
      acc.nnz += Ops<T>::is_negzero(xv);
      const bool fin = Ops<T>::is_finite(xv);
      acc.nfin += fin;
      C cx = Ops<T>::cmp(xv);
      C cm = fin ? cx : acc.mn;
      acc.cmn = (cm < acc.mn) ? 0u : acc.cmn;
      acc.mn = (cm < acc.mn) ? cm : acc.mn;
      acc.cmn += (fin && cm == acc.mn);
      C cM = fin ? cx : acc.mx;
      acc.cmx = (cM > acc.mx) ? 0u : acc.cmx;
      acc.mx = (cM > acc.mx) ? cM : acc.mx;
      acc.cmx += (fin && cM == acc.mx);
      float d = fmaf(Ops<T>::img(xv), acc.sigma, -acc.x0s);
      acc.sum += fin ? d : 0.f;
    };
    stream_x(A.x, geo, false, fn);
    // block reduction of (min, count) and (max, count): smem pairs per warp
    __shared__ C s_m[kWarps], s_M[kWarps];
    __shared__ unsigned long long s_cm[kWarps], s_cM[kWarps];
    C mn = acc.mn, mx = acc.mx;
    unsigned long long cmn = acc.cmn, cmx = acc.cmx;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      C omn = __shfl_xor_sync(0xffffffffu, mn, o);
      unsigned long long ocm = __shfl_xor_sync(0xffffffffu, cmn, o);
      C omx = __shfl_xor_sync(0xffffffffu, mx, o);
      unsigned long long ocM = __shfl_xor_sync(0xffffffffu, cmx, o);
      cmn = omn < mn ? ocm : (omn == mn ? cmn + ocm : cmn);
      mn = omn < mn ? omn : mn;
      cmx = omx > mx ? ocM : (omx == mx ? cmx + ocM : cmx);
      mx = omx > mx ? omx : mx;
    }
    if ((tid & 31) == 0) { s_m[tid >> 5] = mn; s_M[tid >> 5] = mx; s_cm[tid >> 5] = cmn; s_cM[tid >> 5] = cmx; }
    unsigned long long b_nan = block_sum<unsigned long long>(acc.nnan, s_u64);
    unsigned long long b_neg = block_sum<unsigned long long>(acc.nneg, s_u64);
    unsigned long long b_pos = block_sum<unsigned long long>(acc.npos, s_u64);
    unsigned long long b_nz = block_sum<unsigned long long>(acc.nnz, s_u64);
    unsigned long long b_fin = block_sum<unsigned long long>(acc.nfin, s_u64);
    double own = (double)acc.sum / (double)acc.sigma + (double)acc.nfin * (double)acc.x0;
    double b_sum = block_sum<double>(own, s_f64);
    if (tid == 0) {
      C bm = s_m[0], bM = s_M[0];
      unsigned long long bcm = s_cm[0], bcM = s_cM[0];
      for (int w = 1; w < kWarps; ++w) {
        bcm = s_m[w] < bm ? s_cm[w] : (s_m[w] == bm ? bcm + s_cm[w] : bcm);
        bm = s_m[w] < bm ? s_m[w] : bm;
        bcM = s_M[w] > bM ? s_cM[w] : (s_M[w] == bM ? bcM + s_cM[w] : bcM);
        bM = s_M[w] > bM ? s_M[w] : bM;
      }
      StatsPartial sp;
      sp.n_nan = b_nan; sp.n_neginf = b_neg; sp.n_posinf = b_pos; sp.n_negzero = b_nz; sp.n_finite = b_fin;
      sp.mn = (double)cmp_value(bm, T()); sp.mx = (double)cmp_value(bM, T());
      sp.c_mn = bcm; sp.c_mx = bcM; sp.sum = b_sum;
      A.spart[bid] = sp;
    }
  }
  if (!grid_sync(A.ctrl, G)) return;
  stamp();

  // every CTA: reduce the G pass-0 partials in the same order
  __shared__ StatsPartial s_st;
  if (tid == 0) {
    StatsPartial t;
    t.n_nan = t.n_neginf = t.n_posinf = t.n_negzero = t.n_finite = 0;
    t.c_mn = t.c_mx = 0;
    t.mn = INFINITY; t.mx = -INFINITY; t.sum = 0.0;
    for (unsigned int i = 0; i < G; ++i) {
      const StatsPartial* p = &A.spart[i];
      t.n_nan += __ldcg(&p->n_nan); t.n_neginf += __ldcg(&p->n_neginf);
      t.n_posinf += __ldcg(&p->n_posinf); t.n_negzero += __ldcg(&p->n_negzero);
      t.n_finite += __ldcg(&p->n_finite);
      double m = __ldcg(&p->mn), M = __ldcg(&p->mx);
      unsigned long long cm = __ldcg(&p->c_mn), cM = __ldcg(&p->c_mx);
      t.c_mn = m < t.mn ? cm : (m == t.mn ? t.c_mn + cm : t.c_mn);
      t.mn = m < t.mn ? m : t.mn;
      t.c_mx = M > t.mx ? cM : (M == t.mx ? t.c_mx + cM : t.c_mx);
      t.mx = M > t.mx ? M : t.mx;
      t.sum += __ldcg(&p->sum);
    }
    s_st = t;
  }
  __syncthreads();
  const StatsPartial st = s_st;

  if (A.mode == kModeStats) {
    if (bid == 0 && tid == 0) {
      gbs_array_stats o;
      o.n = n;
      o.n_nan = (long long)st.n_nan; o.n_neginf = (long long)st.n_neginf;
      o.n_posinf = (long long)st.n_posinf; o.n_negzero = (long long)st.n_negzero;
      o.n_finite = (long long)st.n_finite;
      const bool any = st.n_finite > 0;
      o.min = any ? st.mn : 0.0; o.max = any ? st.mx : 0.0;
      o.c_le_min = any ? (long long)(st.n_neginf + st.c_mn) : 0;
      o.c_lt_max = any ? (long long)(n - st.n_posinf - st.c_mx - st.n_nan) : 0;
      o.sum = st.sum;
      *A.stats_out = o;
    }
    return;
  }

  // ---------------- trivial resolution and the starting bracket ----------------
  if (tid == 0) {
    BracketState<T> br;
    br.it = 0; br.use_bisect = 0; br.stalled = 0; br.compact = 0; br.phase = 0;
    br.result = T(0); br.sigma = 1.f;
    const long long nneg = (long long)st.n_neginf, npos = (long long)st.n_posinf;
    const long long nnz = (long long)st.n_negzero;
    if (st.n_nan > 0) {
      br.phase = 3;
      br.result = T(NAN);
    } else if (k <= nneg) {
      br.phase = 1; br.result = T(-INFINITY); br.it = GBS_HOW_NEGINF;
    } else if (k > n - npos) {
      br.phase = 1; br.result = T(INFINITY); br.it = GBS_HOW_POSINF;
    } else {
      const T m = (T)st.mn, M = (T)st.mx;
      const long long cle_m = nneg + (long long)st.c_mn;
      const long long clt_M = n - npos - (long long)st.c_mx;
      if (cle_m >= k) {
        br.phase = 1; br.result = zero_signed<T>(m, k, nneg, nnz); br.it = GBS_HOW_MIN;
      } else if (clt_M < k) {
        br.phase = 1; br.result = zero_signed<T>(M, k, clt_M, nnz); br.it = GBS_HOW_MAX;
      } else {
        br.a = m; br.b = M;
        br.cle_a = cle_m; br.clt_b = clt_M; br.cle_b = n - npos;
        const double gL = (double)(cle_m - k) + 0.5;
        const double inner = st.sum - (double)st.c_mn * (double)m - (double)st.c_mx * (double)M;
        br.dF = gL * ((double)M - (double)m) + (double)(clt_M - cle_m) * (double)M - inner;
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
      if (br.use_bisect) {
        U ka = ukey(br.a), kb = ukey(br.b);
        U mid = ka + (kb - ka) / 2;
        t = inside<T>(ukey_value(mid, T()), br.a, br.b);
        if (bid == 0) s_nb++;
      } else {
        const double w = (double)br.b - (double)br.a;
        const double ts = (double)br.a + (gR * w - br.dF) / (gR - gL);
        t = inside<T>(Ops<T>::from_double(ts), br.a, br.b);
        if (bid == 0) s_nk++;
      }
      br.t = t;
      br.sigma = cost_scale((double)Ops<T>::img(t) - (double)Ops<T>::img(br.a), per_thread);
      s_br = br;
    }
    __syncthreads();
    const BracketState<T> br = s_br;
    const C ca = Ops<T>::cmp(br.a), ct = Ops<T>::cmp(br.t), cb = Ops<T>::cmp(br.b);
    const float sig = br.sigma;
    const float tsig = Ops<T>::img(br.t) * sig;
    unsigned int lt = 0, le = 0;
    float S = 0.f;
    auto fn = [&](T xv) {     // step 1.2: the fused cost + count evaluation
      C cx = Ops<T>::cmp(xv);
      lt += (cx < ct);
      le += (cx <= ct);
      bool in = (cx > ca) & (cx < ct);
      float d = fmaf(Ops<T>::img(xv), -sig, tsig);
      S += in ? d : 0.f;
    };
    const bool rev = (pass & 1) == 0;   // pass 0 ran forward
    if (br.compact) {
      if (tid == 0) s_zcnt = 0;
      __syncthreads();
      auto keep = [&](T xv) { C cx = Ops<T>::cmp(xv); return (cx > ca) & (cx <= cb); };
      stream_x_compact(A.x, geo, rev, fn, keep, A.z + (long long)bid * A.region_cap, &s_zcnt);
    } else {
      stream_x(A.x, geo, rev, fn);
    }
    unsigned long long blt = block_sum<unsigned long long>(lt, s_u64);
    unsigned long long ble = block_sum<unsigned long long>(le, s_u64);
    double bS = block_sum<double>((double)S, s_f64);
    const int slot = pass & 1;
    if (tid == 0) {
      PassPartial p;
      p.c_lt = blt; p.c_le = ble; p.c_aux = br.compact ? s_zcnt : 0; p.S = bS;
      A.part[slot * G + bid] = p;
    }
    if (!grid_sync(A.ctrl, G)) return;
    stamp();
    // deterministic grid totals (thread i takes partials i, i+B, ...; then block_sum)
    unsigned long long l0 = 0, l1 = 0, l2 = 0;
    double dS = 0.0;
    for (unsigned int i = tid; i < G; i += kThreads) {
      const PassPartial* p = &A.part[slot * G + i];
      l0 += __ldcg(&p->c_lt); l1 += __ldcg(&p->c_le); l2 += __ldcg(&p->c_aux); dS += __ldcg(&p->S);
    }
    l0 = block_sum<unsigned long long>(l0, s_u64);
    l1 = block_sum<unsigned long long>(l1, s_u64);
    l2 = block_sum<unsigned long long>(l2, s_u64);
    dS = block_sum<double>(dS, s_f64);
    if (tid == 0) {   // steps 1.3-1.4
      BracketState<T> nb = br;
      const long long clt = (long long)l0, cle = (long long)l1;
      const long long pop = br.cle_b - br.cle_a;
      if (bid == 0 && br.it < kMaxIt) s_iter[br.it] = (double)br.t;
      if (clt < k && k <= cle) {
        nb.phase = 1;
        nb.result = zero_signed<T>(br.t, k, clt, (long long)st.n_negzero);
        if (bid == 0 && br.it < kMaxIt) s_pops[br.it] = 0;
        nb.it = br.it + 1;
      } else {
        const double gL = (double)(br.cle_a - k) + 0.5;
        const double dphi = gL * ((double)br.t - (double)br.a) + dS / (double)sig;
        if (cle < k) {
          nb.a = br.t; nb.cle_a = cle; nb.dF = br.dF - dphi;
        } else {
          nb.b = br.t; nb.clt_b = clt; nb.cle_b = cle; nb.dF = dphi;
        }
        const long long npop = nb.cle_b - nb.cle_a;
        if (bid == 0 && br.it < kMaxIt) s_pops[br.it] = npop;
        nb.use_bisect = (!br.use_bisect) && ((double)npop > 0.75 * (double)pop);
        nb.stalled = ((double)npop > 0.875 * (double)pop) ? br.stalled + 1 : 0;
        nb.it = br.it + 1;
        if (br.compact) {
          nb.phase = 2;
          s_tot[0] = l2;   // compacted elements
          if ((long long)l2 != pop) { nb.phase = 4; }
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
  T result = fin.result;
  long long fpop = 0;
  if (fin.phase == 2) {
    // ---------------- exact finish: radix select inside (a, b] ----------------
    const int slot = (pass - 1) & 1;
    // region offsets (exclusive prefix of the per-CTA compaction counts)
    for (unsigned int i = tid; i < G; i += kThreads) s_off[i + 1] = __ldcg(&A.part[slot * G + i].c_aux);
    if (tid == 0) s_off[0] = 0;
    __syncthreads();
    if (tid == 0) {
      for (unsigned int i = 1; i <= G; ++i) s_off[i] += s_off[i - 1];
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
    while (s_known < W) {
      const int known = s_known;
      const U prefix = s_prefix;
      const int nbits = (W - known) < kDigitBits ? (W - known) : kDigitBits;
      const int sh = W - known - nbits;
      const U dmask = (U)((1u << nbits) - 1u);
      for (int i = tid; i < kBins; i += kThreads) s_hist[i] = 0;
      __syncthreads();
      // this CTA's slice of the concatenated regions
      unsigned int r = 0;
      {
        unsigned int lo_r = 0, hi_r = G;   // largest r with s_off[r] <= lo_i
        while (hi_r - lo_r > 1) {
          unsigned int mid = (lo_r + hi_r) / 2;
          if (s_off[mid] <= lo_i) lo_r = mid; else hi_r = mid;
        }
        r = lo_r;
      }
      for (; r < G && s_off[r] < hi_i; ++r) {
        const unsigned long long s0 = s_off[r] > lo_i ? s_off[r] : lo_i;
        const unsigned long long s1 = s_off[r + 1] < hi_i ? s_off[r + 1] : hi_i;
        const T* zr = A.z + (long long)r * A.region_cap;
        const unsigned long long rbase = s_off[r];
        for (unsigned long long i = s0 + tid; i < s1; i += kThreads) {
          const T v = __ldcg(zr + (i - rbase));
          const U key = ukey(v);
          const bool inb = (v > fa) && (v <= fb);
          const bool match = known == 0 || (U)(key >> (W - known)) == prefix;
          if (inb && match) atomicAdd(&s_hist[(unsigned int)(key >> sh) & (unsigned int)dmask], 1u);
        }
      }
      __syncthreads();
      for (int i = tid; i < kBins; i += kThreads)
        if (s_hist[i]) atomicAdd(&A.ghist[rounds * kBins + i], (unsigned long long)s_hist[i]);
      if (!grid_sync(A.ctrl, G)) return;
      stamp();
      if (tid < 32) {   // warp 0: find the digit holding rank s_rank
        unsigned long long h[kBins / 32];
        unsigned long long local = 0;
#pragma unroll
        for (int j = 0; j < kBins / 32; ++j) {
          h[j] = __ldcg(&A.ghist[rounds * kBins + tid * (kBins / 32) + j]);
          local += h[j];
        }
        unsigned long long incl = local;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
          if (tid >= o) incl += y;
        }
        const unsigned long long want = s_rank;
        const unsigned long long excl = incl - local;
        const bool mine = excl < want && want <= incl;
        const unsigned int who = __ballot_sync(0xffffffffu, mine);
        if (mine) {
          unsigned long long c = excl;
          int d = 0;
          for (int j = 0; j < kBins / 32; ++j) {
            if (c + h[j] >= want) { d = tid * (kBins / 32) + j; break; }
            c += h[j];
          }
          s_rank = want - c;
          s_prefix = (U)((prefix << nbits) | (U)d);
          s_known = known + nbits;
        }
        if (who == 0 && tid == 0) {   // no bin holds the rank: inconsistent counts
          atomicCAS(&A.ctrl->status, 0, (int)GBS_EINTERNAL);
          s_known = W;
          s_prefix = 0;
        }
      }
      ++rounds;
      __syncthreads();
    }
    result = ukey_value(s_prefix, T());
  }

  if (bid == 0 && tid == 0) {
    if (fin.phase == 3) atomicCAS(&A.ctrl->status, 0, (int)GBS_ENAN);
    *A.out = result;
    gbs_run_stats* rs = A.rs;
    rs->status = ld_relaxed_i32(&A.ctrl->status);
    rs->how = fin.phase == 3 ? GBS_HOW_NONE
            : fin.phase == 2 ? GBS_HOW_FINISH
            : (pass == 0 ? fin.it : GBS_HOW_HIT);
    rs->passes = 1 + pass;
    rs->kelley_steps = s_nk;
    rs->bisect_steps = s_nb;
    rs->finish_rounds = rounds;
    rs->grid = (int)G;
    rs->learned = 0;
    rs->n = n; rs->k = k;
    rs->finish_pop = fpop;
    const int ni = pass < kMaxIt ? pass : kMaxIt;
    for (int i = 0; i < kMaxIt; ++i) {
      rs->pops[i] = i < ni ? s_pops[i] : 0;
      rs->iterates[i] = i < ni ? s_iter[i] : 0.0;
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
int grid_for(gbs_ctx* c) {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, select_kernel<T>, kThreads, 0) != cudaSuccess) {
    cudaGetLastError();
    occ = 1;
  }
  int bps = c->cfg.blocks_per_sm > 0 ? c->cfg.blocks_per_sm : 2;
  bps = std::max(1, std::min(bps, occ));
  return std::min(kMaxGrid, c->num_sms * bps);
}

template <typename T>
long long region_cap_for(long long n, int grid) {
  const long long vec = vec_of<T>();
  const long long nv_max = n / vec + 1;
  const long long stride = (long long)grid * kThreads;
  return ((nv_max + stride - 1) / stride) * kThreads * vec + 2 * vec;
}

template <typename T>
float stats_sigma(long long n, int grid) {
  const long long vec = vec_of<T>();
  const long long stride = (long long)grid * kThreads;
  const long long per_thread = ((n / vec + 1 + stride - 1) / stride) * vec + 2 * vec;
  int e = 0;
  while ((1ll << e) < per_thread) ++e;
  return std::ldexp(1.0f, -(e + 2));
}

template <typename T>
gbs_status launch_select(gbs_ctx* c, const T* x, long long n, long long k, T* out, int mode,
                                double a, double t, gbs_array_stats* sout, gbs_cost_eval* eout,
                                cudaStream_t stream) {
  DeviceGuard g(c->device);
  if (!g.ok) return GBS_ECUDA;
  const int grid = grid_for<T>(c);
  const long long rcap = region_cap_for<T>(n, grid);
  const size_t zb = mode == kModeSelect ? (size_t)rcap * grid * sizeof(T) : 0;
  gbs_status s = gbs_internal_ensure(c, zb);
  if (s != GBS_OK) return s;
  SelArgs<T> A;
  A.x = x; A.n = n; A.k = k; A.out = out; A.mode = mode;
  A.maxit = c->cfg.maxit > 0 ? c->cfg.maxit : 64;
  if (A.maxit > kMaxIt) A.maxit = kMaxIt;
  A.cap = c->cfg.cap > 0 ? c->cfg.cap : std::max<long long>(n / 16, 4096);
  A.a_eval = a; A.t_eval = t;
  A.sigma_stats = stats_sigma<T>(n, grid);
  A.ctrl = c->ctrl; A.part = c->part; A.spart = c->spart; A.ghist = c->ghist;
  A.z = reinterpret_cast<T*>(c->z); A.region_cap = rcap;
  A.rs = c->rs; A.stats_out = sout; A.eval_out = eout;
  if (cudaMemsetAsync(c->ctrl, 0, sizeof(Ctrl), stream) != cudaSuccess) return GBS_ECUDA;
  if (mode == kModeSelect && cudaMemsetAsync(c->rs, 0, sizeof(gbs_run_stats), stream) != cudaSuccess)
    return GBS_ECUDA;
  void* args[] = {&A};
  cudaError_t e = cudaLaunchCooperativeKernel((const void*)select_kernel<T>, dim3(grid), dim3(kThreads), args,
                                              0, stream);
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
long long select_region_cap_f32(long long n, int grid) { return region_cap_for<float>(n, grid); }
float select_stats_sigma_f32(long long n, int grid) { return stats_sigma<float>(n, grid); }
int select_occupancy_f32() {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, select_kernel<float>, kThreads, 0) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return occ;
}
cudaError_t select_launch_f32(const SelArgs<float>& A, int grid, cudaStream_t stream) {
  SelArgs<float> a = A;
  void* args[] = {&a};
  return cudaLaunchCooperativeKernel((const void*)select_kernel<float>, dim3(grid), dim3(kThreads), args, 0,
                                     stream);
}

gbs_status reserve_select(gbs_ctx* c, long long n, int elem_bytes) {
  DeviceGuard g(c->device);
  if (!g.ok) return GBS_ECUDA;
  if (elem_bytes == 4) {
    const int grid = grid_for<float>(c);
    return gbs_internal_ensure(c, (size_t)region_cap_for<float>(n, grid) * grid * 4);
  }
  const int grid = grid_for<double>(c);
  return gbs_internal_ensure(c, (size_t)region_cap_for<double>(n, grid) * grid * 8);
}

}  // namespace gbs
