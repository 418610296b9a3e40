// Element-level pieces shared by the selection kernels: per-type operations, the
// fused cost + count core of a cutting-plane pass, CTA-wide sums, and the iterate
// guards.
#pragma once

#include <cfloat>
#include <cmath>
#include <cstdint>

#include "common.cuh"

namespace gbs {

// ---------------------------------------------------------------------------------
// Per-type element operations.  cmp(): the value compared against the iterate
// (IEEE float for float32, the unsigned totalOrder key for float64, see CmpOf).  img():
// float32 image used only for the cost partials.
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
  using C = unsigned long long;
  using V = double2;
  static constexpr int kVec = 2;
  static __device__ __forceinline__ C cmp(double x) { return ukey(x); }
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

// ---------------------------------------------------------------------------------
// Per-element cores.
// ---------------------------------------------------------------------------------
// One element of a cutting-plane pass (Algorithm 1, step 1.2; the figure's Objective()):
// lt += [x < t], le += [x <= t], S += [a < x < t] * (t - x) * sigma.
__device__ __forceinline__ void core(float x, float a, float t, float nsig, float tsig, unsigned& lt,
                                     unsigned& le, float& S) {
  asm("{\n\t"
      ".reg .pred p, q, r;\n\t"
      ".reg .f32 d;\n\t"
      "setp.lt.f32 p, %3, %5;\n\t"
      "setp.le.f32 q, %3, %5;\n\t"
      "setp.gt.and.f32 r, %3, %4, p;\n\t"
      "fma.rn.f32 d, %3, %6, %7;\n\t"
      "@p add.u32 %0, %0, 1;\n\t"
      "@q add.u32 %1, %1, 1;\n\t"
      "@r add.f32 %2, %2, d;\n\t"
      "}"
      : "+r"(lt), "+r"(le), "+f"(S)
      : "f"(x), "f"(a), "f"(t), "f"(nsig), "f"(tsig));
}
// float64: comparisons on unsigned totalOrder keys (integer pipes; the thresholds carry
// the IEEE treatment of zeros, see CmpOf), the cost on the truncated float32 image.
// ka = CmpOf::le(a), kt_lt = CmpOf::lt(t), kt_le = CmpOf::le(t).
__device__ __forceinline__ void core(double xv, unsigned long long ka, unsigned long long kt_lt,
                                     unsigned long long kt_le, float nsig, float tsig, unsigned& lt, unsigned& le,
                                     float& S) {
  const uint64_t u = (uint64_t)__double_as_longlong(xv);
  const unsigned long long kx = ukey_bits(u);
  lt += (kx < kt_lt);
  le += (kx <= kt_le);
  const bool in = (kx > ka) & (kx < kt_lt);
  const float d = fmaf(f64_to_f32_trunc(u), nsig, tsig);
  S += in ? d : 0.f;
}
// float64, the fast form: every decision on the high 32 bits of the keys, exact unless an
// element's high word equals a threshold's, when the element takes the comparisons above
// (rare: those elements lie within 2^32 ulps of a or t).  Valid when t is not a zero (one
// key serves "<" and "<="; kt = CmpOf::lt(t) = CmpOf::le(t)) and |a|, |t| < 2^127, so that
// no element of (a, t) lies above float32's range: its float32 image is then formed from
// the high word alone (exponent rebiased, 20 mantissa bits; 0 below the normal range).
__device__ __forceinline__ bool core64_fast_ok(unsigned long long ka, unsigned long long kt_lt,
                                               unsigned long long kt_le) {
  constexpr unsigned long long kLo = 0x381FFFFFFFFFFFFFull, kHi = 0xC7E0000000000000ull;   // keys of -+2^127
  return kt_lt == kt_le && ka > kLo && ka < kHi && kt_lt > kLo && kt_lt < kHi;
}
__device__ __forceinline__ void core64_fast(double xv, unsigned long long ka, unsigned long long kt, uint32_t a_hi,
                                            uint32_t t_hi, float nsig, float tsig, unsigned& lt, unsigned& le,
                                            float& S) {
  const uint64_t u = (uint64_t)__double_as_longlong(xv);
  const uint32_t hi = (uint32_t)(u >> 32);
  const uint32_t khi = hi ^ ((uint32_t)((int32_t)hi >> 31) | 0x80000000u);
  const bool p = khi < t_hi;                 // x < t for certain
  const bool r = p & (khi > a_hi);           // a < x < t for certain
  lt += p;
  le += p;
  const uint32_t fb = (((hi << 3) + 0x40000000u) & 0x7FFFFFFFu) | (hi & 0x80000000u);
  const float xi = (hi & 0x7FFFFFFFu) >= 0x38100000u ? __uint_as_float(fb) : 0.f;
  const float d = fmaf(xi, nsig, tsig);
  S += r ? d : 0.f;
  if ((khi == t_hi) | (khi == a_hi)) {
    const unsigned long long kx = ukey_bits(u);
    if (khi == t_hi) {
      lt += (kx < kt);
      le += (kx <= kt);
    }
    if ((kx > ka) & (kx < kt)) S += fmaf(f64_to_f32_trunc(u), nsig, tsig);
  }
}
// float32: the IEEE comparisons of the inline-PTX core (both thresholds are t itself).
__device__ __forceinline__ void core(float x, float a, float t_lt, float, float nsig, float tsig, unsigned& lt,
                                     unsigned& le, float& S) {
  core(x, a, t_lt, nsig, tsig, lt, le, S);
}

// Shared-memory store at a 32-bit shared-space address.
__device__ __forceinline__ unsigned int smem_u32(const void* p) { return (unsigned int)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void st_shared(unsigned int addr, float v) {
  asm volatile("st.shared.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}
__device__ __forceinline__ void st_shared(unsigned int addr, double v) {
  asm volatile("st.shared.f64 [%0], %1;" ::"r"(addr), "d"(v) : "memory");
}
__device__ __forceinline__ void ld_shared(unsigned int addr, float& v) {
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(addr) : "memory");
}
__device__ __forceinline__ void ld_shared(unsigned int addr, double& v) {
  asm volatile("ld.shared.f64 %0, [%1];" : "=d"(v) : "r"(addr) : "memory");
}

// One element of a compacting cutting-plane pass: core() at (a, t), and an element of
// (a, b] is stored at the shared-memory address `off`, which then moves on by one slot of
// the lane's column (32 elements).  float32: one predicate x > a serves both the cost
// term and the bracket test.
__device__ __forceinline__ void core_keep(float x, float a, float t, float, float b, float nsig, float tsig,
                                          unsigned& lt, unsigned& le, float& S, unsigned& off) {
  asm volatile(
      "{\n\t"
      ".reg .pred p, q, g, r, w;\n\t"
      ".reg .f32 d;\n\t"
      "setp.lt.f32 p, %4, %6;\n\t"
      "setp.le.f32 q, %4, %6;\n\t"
      "setp.gt.f32 g, %4, %5;\n\t"
      "and.pred r, g, p;\n\t"
      "setp.le.and.f32 w, %4, %7, g;\n\t"
      "fma.rn.f32 d, %4, %8, %9;\n\t"
      "@p add.u32 %0, %0, 1;\n\t"
      "@q add.u32 %1, %1, 1;\n\t"
      "@r add.f32 %2, %2, d;\n\t"
      "@w st.shared.f32 [%3], %4;\n\t"
      "@w add.u32 %3, %3, 128;\n\t"
      "}"
      : "+r"(lt), "+r"(le), "+f"(S), "+r"(off)
      : "f"(x), "f"(a), "f"(t), "f"(b), "f"(nsig), "f"(tsig)
      : "memory");
}
// float64: the key comparisons of core(), the bracket test on the same key.
__device__ __forceinline__ void core_keep(double xv, unsigned long long ka, unsigned long long kt_lt,
                                          unsigned long long kt_le, unsigned long long kb_le, float nsig, float tsig,
                                          unsigned& lt, unsigned& le, float& S, unsigned& off) {
  core(xv, ka, kt_lt, kt_le, nsig, tsig, lt, le, S);
  const unsigned long long kx = ukey_bits((uint64_t)__double_as_longlong(xv));
  const bool w = (kx > ka) & (kx <= kb_le);
  if (w) st_shared(off, xv);
  off += w ? 256u : 0u;
}

// One element of a compaction pass without a cut: an element of (a, b] is stored at the
// shared-memory address `off`, which then moves on by one slot of the lane's column.
__device__ __forceinline__ void keep_only(float x, float a, float b, unsigned& off) {
  asm volatile(
      "{\n\t"
      ".reg .pred g, w;\n\t"
      "setp.gt.f32 g, %1, %2;\n\t"
      "setp.le.and.f32 w, %1, %3, g;\n\t"
      "@w st.shared.f32 [%0], %1;\n\t"
      "@w add.u32 %0, %0, 128;\n\t"
      "}"
      : "+r"(off)
      : "f"(x), "f"(a), "f"(b)
      : "memory");
}
__device__ __forceinline__ void keep_only(double xv, unsigned long long ka, unsigned long long kb_le, unsigned& off) {
  const unsigned long long kx = ukey_bits((uint64_t)__double_as_longlong(xv));
  const bool w = (kx > ka) & (kx <= kb_le);
  if (w) st_shared(off, xv);
  off += w ? 256u : 0u;
}



template <typename T> __device__ __forceinline__ typename Ops<T>::C cmp_pos_inf();
template <> __device__ __forceinline__ float cmp_pos_inf<float>() { return INFINITY; }
template <> __device__ __forceinline__ unsigned long long cmp_pos_inf<double>() { return 0xFFF0000000000000ull; }
template <typename T> __device__ __forceinline__ typename Ops<T>::C cmp_neg_inf();
template <> __device__ __forceinline__ float cmp_neg_inf<float>() { return -INFINITY; }
template <> __device__ __forceinline__ unsigned long long cmp_neg_inf<double>() { return 0x000FFFFFFFFFFFFFull; }

// value of a comparison key
__device__ __forceinline__ float cmp_value(float c, float) { return c; }
__device__ __forceinline__ double cmp_value(unsigned long long c, double) { return ukey_value(c, 0.0); }

// Comparison images.  of(x): the image of an element; lt(t) and le(t): thresholds with
// x < t  <=>  of(x) < lt(t)  and  x <= t  <=>  of(x) <= le(t)  (so x > a <=> of(x) > le(a))
// for every non-NaN x under IEEE comparison.  float32 compares the values themselves;
// float64 compares unsigned totalOrder keys, where -0 sorts before +0, so a zero
// threshold takes the key of -0 for "<" and of +0 for "<=".
template <typename T> struct CmpOf;
template <> struct CmpOf<float> {
  static __device__ __forceinline__ float of(float v) { return v; }
  static __device__ __forceinline__ float lt(float v) { return v; }
  static __device__ __forceinline__ float le(float v) { return v; }
};
template <> struct CmpOf<double> {
  static __device__ __forceinline__ unsigned long long of(double v) { return ukey(v); }
  static __device__ __forceinline__ unsigned long long lt(double v) { return v == 0.0 ? ukey(-0.0) : ukey(v); }
  static __device__ __forceinline__ unsigned long long le(double v) { return v == 0.0 ? ukey(0.0) : ukey(v); }
};

// Scalar head and tail of x handled by this thread (the first threads of CTA 0).

struct Sum6 {
  unsigned long long u[5];
  double d;
};
__device__ __forceinline__ Sum6 block_sum6(Sum6 v, Sum6* scratch /* [kWarps + 1] */) {
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
    for (int i = 1; i < kWarps; ++i) {
#pragma unroll
      for (int q = 0; q < 5; ++q) r.u[q] += scratch[i].u[q];
      r.d += scratch[i].d;
    }
    scratch[kWarps] = r;
  }
  __syncthreads();
  return scratch[kWarps];
}

// The same sum, valid in thread 0 only (no broadcast).
__device__ __forceinline__ Sum6 block_sum6_t0(Sum6 v, Sum6* scratch /* [kWarps] */) {
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
  Sum6 r = v;
  if (threadIdx.x == 0) {
    r = scratch[0];
    for (int i = 1; i < kWarps; ++i) {
#pragma unroll
      for (int q = 0; q < 5; ++q) r.u[q] += scratch[i].u[q];
      r.d += scratch[i].d;
    }
  }
  return r;
}


template <typename T>
__device__ __forceinline__ T inside(T tt, T a, T b) {
  if (!(tt > a)) tt = Ops<T>::next_up(a);
  if (!(tt < b)) tt = Ops<T>::next_down(b);
  return tt;
}

// Power-of-two scale keeping per-thread float32 cost partials finite: a thread sums at
// most `per_thread` terms, each at most `width` in magnitude.
// Power-of-two scale sigma of the float32 cost partials: a thread sums at most per_thread
// terms sigma * (t - x) with 0 <= t - x <= width, and sigma * per_thread * width lies in
// [1, 2) (sigma is clamped to [2^-120, 2^120]; see cost_fix_bits for the clamped case).
__device__ __forceinline__ float cost_scale(double width, long long per_thread) {
  const double bound = (double)per_thread * width;
  if (!(bound > 0.0) || !isfinite(bound)) return 1.f;
  int e = -ilogb(bound);
  e = e < -120 ? -120 : (e > 120 ? 120 : e);
  return ldexpf(1.f, e);
}

// Fraction bits of the fixed-point image of the scaled cost sums: 40 when sigma was not
// clamped (a CTA sum of 512 threads is below 2^10, a grid total below 2^21, far inside
// 64 bits); fewer when the clamp left sigma * per_thread * width above 2.
constexpr int kSFixBits = 40;
__device__ __forceinline__ int cost_fix_bits(double width, long long per_thread, float sigma) {
  const double b = (double)per_thread * width * (double)sigma;
  if (!(b >= 2.0) || !isfinite(b)) return kSFixBits;
  return kSFixBits - ilogb(b);
}

template <typename T> __device__ __forceinline__ bool is_neg_zero_bits(T v);
template <> __device__ __forceinline__ bool is_neg_zero_bits<float>(float v) {
  return __float_as_uint(v) == 0x80000000u;
}
template <> __device__ __forceinline__ bool is_neg_zero_bits<double>(double v) {
  return (uint64_t)__double_as_longlong(v) == 0x8000000000000000ull;
}


}  // namespace gbs
