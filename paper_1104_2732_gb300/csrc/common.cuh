// Shared device helpers of the selection kernels: order-preserving keys, the bounded
// grid-wide barrier of the persistent kernels, and warp / block reductions.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "gbselect.h"

namespace gbs {

constexpr int kThreads = 512;          // threads per CTA of the persistent kernels
constexpr int kWarps = kThreads / 32;
constexpr int kDigitBits = 12;         // radix digit of the exact finish
constexpr int kBins = 1 << kDigitBits;
constexpr int kMaxRounds = (64 + kDigitBits - 1) / kDigitBits;   // 64-bit keys
static_assert(kBins % kThreads == 0, "the finish's digit search gives each thread whole bins");
constexpr int kMaxGrid = 2048;         // upper bound on CTAs of a persistent launch
constexpr int kMaxIt = 64;             // length of the per-call iterate record

// Bounded waits: a spinning CTA gives up after this long and flags GBS_ETIMEOUT.
constexpr unsigned long long kWaitLimitNs = 2000000000ull;   // 2 s

// ---------------------------------------------------------------------------------
// Keys.  ukey(): unsigned totalOrder key (-inf < ... < -0 < +0 < ... < +inf) used by
// the radix finish and, for float64, by every comparison of the passes (integer pipes).
// ---------------------------------------------------------------------------------
template <typename T> struct KeyOf;
template <> struct KeyOf<float> {
  using U = uint32_t;
  using S = int32_t;
  static constexpr int kBitsW = 32;
};
template <> struct KeyOf<double> {
  using U = uint64_t;
  using S = int64_t;
  static constexpr int kBitsW = 64;
};

__device__ __host__ __forceinline__ uint32_t bits_of(float v) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(v);
#else
  uint32_t u; memcpy(&u, &v, 4); return u;
#endif
}
__device__ __host__ __forceinline__ uint64_t bits_of(double v) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(v);
#else
  uint64_t u; memcpy(&u, &v, 8); return u;
#endif
}
__device__ __forceinline__ float from_bits(uint32_t u, float) { return __uint_as_float(u); }
__device__ __forceinline__ double from_bits(uint64_t u, double) {
  return __longlong_as_double((long long)u);
}

__device__ __forceinline__ uint32_t ukey(float v) {
  uint32_t u = __float_as_uint(v);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
// float64 totalOrder key from the bits: flip everything for a negative value, the sign
// bit for a positive one (the mask comes from an arithmetic shift of the high word).
__device__ __forceinline__ uint64_t ukey_bits(uint64_t u) {
  const uint32_t m = (uint32_t)((int32_t)(uint32_t)(u >> 32) >> 31);
  return u ^ ((((uint64_t)(m | 0x80000000u)) << 32) | (uint64_t)m);
}
__device__ __forceinline__ uint64_t ukey(double v) { return ukey_bits((uint64_t)__double_as_longlong(v)); }
__device__ __forceinline__ float ukey_value(uint32_t k, float) {
  uint32_t u = (k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k;
  return __uint_as_float(u);
}
__device__ __forceinline__ double ukey_value(uint64_t k, double) {
  uint64_t u = (k & 0x8000000000000000ull) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k;
  return __longlong_as_double((long long)u);
}

// Truncating float32 image of a float64 (exponent clamped to the float range).  It is
// monotone, so t - x >= 0 is kept for x < t; it feeds only the float32 cost partials.
__device__ __forceinline__ float f64_to_f32_trunc(uint64_t u) {
  uint32_t hi = (uint32_t)(u >> 32), lo = (uint32_t)u;
  uint32_t sign = hi & 0x80000000u;
  int e = (int)((hi >> 20) & 0x7FF) - 1023 + 127;
  uint32_t mant = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
  uint32_t fb = e <= 0 ? sign : (e >= 255 ? (sign | 0x7F7FFFFFu) : (sign | ((uint32_t)e << 23) | mant));
  return __uint_as_float(fb);
}

// ---------------------------------------------------------------------------------
// Control block of a persistent launch (zeroed by the host before every launch).
// ---------------------------------------------------------------------------------
struct __align__(128) Ctrl {
  unsigned int bar_count;         // grid barrier: arrivals so far (only grows within a launch)
  unsigned int bar_unused;
  int abort;
  int status;
  unsigned long long w_count;     // work-queue head of the segmented launch
  unsigned long long w_len;       // work-queue length of the segmented launch
  unsigned long long pad[12];
  // totals of a cutting-plane pass, three slots used in rotation: c_lt, c_le, #(x <= a),
  // #(x < b), compacted count, and the cost sum S in fixed point (see kSFixBits)
  unsigned long long acc[3][8];
};

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_relaxed_i32(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier for a cooperative launch.  Returns false (in every thread of the
// CTA) if the wait gave up or another CTA aborted; the caller must then return.  The
// wait is bounded by kWaitLimitNs; on expiry the CTA sets status = GBS_ETIMEOUT and
// abort = 1 so that every other waiter also leaves.
__device__ __forceinline__ unsigned int atom_add_acq_rel_u32(unsigned int* p, unsigned int v) {
  unsigned int old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

// Grid barrier of a cooperative launch.  One acquire-release arrival per CTA on a counter
// that only grows: barrier number e is passed once the counter reaches (e + 1) * nblocks,
// and since no CTA can arrive at barrier e + 1 before barrier e is complete, a CTA reads e
// from the value its own arrival returned.  The wait is bounded: after limit_ns (2 s unless
// given) the CTA records GBS_ETIMEOUT, raises the abort flag and returns false, as does
// every CTA that sees the abort flag raised.
__device__ __forceinline__ bool grid_sync(Ctrl* c, unsigned int nblocks,
                                          unsigned long long limit_ns = kWaitLimitNs) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned int old = atom_add_acq_rel_u32(&c->bar_count, 1u);
    const unsigned int target = (old / nblocks + 1u) * nblocks;
    if (old + 1u != target) {
      const unsigned long long t0 = globaltimer();
      unsigned int polls = 0;
      while (ld_acquire_u32(&c->bar_count) < target) {
        if (ld_relaxed_i32(&c->abort)) { ok = 0; break; }
        if ((++polls & 63u) == 0 && globaltimer() - t0 > limit_ns) {
          atomicCAS(&c->status, 0, (int)GBS_ETIMEOUT);
          atomicExch(&c->abort, 1);
          ok = 0;
          break;
        }
        __nanosleep(20);
      }
    }
    if (ok && ld_relaxed_i32(&c->abort)) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// ---------------------------------------------------------------------------------
// Reductions.
// ---------------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum_f64(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ unsigned int warp_sum_u32(unsigned int v) {
  return __reduce_add_sync(0xffffffffu, v);
}

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v) { return warp_sum_u64(v); }
__device__ __forceinline__ double warp_sum(double v) { return warp_sum_f64(v); }

// Deterministic block sum: warp sums, then every thread adds the per-warp values in
// warp order.  Result valid in every thread.  `scratch` holds kWarps values.
template <typename V>
__device__ __forceinline__ V block_sum(V v, V* scratch) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) scratch[w] = v;
  __syncthreads();
  V r = V(0);
#pragma unroll 4
  for (int i = 0; i < kWarps; ++i) r += scratch[i];
  __syncthreads();
  return r;
}

// Makes `dev` current for the lifetime of the guard.
struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; prev = -1; return; }
    if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

}  // namespace gbs
