// Device-resident loop of a sharded selection: the state of Algorithm 1 (Sec. 3) lives
// in device memory, each shard's pass at the state's (a, t) adds its counts and its cost
// (in fixed point) into a device accumulator, the caller sums the accumulators over the
// processes in place (one small all-reduce, e.g. NCCL), and a one-thread step applies the
// bracket update (steps 1.3-1.4) and the next point (step 1.1) with the same code as the
// host API (shard_sm.cuh).  Every launch is stream-ordered, so passes need no host round
// trip: the host reads the phase back only now and then.  Once the state leaves ITERATE,
// passes and steps do nothing.
#include <algorithm>
#include <cmath>
#include <cstdint>

#include "api_internal.h"
#include "common.cuh"
#include "elem.cuh"
#include "shard_sm.cuh"

namespace gbs {
namespace {

constexpr int kDevPassThreads = 256;

// One shard's pass: c_lt(t), c_le(t), c_le(a) and S = sum over a < x < t of (t - x) (of
// (u(t) - u(x)), u = log1p(x - xmin), for the log driver), on the float32 images of the
// elements, each block's part rounded once to the fixed point of sm::sfix_bits.
template <typename T>
__global__ void __launch_bounds__(kDevPassThreads) shard_pass_kernel(const T* __restrict__ x, long long n,
                                                                     const gbs_shard_state* __restrict__ st,
                                                                     long long* __restrict__ acc) {
  using C = typename Ops<T>::C;
  __shared__ int s_go, s_log, s_fx;
  __shared__ double s_a, s_t, s_xmin;
  __shared__ unsigned long long s_c[3][kDevPassThreads / 32];
  __shared__ double s_S[kDevPassThreads / 32];
  if (threadIdx.x == 0) {
    const gbs_shard_state s = *st;
    s_go = s.phase == GBS_SHARD_ITERATE && acc[4] == 0;
    s_log = s.driver == GBS_DRIVER_LOG;
    s_fx = sm::sfix_bits(&s);
    s_a = s.a;
    s_t = s.t;
    s_xmin = s.xmin;
  }
  __syncthreads();
  if (!s_go) return;
  const T a = (T)s_a, t = (T)s_t;
  const C ca = CmpOf<T>::le(a), ct_lt = CmpOf<T>::lt(t), ct_le = CmpOf<T>::le(t);
  const bool lg = s_log != 0;
  const double xmin = s_xmin;
  const float ft = Ops<T>::img(t);
  const float ut = lg ? (float)log1p((double)t - xmin) : 0.f;
  unsigned int lt = 0, le = 0, lea = 0;
  float S = 0.f;
  auto f = [&](T v) {
    const C cv = CmpOf<T>::of(v);
    lt += cv < ct_lt;
    le += cv <= ct_le;
    lea += cv <= ca;
    if ((cv > ca) & (cv < ct_lt)) S += lg ? ut - log1pf((float)((double)v - xmin)) : ft - Ops<T>::img(v);
  };
  // the scalar head and tail (any alignment), then the 16-byte body with four loads in
  // flight per thread
  using V = typename Ops<T>::V;
  const Geometry<T> geo(x, n);
  const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  if (gtid < geo.head) f(x[gtid]);
  if (gtid < geo.n - geo.tail0) f(x[geo.tail0 + gtid]);
  const V* xv = reinterpret_cast<const V*>(x + geo.head);
  long long i = gtid;
  for (; i + 3 * stride < geo.nv; i += 4 * stride) {
    V r[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) r[u] = load_stream(xv + i + u * stride);
#pragma unroll
    for (int u = 0; u < 4; ++u) Ops<T>::each(r[u], f);
  }
  for (; i < geo.nv; i += stride) {
    const V r = load_stream(xv + i);
    Ops<T>::each(r, f);
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned int r0 = __reduce_add_sync(0xffffffffu, lt), r1 = __reduce_add_sync(0xffffffffu, le),
                     r2 = __reduce_add_sync(0xffffffffu, lea);
  double Sd = (double)S;
  for (int o = 16; o > 0; o >>= 1) Sd += __shfl_xor_sync(0xffffffffu, Sd, o);
  if (lane == 0) { s_c[0][w] = r0; s_c[1][w] = r1; s_c[2][w] = r2; s_S[w] = Sd; }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long c0 = 0, c1 = 0, c2 = 0;
    double Sb = 0.0;
    for (int j = 0; j < kDevPassThreads / 32; ++j) { c0 += s_c[0][j]; c1 += s_c[1][j]; c2 += s_c[2][j]; Sb += s_S[j]; }
    auto* au = reinterpret_cast<unsigned long long*>(acc);
    if (c0) atomicAdd(&au[0], c0);
    if (c1) atomicAdd(&au[1], c1);
    if (c2) atomicAdd(&au[2], c2);
    const long long sf = llrint(ldexp(Sb, s_fx));
    if (sf) atomicAdd(&au[3], (unsigned long long)sf);
  }
}

// The step after the all-reduce: totals -> bracket update -> next point; the
// accumulator is cleared for the next pass.  A failed update or next stops the loop
// with its status in acc[4].
__global__ void shard_step_kernel(gbs_shard_state* st, long long* acc) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  gbs_shard_state s = *st;
  if (acc[4] == 0 && s.phase == GBS_SHARD_ITERATE) {
    gbs_cost_eval e;
    e.c_lt_t = acc[0];
    e.c_le_t = acc[1];
    e.c_le_a = acc[2];
    e.pad = 0;
    e.S = ldexp((double)acc[3], -sm::sfix_bits(&s));
    e.dphi = 0.0;
    gbs_status r = sm::update(&s, &e);
    if (r == GBS_OK && s.phase == GBS_SHARD_ITERATE) r = sm::next(&s);
    if (r == GBS_OK) *st = s;
    else acc[4] = (long long)r;
  }
  acc[0] = acc[1] = acc[2] = acc[3] = 0;
}

template <typename T>
gbs_status pass_dev(gbs_ctx* c, const T* x, int64_t n, const gbs_shard_state* d_state, int64_t* d_acc,
                    void* stream) {
  if (!c || !d_state || !d_acc || n < 0 || (n > 0 && !x)) return GBS_EINVAL;
  if (reinterpret_cast<uintptr_t>(d_acc) % 8 != 0 || reinterpret_cast<uintptr_t>(d_state) % 8 != 0 ||
      reinterpret_cast<uintptr_t>(x) % sizeof(T) != 0)
    return GBS_EINVAL;
  if (n == 0) return GBS_OK;
  DeviceGuard g(c->device);
  if (!g.ok) return GBS_ECUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const long long blocks = std::min<long long>((n + kDevPassThreads - 1) / kDevPassThreads, (long long)c->num_sms * 8);
  shard_pass_kernel<T><<<(unsigned int)blocks, kDevPassThreads, 0, s>>>(x, n, d_state,
                                                                        reinterpret_cast<long long*>(d_acc));
  if (cudaGetLastError() != cudaSuccess) return GBS_ECUDA;
  c->last_stream = s;
  return GBS_OK;
}

}  // namespace
}  // namespace gbs

using namespace gbs;

extern "C" {

gbs_status gbs_shard_pass_dev_f32(gbs_ctx* ctx, const float* x, int64_t n, const gbs_shard_state* d_state,
                                  int64_t* d_acc, void* stream) {
  return pass_dev<float>(ctx, x, n, d_state, d_acc, stream);
}
gbs_status gbs_shard_pass_dev_f64(gbs_ctx* ctx, const double* x, int64_t n, const gbs_shard_state* d_state,
                                  int64_t* d_acc, void* stream) {
  return pass_dev<double>(ctx, x, n, d_state, d_acc, stream);
}
gbs_status gbs_shard_passes_dev_f32(gbs_ctx* ctx, const float* const* shards, const int64_t* lens, int32_t count,
                                   gbs_shard_state* d_state, int64_t* d_acc, int32_t step, void* stream) {
  if (!ctx || count < 0 || (count > 0 && (!shards || !lens))) return GBS_EINVAL;
  for (int32_t i = 0; i < count; ++i) {
    const gbs_status st = pass_dev<float>(ctx, shards[i], lens[i], d_state, d_acc, stream);
    if (st != GBS_OK) return st;
  }
  return step ? gbs_shard_step_dev(ctx, d_state, d_acc, stream) : GBS_OK;
}
gbs_status gbs_shard_passes_dev_f64(gbs_ctx* ctx, const double* const* shards, const int64_t* lens, int32_t count,
                                   gbs_shard_state* d_state, int64_t* d_acc, int32_t step, void* stream) {
  if (!ctx || count < 0 || (count > 0 && (!shards || !lens))) return GBS_EINVAL;
  for (int32_t i = 0; i < count; ++i) {
    const gbs_status st = pass_dev<double>(ctx, shards[i], lens[i], d_state, d_acc, stream);
    if (st != GBS_OK) return st;
  }
  return step ? gbs_shard_step_dev(ctx, d_state, d_acc, stream) : GBS_OK;
}
gbs_status gbs_shard_step_dev(gbs_ctx* ctx, gbs_shard_state* d_state, int64_t* d_acc, void* stream) {
  if (!ctx || !d_state || !d_acc) return GBS_EINVAL;
  if (reinterpret_cast<uintptr_t>(d_acc) % 8 != 0 || reinterpret_cast<uintptr_t>(d_state) % 8 != 0)
    return GBS_EINVAL;
  DeviceGuard g(ctx->device);
  if (!g.ok) return GBS_ECUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  shard_step_kernel<<<1, 32, 0, s>>>(d_state, reinterpret_cast<long long*>(d_acc));
  if (cudaGetLastError() != cudaSuccess) return GBS_ECUDA;
  ctx->last_stream = s;
  return GBS_OK;
}

}  // extern "C"
