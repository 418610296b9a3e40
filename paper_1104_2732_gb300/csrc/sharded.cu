// Selection over a vector split into shards that are reduced separately (on several
// devices, in several processes, or as sub-ranges of one array): Algorithm 1 (Sec. 3)
// with the per-pass totals summed by the caller, as the paper's multi-GPU remark sums
// the per-device reductions on the host.  This file holds the host API of the scalar part
// of the method -- the starting bracket from the pass-0 totals (Sec. 3, step 0), and the
// cutting-plane iterate (step 1.1) and bracket update (steps 1.3-1.4) of shard_sm.cuh --
// and the compaction kernel of the finish.  The per-element passes are the library's own
// gbs_array_stats_* and gbs_cost_pass_* on each shard.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>

#include "api_internal.h"
#include "common.cuh"
#include "elem.cuh"
#include "shard_sm.cuh"

static_assert(sizeof(gbs_shard_state) == 184, "gbs_shard_state layout is part of the C-ABI");
static_assert(sizeof(gbs_array_stats) == 88 && sizeof(gbs_cost_eval) == 48, "C-ABI struct layout");

namespace gbs {
namespace {

using sm::done;
using sm::next_down;
using sm::round_to;

// ---------------------------------------------------------------------------------
// Compaction of (a, b] (the finish of Sec. 3): tiles staged in shared memory, one global
// atomic per tile.
// ---------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) compact_kernel(const T* __restrict__ x, long long n, T a, T b,
                                                      T* __restrict__ z, long long zcap,
                                                      unsigned long long* __restrict__ cnt) {
  // each tile of 4 x 256 elements: the kept ones gathered in shared memory (a warp's
  // ballot and one shared atomic per element slot), then one global atomic reserves the
  // tile's place and the block copies them out with consecutive stores
  using C = typename Ops<T>::C;
  __shared__ T s_buf[4 * 256];
  __shared__ unsigned int s_n;
  __shared__ unsigned long long s_base;
  const C ca = CmpOf<T>::le(a), cb = CmpOf<T>::le(b);
  const int lane = threadIdx.x & 31;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < n; base += 4 * stride) {
    if (threadIdx.x == 0) s_n = 0;
    __syncthreads();
    T v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const long long i = base + u * stride + threadIdx.x;
      v[u] = i < n ? x[i] : T(0);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const long long i = base + u * stride + threadIdx.x;
      bool keep = false;
      if (i < n) {
        const C cv = CmpOf<T>::of(v[u]);
        keep = !Ops<T>::is_nan(v[u]) && (cv > ca) && (cv <= cb);
      }
      const unsigned int m = __ballot_sync(0xffffffffu, keep);
      if (m) {
        unsigned int b0 = 0;
        if (lane == 0) b0 = atomicAdd(&s_n, (unsigned int)__popc(m));
        b0 = __shfl_sync(0xffffffffu, b0, 0);
        if (keep) s_buf[b0 + __popc(m & ((1u << lane) - 1u))] = v[u];
      }
    }
    __syncthreads();
    const unsigned int tn = s_n;
    if (threadIdx.x == 0 && tn) s_base = atomicAdd(cnt, (unsigned long long)tn);
    __syncthreads();
    const unsigned long long b0 = s_base;
    for (unsigned int j = threadIdx.x; j < tn; j += blockDim.x)
      if (b0 + j < (unsigned long long)zcap) z[b0 + j] = s_buf[j];
    __syncthreads();
  }
}

template <typename T>
gbs_status compact(gbs_ctx* c, const T* x, int64_t n, double a, double b, T* z, int64_t zcap, int64_t* count,
                   void* stream) {
  if (!c || !x || !count || n < 1 || zcap < 0 || (zcap > 0 && !z)) return GBS_EINVAL;
  if (!(a < b)) return GBS_EINVAL;
  DeviceGuard g(c->device);
  if (!g.ok) return GBS_ECUDA;
  gbs_status st = gbs_internal_ensure(c, 0);
  if (st != GBS_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  auto* cnt = reinterpret_cast<unsigned long long*>(static_cast<unsigned char*>(c->aux) + 256);
  if (cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), s) != cudaSuccess) return GBS_ECUDA;
  const long long blocks = std::min<long long>((n + 255) / 256, (long long)c->num_sms * 8);
  compact_kernel<T><<<(unsigned int)blocks, 256, 0, s>>>(x, n, (T)a, (T)b, z, zcap, cnt);
  if (cudaGetLastError() != cudaSuccess) return GBS_ECUDA;
  unsigned long long h = 0;
  if (cudaMemcpyAsync(&h, cnt, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess) return GBS_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return GBS_ECUDA;
  *count = (int64_t)h;
  return (int64_t)h > zcap ? GBS_ENOMEM : GBS_OK;
}

// One pass of the log driver: the counts at a and t and S = sum over a < x < t of
// (u(t) - u(x)), u = log1p(x - xmin) in float32; per-CTA records, summed in a fixed order
// by log_pass_total_kernel.
struct LogPart {
  unsigned long long lt, le, lea;
  double S;
};
template <typename T>
__global__ void __launch_bounds__(256) log_pass_kernel(const T* __restrict__ x, long long n, T a, T t, double xmin,
                                                       float ut, LogPart* part) {
  __shared__ LogPart s_p[8];
  using C = typename Ops<T>::C;
  const C ca = CmpOf<T>::le(a), ct_lt = CmpOf<T>::lt(t), ct_le = CmpOf<T>::le(t);
  unsigned int lt = 0, le = 0, lea = 0;
  float S = 0.f;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const T v = x[i];
    const C cv = CmpOf<T>::of(v);
    lt += cv < ct_lt;
    le += cv <= ct_le;
    lea += cv <= ca;
    if ((cv > ca) & (cv < ct_lt)) S += ut - log1pf((float)((double)v - xmin));
  }
  LogPart p;
  p.lt = __reduce_add_sync(0xffffffffu, lt);
  p.le = __reduce_add_sync(0xffffffffu, le);
  p.lea = __reduce_add_sync(0xffffffffu, lea);
  double Sd = (double)S;
  for (int o = 16; o > 0; o >>= 1) Sd += __shfl_xor_sync(0xffffffffu, Sd, o);
  p.S = Sd;
  if ((threadIdx.x & 31) == 0) s_p[threadIdx.x >> 5] = p;
  __syncthreads();
  if (threadIdx.x == 0) {
    LogPart q = s_p[0];
    for (int w = 1; w < 8; ++w) { q.lt += s_p[w].lt; q.le += s_p[w].le; q.lea += s_p[w].lea; q.S += s_p[w].S; }
    part[blockIdx.x] = q;
  }
}

__global__ void log_pass_total_kernel(const LogPart* part, int nparts, long long k, double ua, double ut,
                                      gbs_cost_eval* out) {
  if (threadIdx.x != 0) return;
  LogPart q{0ull, 0ull, 0ull, 0.0};
  for (int i = 0; i < nparts; ++i) { q.lt += part[i].lt; q.le += part[i].le; q.lea += part[i].lea; q.S += part[i].S; }
  gbs_cost_eval e;
  e.c_lt_t = (long long)q.lt; e.c_le_t = (long long)q.le; e.c_le_a = (long long)q.lea; e.pad = 0;
  e.S = q.S;
  e.dphi = ((double)e.c_le_a - (double)k + 0.5) * (ut - ua) + e.S;
  *out = e;
}

template <typename T>
gbs_status cost_pass_log(gbs_ctx* c, const T* x, int64_t n, int64_t k, double a, double t, double xmin,
                         gbs_cost_eval* out, void* stream) {
  if (!c || !x || !out || n < 1 || k < 1 || k > n) return GBS_EINVAL;
  if (!std::isfinite(a) || !std::isfinite(t) || !std::isfinite(xmin) || !((T)a < (T)t) || !(a > xmin - 1.0))
    return GBS_EINVAL;
  DeviceGuard g(c->device);
  if (!g.ok) return GBS_ECUDA;
  gbs_status st = gbs_internal_ensure(c, 0);
  if (st != GBS_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int blocks = (int)std::min<long long>((n + 255) / 256, (long long)c->num_sms * 8);
  auto* part = reinterpret_cast<LogPart*>(static_cast<unsigned char*>(c->aux) + 4096);   // within the 1 MiB area
  const double ua = std::log1p((double)(T)a - xmin), ut = std::log1p((double)(T)t - xmin);
  log_pass_kernel<T><<<blocks, 256, 0, s>>>(x, n, (T)a, (T)t, xmin, (float)ut, part);
  log_pass_total_kernel<<<1, 32, 0, s>>>(part, blocks, k, ua, ut, out);
  if (cudaGetLastError() != cudaSuccess) return GBS_ECUDA;
  c->last_stream = s;
  return GBS_OK;
}

}  // namespace
}  // namespace gbs

using namespace gbs;

extern "C" {

gbs_status gbs_shard_begin(gbs_shard_state* s, int32_t elem_bytes, int64_t n, int64_t k,
                           const gbs_array_stats* total, int64_t cap, int32_t maxit) {
  if (!s || !total || n < 1 || k < 1 || k > n || (elem_bytes != 4 && elem_bytes != 8)) return GBS_EINVAL;
  if (total->n != n || total->n_nan < 0 || total->n_neginf < 0 || total->n_posinf < 0 || total->n_finite < 0 ||
      total->n_nan + total->n_neginf + total->n_posinf + total->n_finite != n)
    return GBS_EINVAL;
  std::memset(s, 0, sizeof(*s));
  s->n = n;
  s->k = k;
  s->cap = cap > 0 ? cap : std::max<int64_t>(n / 16, 4096);
  s->maxit = maxit > 0 ? std::min(maxit, 64) : 64;
  s->elem_bytes = elem_bytes;
  s->n_negzero = total->n_negzero;
  s->n_neginf = total->n_neginf;
  s->dfv = 1;
  s->cle_a = -1;
  s->driver = GBS_DRIVER_KELLEY;
  s->xmin = total->n_finite > 0 ? round_to(total->min, elem_bytes) : 0.0;
  const int64_t nneg = total->n_neginf, npos = total->n_posinf;
  if (total->n_nan > 0) {
    s->phase = GBS_SHARD_NAN;
    s->result = std::numeric_limits<double>::quiet_NaN();
    return GBS_OK;
  }
  if (k <= nneg) {
    done(s, -std::numeric_limits<double>::infinity(), GBS_HOW_NEGINF, -1);
    return GBS_OK;
  }
  if (k > n - npos) {
    done(s, std::numeric_limits<double>::infinity(), GBS_HOW_POSINF, -1);
    return GBS_OK;
  }
  const double m = round_to(total->min, elem_bytes), M = round_to(total->max, elem_bytes);
  if (!(m < M) || k == nneg + 1) {
    // every finite element equal, or the rank of the smallest finite element
    done(s, m, GBS_HOW_MIN, nneg);
    return GBS_OK;
  }
  if (k == n - npos && M != 0.0) {   // the largest finite element (a zero needs its sign)
    done(s, M, GBS_HOW_MAX, -1);
    return GBS_OK;
  }
  s->phase = GBS_SHARD_ITERATE;
  s->b = M;
  s->cle_b = n - npos;
  s->clt_b = n - npos - 1;   // unique-maximum closed form (Sec. 3, step 0) until b moves
  const double a0 = next_down(m, elem_bytes);
  if (std::isfinite(a0)) {
    // (a0, M]: #(x <= a0) = #(x = -inf) exactly, and Phi(M) - Phi(a0) from the sum
    s->a = a0;
    s->cle_a = nneg;
    const double gL = (double)(nneg - k) + 0.5;
    s->dF = gL * (M - a0) + (double)total->n_finite * M - total->sum;
  } else {
    // m is the lowest finite value: (m, M] with #(x <= m) taken from the first pass
    s->a = m;
    s->cle_a = -1;
    s->dfv = 0;
  }
  return GBS_OK;
}

gbs_status gbs_shard_next(gbs_shard_state* s) {
  if (!s) return GBS_EINVAL;
  return sm::next(s);
}

gbs_status gbs_shard_set_driver(gbs_shard_state* s, int32_t driver) {
  if (!s || driver < GBS_DRIVER_KELLEY || driver > GBS_DRIVER_LOG || s->it != 0) return GBS_EINVAL;
  s->driver = driver;
  if (driver == GBS_DRIVER_LOG && s->phase == GBS_SHARD_ITERATE) s->dfv = 0;   // its dF is in u: not known yet
  return GBS_OK;
}

gbs_status gbs_shard_update(gbs_shard_state* s, const gbs_cost_eval* total) {
  if (!s || !total) return GBS_EINVAL;
  return sm::update(s, total);
}

gbs_status gbs_cost_pass_log_f32(gbs_ctx* ctx, const float* x, int64_t n, int64_t k, double a, double t,
                                 double xmin, gbs_cost_eval* out, void* stream) {
  return cost_pass_log<float>(ctx, x, n, k, a, t, xmin, out, stream);
}
gbs_status gbs_cost_pass_log_f64(gbs_ctx* ctx, const double* x, int64_t n, int64_t k, double a, double t,
                                 double xmin, gbs_cost_eval* out, void* stream) {
  return cost_pass_log<double>(ctx, x, n, k, a, t, xmin, out, stream);
}

gbs_status gbs_compact_f32(gbs_ctx* ctx, const float* x, int64_t n, double a, double b, float* z, int64_t z_cap,
                           int64_t* count, void* stream) {
  return compact<float>(ctx, x, n, a, b, z, z_cap, count, stream);
}
gbs_status gbs_compact_f64(gbs_ctx* ctx, const double* x, int64_t n, double a, double b, double* z,
                           int64_t z_cap, int64_t* count, void* stream) {
  return compact<double>(ctx, x, n, a, b, z, z_cap, count, stream);
}

}  // extern "C"
