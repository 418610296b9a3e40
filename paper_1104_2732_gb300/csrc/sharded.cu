// Selection over a vector split into shards that are reduced separately (on several
// devices, in several processes, or as sub-ranges of one array): Algorithm 1 (Sec. 3)
// with the per-pass totals summed by the caller, as the paper's multi-GPU remark sums
// the per-device reductions on the host.  This file holds the scalar part of the method
// as host code -- the starting bracket from the pass-0 totals (Sec. 3, step 0), the
// cutting-plane iterate (step 1.1) and the bracket update (steps 1.3-1.4) -- and the
// compaction kernel of the finish.  The per-element passes are the library's own
// gbs_array_stats_* and gbs_cost_pass_* on each shard.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>

#include "api_internal.h"
#include "common.cuh"
#include "elem.cuh"

static_assert(sizeof(gbs_shard_state) == 184, "gbs_shard_state layout is part of the C-ABI");
static_assert(sizeof(gbs_array_stats) == 88 && sizeof(gbs_cost_eval) == 48, "C-ABI struct layout");

namespace gbs {
namespace {

// ---------------------------------------------------------------------------------
// Host arithmetic on the element grid (float32 or float64).
// ---------------------------------------------------------------------------------
uint64_t host_ukey(double v, int eb) {   // totalOrder key of v as an element of width eb
  if (eb == 4) {
    uint32_t u;
    const float f = (float)v;
    std::memcpy(&u, &f, 4);
    return (u & 0x80000000u) ? (uint64_t)(~u) : (uint64_t)(u | 0x80000000u);
  }
  uint64_t u;
  std::memcpy(&u, &v, 8);
  return (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
}
double host_ukey_value(uint64_t k, int eb) {
  if (eb == 4) {
    const uint32_t kk = (uint32_t)k;
    const uint32_t u = (kk & 0x80000000u) ? (kk & 0x7FFFFFFFu) : ~kk;
    float f;
    std::memcpy(&f, &u, 4);
    return (double)f;
  }
  const uint64_t u = (k & 0x8000000000000000ull) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k;
  double d;
  std::memcpy(&d, &u, 8);
  return d;
}
double round_to(double v, int eb) { return eb == 4 ? (double)(float)v : v; }
double next_up(double v, int eb) {
  return eb == 4 ? (double)std::nextafter((float)v, std::numeric_limits<float>::infinity())
                 : std::nextafter(v, std::numeric_limits<double>::infinity());
}
double next_down(double v, int eb) {
  return eb == 4 ? (double)std::nextafter((float)v, -std::numeric_limits<float>::infinity())
                 : std::nextafter(v, -std::numeric_limits<double>::infinity());
}
// a point of the grid strictly inside (a, b), as close to v as possible
double inside(double v, double a, double b, int eb) {
  double t = round_to(v, eb);
  if (!(t > a)) t = next_up(a, eb);
  if (!(t < b)) t = next_down(b, eb);
  return t;
}

// x_(k) = 0: -0 sorts before +0, so it is -0 when k - #(x < 0) <= #(x = -0)
void finish_zero(gbs_shard_state* s, int64_t clt) {
  if (s->result == 0.0) s->result = (s->k - clt) <= s->n_negzero ? -0.0 : 0.0;
}
void done(gbs_shard_state* s, double v, int32_t how, int64_t clt) {
  s->phase = GBS_SHARD_DONE;
  s->result = v;
  s->how = how;
  if (clt >= 0) finish_zero(s, clt);
}

// Brent's root-finder on g(y) = #(x < y) - k + 1/2 over the bracket (a, b), where
// g(a) = #(x <= a) - k + 1/2 < 0 and g(b) = #(x < b) - k + 1/2 > 0: inverse quadratic
// interpolation through (a, b, the last point evaluated) when their g are distinct, else
// the secant through the ends; the interpolant is taken when it lies strictly inside and
// moves less than half the step before last, else the midpoint (Brent's safeguard).
double brent_point(gbs_shard_state* s, double mid) {
  const double a = s->a, b = s->b;
  if (s->cle_a < 0) return mid;
  const double ga = (double)(s->cle_a - s->k) + 0.5, gb = (double)(s->clt_b - s->k) + 0.5;
  double t;
  const double c = s->px, gc = s->pg;
  const bool iqi = s->it > 0 && c != a && c != b && gc != ga && gc != gb && ga != gb;
  if (iqi) {
    t = a * gb * gc / ((ga - gb) * (ga - gc)) + b * ga * gc / ((gb - ga) * (gb - gc)) +
        c * ga * gb / ((gc - ga) * (gc - gb));
  } else {
    t = a - ga * (b - a) / (gb - ga);
  }
  const double last = s->it > 0 ? s->px : (std::fabs(ga) < std::fabs(gb) ? a : b);
  const bool ok = std::isfinite(t) && t > a && t < b && (s->it < 2 || std::fabs(t - last) < 0.5 * std::fabs(s->step2));
  const double chosen = ok ? t : mid;
  s->step2 = s->step1;
  s->step1 = chosen - last;
  return chosen;
}

// ---------------------------------------------------------------------------------
// Compaction of (a, b] (the finish of Sec. 3): warp ballots, one atomic per warp.
// ---------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) compact_kernel(const T* __restrict__ x, long long n, T a, T b,
                                                      T* __restrict__ z, long long zcap,
                                                      unsigned long long* __restrict__ cnt) {
  using C = typename Ops<T>::C;
  const C ca = CmpOf<T>::le(a), cb = CmpOf<T>::le(b);
  const int lane = threadIdx.x & 31;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < n; base += stride) {
    const long long i = base + threadIdx.x;
    T v = T(0);
    bool keep = false;
    if (i < n) {
      v = x[i];
      const C cv = CmpOf<T>::of(v);
      keep = !Ops<T>::is_nan(v) && (cv > ca) && (cv <= cb);
    }
    const unsigned int m = __ballot_sync(0xffffffffu, keep);
    if (m) {
      unsigned long long b0 = 0;
      if (lane == 0) b0 = atomicAdd(cnt, (unsigned long long)__popc(m));
      b0 = __shfl_sync(0xffffffffu, b0, 0);
      const unsigned long long pos = b0 + (unsigned long long)__popc(m & ((1u << lane) - 1u));
      if (keep && pos < (unsigned long long)zcap) z[pos] = v;
    }
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
  if (!s || s->phase != GBS_SHARD_ITERATE) return GBS_EINVAL;
  const int eb = s->elem_bytes;
  if (s->cle_a >= 0) {
    const int64_t pop = s->cle_b - s->cle_a;
    if (pop <= s->cap || s->it >= s->maxit || s->stalled >= 2) {
      s->phase = GBS_SHARD_COMPACT;
      return GBS_OK;
    }
  }
  const double mid = s->a + 0.5 * (s->b - s->a);   // the bracket's midpoint in value
  double t;
  if (s->driver == GBS_DRIVER_BISECT) {
    t = inside(mid, s->a, s->b, eb);
  } else if (s->driver == GBS_DRIVER_BRENT) {
    t = inside(brent_point(s, mid), s->a, s->b, eb);
  } else if (s->use_bisect || !s->dfv || s->cle_a < 0) {
    const uint64_t ka = host_ukey(s->a, eb), kb = host_ukey(s->b, eb);
    t = inside(host_ukey_value(ka + (kb - ka) / 2, eb), s->a, s->b, eb);
  } else {
    const double gL = (double)(s->cle_a - s->k) + 0.5, gR = (double)(s->clt_b - s->k) + 0.5;
    if (s->driver == GBS_DRIVER_LOG) {   // the tangent intersection in u = log1p(x - xmin)
      const double ua = std::log1p(s->a - s->xmin), ub = std::log1p(s->b - s->xmin);
      const double ut = ua + (gR * (ub - ua) - s->dF) / (gR - gL);
      t = inside(s->xmin + std::expm1(ut), s->a, s->b, eb);
    } else {
      const double w = s->b - s->a;
      t = inside(s->a + (gR * w - s->dF) / (gR - gL), s->a, s->b, eb);
    }
  }
  s->t = t;
  return GBS_OK;
}

gbs_status gbs_shard_set_driver(gbs_shard_state* s, int32_t driver) {
  if (!s || driver < GBS_DRIVER_KELLEY || driver > GBS_DRIVER_LOG || s->it != 0) return GBS_EINVAL;
  s->driver = driver;
  if (driver == GBS_DRIVER_LOG && s->phase == GBS_SHARD_ITERATE) s->dfv = 0;   // its dF is in u: not known yet
  return GBS_OK;
}

gbs_status gbs_shard_update(gbs_shard_state* s, const gbs_cost_eval* total) {
  if (!s || !total || s->phase != GBS_SHARD_ITERATE) return GBS_EINVAL;
  const int64_t k = s->k;
  if (total->c_le_a < 0 || total->c_lt_t < total->c_le_a || total->c_le_t < total->c_lt_t ||
      total->c_le_t > s->n)
    return GBS_EINTERNAL;
  if (s->cle_a < 0) {          // the first pass counted #(x <= m)
    s->cle_a = total->c_le_a;
    if (s->cle_a >= k) {       // x_(k) = m; #(x < m) = #(x = -inf)
      done(s, s->a, GBS_HOW_MIN, s->n_neginf);
      return GBS_OK;
    }
  } else if (total->c_le_a != s->cle_a) {
    return GBS_EINTERNAL;      // the shards did not all see the same array
  }
  s->it++;
  const int64_t clt = total->c_lt_t, cle = total->c_le_t;
  if (clt < k && k <= cle) {   // step 1.3: 0 in dF(t)
    done(s, s->t, GBS_HOW_HIT, clt);
    return GBS_OK;
  }
  const double gL = (double)(s->cle_a - k) + 0.5;
  const double width = s->driver == GBS_DRIVER_LOG ? std::log1p(s->t - s->xmin) - std::log1p(s->a - s->xmin)
                                                   : s->t - s->a;
  const double dphi = gL * width + total->S;
  const int64_t pop = s->cle_b - s->cle_a;
  // the root-finder's memory: the point just evaluated with its g on the side it moves
  s->px = s->t;
  s->pg = cle < k ? (double)(cle - k) + 0.5 : (double)(clt - k) + 0.5;
  if (cle < k) {               // step 1.4: the subgradient at t is negative
    s->a = s->t;
    s->cle_a = cle;
    s->dF = s->dF - dphi;
  } else {
    s->b = s->t;
    s->clt_b = clt;
    s->cle_b = cle;
    s->dF = dphi;
    s->dfv = 1;
  }
  const int64_t npop = s->cle_b - s->cle_a;
  if (s->driver == GBS_DRIVER_KELLEY || s->driver == GBS_DRIVER_LOG) {   // the safeguards of the cutting plane
    const int prev = s->use_bisect;
    s->use_bisect = (!prev) && ((double)npop > 0.75 * (double)pop);
    s->stalled = ((double)npop > 0.875 * (double)pop) ? s->stalled + 1 : 0;
  }
  return GBS_OK;
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
