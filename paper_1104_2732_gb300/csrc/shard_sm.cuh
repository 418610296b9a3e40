// The scalar part of a sharded selection (Algorithm 1, Sec. 3): the next point (step 1.1,
// or a driver's alternative) and the bracket update from the per-pass totals (steps
// 1.3-1.4), as host-and-device functions.  The host API (gbs_shard_next / _update) and
// the device-resident loop (shard_dev.cu) run the same code, so a state advanced on the
// device equals one advanced on the host from the same totals.
#pragma once

#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>

#include "gbselect.h"

#ifdef __CUDACC__
#define GBS_HD __host__ __device__ __forceinline__
#else
#define GBS_HD inline
#endif

namespace gbs {
namespace sm {

GBS_HD uint64_t ukey_of(double v, int eb) {   // totalOrder key of v as an element of width eb
  if (eb == 4) {
    uint32_t u;
    const float f = (float)v;
    memcpy(&u, &f, 4);
    return (u & 0x80000000u) ? (uint64_t)(~u) : (uint64_t)(u | 0x80000000u);
  }
  uint64_t u;
  memcpy(&u, &v, 8);
  return (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
}
GBS_HD double ukey_value_of(uint64_t k, int eb) {
  if (eb == 4) {
    const uint32_t kk = (uint32_t)k;
    const uint32_t u = (kk & 0x80000000u) ? (kk & 0x7FFFFFFFu) : ~kk;
    float f;
    memcpy(&f, &u, 4);
    return (double)f;
  }
  const uint64_t u = (k & 0x8000000000000000ull) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k;
  double d;
  memcpy(&d, &u, 8);
  return d;
}
GBS_HD double round_to(double v, int eb) { return eb == 4 ? (double)(float)v : v; }
GBS_HD double next_up(double v, int eb) {
  return eb == 4 ? (double)nextafterf((float)v, std::numeric_limits<float>::infinity())
                 : nextafter(v, std::numeric_limits<double>::infinity());
}
GBS_HD double next_down(double v, int eb) {
  return eb == 4 ? (double)nextafterf((float)v, -std::numeric_limits<float>::infinity())
                 : nextafter(v, -std::numeric_limits<double>::infinity());
}
// a point of the grid strictly inside (a, b), as close to v as possible
GBS_HD double inside(double v, double a, double b, int eb) {
  double t = round_to(v, eb);
  if (!(t > a)) t = next_up(a, eb);
  if (!(t < b)) t = next_down(b, eb);
  return t;
}

// x_(k) = 0: -0 sorts before +0, so it is -0 when k - #(x < 0) <= #(x = -0)
GBS_HD void finish_zero(gbs_shard_state* s, int64_t clt) {
  if (s->result == 0.0) s->result = (s->k - clt) <= s->n_negzero ? -0.0 : 0.0;
}
GBS_HD void done(gbs_shard_state* s, double v, int32_t how, int64_t clt) {
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
GBS_HD double brent_point(gbs_shard_state* s, double mid) {
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
  const double last = s->it > 0 ? s->px : (fabs(ga) < fabs(gb) ? a : b);
  const bool ok = isfinite(t) && t > a && t < b && (s->it < 2 || fabs(t - last) < 0.5 * fabs(s->step2));
  const double chosen = ok ? t : mid;
  s->step2 = s->step1;
  s->step1 = chosen - last;
  return chosen;
}

// Step 1.1 (or the driver's point): sets t, or moves the state to COMPACT once the
// bracket holds at most cap elements, after maxit iterates or two stalled steps.
GBS_HD gbs_status next(gbs_shard_state* s) {
  if (s->phase != GBS_SHARD_ITERATE) return GBS_EINVAL;
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
    const uint64_t ka = ukey_of(s->a, eb), kb = ukey_of(s->b, eb);
    t = inside(ukey_value_of(ka + (kb - ka) / 2, eb), s->a, s->b, eb);
  } else {
    const double gL = (double)(s->cle_a - s->k) + 0.5, gR = (double)(s->clt_b - s->k) + 0.5;
    if (s->driver == GBS_DRIVER_LOG) {   // the tangent intersection in u = log1p(x - xmin)
      const double ua = log1p(s->a - s->xmin), ub = log1p(s->b - s->xmin);
      const double ut = ua + (gR * (ub - ua) - s->dF) / (gR - gL);
      t = inside(s->xmin + expm1(ut), s->a, s->b, eb);
    } else {
      const double w = s->b - s->a;
      t = inside(s->a + (gR * w - s->dF) / (gR - gL), s->a, s->b, eb);
    }
  }
  s->t = t;
  return GBS_OK;
}

// Steps 1.3-1.4 from the pass totals at (a, t) over every shard.
GBS_HD gbs_status update(gbs_shard_state* s, const gbs_cost_eval* total) {
  if (s->phase != GBS_SHARD_ITERATE) return GBS_EINVAL;
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
  const double width = s->driver == GBS_DRIVER_LOG ? log1p(s->t - s->xmin) - log1p(s->a - s->xmin) : s->t - s->a;
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

// Fraction bits of the fixed-point cost total of a device-resident pass at the state's
// (a, t): every term of S lies in [0, w] (w = t - a, or u(t) - u(a) for the log driver),
// so with n w < 2^e and fx = 61 - e the scaled total stays below 2^61 (int64, with room
// for the rounding of each block's part).
GBS_HD int sfix_bits(const gbs_shard_state* s) {
  const double w = s->driver == GBS_DRIVER_LOG ? log1p(s->t - s->xmin) - log1p(s->a - s->xmin) : s->t - s->a;
  const double bound = (double)s->n * (w > 0.0 ? w : 0.0);
  if (!(bound > 0.0) || !isfinite(bound)) return 0;
  int e = 0;
  frexp(bound, &e);   // bound < 2^e
  int fx = 61 - e;
  if (fx > 1000) fx = 1000;
  if (fx < -1000) fx = -1000;
  return fx;
}

}  // namespace sm
}  // namespace gbs
