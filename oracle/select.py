"""Exact order statistics and the cutting-plane model (CPU oracle, float64).

Test infrastructure only (see the package docstring): the GPU library never calls
this module.  Every function cites the passage of Beliakov, arXiv:1104.2732 that it
restates.  Readings of passages that are garbled or silent:

* Rank.  x_(k) is the k-th smallest element, k 1-based; Med(x) = x_([(n+1)/2])
  (Sec. 1).  Ties, signed zeros and infinities are ordered by IEEE-754 totalOrder
  (-inf < ... < -0 < +0 < ... < +inf); NaN has no rank and is rejected.
* Pinball weights.  Eq. (med_objOS) as printed puts (n-k+1/2) on x_i >= y, which
  makes k = 1 select the maximum.  The reading used here puts (k-1/2) on x_i >= y
  and (n-k+1/2) on x_i < y, so that k = 1 selects the minimum.
* Subgradient sign.  The count formula of Sec. 2 is -f'; Algorithm 1 and the
  figure's code use +f' (g < 0 moves y_L).  The reading is g = f'.
* One-sided slopes.  The tangent at y_L uses the right derivative (from #(x <= y_L)),
  the tangent at y_R the left derivative (from #(x < y_R)) (Sec. 3, step 0).
* Hybrid finish.  After the cutting-plane iterations the elements of the half-open
  bracket (y_L, y_R] are compacted and the (k - #(x <= y_L))-th of them is taken
  (Sec. 3, last paragraph; the open interval and index printed there drop x_(k)
  when it equals y_R).
"""
from __future__ import annotations

import math

import numpy as np

_SIGN = {np.dtype(np.float32): np.uint32(0x80000000),
         np.dtype(np.float64): np.uint64(0x8000000000000000)}
_UINT = {np.dtype(np.float32): np.uint32, np.dtype(np.float64): np.uint64}


def _check_float(x):
    x = np.ascontiguousarray(x)
    if x.dtype not in _SIGN:
        raise TypeError(f"float32 or float64 expected, got {x.dtype}")
    return x


def total_order_key(x):
    """Order-preserving unsigned key of IEEE-754 bits (totalOrder; Sec. 1 ranks).

    Negative values have all bits flipped, non-negative values get the sign bit set,
    so unsigned comparison of keys is -inf < ... < -0 < +0 < ... < +inf.
    """
    x = _check_float(x)
    sign = _SIGN[x.dtype]
    u = x.view(_UINT[x.dtype])
    return np.where((u & sign) != 0, ~u, u | sign)


def key_to_value(keys, dtype):
    """Inverse of :func:`total_order_key`."""
    dtype = np.dtype(dtype)
    sign = _SIGN[dtype]
    k = np.asarray(keys, dtype=_UINT[dtype])
    u = np.where((k & sign) != 0, k & ~sign, ~k)
    return u.astype(_UINT[dtype]).view(dtype)


def _check_rank(x, k):
    n = x.size
    if n < 1:
        raise ValueError("empty input has no order statistic")
    if not (1 <= k <= n):
        raise ValueError(f"rank k={k} outside [1, {n}]")
    if np.isnan(x).any():
        raise ValueError("NaN has no rank")


def select_kth(x, k):
    """x_(k), the k-th smallest element of x (Sec. 1), returned with its exact bits.

    Plain definition: the k-th entry of x in ascending totalOrder.  The library
    selection primitive ``np.partition`` places that entry at index k-1.
    """
    x = _check_float(x)
    k = int(k)
    _check_rank(x, k)
    keys = total_order_key(x)
    kth = np.partition(keys, k - 1)[k - 1]
    return key_to_value(kth, x.dtype)[()]


def select_kth_sorted(x, k):
    """x_(k) by a full sort of the keys (the alternative the paper benchmarks, Sec. 2)."""
    x = _check_float(x)
    k = int(k)
    _check_rank(x, k)
    return key_to_value(np.sort(total_order_key(x))[k - 1], x.dtype)[()]


def median(x):
    """Med(x) = x_([(n+1)/2]) (Sec. 1)."""
    x = _check_float(x)
    return select_kth(x, (x.size + 1) // 2)


def median_rank(n):
    """The rank [(n+1)/2] of the median (Sec. 1)."""
    return (int(n) + 1) // 2


def counts(x, t):
    """(#(x < t), #(x <= t)) under IEEE comparison: the counts that make up the
    subgradient g of Sec. 2 (so -0 == +0 and -inf < t < +inf for finite t)."""
    x = _check_float(x)
    t = x.dtype.type(t)
    return int(np.count_nonzero(x < t)), int(np.count_nonzero(x <= t))


def median_cost(x, y):
    """f(y) = sum_i |x_i - y| (Eq. med_obj), summed exactly and rounded once."""
    x = np.asarray(x, dtype=np.float64)
    return math.fsum(np.abs(x - float(y)).tolist())


def pinball_cost(x, k, y):
    """F(y) = sum_i u(x_i - y) of Eq. (med_objOS) with the weights read as
    u(s) = (k - 1/2) s for s >= 0 and u(s) = -(n - k + 1/2) s for s < 0."""
    x = np.asarray(x, dtype=np.float64)
    n = x.size
    s = x - float(y)
    u = np.where(s >= 0, (k - 0.5) * s, -(n - k + 0.5) * s)
    return math.fsum(u.tolist())


def pinball_subdifferential(x, k, y):
    """The subdifferential of F at y (Sec. 2, Clarke's subdifferential of a sum of
    one-sided linear terms): [n(#(x<y) - k + 1/2), n(#(x<=y) - k + 1/2)].

    Slope of F left of y: every x_i < y contributes +(n-k+1/2) and every x_i >= y
    contributes -(k-1/2); the sum simplifies to n(#(x<y) - k + 1/2).  Right of y the
    same holds with #(x<=y)."""
    n = np.asarray(x).size
    c_lt, c_le = counts(x, y)
    return n * (c_lt - k + 0.5), n * (c_le - k + 0.5)


def is_minimiser(x, k, y):
    """0 in dF(y)  <=>  #(x<y) < k <= #(x<=y)  (Sec. 2, root of 0 in g(y))."""
    lo, hi = pinball_subdifferential(x, k, y)
    return lo <= 0.0 <= hi


def relative_cost(x, k, a, t):
    """Phi(t) - Phi(a) for a < t, where Phi = F / n (Eq. med_objOS scaled by 1/n).

    Phi is piecewise linear with slope #(x<y) - k + 1/2 between data points, so
        Phi(t) - Phi(a) = (#(x<=a) - k + 1/2)(t - a) + sum_{a < x_i < t} (t - x_i).
    Only the elements inside (a, t) enter the sum, which keeps far outliers (Sec. 4,
    Discussion) out of it.
    """
    x = np.asarray(x)
    a64, t64 = float(a), float(t)
    _, c_le_a = counts(x, a)
    inside = x[(x > x.dtype.type(a)) & (x < x.dtype.type(t))].astype(np.float64)
    return (c_le_a - k + 0.5) * (t64 - a64) + math.fsum((t64 - inside).tolist())


def _next_toward(v, direction, dtype):
    return np.nextafter(dtype.type(v), dtype.type(direction))


def _inside(t, a, b, dtype):
    """Round t to the data's floating-point grid strictly inside (a, b) (IEEE)."""
    tt = dtype.type(t)
    if not (tt > dtype.type(a)):
        tt = _next_toward(a, np.inf, dtype)
    if not (tt < dtype.type(b)):
        tt = _next_toward(b, -np.inf, dtype)
    return tt


def _key_midpoint(a, b, dtype):
    ka = int(total_order_key(np.array([a], dtype=dtype))[0])
    kb = int(total_order_key(np.array([b], dtype=dtype))[0])
    return key_to_value((ka + kb) // 2, dtype)[()]


def _zero_sign(value, k, c_lt_v, n_negzero, dtype):
    """x_(k) is zero: it is -0 iff its rank inside the zero run falls among the -0s."""
    if value == 0:
        return dtype.type(-0.0) if (k - c_lt_v) <= n_negzero else dtype.type(0.0)
    return dtype.type(value)


def kelley_select(x, k, cap=None, maxit=64, slow_shrink=0.75, stall=0.875):
    """Hybrid selection: Kelley's cutting plane (Algorithm 1) on the pinball cost,
    then compaction of the bracket and an exact select inside it (Sec. 3).

    Step 0 takes y_L = x_(1), y_R = x_(n) over the finite elements (Sec. 3) with the
    one-sided slopes of :func:`pinball_subdifferential`.  Each iteration computes the
    intersection of the two tangents (step 1.1), evaluates #(x<t), #(x<=t) and
    Phi(t) - Phi(y_L) (step 1.2), stops on 0 in dPhi(t) (step 1.3) and moves y_L or y_R
    by the sign of the subgradient (step 1.4).

    Readings where the paper is silent (the GPU path follows the same rules):
    * t is rounded to the data's grid strictly inside (y_L, y_R).
    * If a cutting-plane step leaves more than ``slow_shrink`` of the bracket's
      elements, the next point is the midpoint of the bracket in totalOrder keys
      (guards against rounding stalls; the result never depends on it).
    * Iterations stop once the bracket holds at most ``cap`` elements: that pass
      also compacts (y_L, y_R], and the answer is selected among them (Sec. 3, last
      paragraph).  The next pass compacts as well once two steps in a row have each
      left more than ``stall`` of the bracket's elements (a heavy run of equal
      values that no iterate hits exactly), and unconditionally after ``maxit``.
    * +-inf enter only the counts; the starting bracket is over finite elements.

    Returns ``(value, info)``; ``info['passes']`` counts full passes over x
    (pass 0 = the min/max/count reduction, then one per evaluated t).
    """
    x = _check_float(x)
    dt = x.dtype
    k = int(k)
    _check_rank(x, k)
    n = x.size
    if cap is None:
        cap = max(1, n // 16)
    info = {"passes": 1, "iterates": [], "pops": [], "steps": [], "how": None}

    # pass 0: extremes of the finite part, infinities, signed zeros (Sec. 3, step 0)
    n_neginf = int(np.count_nonzero(x == -np.inf))
    n_posinf = int(np.count_nonzero(x == np.inf))
    n_negzero = int(np.count_nonzero((x == 0) & np.signbit(x)))
    if k <= n_neginf:
        info["how"] = "neginf"
        return dt.type(-np.inf), info
    if k > n - n_posinf:
        info["how"] = "posinf"
        return dt.type(np.inf), info
    fin = x[np.isfinite(x)]
    m, M = fin.min(), fin.max()
    c_le_m = counts(x, m)[1]
    c_lt_M = counts(x, M)[0]
    if c_le_m >= k:
        info["how"] = "min"
        return _zero_sign(m, k, n_neginf, n_negzero, dt), info
    if c_lt_M < k:
        info["how"] = "max"
        return _zero_sign(M, k, c_lt_M, n_negzero, dt), info

    yL, yR = m, M
    cle_L, clt_R, cle_R = c_le_m, c_lt_M, n - n_posinf
    dF = relative_cost(x, k, yL, yR)           # Phi(y_R) - Phi(y_L)
    use_bisect = False
    stalled = 0
    it = 0
    while True:
        it += 1
        pop = cle_R - cle_L
        compact = pop <= cap or it > maxit or stalled >= 2
        gL = cle_L - k + 0.5                   # right slope at y_L  (< 0)
        gR = clt_R - k + 0.5                   # left slope at y_R   (> 0)
        if use_bisect:
            t = _inside(_key_midpoint(yL, yR, dt), yL, yR, dt)
            info["steps"].append("bisect")
        else:
            w = float(yR) - float(yL)
            t_star = float(yL) + (gR * w - dF) / (gR - gL)     # step 1.1
            t = _inside(t_star, yL, yR, dt)
            info["steps"].append("kelley")
        info["passes"] += 1
        info["iterates"].append(t)
        c_lt, c_le = counts(x, t)              # step 1.2
        dphi = relative_cost(x, k, yL, t)      # Phi(t) - Phi(y_L)
        if c_lt < k <= c_le:                   # step 1.3: 0 in dPhi(t)
            info["how"] = "hit"
            info["pops"].append(0)
            return _zero_sign(t, k, c_lt, n_negzero, dt), info
        if c_le < k:                           # step 1.4: g(t) < 0
            new = dict(yL=t, cle_L=c_le, dF=dF - dphi)
        else:                                  # g(t) > 0
            new = dict(yR=t, clt_R=c_lt, cle_R=c_le, dF=dphi)
        yL = new.get("yL", yL)
        cle_L = new.get("cle_L", cle_L)
        yR = new.get("yR", yR)
        clt_R = new.get("clt_R", clt_R)
        cle_R = new.get("cle_R", cle_R)
        dF = new["dF"]
        new_pop = cle_R - cle_L
        info["pops"].append(new_pop)
        use_bisect = (not use_bisect) and new_pop > slow_shrink * pop
        stalled = stalled + 1 if new_pop > stall * pop else 0
        if compact:
            # compaction of (y_L, y_R] and the exact finish (Sec. 3, hybrid)
            z = x[(x > yL) & (x <= yR)]
            info["how"] = "finish"
            info["finish_pop"] = int(z.size)
            return select_kth(z, k - cle_L), info
