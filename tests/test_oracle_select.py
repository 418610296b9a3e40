"""Pins of the selection oracle against what the paper and the mathematics fix.

CPU only.  Each test pins a part of oracle/select.py to something other than the
oracle itself: hand-worked values, the rank definition by brute force, closed forms
(Sec. 3, step 0), the optimality condition 0 in dF (Sec. 2), permutation invariance
(Sec. 4, Discussion) and textbook special cases.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

from oracle import select as osel
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def _rank_brute(x, k):
    """x_(k) by the rank definition alone: the element e with
    #(key < key(e)) < k <= #(key <= key(e)); no sorting or selection routine."""
    keys = [int(v) for v in osel.total_order_key(np.asarray(x))]
    for i, e in enumerate(keys):
        below = sum(1 for v in keys if v < e)
        upto = sum(1 for v in keys if v <= e)
        if below < k <= upto:
            return np.asarray(x)[i]
    raise AssertionError("no element has rank k")


def _bits(v):
    v = np.asarray(v)
    return v.view(np.uint32 if v.dtype == np.float32 else np.uint64).item()


ALPHABET = [-np.inf, -2.0, -1.0, -0.0, 0.0, 1.0, 1.5, np.inf]


def test_golden_order_statistics_and_costs():
    g = _golden("median_objective_n9.json")
    x = np.array(g["x"], dtype=np.float64)
    for k, v in g["order_statistics"]["k_to_value"].items():
        assert osel.select_kth(x, int(k)) == v
    assert osel.median(x) == g["order_statistics"]["median"]
    for y, f in g["median_cost"]["y_to_f"].items():
        assert osel.median_cost(x, float(y)) == f
    for y, F in g["pinball_k3"]["y_to_F"].items():
        assert osel.pinball_cost(x, 3, float(y)) == F
    # the pinball minimiser over the data is x_(3) = 2 with the corrected weights
    costs = {v: osel.pinball_cost(x, 3, v) for v in set(g["x"])}
    assert min(costs, key=costs.get) == g["pinball_k3"]["minimiser"]


def test_golden_closed_forms_step0():
    g = _golden("median_objective_n9.json")["closed_forms"]
    x = np.array(_golden("median_objective_n9.json")["x"], dtype=np.float64)
    n = x.size
    yL, yR = x.min(), x.max()
    assert math.fsum(x) == g["sum_x"]
    assert osel.median_cost(x, yL) == g["f_yL"] == g["sum_x"] - n * yL
    assert osel.median_cost(x, yR) == g["f_yR"] == n * yR - g["sum_x"]
    # one-sided slopes of sum|x - y| from the counts: right slope #(<=) - #(>)
    c_lt_L, c_le_L = osel.counts(x, yL)
    c_lt_R, c_le_R = osel.counts(x, yR)
    assert c_le_L - (n - c_le_L) == g["right_slope_at_yL"]
    assert c_lt_R - (n - c_lt_R) == g["left_slope_at_yR"] == n - 2


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_brute_force_tiny_alphabet(dtype):
    rng = np.random.default_rng(1)
    for n in range(1, 7):
        for _ in range(60):
            x = rng.choice(ALPHABET, size=n).astype(dtype)
            for k in range(1, n + 1):
                got = osel.select_kth(x, k)
                want = _rank_brute(x, k)
                assert _bits(got) == _bits(want), (x, k)
                assert _bits(osel.select_kth_sorted(x, k)) == _bits(want)


def test_brute_force_all_small_arrays_exhaustive():
    alph = [-np.inf, -0.0, 0.0, 1.0, np.inf]
    for n in range(1, 5):
        for tup in itertools.product(alph, repeat=n):
            x = np.array(tup, dtype=np.float32)
            for k in range(1, n + 1):
                assert _bits(osel.select_kth(x, k)) == _bits(_rank_brute(x, k))


def test_signed_zero_order():
    x = np.array([0.0, -0.0, 0.0, -0.0, -0.0], dtype=np.float32)
    assert [np.signbit(osel.select_kth(x, k)) for k in range(1, 6)] == [True] * 3 + [False] * 2


def test_min_max_special_cases():
    rng = np.random.default_rng(2)
    x = rng.standard_normal(1001).astype(np.float32)
    assert osel.select_kth(x, 1) == x.min()
    assert osel.select_kth(x, x.size) == x.max()
    assert osel.median(x) == np.sort(x)[500]


def test_nan_and_rank_rejected():
    with pytest.raises(ValueError):
        osel.select_kth(np.array([1.0, np.nan], dtype=np.float32), 1)
    with pytest.raises(ValueError):
        osel.select_kth(np.array([1.0], dtype=np.float32), 2)
    with pytest.raises(ValueError):
        osel.select_kth(np.array([], dtype=np.float32), 1)


@pytest.mark.parametrize("k_frac", [0.0, 0.01, 0.5, 0.99, 1.0])
def test_pinball_minimiser_is_order_statistic(k_frac):
    """The minimiser of Eq. (med_objOS) (corrected weights) over y in x is x_(k):
    a swapped weight pair would return x_(n-k+1) instead."""
    rng = np.random.default_rng(3)
    x = np.round(rng.standard_normal(41) * 4).astype(np.float64)   # ties included
    n = x.size
    k = min(n, max(1, int(round(k_frac * n))))
    vals = np.unique(x)
    costs = np.array([osel.pinball_cost(x, k, v) for v in vals])
    assert vals[np.argmin(costs)] == osel.select_kth(x, k)


def test_pinball_reduces_to_median_cost_for_odd_n():
    """k = (n+1)/2 with n odd: u(s) = (n/2)|s|, so F = (n/2) f of Eq. (med_obj)."""
    rng = np.random.default_rng(4)
    x = rng.integers(-50, 50, 21).astype(np.float64)
    n = x.size
    k = (n + 1) // 2
    for y in (-60.0, -3.0, 0.0, 7.5, 60.0):
        assert osel.pinball_cost(x, k, y) == pytest.approx(n / 2 * osel.median_cost(x, y), abs=0)


def test_subdifferential_and_minimiser_condition():
    """0 in dF(y) exactly at y = x_(k) (Sec. 2): checked against finite differences of
    F and against the rank definition."""
    rng = np.random.default_rng(5)
    x = rng.integers(0, 12, 30).astype(np.float64)     # heavy ties
    n = x.size
    for k in (1, 7, 15, 16, 30):
        xk = _rank_brute(x, k)
        for y in np.unique(x):
            lo, hi = osel.pinball_subdifferential(x, k, y)
            h = 1e-3
            assert (osel.pinball_cost(x, k, y) - osel.pinball_cost(x, k, y - h)) / h == pytest.approx(lo, rel=1e-9, abs=1e-6)
            assert (osel.pinball_cost(x, k, y + h) - osel.pinball_cost(x, k, y)) / h == pytest.approx(hi, rel=1e-9, abs=1e-6)
            assert osel.is_minimiser(x, k, y) == (y == xk)
        assert n * 0 == 0


def test_relative_cost_matches_cost_differences():
    """Phi(t) - Phi(a) from the bracket-only sum equals (F(t) - F(a))/n exactly on
    integer data (every sum is exact in float64)."""
    rng = np.random.default_rng(6)
    x = rng.integers(-1000, 1000, 501).astype(np.float64)
    n = x.size
    for k in (1, 100, 251, 500, 501):
        for a, t in [(-1000.0, 1000.0), (-3.0, 17.0), (0.0, 0.5), (-999.5, -998.0), (5.0, 600.0)]:
            want = (osel.pinball_cost(x, k, t) - osel.pinball_cost(x, k, a)) / n
            assert osel.relative_cost(x, k, a, t) == pytest.approx(want, rel=1e-12, abs=1e-9)


def test_relative_cost_at_tied_data_points():
    """Bracket ends on data values with ties: the elements equal to a count in the
    slope #(x <= a), not in the sum over (a, t); those equal to t add t - x = 0.  The
    difference of Eq. (med_objOS) costs fixes the value for every k."""
    x = np.array([-2.0, 0.0, 0.0, 0.0, 1.0, 3.0, 3.0, 5.0, 8.0, 8.0], dtype=np.float64)
    n = x.size
    for k in range(1, n + 1):
        for a, t in [(0.0, 3.0), (-2.0, 8.0), (3.0, 5.0), (0.0, 8.0), (1.0, 3.0)]:
            want = (osel.pinball_cost(x, k, t) - osel.pinball_cost(x, k, a)) / n
            assert osel.relative_cost(x, k, a, t) == pytest.approx(want, rel=1e-12, abs=1e-12)
    # k = 5, (a, t) = (0, 3): slope #(x <= 0) - 5 + 1/2 = -1/2 over width 3, plus 3 - 1 = 2
    assert osel.relative_cost(x, 5, 0.0, 3.0) == -1.5 + 2.0


def test_relative_cost_ignores_far_outliers():
    x = np.array([1.0, 2.0, 3.0, 4.0, 1e30, -1e30], dtype=np.float64)
    # only 2 and 3 lie strictly inside (1.5, 3.5)
    want = (osel.counts(x, 1.5)[1] - 3 + 0.5) * 2.0 + (3.5 - 2.0) + (3.5 - 3.0)
    assert osel.relative_cost(x, 3, 1.5, 3.5) == want


def test_key_roundtrip_and_order():
    vals = np.array([-np.inf, -3.0, -1e-40, -0.0, 0.0, 1e-45, 2.0, np.inf], dtype=np.float32)
    keys = osel.total_order_key(vals)
    assert np.all(np.diff(keys.astype(np.int64)) > 0)
    assert _bits(osel.key_to_value(keys, np.float32)[3]) == 0x80000000
    assert np.array_equal(osel.key_to_value(keys, np.float32).view(np.uint32), vals.view(np.uint32))
    d = np.array([-np.inf, -1.0, -0.0, 0.0, 5e-324, np.inf])
    kd = osel.total_order_key(d)
    assert np.all(np.diff(kd.astype(object)) > 0)


@pytest.mark.parametrize("dist", synth.PAPER_DISTRIBUTIONS)
def test_kelley_model_matches_definition(dist):
    x = synth.paper_distribution(dist, 20000, seed=7)
    for k in (1, 200, 10000, 19800, 20000):
        got, info = osel.kelley_select(x, k, cap=500)
        assert _bits(got) == _bits(osel.select_kth(x, k))
        assert info["passes"] <= 40


def test_kelley_model_ties_infinities_zeros():
    x = synth.heavy_mixture("mixture", 30000, seed=8)
    for k in (1, 5, 6, 300, 15000, 29700, 29995, 29996, 30000):
        got, _ = osel.kelley_select(x, k, cap=200)
        assert _bits(got) == _bits(osel.select_kth(x, k))
    z = np.array([0.0, -0.0] * 50 + [1.0, -1.0] * 10, dtype=np.float32)
    for k in range(1, z.size + 1, 7):
        assert _bits(osel.kelley_select(z, k, cap=4)[0]) == _bits(osel.select_kth(z, k))


def test_kelley_model_exhaustive_small_alphabet():
    """Every array of length <= 4 over {-inf, -1, -0, +0, 2, +inf} and every rank: the
    hybrid selection returns the rank definition's element, sign of zero included
    (the early exits at the extremes and at +-inf reach every branch here)."""
    alph = [-np.inf, -1.0, -0.0, 0.0, 2.0, np.inf]
    for n in range(1, 5):
        for tup in itertools.product(alph, repeat=n):
            x = np.array(tup, dtype=np.float32)
            for k in range(1, n + 1):
                got, _ = osel.kelley_select(x, k, cap=1)
                assert _bits(got) == _bits(_rank_brute(x, k)), (tup, k)


def test_kelley_model_integer_ties_every_rank():
    """Small integer arrays with heavy ties, every rank: the result is the rank
    definition's element, and after every step the bracket (y_L, y_R] rebuilt from the
    iterates by the rule of step 1.4 holds exactly the recorded number of elements.
    Iterates that land on a run of equal values below x_(k) occur in this set."""
    rng = np.random.default_rng(17)
    tied_low = 0
    for _ in range(300):
        n = int(rng.integers(5, 40))
        x = rng.integers(0, 6, n).astype(np.float64)
        for k in range(1, n + 1):
            got, info = osel.kelley_select(x, k, cap=1)
            assert got == _rank_brute(x, k), (x.tolist(), k)
            lo, hi = x.min(), x.max()   # step 0: the extremes
            for t, pop in zip(info["iterates"], info["pops"]):
                below, upto = np.count_nonzero(x < t), np.count_nonzero(x <= t)
                if below < k <= upto:
                    break
                if upto < k:
                    lo = t
                    tied_low += below < upto
                else:
                    hi = t
                assert pop == np.count_nonzero((x > lo) & (x <= hi)), (x.tolist(), k)
    assert tied_low > 0


def test_kelley_model_permutation_invariant():
    """Sec. 4 (Discussion): the cost is invariant under permutations of x."""
    x = synth.paper_distribution("mix4", 5000, seed=9)
    base = osel.kelley_select(x, 2500, cap=50)
    for perm in (np.sort(x), np.sort(x)[::-1].copy(), np.random.default_rng(1).permutation(x)):
        got = osel.kelley_select(perm, 2500, cap=50)
        assert _bits(got[0]) == _bits(base[0])
        assert got[1]["passes"] == base[1]["passes"]


def test_kelley_model_outlier_insensitive():
    """Sec. 4 (Discussion): the cutting plane is not slowed by a few huge values,
    unlike bisection on the data's range."""
    x = synth.paper_distribution("normal", 50000, seed=10).astype(np.float64)
    base = osel.kelley_select(x, 25000, cap=100)[1]["passes"]
    for big in (1e9, 1e20, 3e38):
        y = x.copy()
        y[:3] = big
        val, info = osel.kelley_select(y, 25000, cap=100)
        assert val == osel.select_kth(y, 25000)
        assert info["passes"] <= base + 3


def test_order_statistics_commute_with_monotone_transforms():
    """Sec. 4 (Discussion): order statistics are invariant under monotone transforms,
    x_(k) of F(x) = F(x_(k)) for increasing F; a decreasing F maps the rank k to
    n - k + 1 (so a reversed rank convention fails here)."""
    x = synth.paper_distribution("mix3", 4001, seed=12).astype(np.float64)
    n = x.size
    incr = (np.exp, np.cbrt, lambda v: 3.0 * v - 7.0, np.arcsinh)
    decr = (lambda v: -v, lambda v: np.exp(-v))
    for k in (1, 2, 40, 2001, 3960, 4000, 4001):
        base = osel.select_kth(x, k)
        base_rev = osel.select_kth(x, n - k + 1)
        for F in incr:
            assert _bits(osel.select_kth(F(x), k)) == _bits(F(base))
            assert _bits(osel.kelley_select(F(x), k, cap=32)[0]) == _bits(F(base))
        for F in decr:
            assert _bits(osel.select_kth(F(x), k)) == _bits(F(base_rev))
            assert _bits(osel.kelley_select(F(x), k, cap=32)[0]) == _bits(F(base_rev))


@pytest.mark.parametrize("dist", synth.PAPER_DISTRIBUTIONS)
def test_kelley_model_bracket_shrinks_as_reported(dist):
    """Sec. 3 reports fewer than 30 iterations in its experiments and, at n = 2^25,
    fewer than 2^19 elements (1/64 of them) left in the bracket after 7 iterations.
    A soft pin (the paper's arrays differ): on the Sec. 4.1 distributions at n = 2^20,
    for the median and the 1 % rank, 7 iterates leave under n/64 elements and the
    model runs to a one-element bracket in under 30 passes."""
    n = 1 << 20
    x = synth.paper_distribution(dist, n, seed=3)
    for k in ((n + 1) // 2, n // 100):
        _, info = osel.kelley_select(x, k, cap=1, maxit=200)
        if info["how"] == "hit":
            assert info["passes"] < 30
            continue
        assert info["pops"][6] < n / 64, info["pops"][:8]
        assert info["passes"] < 30


def test_kelley_model_first_step_is_tangent_intersection():
    """Step 1.1: on the hand-worked n = 9 example the first iterate is the
    intersection of the tangents at x_(1) and x_(n)."""
    g = _golden("median_objective_n9.json")
    x = np.array(g["x"], dtype=np.float64)
    k = 5
    _, info = osel.kelley_select(x, k, cap=1)
    # tangents of Phi = F/n: slopes (#(x<=1) - k + 1/2) = -2.5, (#(x<9) - k + 1/2) = 3.5;
    # Phi(9) - Phi(1) = -2.5*8 + sum_{1<x<9}(9 - x) = -20 + 29 = 9, which is also
    # (F(9) - F(1))/n = (4.5*45 - 4.5*27)/9 with F = (n/2) f for odd n
    t_star = 1 + (3.5 * 8 - 9) / (3.5 + 2.5)
    assert info["iterates"][0] == pytest.approx(t_star)
