"""Pins of the LMS / LTS oracle (Sec. 5) by brute force and special cases. CPU only."""
import itertools
import math

import numpy as np
import pytest

from oracle import regression as oreg
from oracle import select as osel
import synth


def test_lts_is_min_over_h_subsets_brute_force():
    """The LTS objective is the smallest sum of squares over all h-subsets of the
    residuals (Sec. 5: the model is fitted to the retained h observations); that
    minimum is the sum of the h smallest."""
    rng = np.random.default_rng(11)
    for n in range(1, 9):
        s = np.round(rng.standard_normal(n) * 3, 1) ** 2
        for h in range(1, n + 1):
            brute = min(math.fsum(s[list(c)]) for c in itertools.combinations(range(n), h))
            assert oreg.lts(s, h) == pytest.approx(brute, rel=1e-15, abs=0)
            assert oreg.lts_rho_form(s, h) == pytest.approx(brute, rel=1e-15, abs=0)


def test_rho_form_with_ties():
    """Eq. (med_reg): with a run of values equal to q the weights a/b split it."""
    s = np.array([4.0, 1.0, 4.0, 4.0, 9.0, 0.0, 4.0])
    for h in range(1, s.size + 1):
        assert oreg.lts_rho_form(s, h) == math.fsum(sorted(s)[:h])


def test_lms_brute_force_rank():
    rng = np.random.default_rng(12)
    for n in range(1, 10):
        r = rng.standard_normal(n)
        s = r * r
        k = (n + 1) // 2
        # rank definition: #(s < v) < k <= #(s <= v)
        v = oreg.lms(s, k)
        assert np.count_nonzero(s < v) < k <= np.count_nonzero(s <= v)
        # LMS = Med(|r|)^2 (reading of "Med(r_i)^2")
        assert v == pytest.approx(float(osel.median(np.abs(r))) ** 2, rel=0, abs=0)


def test_p1_theta0_is_median_of_y_squared():
    y = synth.uniform(999, seed=13).astype(np.float64) - 0.5
    X = np.ones((999, 1))
    lms, lts = oreg.lms_lts(X, y, np.zeros((1, 1)), k=500, h=500)
    assert lms[0] == osel.select_kth(y * y, 500)
    assert lts[0] == pytest.approx(math.fsum(np.sort(y * y)[:500]), rel=1e-15)


def test_exact_fit_candidate_has_zero_residuals_on_its_subset():
    X, y, _ = synth.regression(200, 3, seed=14)
    th = synth.elemental_thetas(X, y, 4, seed=15)
    r = oreg.residuals(X, y, th)
    # each candidate fits at least p observations to float32 rounding
    for c in range(4):
        assert np.count_nonzero(np.abs(r[:, c]) < 1e-3) >= 3


def test_residual_sign_and_shape():
    X = np.array([[1.0, 2.0], [3.0, 4.0]], dtype=np.float32)
    y = np.array([5.0, 6.0], dtype=np.float32)
    th = np.array([[1.0, 0.0], [1.0, 1.0]], dtype=np.float32)
    r = oreg.residuals(X, y, th)
    assert r.tolist() == [[2.0, 3.0], [-1.0, 2.0]]


def test_extreme_ranks_and_row_permutation():
    """LTS with h = n is the full sum of squares and with h = 1 the smallest square; LMS at
    k = 1 and k = n are the smallest and largest squares; both objectives are invariant
    under a permutation of the rows (Sec. 5: they depend on the residuals' multiset)."""
    X, y, _ = synth.regression(301, 4, seed=16)
    th = synth.elemental_thetas(X, y, 3, seed=17)
    r = oreg.residuals(X, y, th)
    s = r * r
    n = s.shape[0]
    for c in range(3):
        sc = s[:, c]
        assert oreg.lts(sc, n) == pytest.approx(math.fsum(sc.tolist()), rel=1e-15)
        assert oreg.lts(sc, 1) == sc.min()
        assert oreg.lms(sc, 1) == sc.min() and oreg.lms(sc, n) == sc.max()
    perm = np.random.default_rng(18).permutation(n)
    a = oreg.lms_lts(X, y, th, k=151, h=153)
    b = oreg.lms_lts(X[perm], y[perm], th, k=151, h=153)
    assert np.array_equal(a[0], b[0])
    assert np.allclose(a[1], b[1], rtol=1e-15, atol=0)


# ---------------------------------------------------------------------------------
# The estimator search: rho weights, C-steps, LMS / LTS search (Sec. 5).
# ---------------------------------------------------------------------------------
from fractions import Fraction


def test_rho_weights_sum_to_h_and_give_the_lts_objective():
    """The Eq. (med_reg) weights total exactly h (a/b of the tied values counted as an
    exact rational) and weight the squares to the sum of the h smallest, ties included."""
    rng = np.random.default_rng(40)
    for n in (1, 2, 7, 30):
        s = np.round(rng.standard_normal(n), 1) ** 2       # many ties
        for h in range(1, n + 1):
            rho = oreg.rho_weights(s, h)
            q = osel.select_kth(s, h)
            b = int(np.count_nonzero(s == q))
            total = int(np.count_nonzero(s < q)) + Fraction(h - int(np.count_nonzero(s < q)), b) * b
            assert total == h
            a = h - int(np.count_nonzero(s < q))
            assert np.all(rho[s < q] == 1.0) and np.all(rho[s > q] == 0.0) and np.all(rho[s == q] == a / b)
            assert math.fsum((rho * s).tolist()) == pytest.approx(math.fsum(np.sort(s)[:h].tolist()), rel=1e-14)


def test_float32_residuals_follow_their_stated_order():
    """The retained rows are decided on float32 squares formed term by term (no fused
    multiply-add): a scalar loop of that definition gives the same bits, and the squares
    lie within the float32 rounding bound of the float64 residuals."""
    X, y, _ = synth.regression(300, 5, seed=41)
    th = synth.elemental_thetas(X, y, 1, seed=42)[:, 0]
    s = oreg.squared_residuals_f32(X, y, th)
    for i in range(0, 300, 37):
        acc = np.float32(0.0)
        for j in range(5):
            acc = np.float32(acc + np.float32(X[i, j] * th[j]))
        r = np.float32(y[i] - acc)
        assert np.float32(r * r).view(np.uint32) == s[i].view(np.uint32)
    r64 = oreg.residuals(X, y, th)[:, 0]
    bound = 2 * np.abs(r64) * 7 * 2.0 ** -24 * (np.abs(y) + np.abs(X.astype(np.float64)) @ np.abs(th.astype(np.float64))) \
        + 2.0 ** -23 * r64 ** 2 + 1e-30
    assert np.all(np.abs(s - r64 ** 2) <= 2 * bound)


def test_c_step_with_all_rows_retained_is_ordinary_least_squares():
    """h = n gives every row the weight 1: one C-step is the least-squares fit of all the
    data (numpy.linalg.lstsq), rounded to float32."""
    X, y, _ = synth.regression(500, 4, seed=43, contamination=0.0)
    th0 = np.zeros(4, dtype=np.float32)
    got = oreg.c_step(X, y, th0, h=500)
    want = np.linalg.lstsq(X.astype(np.float64), y.astype(np.float64), rcond=None)[0]
    assert np.allclose(got, want.astype(np.float32), rtol=2e-6, atol=1e-7)


def _clean_plus_outliers(n, p, n_good, seed):
    """y = X beta exactly (float32, zero residual up to rounding) on the first n_good
    rows; the rest are far outliers."""
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, p)).astype(np.float32)
    beta = rng.integers(-3, 4, p).astype(np.float32)       # small integers: X beta exact in float32
    X[:n_good] = np.round(X[:n_good] * 8) / 8
    y = (X.astype(np.float64) @ beta.astype(np.float64)).astype(np.float32)
    y[n_good:] += rng.uniform(50.0, 100.0, n - n_good).astype(np.float32)
    return X, y, beta


def test_c_step_fixed_point_and_recovery_of_the_clean_model():
    """With 70% of the rows fitted exactly by beta and h no larger than them, beta is a
    fixed point of the C-step (its h smallest squares are zeros), its LTS objective is 0,
    and C-steps from a perturbed start recover it."""
    X, y, beta = _clean_plus_outliers(400, 3, 280, seed=44)
    h = 210
    assert np.array_equal(oreg.c_step(X, y, beta, h), beta)
    assert oreg.lts_objective_f32(X, y, beta, h) == 0.0
    start = beta + np.float32(0.05) * np.array([1.0, -1.0, 0.5], dtype=np.float32)
    th, F, kept = oreg.c_steps(X, y, start, h, max_steps=30)
    assert kept >= 1 and F == 0.0 and np.array_equal(th, beta)
    # from the fixed point no refit lowers the objective: none is kept
    th, F, kept = oreg.c_steps(X, y, beta, h, max_steps=30)
    assert kept == 0 and F == 0.0 and np.array_equal(th, beta)


def test_c_steps_never_increase_the_objective():
    """The C-step's objective cannot increase (the h smallest squares at the refit sum to
    at most its rho-weighted fit); checked step by step on contaminated data from
    elemental starts."""
    X, y, _ = synth.regression(2000, 4, seed=45)
    ths = synth.elemental_thetas(X, y, 6, seed=46).T
    h = (2000 + 4 + 1) // 2
    for th in ths:
        F = oreg.lts_objective_f32(X, y, th, h)
        for _ in range(6):
            th = oreg.c_step(X, y, th, h)
            Fn = oreg.lts_objective_f32(X, y, th, h)
            assert Fn <= F * (1 + 1e-12)
            F = Fn


def test_lts_brute_force_optimum_is_a_c_step_fixed_point():
    """Tiny problems, all h-subsets: the LTS minimum is the least-squares fit of the best
    h-subset; that fit is a fixed point of the C-step, and the search from every elemental
    start reaches no lower objective than it."""
    rng = np.random.default_rng(47)
    for trial in range(6):
        n, p, h = 9, 2, 6
        X = np.round(rng.standard_normal((n, p)) * 4).astype(np.float32) / 4
        y = np.round(rng.standard_normal(n) * 4).astype(np.float32) / 4
        y[:3] += 20
        best = None
        for sub in itertools.combinations(range(n), h):
            idx = list(sub)
            th = np.linalg.lstsq(X[idx].astype(np.float64), y[idx].astype(np.float64), rcond=None)[0]
            th32 = th.astype(np.float32)
            F = oreg.lts_objective_f32(X, y, th32, h)
            if best is None or F < best[1]:
                best = (th32, F)
        th_fix = oreg.c_step(X, y, best[0], h)
        assert np.allclose(th_fix, best[0], rtol=1e-5, atol=1e-6)
        starts = np.array([np.linalg.solve(X[[i, j]].astype(np.float64), y[[i, j]].astype(np.float64))
                           for i, j in itertools.combinations(range(n), 2)
                           if abs(np.linalg.det(X[[i, j]].astype(np.float64))) > 1e-9], dtype=np.float32)
        _, F_search, _ = oreg.lts_search(X, y, starts, h, n_refine=len(starts), max_steps=20)
        assert F_search >= best[1] * (1 - 1e-6) - 1e-9


def test_lms_search_is_the_least_objective():
    X, y, _ = synth.regression(3001, 3, seed=48)
    ths = synth.elemental_thetas(X, y, 40, seed=49).T
    k = 1501
    c, v = oreg.lms_search(X, y, ths, k)
    vals = [osel.select_kth(oreg.residuals(X, y, t)[:, 0] ** 2, k) for t in ths]
    assert v == min(vals) and c == vals.index(min(vals))
