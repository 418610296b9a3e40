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
