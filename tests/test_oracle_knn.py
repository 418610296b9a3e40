"""Pins of the kNN oracle (Sec. 5, last application) by brute force over neighbour sets,
closed forms and invariances.  CPU only."""
import itertools
import math

import numpy as np
import pytest

from oracle import knn as ok


def _d2_loop(X, q):
    """Squared distances by plain loops (independent of the oracle's einsum)."""
    return [sum((float(q[t]) - float(x[t])) ** 2 for t in range(len(q))) for x in X]


def _nearest_sets(d2, k):
    """Every k-subset that is a valid set of k nearest points (ties broken any way)."""
    n = len(d2)
    sets = []
    for S in itertools.combinations(range(n), k):
        inside = max(d2[i] for i in S)
        outside = min((d2[i] for i in range(n) if i not in S), default=math.inf)
        if inside <= outside:
            sets.append(S)
    return sets


def _w(d, kind, eps=1e-6):
    return 1.0 if kind == "uniform" else 1.0 / (d + eps)


def test_squared_distances_hand_worked():
    X = np.array([[0.0, 0.0], [3.0, 4.0], [1.0, 1.0]])
    assert ok.squared_distances(X, np.array([[0.0, 0.0]])).tolist() == [[0.0, 25.0, 2.0]]
    assert ok.squared_distances(X, np.array([[1.0, 1.0]])).tolist() == [[2.0, 13.0, 0.0]]


def test_indicator_is_inclusion_frequency_over_tie_breaks():
    """rho_i equals the fraction of valid k-nearest sets that contain point i, so the
    rho sum to exactly k (Eq. (med_reg) weights at the order statistic)."""
    rng = np.random.default_rng(40)
    for _ in range(200):
        n = int(rng.integers(1, 9))
        d2 = rng.integers(0, 4, n).astype(np.float64)      # heavy ties
        for k in range(1, n + 1):
            sets = _nearest_sets(list(d2), k)
            freq = np.array([sum(i in S for S in sets) / len(sets) for i in range(n)])
            rho = ok.indicator(d2, k)
            assert np.allclose(rho, freq, rtol=0, atol=1e-15), (d2, k)
            assert math.fsum(rho.tolist()) == pytest.approx(k, abs=1e-12)


@pytest.mark.parametrize("kind", ["uniform", "inverse"])
def test_regression_is_the_mean_over_tie_breaks(kind):
    """The prediction equals the plain kNN estimate sum_S w_i f_i / sum_S w_i averaged
    over every valid set S of k nearest points (tied points share one distance, so the
    denominator is the same for every S)."""
    rng = np.random.default_rng(41)
    for _ in range(60):
        n = int(rng.integers(2, 8))
        X = rng.integers(-2, 3, (n, 2)).astype(np.float64)   # lattice points: tied distances
        f = rng.normal(size=n)
        Q = rng.integers(-2, 3, (3, 2)).astype(np.float64)
        for k in range(1, n + 1):
            got = ok.regress(X, f, Q, k, kind)
            for j, q in enumerate(Q):
                d2 = _d2_loop(X, q)
                ests = []
                for S in _nearest_sets(d2, k):
                    ws = [_w(math.sqrt(d2[i]), kind) for i in S]
                    ests.append(sum(w * f[i] for w, i in zip(ws, S)) / sum(ws))
                assert got[j] == pytest.approx(sum(ests) / len(ests), rel=1e-12, abs=1e-12), (kind, k)


def test_votes_are_the_mean_over_tie_breaks():
    rng = np.random.default_rng(42)
    for _ in range(60):
        n = int(rng.integers(2, 8))
        X = rng.integers(-2, 3, (n, 2)).astype(np.float64)
        lab = rng.integers(0, 3, n)
        Q = rng.integers(-2, 3, (2, 2)).astype(np.float64)
        for k in range(1, n + 1):
            V = ok.votes(X, lab, Q, k, 3)
            for j, q in enumerate(Q):
                sets = _nearest_sets(_d2_loop(X, q), k)
                mean = np.array([sum(sum(lab[i] == c for i in S) for S in sets) / len(sets) for c in range(3)])
                assert np.allclose(V[j], mean, rtol=0, atol=1e-12)


def test_without_ties_matches_sorting():
    """Continuous data (no tied distances): the k nearest by a full sort of the
    distances, the textbook method the paper replaces."""
    rng = np.random.default_rng(43)
    X = rng.normal(size=(300, 5))
    f = rng.normal(size=300)
    lab = rng.integers(0, 4, 300)
    Q = rng.normal(size=(7, 5))
    for k in (1, 2, 17, 150, 300):
        for kind in ("uniform", "inverse"):
            got = ok.regress(X, f, Q, k, kind)
            for j, q in enumerate(Q):
                d = np.sqrt(np.array(_d2_loop(X, q)))
                idx = np.argsort(d)[:k]
                w = np.array([_w(d[i], kind) for i in idx])
                assert got[j] == pytest.approx(float(w @ f[idx] / w.sum()), rel=1e-12)
        cls = ok.classify(X, lab, Q, k, 4)
        for j, q in enumerate(Q):
            idx = np.argsort(np.array(_d2_loop(X, q)))[:k]
            counts = np.bincount(lab[idx], minlength=4)
            assert cls[j] == int(np.argmax(counts))


def test_closed_forms_k_one_and_k_all():
    rng = np.random.default_rng(44)
    X = rng.normal(size=(50, 3))
    f = rng.normal(size=50)
    Q = rng.normal(size=(5, 3))
    # k = n with uniform weights: the mean of every ordinate
    assert np.allclose(ok.regress(X, f, Q, 50), math.fsum(f.tolist()) / 50, rtol=1e-14, atol=0)
    # k = 1: the ordinate of the nearest point, whatever the weight
    for kind in ("uniform", "inverse"):
        got = ok.regress(X, f, Q, 1, kind)
        for j, q in enumerate(Q):
            d2 = _d2_loop(X, q)
            assert got[j] == f[int(np.argmin(d2))]
    # a query on a training point with k = 1 returns that point's ordinate
    assert ok.regress(X, f, X[7:8], 1, "inverse")[0] == f[7]


def test_rigid_motion_and_row_permutation_invariance():
    """Distances, hence predictions, do not change under a rotation plus translation of
    every point, nor under a permutation of the training rows."""
    rng = np.random.default_rng(45)
    X = rng.normal(size=(200, 4))
    f = rng.normal(size=200)
    lab = rng.integers(0, 3, 200)
    Q = rng.normal(size=(6, 4))
    R, _ = np.linalg.qr(rng.normal(size=(4, 4)))
    t = rng.normal(size=4)
    for k in (1, 9, 100):
        base = ok.regress(X, f, Q, k, "inverse")
        moved = ok.regress(X @ R.T + t, f, Q @ R.T + t, k, "inverse")
        assert np.allclose(moved, base, rtol=1e-9, atol=1e-12)
        perm = rng.permutation(200)
        assert np.array_equal(ok.regress(X[perm], f[perm], Q, k, "inverse"), base)
        assert np.array_equal(ok.classify(X[perm], lab[perm], Q, k, 3), ok.classify(X, lab, Q, k, 3))


def test_class_ties_go_to_the_smallest_label():
    X = np.array([[1.0], [-1.0], [2.0], [-2.0]])
    lab = np.array([2, 1, 0, 0])
    # k = 2 around 0: one vote each for classes 1 and 2 -> class 1
    assert ok.classify(X, lab, np.array([[0.0]]), 2, 3).tolist() == [1]
    # k = 4: class 0 has two votes
    assert ok.classify(X, lab, np.array([[0.0]]), 4, 3).tolist() == [0]


def test_knn_problem_recipe():
    """The seeded kNN inputs: shapes, dtypes, determinism, and lattice coordinates that
    are integers (so float32 squared distances are exact for |coordinates| < 2^11)."""
    import synth
    X, Q, f, lab = synth.knn_problem(1000, 8, 16, 5, seed=3)
    assert X.shape == (1000, 8) and Q.shape == (16, 8) and f.shape == (1000,) and lab.shape == (1000,)
    assert X.dtype == Q.dtype == f.dtype == np.float32 and lab.dtype == np.int32
    assert set(np.unique(lab)) <= set(range(5))
    X2, Q2, f2, lab2 = synth.knn_problem(1000, 8, 16, 5, seed=3)
    assert np.array_equal(X, X2) and np.array_equal(Q, Q2) and np.array_equal(f, f2) and np.array_equal(lab, lab2)
    XL, QL, _, _ = synth.knn_problem(1000, 8, 16, 5, seed=3, lattice=True)
    assert np.array_equal(XL, np.rint(XL)) and np.array_equal(QL, np.rint(QL))
    assert np.abs(XL).max() < 2 ** 11
    d32 = ((QL[0][None, :] - XL) ** 2).sum(axis=1, dtype=np.float32)
    assert np.array_equal(d32.astype(np.float64), ok.squared_distances(XL, QL[:1])[0])


def test_vote_totals_are_exact_fractions():
    """Three points below d_(k) and three tied at d_(k) with k = 4: each tied point counts
    1/3, so class 1 (one below, three tied) and class 0 (two below) both score exactly 2,
    and the tie goes to class 0."""
    from fractions import Fraction
    X = np.array([[1.0], [-1.0], [-1.0], [2.0], [-2.0], [2.0]])
    lab = np.array([1, 0, 0, 1, 1, 1])
    Q = np.array([[0.0]])
    assert ok.exact_votes(X, lab, Q, 4, 2) == [[Fraction(2), Fraction(2)]]
    assert ok.classify(X, lab, Q, 4, 2).tolist() == [0]
    assert ok.exact_votes(X, lab, Q, 5, 2) == [[Fraction(2), Fraction(1) + 3 * Fraction(2, 3)]]
    assert ok.classify(X, lab, Q, 5, 2).tolist() == [1]


def test_float32_distances_follow_their_stated_order():
    """squared_distances_f32: every entry equals a scalar float32 loop of the stated
    definition (diff = q_t - x_t, acc = acc + diff * diff, t = 0..p-1, no fused
    multiply-add); it lies within (p + 2) * 2^-24 of the float64 distance; on integer
    lattice data it is exact."""
    rng = np.random.default_rng(46)
    X = (rng.normal(size=(40, 6)) * 3).astype(np.float32)
    Q = (rng.normal(size=(5, 6)) * 3).astype(np.float32)
    D32 = ok.squared_distances_f32(X, Q)
    assert D32.dtype == np.float32
    for j in range(5):
        for i in range(40):
            acc = np.float32(0.0)
            for t in range(6):
                d = np.float32(Q[j, t]) - np.float32(X[i, t])
                acc = np.float32(acc + np.float32(d * d))
            assert D32[j, i] == acc
    D64 = ok.squared_distances(X, Q)
    assert np.all(np.abs(D32.astype(np.float64) - D64) <= (6 + 2) * 2.0 ** -24 * D64 + 1e-30)
    import synth
    XL, QL, _, _ = synth.knn_problem(500, 8, 4, 3, seed=9, lattice=True)
    assert np.array_equal(ok.squared_distances_f32(XL, QL).astype(np.float64), ok.squared_distances(XL, QL))


def test_from_distances_entry_points_agree():
    rng = np.random.default_rng(47)
    X = rng.integers(-3, 4, (60, 3)).astype(np.float64)
    f = rng.normal(size=60)
    lab = rng.integers(0, 4, 60)
    Q = rng.integers(-3, 4, (4, 3)).astype(np.float64)
    D2 = ok.squared_distances(X, Q)
    for k in (1, 7, 30, 60):
        assert np.array_equal(ok.regress_d2(D2, f, k, "inverse"), ok.regress(X, f, Q, k, "inverse"))
        assert ok.exact_votes_d2(D2, lab, k, 4) == ok.exact_votes(X, lab, Q, k, 4)
        assert np.array_equal(ok.classify_d2(D2, lab, k, 4), ok.classify(X, lab, Q, k, 4))
