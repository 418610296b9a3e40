"""GPU parity of kNN regression and classification through d_(k) (Sec. 5, last
application) against the float64 oracle.

Which points are the k nearest is decided on float32 squared distances formed in the
order oracle.knn.squared_distances_f32 states, so d_(k)^2, the tie shares, the class
votes (exact rationals, compared after their single rounding) and the predicted classes
must equal the oracle's bit for bit.  The regression is a ratio of float64 sums of the
same terms in another order: it must lie within the rounding bound of those sums,
2 (K + 8) 2^-53 (sum rho w |f| + |pred| sum rho w) / sum rho w + 4 * 2^-53 |pred| over the
K points with a non-zero indicator, computed here from the oracle's own terms."""
import math

import numpy as np
import pytest
import torch

import synth
from oracle import knn as oknn
from oracle import select as osel

pytestmark = pytest.mark.gpu

U53 = 2.0 ** -53


@pytest.fixture(scope="module")
def ctx(lib):
    c = lib.Context()
    yield c
    c.close()


def bits32(v):
    return np.asarray(v, dtype=np.float32).view(np.uint32)


def bits64(v):
    return np.asarray(v, dtype=np.float64).view(np.uint64)


def oracle_rows(D2, k):
    """Per query: d_(k)^2 and the indicator rho (float64) from the oracle."""
    kth = np.array([osel.select_kth(D2[j].astype(np.float32), k) for j in range(D2.shape[0])], dtype=np.float32)
    rho = np.stack([oknn.indicator(D2[j], k) for j in range(D2.shape[0])])
    return kth, rho


def regress_bound(D2, rho, f, pred, kind, eps):
    w = oknn.weight(np.sqrt(D2), kind, eps)
    rw = rho * w
    K = np.count_nonzero(rho, axis=1)
    num_abs = (rw * np.abs(f.astype(np.float64))[None, :]).sum(axis=1)
    den = rw.sum(axis=1)
    return 2 * (K + 8) * U53 * (num_abs + np.abs(pred) * den) / den + 4 * U53 * np.abs(pred)


def run_case(ctx, X, Q, f, labels, C, k, kinds=("uniform", "inverse"), eps=1e-6):
    Xt, Qt = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    D2 = oknn.squared_distances_f32(X, Q).astype(np.float64)
    kth64, rho = oracle_rows(D2, k)
    for kind in kinds:
        pred, kth = ctx.knn_regress(Xt, torch.from_numpy(f).cuda(), Qt, k, weight=kind, eps=eps)
        st = ctx.last_stats()
        assert st["status"] == 0
        assert np.array_equal(bits32(kth.cpu().numpy()), bits32(kth64)), kind
        want = oknn.regress_d2(D2, f, k, kind, eps)
        got = pred.cpu().numpy()
        tol = regress_bound(D2, rho, f, want, kind, eps)
        err = np.abs(got - want)
        j = int(np.argmax(err / tol))
        assert np.all(err <= tol), (kind, j, got[j], want[j], tol[j])
    cls, votes, kth = ctx.knn_classify(Xt, torch.from_numpy(labels).cuda(), C, Qt, k)
    assert ctx.last_stats()["status"] == 0
    assert np.array_equal(bits32(kth.cpu().numpy()), bits32(kth64))
    exact = oknn.exact_votes_d2(D2, labels, k, C)
    want_votes = np.array([[float(v) for v in row] for row in exact])
    assert np.array_equal(bits64(votes.cpu().numpy()), bits64(want_votes))
    assert np.array_equal(cls.cpu().numpy(), oknn.classify_d2(D2, labels, k, C))


@pytest.mark.parametrize("start", [0, 1])
@pytest.mark.parametrize("p,k", [(8, 1), (8, 17), (3, 500), (13, 35000), (32, 70001)])
def test_knn_matches_oracle_gaussian(ctx, start, p, k):
    """Gaussian clusters, n = 70001 (the sampled start applies from 65536 rows; the row
    count is ragged against tiles and chunks), 37 queries; both routes."""
    X, Q, f, labels = synth.knn_problem(70001, p, 37, 7, seed=300 + p)
    k = min(k, X.shape[0])
    ctx.set_config(knn_start=start)
    try:
        run_case(ctx, X, Q, f, labels, 7, k)
    finally:
        ctx.set_config(knn_start=0)


@pytest.mark.parametrize("start", [0, 1])
@pytest.mark.parametrize("k", [1, 64, 3000])
def test_knn_matches_oracle_on_lattice_ties(ctx, start, k):
    """Integer coordinates: exact distances with long runs of ties, so d_(k) is shared by
    many points and the tie shares a/b of Eq. (med_reg) decide the votes."""
    X, Q, f, labels = synth.knn_problem(80000, 4, 29, 5, seed=310 + k, lattice=True)
    ctx.set_config(knn_start=start)
    try:
        run_case(ctx, X, Q, f, labels, 5, k)
    finally:
        ctx.set_config(knn_start=0)


def test_knn_many_queries_ragged_blocks(ctx):
    """1037 queries (more than one query block of the pass, ragged), p = 5."""
    X, Q, f, labels = synth.knn_problem(66000, 5, 1037, 11, seed=320)
    run_case(ctx, X, Q, f, labels, 11, 100, kinds=("inverse",))


@pytest.mark.parametrize("n,p,m,k", [(1, 1, 1, 1), (5, 2, 3, 5), (1000, 7, 19, 999), (4099, 16, 64, 50)])
def test_knn_small_problems(ctx, n, p, m, k):
    """Below 65536 rows every query takes the plain form."""
    X, Q, f, labels = synth.knn_problem(n, p, m, 3, seed=330 + n, lattice=(n == 5))
    run_case(ctx, X, Q, f, labels, 3, k)


def test_knn_all_points_equal(ctx):
    """Every distance of a query ties: the k nearest are k/n of each point."""
    n, p, m = 70000, 4, 9
    X = np.full((n, p), 1.5, dtype=np.float32)
    rng = np.random.default_rng(340)
    Q = rng.normal(size=(m, p)).astype(np.float32)
    f = rng.normal(size=n).astype(np.float32)
    labels = rng.integers(0, 4, n).astype(np.int32)
    for start in (0, 1):
        ctx.set_config(knn_start=start)
        try:
            run_case(ctx, X, Q, f, labels, 4, 1234)
        finally:
            ctx.set_config(knn_start=0)


def test_knn_bench_size_sampled_queries(ctx):
    """The benchmark problem (n = 2^20, p = 8, 4096 queries, k = 256, 16 classes) in the
    benchmark's launch; 24 queries checked against the oracle one by one."""
    n, p, m, k, C = 1 << 20, 8, 4096, 256, 16
    X, Q, f, labels = synth.knn_problem(n, p, m, C, seed=350)
    Xt, Qt, ft, lt = (torch.from_numpy(a).cuda() for a in (X, Q, f, labels))
    pred, kth = ctx.knn_regress(Xt, ft, Qt, k, weight="inverse")
    cls, votes, kth2 = ctx.knn_classify(Xt, lt, C, Qt, k)
    assert ctx.last_stats()["status"] == 0
    pick = np.random.default_rng(351).choice(m, 24, replace=False)
    D2 = oknn.squared_distances_f32(X, Q[pick]).astype(np.float64)
    kth64, rho = oracle_rows(D2, k)
    assert np.array_equal(bits32(kth.cpu().numpy()[pick]), bits32(kth64))
    assert np.array_equal(bits32(kth2.cpu().numpy()[pick]), bits32(kth64))
    want = oknn.regress_d2(D2, f, k, "inverse", 1e-6)
    tol = regress_bound(D2, rho, f, want, "inverse", 1e-6)
    assert np.all(np.abs(pred.cpu().numpy()[pick] - want) <= tol)
    exact = oknn.exact_votes_d2(D2, labels, k, C)
    want_votes = np.array([[float(v) for v in row] for row in exact])
    assert np.array_equal(bits64(votes.cpu().numpy()[pick]), bits64(want_votes))
    assert np.array_equal(cls.cpu().numpy()[pick], oknn.classify_d2(D2, labels, k, C))
    # every query: exactly k points count (sum of its votes) and the class has the top vote
    v = votes.cpu().numpy()
    assert np.allclose(v.sum(axis=1), k, rtol=1e-12, atol=0)
    assert np.all(v[np.arange(m), cls.cpu().numpy()] == v.max(axis=1))


def test_knn_rejects_non_finite_and_bad_labels(ctx, lib):
    X, Q, f, labels = synth.knn_problem(70000, 4, 8, 3, seed=360)
    Xb = X.copy()
    Xb[123, 2] = np.nan
    pred, kth = ctx.knn_regress(torch.from_numpy(Xb).cuda(), torch.from_numpy(f).cuda(), torch.from_numpy(Q).cuda(), 10)
    assert ctx.last_stats(raise_on_error=False)["status"] == lib.GBS_ENAN
    assert np.all(np.isnan(pred.cpu().numpy())) and np.all(np.isnan(kth.cpu().numpy()))
    Qb = Q.copy()
    Qb[3, 0] = np.inf
    cls, votes, _ = ctx.knn_classify(torch.from_numpy(X).cuda(), torch.from_numpy(labels).cuda(), 3,
                                     torch.from_numpy(Qb).cuda(), 10)
    assert ctx.last_stats(raise_on_error=False)["status"] == lib.GBS_ENAN
    assert np.all(cls.cpu().numpy() == -1)
    bad = labels.copy()
    bad[77] = 3
    ctx.knn_classify(torch.from_numpy(X).cuda(), torch.from_numpy(bad).cuda(), 3, torch.from_numpy(Q).cuda(), 10)
    assert ctx.last_stats(raise_on_error=False)["status"] == lib.GBS_EINVAL
    # the context stays usable
    run_case(ctx, X[:5000], Q, f[:5000], labels[:5000], 3, 10, kinds=("uniform",))
