"""GPU parity of the single-array selection path against the CPU oracle.

Every selection must be bit-identical to oracle.select.select_kth (the plain
definition x_(k), Sec. 1).  Counts of the fused pass are exact integers; the float
cost partials are compared within the bound stated in each test.  Calls go through
the C-ABI (ctypes binding).
"""
import math

import numpy as np
import pytest
import torch

import synth
from oracle import select as osel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(lib):
    c = lib.Context()
    yield c
    c.close()


def bits(v):
    v = np.asarray(v)
    return v.view(np.uint32 if v.dtype == np.float32 else np.uint64).item()


def gpu_select(ctx, x_np, k, offset=0):
    """Select on a device copy of x_np placed `offset` elements into its buffer."""
    buf = torch.empty(x_np.size + offset, dtype=torch.from_numpy(x_np[:0]).dtype, device="cuda")
    x = buf[offset:]
    x.copy_(torch.from_numpy(x_np))
    r = ctx.select_kth(x, k)
    st = ctx.last_stats()
    return r.cpu().numpy()[0], st


def check(ctx, x_np, ks, offset=0):
    for k in ks:
        got, st = gpu_select(ctx, x_np, k, offset)
        want = osel.select_kth(x_np, k)
        assert bits(got) == bits(want), (x_np.dtype, x_np.size, k, got, want, st["how"], st["passes"])


def ranks(n):
    ks = {1, 2, max(1, n // 100), (n + 1) // 2, max(1, (99 * n) // 100), max(1, n - 1), n}
    return sorted(k for k in ks if 1 <= k <= n)


# ----------------------------------------------------------------------------- pass 0
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_array_stats_parity(ctx, dtype):
    x = synth.heavy_mixture("mixture", 100003, seed=31, dtype=dtype)
    x[:3] = 0.0
    x[3:5] = -0.0
    st = ctx.array_stats(torch.from_numpy(x).cuda())
    fin = x[np.isfinite(x)]
    assert st["n"] == x.size
    assert st["n_nan"] == 0
    assert st["n_neginf"] == np.count_nonzero(x == -np.inf)
    assert st["n_posinf"] == np.count_nonzero(x == np.inf)
    assert st["n_negzero"] == np.count_nonzero((x == 0) & np.signbit(x))
    assert st["n_finite"] == fin.size
    assert st["min"] == fin.min() and st["max"] == fin.max()
    assert st["c_le_min"] == np.count_nonzero(x <= fin.min())
    assert st["c_lt_max"] == np.count_nonzero(x < fin.max())
    # float32 partials per thread, float64 across: relative bound 1e-4 of sum |x|
    ref = math.fsum(fin.astype(np.float64).tolist())
    assert abs(st["sum"] - ref) <= 1e-4 * math.fsum(np.abs(fin.astype(np.float64)).tolist())


def test_array_stats_nan_count(ctx):
    x = synth.uniform(5000, seed=32)
    x[[7, 4000]] = np.nan
    st = ctx.array_stats(torch.from_numpy(x).cuda())
    assert st["n_nan"] == 2


# ----------------------------------------------------------------------------- one fused pass
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_cost_pass_parity(ctx, dtype):
    """Counts exact; S = sum_{a<x<t}(t - x) within the float32-accumulation bound
    (per-thread partials of at most ~1000 terms: relative 1e-4 of the sum of the
    terms), plus, for float64 input, the 2^-23 relative error of its float32 image."""
    rng = np.random.default_rng(33)
    x = synth.paper_distribution("mix4", 300007, seed=34, dtype=dtype)
    xt = torch.from_numpy(x).cuda()
    n = x.size
    for _ in range(12):
        a, t = np.sort(rng.uniform(-1, 102, 2))
        a, t = dtype(a), dtype(t)
        k = int(rng.integers(1, n + 1))
        e = ctx.cost_pass(xt, k, float(a), float(t))
        c_lt, c_le = osel.counts(x, t)
        assert e["c_lt_t"] == c_lt and e["c_le_t"] == c_le
        assert e["c_le_a"] == osel.counts(x, a)[1]
        inside = x[(x > a) & (x < t)].astype(np.float64)
        S = math.fsum((float(t) - inside).tolist())
        tol = 1e-4 * S + (2.0 ** -22 * math.fsum((abs(float(t)) + np.abs(inside)).tolist())
                          if dtype == np.float64 else 0.0) + 1e-30
        assert abs(e["S"] - S) <= tol
        assert abs(e["dphi"] - osel.relative_cost(x, k, a, t)) <= tol + 1e-9 * abs(e["dphi"])


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_cost_pass_zero_thresholds_follow_ieee(ctx, dtype):
    """Thresholds at -0 and +0 on data full of signed zeros: #(x < t), #(x <= t) and
    #(x <= a) are the IEEE counts (-0 == +0), whatever the sign of the zero threshold
    (float64 compares totalOrder keys, whose zero thresholds carry the IEEE rule)."""
    rng = np.random.default_rng(35)
    n = 100003
    vals = np.array([-0.0, 0.0, -1.5, 2.5, -np.inf, np.inf, 1e-300 if dtype == np.float64 else 1e-38,
                     -(1e-300 if dtype == np.float64 else 1e-38)], dtype=dtype)
    x = vals[rng.integers(0, vals.size, n)]
    xt = torch.from_numpy(x).cuda()
    for a, t in ((-1.0, -0.0), (-1.0, 0.0), (-0.0, 1.0), (0.0, 1.0), (-2.0, 3.0)):
        a, t = dtype(a), dtype(t)
        e = ctx.cost_pass(xt, 1, float(a), float(t))
        assert e["c_lt_t"] == int(np.count_nonzero(x < t)), (a, t)
        assert e["c_le_t"] == int(np.count_nonzero(x <= t)), (a, t)
        assert e["c_le_a"] == int(np.count_nonzero(x <= a)), (a, t)
    for k in (1, n // 3, n // 2, (2 * n) // 3, n):
        got = ctx.select_kth(xt, k).cpu().numpy()[0]
        assert np.asarray(got).view(np.uint64 if dtype == np.float64 else np.uint32) == \
            np.asarray(osel.select_kth(x, k)).view(np.uint64 if dtype == np.float64 else np.uint32)


def test_cost_pass_rejects_bad_bracket(ctx, lib):
    x = torch.zeros(10, device="cuda")
    with pytest.raises(lib.GbsError):
        ctx.cost_pass(x, 1, 1.0, 1.0)
    with pytest.raises(lib.GbsError):
        ctx.cost_pass(x, 11, 0.0, 1.0)


# ----------------------------------------------------------------------------- selection
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("dist", synth.PAPER_DISTRIBUTIONS)
def test_select_paper_distributions(ctx, dist, dtype):
    for n in (1000, 4099, 100003):
        check(ctx, synth.paper_distribution(dist, n, seed=35 + n, dtype=dtype), ranks(n))


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_select_small_sizes_every_rank(ctx, dtype):
    rng = np.random.default_rng(36)
    for n in (1, 2, 3, 4, 5, 7, 8, 9, 17, 33, 64):
        x = rng.integers(-4, 5, n).astype(dtype)
        check(ctx, x, range(1, n + 1))


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("offset", [1, 2, 3])
def test_select_unaligned_and_ragged(ctx, dtype, offset):
    x = synth.paper_distribution("normal", 2 ** 20 + 5, seed=37, dtype=dtype)
    check(ctx, x, ranks(x.size), offset=offset)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("family", synth.HEAVY_FAMILIES)
def test_select_heavy_tails_duplicates_infinities(ctx, family, dtype):
    x = synth.heavy_mixture(family, 2 ** 20 + 3, seed=38, dtype=dtype)
    n = x.size
    check(ctx, x, ranks(n) + [5, 6, n - 5, n - 4])


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_select_edge_cases(ctx, dtype):
    inf = np.inf
    cases = [
        np.full(1, 3.5), np.full(1000, 2.0), np.full(777, -inf), np.full(10, inf),
        np.array([inf, -inf] * 50), np.array([0.0, -0.0] * 500 + [1.0]),
        np.array([-0.0] * 300 + [0.0] * 200 + [-1.0, 1.0] * 10),
        np.concatenate([np.full(5000, 1.0), np.full(5000, 2.0)]),
        np.array([5e-324 if dtype == np.float64 else 1e-45] * 7 + [0.0] * 5 + [-0.0] * 3),
    ]
    for c in cases:
        x = c.astype(dtype)
        check(ctx, x, sorted(set(list(range(1, min(x.size, 12) + 1)) + ranks(x.size))))


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_select_monotone_transforms(ctx, dtype):
    """Sec. 4 (Discussion): order statistics commute with monotone transforms.  exp of the
    heavy-tailed mixture (long runs of +0 and +inf from under- and overflow), its cube and
    its reflection: the GPU's x_(k) of F(x) equals the oracle's bit for bit, and equals
    F(x_(k)) (x_(n-k+1) for the reflection)."""
    x = synth.heavy_mixture("mixture", 200003, seed=47, dtype=dtype)
    n = x.size
    with np.errstate(over="ignore", under="ignore"):
        images = [(np.exp(x), False), (x * x * x, False), (-x, True)]
    for Fx, reverse in images:
        Fx = np.ascontiguousarray(Fx.astype(dtype))
        for k in ranks(n):
            got, st = gpu_select(ctx, Fx, k)
            want = osel.select_kth(Fx, k)
            assert bits(got) == bits(want), (dtype, k, got, want, st["how"])
            # F(x_(k)) read from the same transformed array (an element equal to x_(k))
            base = osel.select_kth(x, n - k + 1 if reverse else k)
            assert got == Fx[np.flatnonzero(x == base)[0]], (dtype, k)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_select_huge_outliers_do_not_add_passes(ctx, dtype):
    """Sec. 4 (Discussion): a few values of 1e9 or more leave the cutting plane's pass
    count essentially unchanged."""
    x = synth.paper_distribution("normal", 2 ** 21, seed=39, dtype=dtype)
    k = (x.size + 1) // 2
    _, base = gpu_select(ctx, x, k)
    big = (1e9, 1e20, 3e38) if dtype == np.float32 else (1e9, 1e20, 1e300)
    for b in big:
        y = x.copy()
        y[:3] = b
        got, st = gpu_select(ctx, y, k)
        assert bits(got) == bits(osel.select_kth(y, k))
        assert st["passes"] <= base["passes"] + 3


@pytest.mark.parametrize("cap", [0, 64])
def test_select_f64_clustered_within_one_high_word(ctx, cap):
    """float64 passes decide on the keys' high 32 bits and take exact comparisons for the
    elements that share a threshold's high word: here most elements lie within 2^32 ulps
    of 1.0 and of -3.0 (so every iterate inside a cluster shares its high word with them),
    with ties, zeros and a few spread values; results bit-exact for every rank."""
    rng = np.random.default_rng(47)
    n = 400_003
    ulps = rng.integers(0, 1 << 31, n)
    x = np.where(rng.random(n) < 0.5, 1.0 + ulps * 2.0 ** -52, -3.0 - ulps * 2.0 ** -51)
    x[::97] = 1.0 + 12345 * 2.0 ** -52            # ties inside the cluster
    x[::1009] = 0.0
    x[::1013] = -0.0
    x[:50] = rng.standard_normal(50) * 1e3        # a few values outside the clusters
    ctx.set_config(cap=cap)
    try:
        check(ctx, x, (1, 77, n // 3, n // 2, (n + 1) // 2, 2 * n // 3, n - 5, n))
    finally:
        ctx.set_config(cap=0)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("cap", [64, 20000, 150000])
def test_compaction_and_finish_paths(ctx, dtype, cap):
    """The compacting pass after the first (keep only, the finish's first-round histogram
    formed as it keeps) and the finish's rounds: caps from 64 (a late compaction of a
    narrow bracket) to n/2 (a wide one whose finish takes a third round and reads the
    second-level copy), on data with heavy ties, runs of -0 and +0 (bracket ends at a
    zero take the exact key tests), infinities and a dense cluster; every rank exact."""
    rng = np.random.default_rng(48)
    n = 300_007
    x = rng.standard_normal(n)
    x[rng.choice(n, n // 10, replace=False)] = 0.0
    x[rng.choice(n, n // 10, replace=False)] = -0.0
    x[rng.choice(n, n // 20, replace=False)] = 0.75
    x[:9] = np.inf
    x[9:17] = -np.inf
    x[17:5017] = 1.0 + rng.integers(0, 4096, 5000) * 2.0 ** -20
    x = x.astype(dtype)
    ctx.set_config(cap=cap)
    try:
        ks = sorted({18, 1000, n // 3, int(np.count_nonzero(x < 0)) + 1, int(np.count_nonzero(x <= 0)),
                     (n + 1) // 2, int(np.count_nonzero(x < 0.75)) + 1, int(np.count_nonzero(x <= 0.75)),
                     2 * n // 3, n - 5000, n - 9})
        check(ctx, x, ks)
    finally:
        ctx.set_config(cap=0)


def test_select_nan_reports_enan(ctx, lib):
    x = torch.from_numpy(synth.uniform(1000, seed=40)).cuda()
    x[17] = float("nan")
    r = ctx.select_kth(x, 500)
    with pytest.raises(lib.GbsError) as ei:
        ctx.last_stats()
    assert ei.value.status == lib.GBS_ENAN
    assert torch.isnan(r).all()
    # the context stays usable
    y = torch.from_numpy(synth.uniform(1000, seed=40)).cuda()
    ctx.select_kth(y, 500)
    assert ctx.last_stats()["status"] == 0


def test_select_rejects_bad_rank(ctx, lib):
    x = torch.zeros(10, device="cuda")
    for k in (0, 11, -1):
        with pytest.raises(lib.GbsError):
            ctx.select_kth(x, k)


def test_permutation_invariance(ctx):
    """Sec. 4 (Discussion): same result for random, sorted and reverse-sorted x."""
    x = synth.paper_distribution("mix5", 500001, seed=41)
    k = 250001
    want = bits(osel.select_kth(x, k))
    for perm in (x, np.sort(x), np.sort(x)[::-1].copy()):
        got, _ = gpu_select(ctx, perm, k)
        assert bits(got) == want


def test_cap_and_maxit_variants_same_result(ctx):
    x = synth.heavy_mixture("lognormal", 300001, seed=42)
    ks = ranks(x.size)
    try:
        for cfg in ({"cap": 1}, {"cap": 10 ** 9}, {"cap": 100, "maxit": 2}, {"maxit": 1}, {"blocks_per_sm": 1}):
            ctx.set_config(**{**{"cap": 0, "maxit": 0, "blocks_per_sm": 0}, **cfg})
            check(ctx, x, ks)
    finally:
        ctx.set_config(cap=0, maxit=0, blocks_per_sm=0)


def test_pass_count_matches_cutting_plane_model(ctx):
    """Soft pin: with the same cap the GPU needs about as many passes as the float64
    model of Algorithm 1 (iterates differ only by float32 partial sums)."""
    n = 2 ** 20
    for dist in ("uniform", "normal", "mix1", "mix4"):
        x = synth.paper_distribution(dist, n, seed=43)
        k = (n + 1) // 2
        _, info = osel.kelley_select(x, k, cap=n // 16)
        ctx.set_config(cap=n // 16)
        try:
            got, st = gpu_select(ctx, x, k)
        finally:
            ctx.set_config(cap=0)
        assert bits(got) == bits(osel.select_kth(x, k))
        assert abs(st["passes"] - info["passes"]) <= 2, (dist, st["passes"], info["passes"])


def test_first_iterates_match_cutting_plane_model(ctx):
    """Pin of the iterate values (Algorithm 1, step 1.1): on continuous data (unique
    extremes) the GPU's first two tangent intersections equal the float64 model's within
    1e-5 of the starting bracket's width; they differ only by the rounding of float32
    partial sums (a swapped slope, a wrong sign or a dropped term moves them by a sizeable
    part of the bracket)."""
    n = 2 ** 20
    for dist in ("uniform", "normal"):
        x = synth.paper_distribution(dist, n, seed=44)
        k = (n + 1) // 2
        _, info = osel.kelley_select(x, k, cap=n // 64)
        ctx.set_config(cap=n // 64)
        try:
            got, st = gpu_select(ctx, x, k)
        finally:
            ctx.set_config(cap=0)
        assert bits(got) == bits(osel.select_kth(x, k))
        width = float(x.max()) - float(x.min())
        for i in range(2):
            assert abs(st["iterates"][i] - info["iterates"][i]) <= 1e-5 * width, (dist, i, st["iterates"][:3],
                                                                                  info["iterates"][:3])


def test_bounded_wait_gives_up_and_context_stays_usable(ctx, lib):
    """Failure path without a fault: a grid-barrier wait that cannot complete gives up after
    its bound (2 ms here, 2 s in the kernels) and records GBS_ETIMEOUT; the context then
    selects correctly."""
    import time
    t0 = time.perf_counter()
    assert ctx.check_wait_timeout(2_000_000) == lib.GBS_ETIMEOUT
    assert time.perf_counter() - t0 < 5.0
    x = synth.heavy_mixture("mixture", 300_001, seed=45)
    k = 150_001
    got, _ = gpu_select(ctx, x, k)
    assert bits(got) == bits(osel.select_kth(x, k))


def test_median_entry_point(ctx):
    x = synth.uniform(1_000_000, seed=0)
    got = ctx.median(torch.from_numpy(x).cuda()).cpu().numpy()[0]
    assert bits(got) == bits(osel.median(x))
    x64 = synth.uniform(999_999, seed=0, dtype=np.float64)
    got = ctx.median(torch.from_numpy(x64).cuda()).cpu().numpy()[0]
    assert bits(got) == bits(osel.median(x64))


def test_non_default_stream(ctx):
    x = torch.from_numpy(synth.uniform(2 ** 20 + 1, seed=44)).cuda()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        r = ctx.select_kth(x, 12345, stream=s)
    s.synchronize()
    assert bits(r.cpu().numpy()[0]) == bits(osel.select_kth(x.cpu().numpy(), 12345))


# ----------------------------------------------------------------------------- full size
def test_full_size_single_array_f32(ctx):
    """n = 2^27 float32 mixture with duplicates and +-inf (the benchmark workload), the
    five ranks of the benchmark, in the launch configuration the benchmark times."""
    x = synth.heavy_mixture("mixture", 2 ** 27, seed=4)
    n = x.size
    xt = torch.from_numpy(x).cuda()
    keys = osel.total_order_key(x)
    for k in (1, n // 100, (n + 1) // 2, (99 * n) // 100, n):
        r = ctx.select_kth(xt, k).cpu().numpy()[0]
        want = osel.key_to_value(np.partition(keys, k - 1)[k - 1], np.float32)[()]
        assert bits(r) == bits(want), k


def test_full_size_single_array_f64(ctx):
    x = synth.heavy_mixture("cauchy", 2 ** 26, seed=3, dtype=np.float64)
    n = x.size
    xt = torch.from_numpy(x).cuda()
    for k in (n // 100, (n + 1) // 2, (99 * n) // 100):
        r = ctx.select_kth(xt, k).cpu().numpy()[0]
        assert bits(r) == bits(osel.select_kth(x, k)), k


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_whole_array_compaction_fills_every_region(ctx, dtype):
    """cap >= n: the first cutting-plane pass compacts (almost) all of x, so every CTA's
    compaction region is filled to its bound; sizes straddle chunk boundaries."""
    try:
        ctx.set_config(cap=10 ** 12)
        for n in (4099, 8192 * 3 + 1, 300007, 2 ** 21 + 7):
            x = synth.paper_distribution("normal", n, seed=60 + n, dtype=dtype)
            for offset in (0, 1):
                check(ctx, x, [1, 2, n // 3, (n + 1) // 2, n - 1, n], offset=offset)
    finally:
        ctx.set_config(cap=0)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_beyond_2_31_elements_rank_property(ctx, dtype):
    """n = 2^31 + 5 elements (8 or 16 GiB, past every 32-bit element index), read from an
    offset of one element: the result satisfies the rank definition of Sec. 1,
    #(x < v) < k <= #(x <= v), with the counts taken by torch on the device.  float32:
    rounded normals (runs of ~10^7 equal values, +-0) with +-inf; float64: plain normals."""
    n = 2 ** 31 + 5
    g = torch.Generator(device="cuda")
    g.manual_seed(71)
    buf = torch.empty(n + 1, dtype=dtype, device="cuda")
    x = buf[1:]
    x.normal_(generator=g)
    if dtype == torch.float32:
        x.mul_(4.0).round_()
        x[:: 2 ** 24] = float("inf")
        x[7:: 2 ** 24] = float("-inf")
    for k in (1, n // 3, (n + 1) // 2, n - 7, n):
        v = ctx.select_kth(x, k)
        lt = int((x < v).sum())
        le = int((x <= v).sum())
        assert lt < k <= le, (dtype, k, v.item(), lt, le, ctx.last_stats()["how"])
    del x, buf
    torch.cuda.empty_cache()
