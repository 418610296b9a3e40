"""GPU parity of the LMS / LTS objectives (Sec. 5) against the float64 oracle.

Tolerance: each LMS and LTS must be within 1e-5 relative of the float64 oracle.  The
squared residuals are float32 (split-precision TF32 x 3 or float32 FMAs); order
statistics are 1-Lipschitz in the sup norm, so |LMS - LMS64| <= max_i |s_i - s64_i|
and |LTS - LTS64| <= h max_i |s_i - s64_i|: the tests also check the GPU's residuals
against float64 and that the GPU's selection on its own residuals is bit-exact.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import regression as oreg
from oracle import select as osel

pytestmark = pytest.mark.gpu

REL = 1e-5
# LTS sums: float32 partials of at most a few hundred terms per thread, float64 beyond
SUM_REL = 2e-6


def resid_bound(X, y, th, p, precision):
    """Bound on |s_gpu - s64| per element: the residual's error is at most
    c * (|y| + sum_j |x_j theta_j|), c = (p+2) u for float32 FMAs and additionally
    4 * 2^-22 for the TF32 x 3 products (u = 2^-24); squaring doubles it."""
    u = 2.0 ** -24
    c = (p + 2) * u + (4 * 2.0 ** -22 if precision == 1 else 0.0)
    scale = (np.abs(y)[None, :].astype(np.float64)
             + (np.abs(X.astype(np.float64)) @ np.abs(th.T.astype(np.float64))).T)
    r64 = np.abs(oreg.residuals(X, y, th.T)).T
    d = c * scale
    return 2 * d * (r64 + d) + u * r64 * r64 + 1e-30


@pytest.fixture(scope="module")
def ctx(lib):
    c = lib.Context()
    yield c
    c.close()


def problem(n, p, C, seed):
    X, y, _ = synth.regression(n, p, seed)
    th = synth.elemental_thetas(X, y, C, seed + 1)          # (p, C)
    return X, y, np.ascontiguousarray(th.T)                   # theta as (C, p)


def to_dev(*arrs):
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs]


@pytest.mark.parametrize("precision", [0, 1])
def test_residuals_match_float64(ctx, precision):
    X, y, th = problem(5003, 8, 70, seed=90)
    Xt, yt, tt = to_dev(X, y, th)
    S = ctx.residual_sq(Xt, yt, tt, precision=precision).cpu().numpy()
    r64 = oreg.residuals(X, y, th.T)                           # (n, C)
    s64 = (r64 * r64).T
    assert np.all(np.abs(S - s64) <= resid_bound(X, y, th, 8, precision))


@pytest.mark.parametrize("p", [1, 3, 8, 12, 16])
def test_residual_tensor_core_layout(ctx, p):
    """TF32 x 3 and float32 FMA residuals agree for every p (fragment layout check)."""
    X, y, th = problem(777, p, 37, seed=91)
    Xt, yt, tt = to_dev(X, y, th)
    a = ctx.residual_sq(Xt, yt, tt, precision=0).cpu().numpy()
    b = ctx.residual_sq(Xt, yt, tt, precision=1).cpu().numpy()
    s64 = (oreg.residuals(X, y, th.T) ** 2).T
    assert np.all(np.abs(a - s64) <= resid_bound(X, y, th, p, 0))
    assert np.all(np.abs(b - s64) <= resid_bound(X, y, th, p, 1))


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("batched", [False, True])
def test_lms_lts_match_float64_oracle(ctx, precision, batched):
    n, p, C = 20001, 8, 96
    X, y, th = problem(n, p, C, seed=92)
    k, h = (n + 1) // 2, (n + p + 1) // 2
    Xt, yt, tt = to_dev(X, y, th)
    lms, lts = ctx.lms_lts(Xt, yt, tt, k=k, h=h, precision=precision, batched=batched)
    assert ctx.last_stats()["status"] == 0
    lms, lts = lms.cpu().numpy(), lts.cpu().numpy()
    want_lms, want_lts = oreg.lms_lts(X, y, th.T, k, h)
    assert np.all(np.abs(lms - want_lms) <= REL * np.abs(want_lms)), np.max(np.abs(lms / want_lms - 1))
    assert np.all(np.abs(lts - want_lts) <= REL * np.abs(want_lts)), np.max(np.abs(lts / want_lts - 1))
    # the selection itself is exact on the GPU's own residuals
    S = ctx.residual_sq(Xt, yt, tt, precision=precision).cpu().numpy()
    for c in range(0, C, 7):
        assert np.float32(lms[c]).view(np.uint32) == np.float32(osel.select_kth(S[c], k)).view(np.uint32)
        assert lts[c] == pytest.approx(oreg.lts(S[c], h), rel=SUM_REL)


def test_lms_lts_special_case_theta_zero(ctx):
    """p = 1, theta = 0: the residuals are y, LMS = median(y^2) exactly."""
    n = 9999
    y = synth.uniform(n, seed=93) - np.float32(0.5)
    X = np.ones((n, 1), np.float32)
    th = np.zeros((3, 1), np.float32)
    Xt, yt, tt = to_dev(X, y, th)
    for batched in (False, True):
        lms, lts = ctx.lms_lts(Xt, yt, tt, k=(n + 1) // 2, h=(n + 1) // 2, precision=1, batched=batched)
        s32 = (y * y).astype(np.float32)
        assert lms.cpu().numpy()[0] == osel.select_kth(s32, (n + 1) // 2)
        assert lts.cpu().numpy()[0] == pytest.approx(oreg.lts(s32, (n + 1) // 2), rel=SUM_REL)


def test_lms_lts_ranks_far_apart(ctx):
    """h far from k: the LMS rank lies outside the compacted bracket, the second batched
    select must supply it."""
    n, p, C = 50000, 4, 40
    X, y, th = problem(n, p, C, seed=94)
    Xt, yt, tt = to_dev(X, y, th)
    k, h = n // 10, (9 * n) // 10
    lms, lts = ctx.lms_lts(Xt, yt, tt, k=k, h=h, precision=1, batched=True)
    S = ctx.residual_sq(Xt, yt, tt, precision=1).cpu().numpy()
    for c in range(C):
        assert np.float32(lms.cpu().numpy()[c]).view(np.uint32) == np.float32(osel.select_kth(S[c], k)).view(np.uint32)
        assert lts.cpu().numpy()[c] == pytest.approx(oreg.lts(S[c], h), rel=SUM_REL)


def test_lms_lts_full_size_sampled(ctx):
    """The benchmark problem: n = 1e6, p = 8, 30% contaminated rows, 2048 elemental
    candidates; 12 sampled candidates against the float64 oracle."""
    n, p, C = 1_000_000, 8, 2048
    X, y, th = problem(n, p, C, seed=6)
    k, h = (n + 1) // 2, (n + p + 1) // 2
    Xt, yt, tt = to_dev(X, y, th)
    lms, lts = ctx.lms_lts(Xt, yt, tt, k=k, h=h, precision=1, batched=True)
    lms, lts = lms.cpu().numpy(), lts.cpu().numpy()
    rng = np.random.default_rng(95)
    for c in rng.choice(C, 12, replace=False):
        wl, wt = oreg.lms_lts(X, y, th[c:c + 1].T, k, h)
        assert abs(lms[c] - wl[0]) <= REL * abs(wl[0])
        assert abs(lts[c] - wt[0]) <= REL * abs(wt[0])


def test_lms_lts_rejects_bad_arguments(ctx, lib):
    X, y, th = problem(100, 8, 4, seed=96)
    Xt, yt, tt = to_dev(X, y, th)
    with pytest.raises(lib.GbsError):
        ctx.lms_lts(Xt, yt, tt, k=0, h=50)
    with pytest.raises(lib.GbsError):
        ctx.lms_lts(Xt, yt, tt, k=50, h=101)
    X17 = torch.zeros(10, 17, device="cuda")
    with pytest.raises(lib.GbsError):
        ctx.residual_sq(X17, torch.zeros(10, device="cuda"), torch.zeros(2, 17, device="cuda"))


# ---------------------------------------------------------------- fused form
def check_against_oracle(lms, lts, X, y, th, k, h, cands=None):
    cands = range(th.shape[0]) if cands is None else cands
    for c in cands:
        wl, wt = oreg.lms_lts(X, y, th[c:c + 1].T, k, h)
        assert abs(lms[c] - wl[0]) <= REL * abs(wl[0]), (c, lms[c], wl[0])
        assert abs(lts[c] - wt[0]) <= REL * abs(wt[0]), (c, lts[c], wt[0])


@pytest.mark.parametrize("p,C", [(8, 96), (8, 130), (3, 37), (1, 5), (12, 37), (16, 20)])
def test_fused_matches_float64_oracle(ctx, p, C):
    """Residuals recomputed in every pass (never written): within 1e-5 of the float64
    oracle for every candidate; C not a multiple of the 128 candidates of a CTA."""
    n = 20001 if p == 8 else 7777
    X, y, th = problem(n, p, C, seed=97 + p)
    k, h = (n + 1) // 2, (n + p + 1) // 2
    Xt, yt, tt = to_dev(X, y, th)
    lms, lts, passes = ctx.lms_lts_fused(Xt, yt, tt, k=k, h=h)
    lms, lts = lms.cpu().numpy(), lts.cpu().numpy()
    assert 2 <= passes <= 66
    want_lms, want_lts = oreg.lms_lts(X, y, th.T, k, h)
    assert np.all(np.abs(lms - want_lms) <= REL * np.abs(want_lms)), np.max(np.abs(lms / want_lms - 1))
    assert np.all(np.abs(lts - want_lts) <= REL * np.abs(want_lts)), np.max(np.abs(lts / want_lts - 1))


def test_fused_theta_zero_is_exact(ctx):
    """p = 1, theta = 0: s = y^2 exactly, so LMS is the exact order statistic of y^2."""
    n = 9999
    y = synth.uniform(n, seed=93) - np.float32(0.5)
    X = np.ones((n, 1), np.float32)
    th = np.zeros((3, 1), np.float32)
    Xt, yt, tt = to_dev(X, y, th)
    k = (n + 1) // 2
    lms, lts, _ = ctx.lms_lts_fused(Xt, yt, tt, k=k, h=k)
    s32 = (y * y).astype(np.float32)
    assert np.all(lms.cpu().numpy() == osel.select_kth(s32, k))
    assert lts.cpu().numpy() == pytest.approx(oreg.lts(s32, k), rel=SUM_REL)


def test_fused_exact_fit_all_residuals_zero(ctx):
    """y = X theta exactly (small integers): every residual is 0, LMS = LTS = 0."""
    rng = np.random.default_rng(98)
    n, p = 4096, 4
    X = rng.integers(-3, 4, (n, p)).astype(np.float32)
    th = rng.integers(-3, 4, (2, p)).astype(np.float32)
    y = (X @ th[0]).astype(np.float32)
    Xt, yt, tt = to_dev(X, y, th)
    lms, lts, _ = ctx.lms_lts_fused(Xt, yt, tt)
    assert lms.cpu().numpy()[0] == 0.0 and lts.cpu().numpy()[0] == 0.0
    check_against_oracle(lms.cpu().numpy(), lts.cpu().numpy(), X, y, th, (n + 1) // 2, (n + p + 1) // 2, [1])


def test_fused_ranks_far_apart_use_the_batched_form(ctx):
    """k and h far apart: the bracket holding both exceeds the compaction buffer, so the
    candidates are finished by the materialising batched form; results still match."""
    n, p, C = 200000, 4, 20
    X, y, th = problem(n, p, C, seed=94)
    Xt, yt, tt = to_dev(X, y, th)
    k, h = n // 10, (9 * n) // 10
    lms, lts, _ = ctx.lms_lts_fused(Xt, yt, tt, k=k, h=h)
    check_against_oracle(lms.cpu().numpy(), lts.cpu().numpy(), X, y, th, k, h)


@pytest.mark.parametrize("p,C,n", [(8, 256, 300_000), (12, 40, 70_001)])
def test_fused_sampled_start_matches_plain_start(ctx, p, C, n):
    """Brackets proposed by the candidates' order statistics on 8192 sampled rows (compacted
    and checked by counts in one pass) against the start from the extremes: the same LMS
    values bit for bit (both select from the same recomputed residuals), LTS within
    rounding of the sum below the bracket, fewer passes, and both within the oracle's
    bound; p = 12 runs the two-block (K = 16) product."""
    X, y, th = problem(n, p, C, seed=96)
    Xt, yt, tt = to_dev(X, y, th)
    k, h = (n + 1) // 2, (n + p + 1) // 2
    try:
        ctx.set_config(lms_start=1)
        lp, tp, pp = ctx.lms_lts_fused(Xt, yt, tt, k=k, h=h)
        ctx.set_config(lms_start=0)
        ls, ts, ps = ctx.lms_lts_fused(Xt, yt, tt, k=k, h=h)
    finally:
        ctx.set_config(lms_start=0)
    lp, tp, ls, ts = (a.cpu().numpy() for a in (lp, tp, ls, ts))
    assert np.array_equal(lp.view(np.uint32), ls.view(np.uint32))
    assert np.all(np.abs(ts - tp) <= 1e-6 * np.abs(tp))
    assert ps < pp, (ps, pp)
    check_against_oracle(ls, ts, X, y, th, k, h, [0, C // 2, C - 1])


def test_fused_nan_row_matches_batched_form(ctx):
    n, p, C = 5000, 8, 6
    X, y, th = problem(n, p, C, seed=99)
    X[17, 2] = np.nan
    Xt, yt, tt = to_dev(X, y, th)
    lms, lts, _ = ctx.lms_lts_fused(Xt, yt, tt)
    assert np.all(np.isnan(lms.cpu().numpy()))


def test_fused_nan_row_sampled_start(ctx):
    """A NaN in X on a problem large enough for the sampled start: the one-pass route sees
    its counts fall short of n and hands every candidate to the batched form (NaN results);
    an infinite square (huge y) leaves the objectives finite and exact."""
    n, p, C = 70_001, 8, 12
    X, y, th = problem(n, p, C, seed=98)
    Xn = X.copy()
    Xn[31_337, 5] = np.nan
    lms, lts, passes = ctx.lms_lts_fused(*to_dev(Xn, y, th))
    assert passes == 1 and np.all(np.isnan(lms.cpu().numpy()))
    yi = y.copy()
    yi[4242] = np.float32(3e38)     # its square overflows to +inf
    k, h = (n + 1) // 2, (n + p + 1) // 2
    lms, lts, _ = ctx.lms_lts_fused(*to_dev(X, yi, th), k=k, h=h)
    check_against_oracle(lms.cpu().numpy(), lts.cpu().numpy(), X, yi, th, k, h, [0, 5, 11])


def test_fused_full_size_against_oracle_and_batched(ctx):
    """The benchmark problem (n = 1e6, p = 8, 30% contaminated rows, 2048 candidates):
    12 sampled candidates against the float64 oracle, every candidate within 2e-5 of the
    materialising TF32 x 3 batched form (each is within 1e-5 of float64)."""
    n, p, C = 1_000_000, 8, 2048
    X, y, th = problem(n, p, C, seed=6)
    k, h = (n + 1) // 2, (n + p + 1) // 2
    Xt, yt, tt = to_dev(X, y, th)
    lms, lts, passes = ctx.lms_lts_fused(Xt, yt, tt, k=k, h=h)
    lms, lts = lms.cpu().numpy(), lts.cpu().numpy()
    assert passes <= 20
    bl, bt = ctx.lms_lts(Xt, yt, tt, k=k, h=h, precision=1, batched=True)
    bl, bt = bl.cpu().numpy(), bt.cpu().numpy()
    assert np.all(np.abs(lms - bl) <= 2 * REL * np.abs(bl))
    assert np.all(np.abs(lts - bt) <= 2 * REL * np.abs(bt))
    rng = np.random.default_rng(95)
    check_against_oracle(lms, lts, X, y, th, k, h, rng.choice(C, 12, replace=False))
