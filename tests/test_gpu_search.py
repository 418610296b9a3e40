"""GPU parity of the LMS / LTS estimator search (Sec. 5) against the float64 oracle.

C-steps decide the retained rows on float32 squared residuals formed in the oracle's
stated order, so both sides retain the same rows; the refits differ only by the float64
rounding of the normal equations' sums and solve (about 1e-15 relative), far below the
float32 rounding of the coefficients, so the coefficients and the refit counts must be
equal and the objectives (float64 sums of the same float32 squares in other orders)
within h * 2^-52 relative.  The candidates' LMS / LTS objectives come from the fused
tensor-core form, within 1e-5 of the oracle's (the library's stated bound), so a choice
between candidates whose oracle objectives lie that close is accepted either way."""
import numpy as np
import pytest
import torch

import synth
from oracle import regression as oreg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(lib):
    c = lib.Context()
    yield c
    c.close()


def cuda(*arrs):
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs]


@pytest.mark.parametrize("n,p,seed", [(20001, 3, 60), (12345, 8, 61), (5000, 16, 62)])
def test_csteps_match_oracle(ctx, n, p, seed):
    X, y, _ = synth.regression(n, p, seed)
    th = np.ascontiguousarray(synth.elemental_thetas(X, y, 6, seed + 100).T)     # (C, p)
    h = (n + p + 1) // 2
    Xt, yt, tt = cuda(X, y, th)
    th_out, obj, refits = ctx.lts_csteps(Xt, yt, tt, h=h, max_steps=8)
    th_out, obj, refits = th_out.cpu().numpy(), obj.cpu().numpy(), refits.cpu().numpy()
    for c in range(th.shape[0]):
        t_o, F_o, kept = oreg.c_steps(X, y, th[c], h, 8)
        assert refits[c] == kept, (c, refits[c], kept)
        assert np.array_equal(th_out[c].view(np.uint32), t_o.view(np.uint32)), (c, th_out[c], t_o)
        assert obj[c] == pytest.approx(F_o, rel=h * 2.0 ** -52, abs=0), c


def test_csteps_zero_refits_and_exact_model(ctx):
    """max_steps = 0 reports each start's own objective; on data that 70% of the rows fit
    exactly, C-steps from a perturbed start reach that model with objective 0."""
    n, p = 4000, 3
    rng = np.random.default_rng(63)
    X = (np.round(rng.standard_normal((n, p)) * 8) / 8).astype(np.float32)
    beta = np.array([2.0, -1.0, 3.0], dtype=np.float32)
    y = (X.astype(np.float64) @ beta.astype(np.float64)).astype(np.float32)
    y[2800:] += rng.uniform(50, 100, n - 2800).astype(np.float32)
    h = 2100
    start = (beta + np.float32(0.05) * np.array([1, -1, 0.5], dtype=np.float32))[None, :]
    Xt, yt, st = cuda(X, y, start)
    th0, obj0, ref0 = ctx.lts_csteps(Xt, yt, st, h=h, max_steps=0)
    assert ref0.item() == 0 and np.array_equal(th0.cpu().numpy(), start)
    assert obj0.item() == pytest.approx(oreg.lts_objective_f32(X, y, start[0], h), rel=h * 2.0 ** -52)
    th1, obj1, ref1 = ctx.lts_csteps(Xt, yt, st, h=h, max_steps=30)
    assert obj1.item() == 0.0 and np.array_equal(th1.cpu().numpy()[0], beta) and ref1.item() >= 1


def test_search_matches_oracle(ctx):
    n, p, C = 30001, 4, 64
    X, y, beta = synth.regression(n, p, 64)
    th = np.ascontiguousarray(synth.elemental_thetas(X, y, C, 65).T)
    k, h = (n + 1) // 2, (n + p + 1) // 2
    Xt, yt, tt = cuda(X, y, th)
    out = {kk: v.cpu().numpy() for kk, v in ctx.lms_lts_search(Xt, yt, tt, k=k, h=h, n_refine=5, max_steps=10).items()}
    # LMS: the candidate of least objective (any candidate within the 1e-5 bound of it)
    lms_vals = np.array([oreg.lms((oreg.residuals(X, y, t) ** 2)[:, 0], k) for t in th])
    ci = int(out["lms_index"][0])
    assert lms_vals[ci] <= lms_vals.min() * (1 + 2e-5)
    assert np.array_equal(out["lms_theta"], th[ci])
    assert out["lms_value"][0] == pytest.approx(lms_vals[ci], rel=1e-5)
    # LTS: the refined set is the oracle's when its ranks are separated by more than 1e-5
    lts_vals = np.array([oreg.lts((oreg.residuals(X, y, t) ** 2)[:, 0], h) for t in th])
    srt = np.sort(lts_vals)
    assert srt[5] > srt[4] * (1 + 1e-4), "refined set not separated: choose another seed"
    t_o, F_o, order = oreg.lts_search(X, y, th, h, 5, 10)
    assert out["lts_index"][0] in order
    assert np.array_equal(out["lts_theta"].view(np.uint32), t_o.view(np.uint32))
    assert out["lts_value"][0] == pytest.approx(F_o, rel=h * 2.0 ** -52)
    # the estimate is close to the uncontaminated model, and no worse than any start
    assert out["lts_value"][0] <= lts_vals.min() * (1 + 1e-5)
    assert np.max(np.abs(out["lts_theta"] - beta)) < 0.1


def test_search_bench_size(ctx):
    """The benchmark problem (n = 1e6, p = 8, 2048 candidates, 10 refined, 20 refits at
    most): the LTS result is reproduced by the oracle's C-steps from the chosen start and
    its objective by the oracle's evaluation; the LMS choice is checked on a sample."""
    n, p, C = 1_000_000, 8, 2048
    X, y, beta = synth.regression(n, p, 6)
    th = np.ascontiguousarray(synth.elemental_thetas(X, y, C, 7).T)
    k, h = (n + 1) // 2, (n + p + 1) // 2
    Xt, yt, tt = cuda(X, y, th)
    out = {kk: v.cpu().numpy() for kk, v in ctx.lms_lts_search(Xt, yt, tt, k=k, h=h, n_refine=10, max_steps=20).items()}
    start = int(out["lts_index"][0])
    t_o, F_o, _ = oreg.c_steps(X, y, th[start], h, 20)
    assert np.array_equal(out["lts_theta"].view(np.uint32), t_o.view(np.uint32))
    assert out["lts_value"][0] == pytest.approx(F_o, rel=h * 2.0 ** -52)
    assert np.max(np.abs(out["lts_theta"] - beta)) < 0.05
    ci = int(out["lms_index"][0])
    sample = np.random.default_rng(66).choice(C, 24, replace=False)
    v_ci = oreg.lms((oreg.residuals(X, y, th[ci]) ** 2)[:, 0], k)
    for c in sample:
        assert v_ci <= oreg.lms((oreg.residuals(X, y, th[c]) ** 2)[:, 0], k) * (1 + 2e-5)
