"""The paper's alternatives to Kelley's cutting plane (Sec. 2; Sec. 4 Tables 1-2 and
Discussion): bisection and Brent's root-finder on 0 in g(y), and Kelley's method on the
monotone image u = log(1 + x - x_(1)).  They drive the library's sharded state machine,
so the exact finish is shared and every driver must return the oracle's x_(k) bit for
bit; they differ in the passes taken.  The Discussion reports that only the cutting
plane is insensitive to a few huge elements: here the pass counts of the cutting plane
(and of its log variant) stay flat as one outlier grows from 1e3 to 3e38, while
bisection's grow with the logarithm of the data's range.  CPU tests use float64 numpy
passes by definition (test infrastructure); the GPU tests use the library's kernels."""
import math

import numpy as np
import pytest

import synth
from oracle import select as osel
from test_sharded import NumpyBackend, bits, gbs

DRIVERS = ("kelley", "bisect", "brent", "log")


class LogNumpyBackend(NumpyBackend):
    """NumpyBackend with the log driver's pass by its definition, in float64."""

    def cost_pass_log(self, x, a, t, xmin):
        a, t = x.dtype.type(a), x.dtype.type(t)
        inner = x[(x > a) & (x < t)].astype(np.float64)
        ut = math.log1p(float(t) - xmin)
        return {"c_lt_t": int((x < t).sum()), "c_le_t": int((x <= t).sum()), "c_le_a": int((x <= a).sum()),
                "S": float(np.sum(ut - np.log1p(inner - xmin)))}


def outlier_array(n, big, seed, dtype=np.float32):
    x = synth.paper_distribution("normal", n, seed, dtype=dtype)
    if big is not None:
        x[n // 3] = dtype(big)
    return x


@pytest.mark.parametrize("driver", DRIVERS)
@pytest.mark.parametrize("big", [None, 1e9, 1e20, 3e38])
def test_drivers_match_oracle(driver, big):
    g = gbs()
    from paper_1104_2732_gb300.sharded import select_kth_sharded
    x = outlier_array(20001, big, seed=70)
    for k in (1, 200, 10001, 19999, 20001):
        shards = np.array_split(x, 3)
        r = select_kth_sharded(shards, k, LogNumpyBackend(), elem_bytes=4, driver=driver)
        assert bits(r, np.float32) == bits(osel.select_kth(x, k), np.float32), (driver, big, k)


@pytest.mark.parametrize("driver", DRIVERS)
def test_drivers_on_ties_infinities_and_zeros(driver):
    g = gbs()
    from paper_1104_2732_gb300.sharded import select_kth_sharded
    x = synth.heavy_mixture("mixture", 30011, seed=71)
    x[::97] = np.float32(-0.0)
    x[::101] = np.float32(0.0)
    for k in (1, 6, 300, 15006, 29000, 30011):
        r = select_kth_sharded(np.array_split(x, 4), k, LogNumpyBackend(), elem_bytes=4, driver=driver)
        assert bits(r, np.float32) == bits(osel.select_kth(x, k), np.float32), (driver, k)


def passes(driver, big, n=20001, cap=64):
    from paper_1104_2732_gb300.sharded import select_kth_sharded
    x = outlier_array(n, big, seed=72)
    trace = []
    select_kth_sharded([x], (n + 1) // 2, LogNumpyBackend(), elem_bytes=4, cap=cap, trace=trace, driver=driver)
    return len(trace)


def test_only_the_cutting_plane_ignores_a_huge_outlier():
    """Sec. 4 Discussion, on a small cap (so the iterations, not the finish, do the work):
    with one element grown from none to 1e3, 1e9, 1e20 and 3e38, the cutting plane and its
    log variant need no more passes than without it (at most two more), while bisection
    and Brent's root-finder need more passes as the range grows (here 10 -> 64 and
    5 -> 64, the iteration limit)."""
    g = gbs()
    bigs = [None, 1e3, 1e9, 1e20, 3e38]
    got = {d: [passes(d, b) for b in bigs] for d in DRIVERS}
    for d in ("kelley", "log"):
        assert max(got[d]) <= got[d][0] + 2, got
    for d in ("bisect", "brent"):
        assert got[d][3] >= got[d][0] + 20 and got[d][4] >= got[d][3], got
    assert got["kelley"][4] < got["bisect"][4] and got["kelley"][4] < got["brent"][4]


def test_set_driver_checks():
    g = gbs()
    import ctypes as C
    st = g.gbs_shard_state()
    tot = g.gbs_array_stats()
    tot.n, tot.n_finite, tot.min, tot.max, tot.sum = 10, 10, 0.0, 9.0, 45.0
    assert g.gbs_shard_begin(C.byref(st), 4, 10, 5, C.byref(tot), 0, 0) == g.GBS_OK
    assert g.gbs_shard_set_driver(C.byref(st), 4) == g.GBS_EINVAL
    assert g.gbs_shard_set_driver(C.byref(st), -1) == g.GBS_EINVAL
    assert g.gbs_shard_set_driver(C.byref(st), g.GBS_DRIVER_BRENT) == g.GBS_OK and st.driver == 2
    assert g.gbs_shard_next(C.byref(st)) == g.GBS_OK
    st.it = 1   # a state that has iterated keeps its driver
    assert g.gbs_shard_set_driver(C.byref(st), g.GBS_DRIVER_KELLEY) == g.GBS_EINVAL


@pytest.mark.gpu
@pytest.mark.parametrize("driver", DRIVERS)
def test_drivers_on_gpu_shards(lib, driver):
    import torch
    from paper_1104_2732_gb300.sharded import GpuBackend, select_kth_sharded
    ctx = lib.Context()
    try:
        for big, dt in ((None, np.float32), (1e20, np.float32), (3e38, np.float32), (1e300, np.float64)):
            x = outlier_array(1 << 20, big, seed=73, dtype=dt)
            shards = [torch.from_numpy(p).cuda() for p in np.array_split(x, 3)]
            for k in (1, 10486, (x.size + 1) // 2, x.size):
                r = select_kth_sharded(shards, k, GpuBackend(ctx), elem_bytes=x.itemsize, driver=driver)
                assert bits(r, dt) == bits(osel.select_kth(x, k), dt), (driver, big, k)
    finally:
        ctx.close()


@pytest.mark.gpu
def test_log_pass_matches_its_definition(lib):
    """Counts exact; the log-coordinate cost within the float32 rounding of its terms
    (each u(t) - u(x) within 4 ulps of u's scale, summed)."""
    import torch
    ctx = lib.Context()
    try:
        for dt in (np.float32, np.float64):
            x = outlier_array(300001, 1e20, seed=74, dtype=dt)
            xt = torch.from_numpy(x).cuda()
            xmin = float(x.min())
            for a, t in ((-1.0, 0.5), (0.0, 3.0), (-2.5, 1e21)):
                got = ctx.cost_pass_log(xt, 150001, a, t, xmin)
                want = LogNumpyBackend().cost_pass_log(x, a, t, xmin)
                for f in ("c_lt_t", "c_le_t", "c_le_a"):
                    assert got[f] == want[f], (dt, a, t, f)
                inner = int(want["c_lt_t"] - want["c_le_a"])
                ut = math.log1p(float(dt(t)) - xmin)
                tol = inner * 8 * 2.0 ** -24 * max(1.0, abs(ut)) + 1e-6 * abs(want["S"])
                assert abs(got["S"] - want["S"]) <= tol, (dt, a, t, got["S"], want["S"])
    finally:
        ctx.close()
