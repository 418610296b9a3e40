"""GPU parity of the segmented batched select against the CPU oracle.

Every segment's result must be bit-identical to oracle.select.select_kth on that
segment.  Calls go through the C-ABI (ctypes binding).
"""
import os

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


def bits(a):
    return np.asarray(a, dtype=np.float32).view(np.uint32)


def make_batch(sizes, seed, gen=None):
    rng = np.random.default_rng(seed)
    parts = []
    for i, n in enumerate(sizes):
        if gen is None:
            parts.append((rng.standard_normal(n) * 10 ** rng.uniform(-3, 3) + rng.uniform(-100, 100)).astype(np.float32))
        else:
            parts.append(gen(i, n, rng))
    off = np.zeros(len(sizes) + 1, dtype=np.int64)
    off[1:] = np.cumsum(sizes)
    x = np.concatenate(parts) if parts else np.zeros(0, np.float32)
    return x, off


def run(ctx, x, off, k=None):
    xt = torch.from_numpy(x).cuda()
    ot = torch.from_numpy(off).cuda()
    kt = torch.from_numpy(k).cuda() if k is not None else None
    out = ctx.select_segmented(xt, ot, kt)
    return out.cpu().numpy()


def expect(x, off, k=None):
    S = off.size - 1
    want = np.empty(S, dtype=np.float32)
    for s in range(S):
        seg = x[off[s]:off[s + 1]]
        kk = int(k[s]) if k is not None else (seg.size + 1) // 2
        want[s] = osel.select_kth(seg, kk)
    return want


# sizes around every shared-memory capacity of the launch variants
EDGE_SIZES = [1, 2, 3, 7, 100, 1000, 4095, 12287, 12288, 12289, 24575, 24576, 24577, 49151, 49152, 49153,
              100003, 300001]


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_segmented_medians_every_variant(ctx, variant):
    x, off = make_batch(EDGE_SIZES, seed=70)
    ctx.set_segmented_variant(variant)
    try:
        got = run(ctx, x, off)
        assert ctx.last_stats()["status"] == 0
    finally:
        ctx.set_segmented_variant(1)
    assert np.array_equal(bits(got), bits(expect(x, off)))


def test_segmented_random_ranks(ctx):
    rng = np.random.default_rng(71)
    sizes = list(rng.integers(1, 200_000, 300))
    x, off = make_batch(sizes, seed=72)
    k = np.array([rng.integers(1, n + 1) for n in sizes], dtype=np.int64)
    got = run(ctx, x, off, k)
    assert np.array_equal(bits(got), bits(expect(x, off, k)))


def test_segmented_extreme_ranks_and_ties(ctx):
    def gen(i, n, rng):
        v = rng.integers(-3, 4, n).astype(np.float32)          # heavy ties
        if n > 10:
            v[:3] = [np.inf, -np.inf, -0.0]
            v[3:6] = 0.0
        return v
    sizes = [5, 11, 50_000, 20_000, 70_001, 12_300, 13]
    x, off = make_batch(sizes, seed=73, gen=gen)
    for mode in ("first", "second", "last", "mid"):
        k = np.array([{"first": 1, "second": min(2, n), "last": n, "mid": (n + 1) // 2}[mode] for n in sizes],
                     dtype=np.int64)
        got = run(ctx, x, off, k)
        assert np.array_equal(bits(got), bits(expect(x, off, k))), mode


def test_segmented_heavy_tailed_segments(ctx):
    def gen(i, n, rng):
        return synth.heavy_mixture(synth.HEAVY_FAMILIES[i % 4], n, seed=int(rng.integers(1 << 30)))
    sizes = [60_000, 250_000, 1_000_000, 30_000, 500_000, 2_000_000]
    x, off = make_batch(sizes, seed=74, gen=gen)
    for frac in (0.01, 0.5, 0.99):
        k = np.array([max(1, int(frac * n)) for n in sizes], dtype=np.int64)
        got = run(ctx, x, off, k)
        assert np.array_equal(bits(got), bits(expect(x, off, k))), frac


def test_segmented_brackets_compacted_in_device_memory(ctx):
    """Segments of 2e5 to 9e5 elements reach a bracket of at most n/4 elements while it is
    still larger than shared memory: it is compacted into the CTA's device-memory region
    and the finish gathers the chosen digit into shared memory.  Few distinct values (a
    digit bucket larger than shared memory), signed zeros and a normal sample."""
    def gen(i, n, rng):
        kind = i % 3
        if kind == 0:   # 3000 distinct values, each repeated
            return rng.choice(rng.standard_normal(3000).astype(np.float32), n)
        if kind == 1:   # zeros of both signs among a narrow normal sample
            v = (rng.standard_normal(n) * 1e-3).astype(np.float32)
            v[rng.random(n) < 0.2] = 0.0
            v[rng.random(n) < 0.2] = -0.0
            return v
        return (rng.standard_normal(n) * 50.0 + 7.0).astype(np.float32)
    sizes = [200_003, 450_000, 900_001, 333_333, 600_000, 250_000]
    x, off = make_batch(sizes, seed=81, gen=gen)
    for frac in (0.001, 0.3, 0.5, 0.97):
        k = np.array([max(1, int(frac * n)) for n in sizes], dtype=np.int64)
        got = run(ctx, x, off, k)
        assert np.array_equal(bits(got), bits(expect(x, off, k))), frac
    passes = ctx.segmented_passes(len(sizes))
    assert all(2 <= p <= 40 for p in passes), passes


MODEL = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1104_2732_gb300",
                     "bracket_model.bin")


@pytest.mark.skipif(not os.path.exists(MODEL), reason="no trained model in the package")
def test_segmented_learned_medians(lib):
    """Medians with learned starting brackets (proposal in the CTA, lean first pass,
    straight to the finish when the check holds): identical to the oracle, fewer passes on
    the large segments than the plain start, and a NaN in a large segment still reported."""
    def gen(i, n, rng):
        fam = synth.HEAVY_FAMILIES[i % 4]
        return synth.heavy_mixture(fam, n, seed=int(rng.integers(1 << 30))) * np.float32(10 ** rng.uniform(-2, 2))
    sizes = [70_000, 300_000, 1_000_000, 5_000, 131_072, 65_536, 800_001, 40_000, 450_000]
    x, off = make_batch(sizes, seed=82, gen=gen)
    plain = lib.Context()
    learned = lib.Context()
    learned.load_bracket_model(MODEL)
    learned.set_config(use_learned=1)
    try:
        want = expect(x, off)
        got_p = run(plain, x, off)
        got_l = run(learned, x, off)
        assert np.array_equal(bits(got_l), bits(want))
        assert np.array_equal(bits(got_p), bits(want))
        big = np.array(sizes) >= 65_536
        pp = np.array(plain.segmented_passes(len(sizes)))[big]
        pl = np.array(learned.segmented_passes(len(sizes)))[big]
        assert pl.mean() < pp.mean(), (pl, pp)
        # explicit ranks other than the median take the plain start
        k = np.array([max(1, n // 3) for n in sizes], dtype=np.int64)
        assert np.array_equal(bits(run(learned, x, off, k)), bits(expect(x, off, k)))
        y = x.copy()
        y[off[2] + 12345] = np.nan
        got = run(learned, y, off)
        with pytest.raises(lib.GbsError) as ei:
            learned.last_stats()
        assert ei.value.status == lib.GBS_ENAN
        assert np.isnan(got[2])
        assert np.array_equal(bits(np.delete(got, 2)), bits(np.delete(want, 2)))
    finally:
        plain.close()
        learned.close()


def _altered_model(path, centre_shift=0.0, log_width_shift=0.0):
    """A copy of the shipped model with the output biases moved (file layout: 8-byte
    magic, 5 u32 header words, u64 Adam step, then the parameters; the last two are the
    biases of the centre c and of the log half-width omega)."""
    raw = bytearray(open(MODEL, "rb").read())
    n_params = int(np.frombuffer(bytes(raw[8:28]), dtype=np.uint32)[4])
    params = np.frombuffer(bytes(raw[36:36 + 4 * n_params]), dtype=np.float32).copy()
    params[-2] += np.float32(centre_shift)
    params[-1] += np.float32(log_width_shift)
    raw[36:36 + 4 * n_params] = params.tobytes()
    with open(path, "wb") as fh:
        fh.write(bytes(raw))
    return path


@pytest.mark.skipif(not os.path.exists(MODEL), reason="no trained model in the package")
@pytest.mark.parametrize("shift", [(20.0, 0.0), (0.0, 12.0)], ids=["missed", "too-wide"])
def test_segmented_learned_fallbacks(lib, tmp_path, shift):
    """Proposals that miss the median (centre moved 20 sigma) take the plain path after the
    lean pass; proposals holding the whole segment finish from a device-memory bracket
    when it fits the CTA's share and otherwise take the plain path.  Results identical to
    the oracle either way."""
    def gen(i, n, rng):
        return (rng.standard_normal(n) * 3.0 + rng.uniform(-5, 5)).astype(np.float32)
    sizes = [20_000, 150_000, 600_000, 13_000, 260_000]
    x, off = make_batch(sizes, seed=83, gen=gen)
    c = lib.Context()
    try:
        c.load_bracket_model(_altered_model(str(tmp_path / "m.bin"), *shift))
        c.set_config(use_learned=1)
        got = run(c, x, off)
        assert np.array_equal(bits(got), bits(expect(x, off)))
        passes = np.array(c.segmented_passes(len(sizes)))
        large = np.array(sizes) > c.segmented_variant()["smem_cap"]   # the others stay in shared memory
        assert large.sum() >= 3
        if shift[0] != 0.0:
            assert (passes[large] >= 3).all(), passes   # lean pass + pass 0 + at least one cut
    finally:
        c.close()


def test_segmented_invalid_segments_are_flagged(ctx, lib):
    x, off = make_batch([10, 0, 10], seed=75)
    got = run(ctx, x, off)
    with pytest.raises(lib.GbsError) as ei:
        ctx.last_stats()
    assert ei.value.status == lib.GBS_EINVAL
    assert np.isnan(got[1])
    assert bits(got[0]) == bits(expect(x[:10], np.array([0, 10]))[0])
    y, off2 = make_batch([1000, 1000], seed=76)
    y[1500] = np.nan
    got = run(ctx, y, off2)
    with pytest.raises(lib.GbsError) as ei:
        ctx.last_stats()
    assert ei.value.status == lib.GBS_ENAN
    assert np.isnan(got[1]) and not np.isnan(got[0])


def test_segmented_autotune_and_passes(ctx):
    sizes = list(synth.segment_sizes(256, seed=77))
    x, off = make_batch(sizes, seed=78)
    xt, ot = torch.from_numpy(x).cuda(), torch.from_numpy(off).cuda()
    out = torch.empty(len(sizes), device="cuda")
    chosen, ms = ctx.autotune_segmented(xt, ot, None, out)
    assert 0 <= chosen < len(ms) and ms[chosen] > 0 and ms[chosen] == min(m for m in ms if m > 0)
    assert np.array_equal(bits(out.cpu().numpy()), bits(expect(x, off)))
    passes = ctx.segmented_passes(len(sizes))
    cap = ctx.segmented_variant()["smem_cap"]
    for n, p in zip(sizes, passes):
        assert (p == 1) if n <= cap else (p >= 2)
    ctx.set_segmented_variant(1)


def test_segmented_graph_capture_replay(ctx):
    sizes = list(synth.segment_sizes(128, seed=79))
    x, off = make_batch(sizes, seed=80)
    xt, ot = torch.from_numpy(x).cuda(), torch.from_numpy(off).cuda()
    out = torch.zeros(len(sizes), device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ctx.select_segmented(xt, ot, None, out, stream=s)   # sizes the workspace before capture
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        ctx.select_segmented(xt, ot, None, out, stream=s)
    out.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert np.array_equal(bits(out.cpu().numpy()), bits(expect(x, off)))
    # replay on new data of the same shape
    x2, _ = make_batch(sizes, seed=81)
    xt.copy_(torch.from_numpy(x2))
    g.replay()
    torch.cuda.synchronize()
    assert np.array_equal(bits(out.cpu().numpy()), bits(expect(x2, off)))


def test_segmented_full_size_batch_sampled(ctx):
    """The benchmark batch: 4096 normal arrays, sizes log-uniform in [1e3, 1e6]; every
    segment above the largest shared-memory capacity and a random sample of the rest are
    checked against the oracle."""
    x, off = synth.segmented(4096, seed=5)
    sizes = np.diff(off)
    got = run(ctx, x, off)
    rng = np.random.default_rng(82)
    check = set(np.nonzero(sizes > 49152)[0][:200].tolist()) | set(rng.choice(4096, 200, replace=False).tolist())
    for s in sorted(check):
        seg = x[off[s]:off[s + 1]]
        assert bits(got[s]) == bits(np.float32(osel.select_kth(seg, (seg.size + 1) // 2))), s


def test_batch_beyond_2_31_elements_rank_property(ctx):
    """4096 segments of 524291 float32 elements (2^31 + 12288 in all, so the later
    segments start past every 32-bit element offset), medians and a low rank: every
    result satisfies the rank definition #(x_s < v_s) < k_s <= #(x_s <= v_s) of Sec. 1,
    counted by torch on the device.  Rounded normals with per-segment scales give runs of
    equal values and +-0."""
    S, m = 4096, 524291
    g = torch.Generator(device="cuda")
    g.manual_seed(73)
    x = torch.empty(S * m, dtype=torch.float32, device="cuda")
    x.normal_(generator=g)
    X = x.view(S, m)
    scale = torch.pow(10.0, torch.linspace(-1.0, 2.0, S, device="cuda"))
    X.mul_(scale[:, None]).round_()
    off = torch.arange(S + 1, dtype=torch.int64, device="cuda") * m
    for kk in (None, torch.full((S,), m // 100, dtype=torch.int64, device="cuda")):
        out = ctx.select_segmented(x, off, kk)
        k = torch.full((S,), (m + 1) // 2, dtype=torch.int64, device="cuda") if kk is None else kk
        lt = (X < out[:, None]).sum(1)
        le = (X <= out[:, None]).sum(1)
        bad = ~((lt < k) & (k <= le))
        assert int(bad.sum()) == 0, int(bad.nonzero()[0])
    del X, x
    torch.cuda.empty_cache()
