"""Sharded selection: the library's host state machine (gbs_shard_begin / _next /
_update) driven over shards whose per-pass results are summed between passes (Sec. 4,
data distributed over several GPUs).  On the CPU the per-shard passes come from a
float64 numpy restatement of the pass definitions (counts and the cost term of
Algorithm 1, step 1.2); the results must equal the oracle's selection bit for bit,
in one process and across two gloo ranks.  The GPU test runs the same driver with the
library's kernels on shards of one device."""
import os
import socket

import numpy as np
import pytest

import synth
from oracle import select as osel


def gbs():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1104_2732_gb300 as g
    return g


class NumpyBackend:
    """Per-shard passes by their definitions, in float64 (test infrastructure)."""

    def stats(self, x):
        fin = x[np.isfinite(x)]
        return {"n": x.size, "n_nan": int(np.isnan(x).sum()), "n_neginf": int((x == -np.inf).sum()),
                "n_posinf": int((x == np.inf).sum()), "n_negzero": int(((x == 0) & np.signbit(x)).sum()),
                "n_finite": int(fin.size), "min": float(fin.min()) if fin.size else 0.0,
                "max": float(fin.max()) if fin.size else 0.0, "sum": float(np.sum(fin, dtype=np.float64))}

    def cost_pass(self, x, a, t):
        a, t = x.dtype.type(a), x.dtype.type(t)
        inner = x[(x > a) & (x < t)].astype(np.float64)
        return {"c_lt_t": int((x < t).sum()), "c_le_t": int((x <= t).sum()), "c_le_a": int((x <= a).sum()),
                "S": float(np.sum(float(t) - inner))}

    def compact(self, x, a, b):
        a, b = x.dtype.type(a), x.dtype.type(b)
        return x[(x > a) & (x <= b)]

    def concat(self, zs):
        return np.concatenate([np.asarray(z) for z in zs])

    def empty(self, elem_bytes):
        return np.empty(0, dtype=np.float32 if elem_bytes == 4 else np.float64)

    def select(self, z, r):
        return float(osel.select_kth(z, r))


def bits(v, dt):
    return np.asarray(v, dtype=dt).view(np.uint64 if dt == np.float64 else np.uint32)


def split(x, parts, seed):
    rng = np.random.default_rng(seed)
    cuts = np.sort(rng.choice(np.arange(1, x.size), parts - 1, replace=False))
    return np.split(x, cuts)


ARRAYS = [
    ("uniform", lambda: synth.uniform(20000, seed=1)),
    ("mixture", lambda: synth.heavy_mixture("mixture", 30011, seed=2)),
    ("cauchy64", lambda: synth.heavy_mixture("cauchy", 20003, seed=3, dtype=np.float64)),
    ("zeros", lambda: np.array([0.0, -0.0] * 3000 + [1.0, -1.0] * 10, dtype=np.float32)),
    ("dups", lambda: np.repeat(np.arange(50, dtype=np.float32), 400)),
]


@pytest.mark.parametrize("name,make", ARRAYS)
def test_sharded_matches_oracle(name, make):
    g = gbs()
    from paper_1104_2732_gb300.sharded import select_kth_sharded
    x = make()
    n = x.size
    eb = x.dtype.itemsize
    for parts in (1, 3):
        shards = split(x, parts, seed=7) if parts > 1 else [x]
        for k in sorted({1, 2, n // 100 + 1, (n + 1) // 2, n - n // 100, n - 1, n}):
            got = select_kth_sharded(shards, k, NumpyBackend(), elem_bytes=eb, cap=max(64, n // 64))
            want = osel.select_kth(x, k)
            assert bits(got, x.dtype) == bits(want, x.dtype), (name, parts, k, got, want)
    # a NaN has no rank
    y = x.copy()
    y[5] = np.nan
    with pytest.raises(g.GbsError):
        select_kth_sharded([y[:100], y[100:]], 1, NumpyBackend(), elem_bytes=eb)


def test_sharded_empty_and_single_element_shards():
    """Empty shards anywhere in the list, single-element shards, and data that are all
    infinite: the result is the single-array one bit for bit."""
    gbs()
    from paper_1104_2732_gb300.sharded import select_kth_sharded
    x = synth.heavy_mixture("mixture", 5001, seed=2)
    layouts = ([x[:0], x], [x, x[:0]], [x[:0], x[:10], x[10:10], x[10:]], [x[:1], x[1:]], [x[:1], x[1:2], x[2:]])
    for shards in layouts:
        for k in (1, 2, 2500, 5000, 5001):
            got = select_kth_sharded(shards, k, NumpyBackend(), elem_bytes=4, cap=64)
            assert bits(got, np.float32) == bits(osel.select_kth(x, k), np.float32), (len(shards), k)
    y = np.array([np.inf] * 3 + [-np.inf] * 2, dtype=np.float32)
    for k in range(1, 6):
        got = select_kth_sharded([y[:2], y[2:], y[:0]], k, NumpyBackend(), elem_bytes=4)
        assert bits(got, np.float32) == bits(osel.select_kth(y, k), np.float32), k


def test_sharded_no_elements_at_all_is_rejected():
    g = gbs()
    from paper_1104_2732_gb300.sharded import select_kth_sharded
    e = np.empty(0, dtype=np.float32)
    for shards in ([], [e, e]):
        with pytest.raises(g.GbsError):
            select_kth_sharded(shards, 1, NumpyBackend(), elem_bytes=4)


def test_state_machine_rejects_bad_totals():
    g = gbs()
    import ctypes as C
    st = g.gbs_shard_state()
    tot = g.gbs_array_stats()
    tot.n = 10
    tot.n_finite = 9                      # counts do not add up to n
    assert g.gbs_shard_begin(C.byref(st), 4, 10, 3, C.byref(tot), 0, 0) == g.GBS_EINVAL
    tot.n_finite = 10
    tot.min, tot.max = 0.0, 1.0
    assert g.gbs_shard_begin(C.byref(st), 4, 10, 11, C.byref(tot), 0, 0) == g.GBS_EINVAL
    assert g.gbs_shard_begin(C.byref(st), 4, 10, 5, C.byref(tot), 4, 0) == g.GBS_OK
    assert st.phase == g.GBS_SHARD_ITERATE and st.cle_a == 0 and st.cle_b == 10
    ev = g.gbs_cost_eval()
    ev.c_le_a = 3                         # the shards disagree with the state's #(x <= a)
    ev.c_lt_t, ev.c_le_t = 4, 5
    assert g.gbs_shard_next(C.byref(st)) == g.GBS_OK
    assert g.gbs_shard_update(C.byref(st), C.byref(ev)) == g.GBS_EINTERNAL


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


GLOO_RANKS = (1, 400, 20005, 39000, 40009)


def _gloo_data(layout):
    if layout in ("two_each", "three_uneven"):
        return synth.heavy_mixture("mixture", 40009, seed=11)
    return synth.heavy_mixture("cauchy", 40009, seed=12, dtype=np.float64)


def _rank_main(rank, world, port, out, layout):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import paper_1104_2732_gb300  # noqa: F401  (built by the parent)
        from paper_1104_2732_gb300.sharded import TorchComm, select_kth_sharded
        x = _gloo_data(layout)
        if layout == "two_each":
            own = split(x, 4, seed=3)[rank * 2:(rank + 1) * 2]     # two shards per rank
        elif layout == "three_uneven":
            parts = split(x, 4, seed=5)                            # ranks hold 3, 0 and 1 shards
            own = parts[:3] if rank == 0 else ([] if rank == 1 else parts[3:])
        else:
            own = [x] if rank == 0 else []                        # rank 1 holds no element
        res = []
        for k in GLOO_RANKS:
            res.append(select_kth_sharded(own, k, NumpyBackend(), TorchComm(), elem_bytes=x.itemsize, cap=1000))
        out.put((rank, res))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("layout,world", [("two_each", 2), ("one_rank_empty", 2), ("three_uneven", 3)])
def test_sharded_gloo_ranks(layout, world):
    """gloo ranks on the CPU: two shards on each of two ranks (float32); every element on
    rank 0 and none on rank 1 (float64); three ranks holding 3, 0 and 1 uneven shards
    (float32).  Every rank returns the single-array result."""
    gbs()
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q, layout)) for r in range(world)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=240) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    x = _gloo_data(layout)
    want = [osel.select_kth(x, k) for k in GLOO_RANKS]
    for r in range(world):
        assert [bits(v, x.dtype) for v in got[r]] == [bits(v, x.dtype) for v in want]


@pytest.mark.gpu
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_sharded_gpu_shards_match_oracle(lib, dtype):
    import torch
    from paper_1104_2732_gb300.sharded import GpuBackend, select_kth_sharded
    ctx = lib.Context()
    try:
        for fam, n in (("normal", 1 << 20), ("mixture", 3_000_017), ("lognormal", 777_777)):
            x = synth.heavy_mixture(fam, n, seed=21, dtype=dtype)
            parts = split(x, 3, seed=5) + [x[:7]]          # uneven shards, one tiny
            shards = [torch.from_numpy(np.ascontiguousarray(p)).cuda() for p in parts[:3]]
            for k in (1, n // 100, (n + 1) // 2, n - n // 100, n):
                got = select_kth_sharded(shards, k, GpuBackend(ctx), elem_bytes=x.dtype.itemsize)
                want = osel.select_kth(x, k)
                assert bits(got, x.dtype) == bits(want, x.dtype), (fam, k, got, want)
    finally:
        ctx.close()


class _FailingBackend(NumpyBackend):
    """Raises on its third cost pass (a host-side failure of one rank between passes)."""

    def __init__(self):
        self.calls = 0

    def cost_pass(self, x, a, t):
        self.calls += 1
        if self.calls == 3:
            raise RuntimeError("injected failure on this rank")
        return super().cost_pass(x, a, t)


def _failing_rank_main(rank, world, port, out):
    import datetime
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=10))
    import paper_1104_2732_gb300  # noqa: F401  (built by the parent)
    from paper_1104_2732_gb300.sharded import TorchComm, select_kth_sharded
    x = synth.heavy_mixture("mixture", 40009, seed=11)
    own = split(x, 2, seed=3)[rank:rank + 1]
    backend = _FailingBackend() if rank == 1 else NumpyBackend()
    try:
        select_kth_sharded(own, 20005, backend, TorchComm(), elem_bytes=4, cap=10)
        out.put((rank, "finished"))
    except Exception as e:   # the injected failure (rank 1) or the failed collective (rank 0)
        out.put((rank, type(e).__name__))
    # no destroy_process_group: the peer may be gone


def test_sharded_rank_failure_surfaces_on_the_other_rank():
    """A rank that fails between passes (an exception on the host, no GPU involved) ends
    the other rank's next collective with an error within the process group's timeout,
    instead of leaving it waiting."""
    gbs()
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_failing_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=30)
        if p.is_alive():
            p.kill()
    assert got[1] == "RuntimeError"
    assert got[0] != "finished"
