"""The device-resident sharded loop (select_kth_sharded_device): per pass, every shard
adds its counts and fixed-point cost into one int64[8] accumulator, the ranks all-reduce
it in place, and a one-thread step applies the bracket update and the next point of
Algorithm 1 (Sec. 3) to the state held in device memory.

CPU: the loop's host logic over two and three gloo ranks, with a stand-in context whose
pass and step follow the entry points' stated semantics in numpy (counts by definition,
the cost's fixed point of the header, the host state machine for the step); every rank
must return the oracle's element bit for bit.  GPU: the library's kernels, with no
process group and with an NCCL group of one rank; results equal the oracle's and the
host-driven loop's."""
import ctypes as C
import math
import os

import numpy as np
import pytest

import synth
from oracle import select as osel
from test_sharded import _free_port, bits, gbs, split

RANKS = (1, 400, 20005, 39000, 40009)


def sfix_bits(st):
    """fx of the header: 61 - e with n (t - a) < 2^e (w in u = log1p(x - xmin) for the log
    driver)."""
    g = gbs()
    if st.driver == g.GBS_DRIVER_LOG:
        w = math.log1p(st.t - st.xmin) - math.log1p(st.a - st.xmin)
    else:
        w = st.t - st.a
    bound = st.n * max(w, 0.0)
    if not (0.0 < bound < math.inf):
        return 0
    _, e = math.frexp(bound)
    return max(-1000, min(1000, 61 - e))


class FakeDeviceCtx:
    """Stand-in for a Context on CPU tensors: the device-loop calls by their stated
    semantics (test infrastructure), the rest by the oracle."""

    def __init__(self):
        import torch
        self.device = 0
        self.torch_device = torch.device("cpu")
        self.g = gbs()

    def _state(self, d_state):
        return self.g.gbs_shard_state.from_buffer_copy(bytes(d_state.numpy()))

    def array_stats(self, x):
        from test_sharded import NumpyBackend
        return NumpyBackend().stats(x.numpy())

    def compact(self, x, a, b):
        import torch
        v = x.numpy()
        a, b = v.dtype.type(a), v.dtype.type(b)
        return torch.from_numpy(np.ascontiguousarray(v[(v > a) & (v <= b)]))

    def select_kth(self, z, r):
        import torch
        return torch.tensor([osel.select_kth(z.numpy(), r)], dtype=torch.float64)

    def shard_pass_dev(self, x, d_state, d_acc):
        st = self._state(d_state)
        if st.phase != self.g.GBS_SHARD_ITERATE or int(d_acc[4]) != 0:
            return
        v = x.numpy()
        a, t = v.dtype.type(st.a), v.dtype.type(st.t)
        inner = v[(v > a) & (v < t)].astype(np.float64)
        if st.driver == self.g.GBS_DRIVER_LOG:
            S = float(np.sum(math.log1p(float(t) - st.xmin) - np.log1p(inner - st.xmin)))
        else:
            S = float(np.sum(float(t) - inner))
        d_acc[0] += int((v < t).sum())
        d_acc[1] += int((v <= t).sum())
        d_acc[2] += int((v <= a).sum())
        d_acc[3] += int(round(math.ldexp(S, sfix_bits(st))))

    def shard_passes_dev(self, shards, d_state, d_acc, step=False):
        def run():
            for x in shards:
                self.shard_pass_dev(x, d_state, d_acc)
            if step:
                self.shard_step_dev(d_state, d_acc)
        return run

    def shard_step_dev(self, d_state, d_acc):
        import torch
        g = self.g
        st = self._state(d_state)
        if int(d_acc[4]) == 0 and st.phase == g.GBS_SHARD_ITERATE:
            e = g.gbs_cost_eval()
            e.c_lt_t, e.c_le_t, e.c_le_a = int(d_acc[0]), int(d_acc[1]), int(d_acc[2])
            e.S = math.ldexp(float(int(d_acc[3])), -sfix_bits(st))
            r = g.gbs_shard_update(C.byref(st), C.byref(e))
            if r == g.GBS_OK and st.phase == g.GBS_SHARD_ITERATE:
                r = g.gbs_shard_next(C.byref(st))
            if r == g.GBS_OK:
                d_state.copy_(torch.frombuffer(bytearray(bytes(st)), dtype=torch.uint8))
            else:
                d_acc[4] = r
        d_acc[:4] = 0


def _data(layout):
    if layout == "two_each":
        return synth.heavy_mixture("mixture", 40009, seed=11)
    return synth.heavy_mixture("cauchy", 40009, seed=12, dtype=np.float64)


def _rank_main(rank, world, port, out, layout, driver):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_1104_2732_gb300.sharded import select_kth_sharded_device
        x = _data(layout)
        if layout == "two_each":
            own = split(x, 2 * world, seed=3)[rank * 2:(rank + 1) * 2]
        else:
            own = [x] if rank == 0 else []                      # the other ranks hold nothing
        own = [torch.from_numpy(np.ascontiguousarray(p)) for p in own]
        res = []
        for k in RANKS:
            info = {}
            res.append(select_kth_sharded_device(own, k, FakeDeviceCtx(), elem_bytes=x.itemsize, cap=1000,
                                                 driver=driver, check_every=3, info=info))
        out.put((rank, res))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("layout,world,driver", [("two_each", 2, "kelley"), ("one_rank_holds_all", 3, "kelley"),
                                                 ("two_each", 2, "log")])
def test_device_loop_over_gloo_ranks(layout, world, driver):
    gbs()
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q, layout, driver)) for r in range(world)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=240) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    x = _data(layout)
    want = [osel.select_kth(x, k) for k in RANKS]
    for r in range(world):
        assert [bits(v, x.dtype) for v in got[r]] == [bits(v, x.dtype) for v in want], (r, got[r], want)


def test_fixed_point_bits_bound_the_total():
    """The cost total at fx stays below 2^61 for any data in (a, t): n terms of at most w."""
    g = gbs()
    st = g.gbs_shard_state()
    for n, a, t in ((10, 0.0, 1.0), (1 << 40, -1e30, 3e38), (5, 1.0, 1.0 + 2 ** -40), (1 << 31, -2.5, 7.0)):
        st.n, st.a, st.t, st.driver = n, a, t, g.GBS_DRIVER_KELLEY
        fx = sfix_bits(st)
        assert n * (t - a) * 2.0 ** fx < 2.0 ** 61
        assert n * (t - a) * 2.0 ** fx >= 2.0 ** 60                 # and uses the range


@pytest.mark.gpu
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("driver", ["kelley", "log", "bisect"])
def test_device_loop_matches_oracle_on_gpu(lib, dtype, driver):
    import torch
    from paper_1104_2732_gb300.sharded import GpuBackend, select_kth_sharded, select_kth_sharded_device
    ctx = lib.Context()
    try:
        for fam, n in (("mixture", 3_000_017), ("lognormal", 777_777)):
            x = synth.heavy_mixture(fam, n, seed=31, dtype=dtype)
            parts = split(x, 3, seed=6)
            shards = [torch.from_numpy(np.ascontiguousarray(p)).cuda() for p in parts] + \
                     [torch.empty(0, dtype=shards_dtype(dtype), device="cuda")]
            for k in (1, n // 100, (n + 1) // 2, n - n // 100, n):
                info = {}
                got = select_kth_sharded_device(shards, k, ctx, elem_bytes=x.itemsize, driver=driver, info=info)
                want = osel.select_kth(x, k)
                assert bits(got, dtype) == bits(want, dtype), (fam, k, driver, got, want)
                host = select_kth_sharded(shards, k, GpuBackend(ctx), elem_bytes=x.itemsize, driver=driver)
                assert bits(host, dtype) == bits(got, dtype)
    finally:
        ctx.close()


def shards_dtype(dtype):
    import torch
    return torch.float32 if dtype == np.float32 else torch.float64


@pytest.mark.gpu
def test_device_loop_with_nccl_group_of_one(lib):
    """The all-reduce path with NCCL (a group of one rank on this device)."""
    import torch
    import torch.distributed as dist
    from paper_1104_2732_gb300.sharded import TorchComm, select_kth_sharded_device
    dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{_free_port()}", rank=0, world_size=1,
                            device_id=torch.device("cuda", 0))
    ctx = lib.Context()
    try:
        assert TorchComm().device.type == "cuda"          # NCCL reduces device tensors
        x = synth.heavy_mixture("mixture", 2_000_003, seed=32)
        shards = [torch.from_numpy(np.ascontiguousarray(p)).cuda() for p in split(x, 4, seed=7)]
        for k in (20_000, 1_000_002, 1_990_000):           # ranks past the 5 -inf: they iterate
            info = {}
            got = select_kth_sharded_device(shards, k, ctx, elem_bytes=4, info=info)
            assert bits(got, np.float32) == bits(osel.select_kth(x, k), np.float32), k
            assert info["passes"] >= 1
    finally:
        ctx.close()
        dist.destroy_process_group()


@pytest.mark.gpu
def test_device_entry_points_check_arguments(lib):
    import torch
    g = gbs()
    ctx = lib.Context()
    try:
        st = torch.zeros(C.sizeof(g.gbs_shard_state), dtype=torch.uint8, device="cuda")
        acc = torch.zeros(8, dtype=torch.int64, device="cuda")
        x = torch.zeros(16, device="cuda")
        P = C.c_void_p
        h = ctx._h
        assert g.gbs_shard_pass_dev_f32(h, P(x.data_ptr()), -1, P(st.data_ptr()), P(acc.data_ptr()), None) == g.GBS_EINVAL
        assert g.gbs_shard_pass_dev_f32(h, P(x.data_ptr()), 16, None, P(acc.data_ptr()), None) == g.GBS_EINVAL
        assert g.gbs_shard_pass_dev_f32(h, P(x.data_ptr()), 16, P(st.data_ptr()), P(acc.data_ptr() + 4), None) == g.GBS_EINVAL
        assert g.gbs_shard_step_dev(h, P(st.data_ptr()), None, None) == g.GBS_EINVAL
        assert g.gbs_shard_pass_dev_f32(h, P(x.data_ptr()), 0, P(st.data_ptr()), P(acc.data_ptr()), None) == g.GBS_OK
        # a state that is not ITERATE: both calls leave the accumulator alone
        st.view(torch.int32)[g.gbs_shard_state.phase.offset // 4] = g.GBS_SHARD_DONE
        acc.fill_(7)
        acc[4] = 0
        assert g.gbs_shard_pass_dev_f32(h, P(x.data_ptr()), 16, P(st.data_ptr()), P(acc.data_ptr()), None) == g.GBS_OK
        torch.cuda.synchronize()
        assert acc[:4].tolist() == [7, 7, 7, 7]
    finally:
        ctx.close()
