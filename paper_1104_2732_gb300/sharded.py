"""Selection over a vector split into shards: Algorithm 1 (Sec. 3) with the per-pass
results of the shards summed between passes, as the paper's multi-GPU remark (Sec. 4)
sums the per-device reductions on the host.

The scalar steps are the library's host functions ``gbs_shard_begin`` /
``gbs_shard_next`` / ``gbs_shard_update`` (include/gbselect.h); every per-element pass
runs on a shard through a *backend*, and the per-pass totals are formed by a *comm*:

* backend (per-shard work): ``stats(x) -> dict`` (the gbs_array_stats fields),
  ``cost_pass(x, a, t) -> dict`` (c_lt_t, c_le_t, c_le_a, S), ``cost_pass_log(x, a, t,
  xmin)`` (the same with S in the coordinates u = log1p(x - xmin), for the log driver),
  ``compact(x, a, b) ->
  shard's elements of (a, b]``, ``select(z, r) -> z_(r)``, ``concat(list)`` and
  ``empty(elem_bytes)`` (a set of no elements, for a process that holds none).
  :class:`GpuBackend` runs them with a :class:`~paper_1104_2732_gb300.Context`.
* comm (totals over processes): ``sum_i64``, ``sum_f64``, ``min_f64``, ``max_f64`` on
  lists of numbers and ``gather(z)`` of the compacted sets.  :class:`LocalComm` is one
  process holding every shard (host-simulated shards); :class:`TorchComm` uses
  ``torch.distributed`` (one or more shards per rank; the collectives are one small
  all-reduce per pass and one all-gather of at most cap elements at the end).

:func:`select_kth_sharded_device` keeps the cutting-plane loop on the device instead:
the state lives in device memory, each pass adds the shards' counts and fixed-point
cost into one device accumulator that the ranks all-reduce in place, and a one-thread
step advances the state with the host API's own code (no host round trip per pass).

The result equals the single-array result bit for bit.
"""
from __future__ import annotations

import ctypes as C
import math

from . import (DRIVERS, GBS_DRIVER_LOG, GBS_EINTERNAL, GBS_OK, GBS_SHARD_COMPACT, GBS_SHARD_DONE,
               GBS_SHARD_ITERATE, GBS_SHARD_NAN, GBS_ENAN, GbsError, gbs_array_stats, gbs_cost_eval, gbs_shard_begin, gbs_shard_next,
               gbs_shard_set_driver, gbs_shard_state, gbs_shard_update)

_STAT_SUMS = ("n", "n_nan", "n_neginf", "n_posinf", "n_negzero", "n_finite")
_EVAL_SUMS = ("c_lt_t", "c_le_t", "c_le_a")


def _check(status, what):
    if status != GBS_OK:
        raise GbsError(status, what)


class LocalComm:
    """Every shard lives in this process: the totals are the local sums."""

    def sum_i64(self, v):
        return [int(a) for a in v]

    def sum_f64(self, v):
        return [float(a) for a in v]

    def min_f64(self, v):
        return [float(a) for a in v]

    def max_f64(self, v):
        return [float(a) for a in v]

    def gather(self, z, backend):
        return z


class TorchComm:
    """Totals over the ranks of a torch.distributed process group; ``device`` is where
    the small reduction tensors live: by default the current CUDA device when the group's
    backend is NCCL (which reduces device tensors only), else the CPU (gloo)."""

    def __init__(self, group=None, device=None):
        import torch
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        if device is None:
            nccl = dist.get_backend(group) == "nccl"
            device = torch.device("cuda", torch.cuda.current_device()) if nccl else torch.device("cpu")
        self.device = device

    def _reduce(self, v, dtype, op):
        import torch
        t = torch.tensor(v, dtype=dtype, device=self.device)
        self.dist.all_reduce(t, op=op, group=self.group)
        return t.cpu().tolist()

    def sum_i64(self, v):
        import torch
        return [int(a) for a in self._reduce(v, torch.int64, self.dist.ReduceOp.SUM)]

    def sum_f64(self, v):
        import torch
        return self._reduce(v, torch.float64, self.dist.ReduceOp.SUM)

    def min_f64(self, v):
        import torch
        return self._reduce(v, torch.float64, self.dist.ReduceOp.MIN)

    def max_f64(self, v):
        import torch
        return self._reduce(v, torch.float64, self.dist.ReduceOp.MAX)

    def gather(self, z, backend):
        """Concatenation over the ranks (rank order) of each rank's compacted set."""
        import numpy as np
        import torch
        if not isinstance(z, torch.Tensor):
            z = torch.from_numpy(np.ascontiguousarray(z))
        world = self.dist.get_world_size(self.group)
        n = torch.tensor([z.numel()], dtype=torch.int64, device=self.device)
        sizes = [torch.zeros_like(n) for _ in range(world)]
        self.dist.all_gather(sizes, n, group=self.group)
        sizes = [int(s.item()) for s in sizes]
        m = max(sizes)
        buf = torch.zeros(m, dtype=z.dtype, device=z.device)
        buf[:z.numel()] = z
        parts = [torch.zeros_like(buf) for _ in range(world)]
        self.dist.all_gather(parts, buf, group=self.group)
        return backend.concat([p[:s] for p, s in zip(parts, sizes)])


class GpuBackend:
    """Per-shard passes with the library's kernels (shards: contiguous CUDA tensors)."""

    def __init__(self, ctx):
        self.ctx = ctx

    def stats(self, x):
        return self.ctx.array_stats(x)

    def cost_pass(self, x, a, t):
        return self.ctx.cost_pass(x, 1, a, t)

    def cost_pass_log(self, x, a, t, xmin):
        return self.ctx.cost_pass_log(x, 1, a, t, xmin)

    def compact(self, x, a, b):
        return self.ctx.compact(x, a, b)

    def concat(self, zs):
        import torch
        return torch.cat(list(zs)) if zs else None

    def empty(self, elem_bytes):
        import torch
        return torch.empty(0, dtype=torch.float32 if elem_bytes == 4 else torch.float64,
                           device=self.ctx.torch_device)

    def select(self, z, r):
        return float(self.ctx.select_kth(z, r).item())


def _begin(shards, k, backend, comm, elem_bytes, cap, maxit, driver):
    """Pass 0 on every shard (Sec. 3, step 0), its totals over the shards and processes,
    and the state of gbs_shard_begin with the chosen driver."""
    st = [backend.stats(s) for s in shards]
    sums = comm.sum_i64([sum(int(r[f]) for r in st) for f in _STAT_SUMS])
    fin = [r for r in st if int(r["n_finite"]) > 0]
    total = gbs_array_stats()
    for f, v in zip(_STAT_SUMS, sums):
        setattr(total, f, v)
    total.sum = comm.sum_f64([math.fsum(float(r["sum"]) for r in fin)])[0]
    total.min = comm.min_f64([min((float(r["min"]) for r in fin), default=math.inf)])[0]
    total.max = comm.max_f64([max((float(r["max"]) for r in fin), default=-math.inf)])[0]
    if total.n_finite == 0:
        total.min = total.max = 0.0
    state = gbs_shard_state()
    _check(gbs_shard_begin(C.byref(state), int(elem_bytes), total.n, int(k), C.byref(total), int(cap), int(maxit)),
           "gbs_shard_begin")
    _check(gbs_shard_set_driver(C.byref(state), DRIVERS[driver]), "gbs_shard_set_driver")
    return state


def _finish(state, shards, k, backend, comm, elem_bytes):
    """The end of a sharded selection: the result, or the finish over (a, b] (Sec. 3)."""
    if state.phase == GBS_SHARD_NAN:
        raise GbsError(GBS_ENAN, "select_kth_sharded")
    if state.phase == GBS_SHARD_DONE:
        return state.result
    assert state.phase == GBS_SHARD_COMPACT
    local = [backend.compact(s, state.a, state.b) for s in shards]
    z = comm.gather(backend.concat(local) if local else backend.empty(elem_bytes), backend)
    r = int(k - state.cle_a)
    return backend.select(z, r)


def select_kth_sharded_device(shards, k, ctx, group=None, elem_bytes=4, cap=0, maxit=0, driver="kelley",
                              check_every=4, info=None):
    """x_(k) of the concatenation of the shards of every rank, with the cutting-plane
    loop resident on the device: per pass, each shard's gbs_shard_pass_dev adds its
    counts and fixed-point cost into one device int64[8]; with a process group the ranks
    sum it in place by one all_reduce (NCCL on the device, stream-ordered); then
    gbs_shard_step_dev updates the device state.  Nothing returns to the host during a
    pass: the phase is read back every ``check_every`` passes.  Pass 0 and the finish
    (compaction, one all_gather, select) are as in :func:`select_kth_sharded`.

    ``shards``: this rank's CUDA tensors on ``ctx``'s device (any number, empty allowed).
    ``group``: a torch.distributed group, or None for the default group when one is
    initialised (else this process alone).  ``info`` (a dict) receives the passes taken.
    The result equals the single-array result bit for bit."""
    import torch
    import torch.distributed as dist
    backend = GpuBackend(ctx)
    distributed = group is not None or (dist.is_available() and dist.is_initialized())
    comm = TorchComm(group) if distributed else LocalComm()
    shards = [s for s in shards if s is not None and len(s) > 0]
    state = _begin(shards, k, backend, comm, elem_bytes, cap, maxit, driver)
    if state.phase == GBS_SHARD_ITERATE:
        _check(gbs_shard_next(C.byref(state)), "gbs_shard_next")
    passes = 0
    if state.phase == GBS_SHARD_ITERATE:
        dev = ctx.torch_device
        nbytes = C.sizeof(gbs_shard_state)
        d_state = torch.frombuffer(bytearray(bytes(state)), dtype=torch.uint8).to(dev)
        d_acc = torch.zeros(8, dtype=torch.int64, device=dev)
        limit = int(state.maxit) + 2 * check_every + 2   # passes before the state must have left ITERATE
        # one ABI call a pass over this rank's shards (and the step with it when alone)
        run = ctx.shard_passes_dev(shards, d_state, d_acc, step=not distributed) if shards else None
        while True:
            for _ in range(check_every):
                if distributed:
                    if run is not None:
                        run()
                    dist.all_reduce(d_acc[:4], group=group)
                    ctx.shard_step_dev(d_state, d_acc)
                else:
                    run()
                passes += 1
            raw = d_state.cpu().numpy().tobytes()
            status = int(d_acc[4].item())
            if status != 0:
                raise GbsError(status, "gbs_shard_step_dev")
            state = gbs_shard_state.from_buffer_copy(raw[:nbytes])
            if state.phase != GBS_SHARD_ITERATE:
                break
            if passes > limit:
                raise GbsError(GBS_EINTERNAL, "select_kth_sharded_device")
    if info is not None:
        info["passes"] = int(state.it)
        info["launched_passes"] = passes
    return _finish(state, shards, k, backend, comm, elem_bytes)


def select_kth_sharded(shards, k, backend, comm=None, elem_bytes=4, cap=0, maxit=0, trace=None, driver="kelley"):
    """x_(k) of the concatenation of the shards of every process (1-based k).

    ``shards``: this process's shards (any number, empty ones allowed: a process with no
    element still takes part in every collective, with zero counts and an empty set at
    the gather); ``k`` is the rank in the whole vector.  ``driver`` picks the next point:
    "kelley" (the cutting plane, Algorithm 1), "bisect", "brent" (root-finding on the
    subgradient) or "log" (Kelley on u = log1p(x - xmin)), the paper's comparisons; the
    result does not depend on it.  Returns a Python float holding the element (``-0.0``
    kept)."""
    comm = comm or LocalComm()
    shards = [s for s in shards if s is not None and len(s) > 0]
    state = _begin(shards, k, backend, comm, elem_bytes, cap, maxit, driver)
    log = state.driver == GBS_DRIVER_LOG
    # cutting-plane passes (Algorithm 1, steps 1.1-1.4)
    while state.phase == GBS_SHARD_ITERATE:
        _check(gbs_shard_next(C.byref(state)), "gbs_shard_next")
        if state.phase != GBS_SHARD_ITERATE:
            break
        a, t = state.a, state.t
        ev = [backend.cost_pass_log(s, a, t, state.xmin) if log else backend.cost_pass(s, a, t) for s in shards]
        tot = gbs_cost_eval()
        for f, v in zip(_EVAL_SUMS, comm.sum_i64([sum(int(r[f]) for r in ev) for f in _EVAL_SUMS])):
            setattr(tot, f, v)
        tot.S = comm.sum_f64([math.fsum(float(r["S"]) for r in ev)])[0]
        if trace is not None:
            trace.append(t)
        _check(gbs_shard_update(C.byref(state), C.byref(tot)), "gbs_shard_update")
    return _finish(state, shards, k, backend, comm, elem_bytes)
