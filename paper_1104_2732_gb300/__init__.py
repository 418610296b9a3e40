"""Python binding of libgbselect (exact order statistics on GB300).

Argument marshalling only: every step of the selection runs in the library's CUDA
kernels.  The raw C entry points are exposed under their C names (``gbs_select_kth_f32``
and so on, see include/gbselect.h); :class:`Context` wraps them for torch tensors.
Importing fails loudly if the library has not been built (``python
paper_1104_2732_gb300/build.py``); there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libgbselect.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python paper_1104_2732_gb300/build.py`")
_lib = C.CDLL(LIB_PATH)

# ------------------------------------------------------------------ status codes
GBS_OK, GBS_EINVAL, GBS_ENAN, GBS_ENOMEM, GBS_ECUDA, GBS_ETIMEOUT, GBS_EINTERNAL = range(7)
HOW = {0: "none", 1: "neginf", 2: "posinf", 3: "min", 4: "max", 5: "hit", 6: "finish"}


class GbsError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = int(status)
        msg = _lib.gbs_status_string(self.status).decode()
        super().__init__(f"{what}: {msg} (status {self.status})" if what else msg)


# ------------------------------------------------------------------ structures
class gbs_config(C.Structure):
    _fields_ = [("cap", C.c_int64), ("maxit", C.c_int32), ("blocks_per_sm", C.c_int32),
                ("use_learned", C.c_int32), ("lms_start", C.c_int32), ("knn_start", C.c_int32),
                ("reserved", C.c_int32 * 5)]


class gbs_run_stats(C.Structure):
    _fields_ = [("status", C.c_int32), ("how", C.c_int32), ("passes", C.c_int32),
                ("kelley_steps", C.c_int32), ("bisect_steps", C.c_int32), ("finish_rounds", C.c_int32),
                ("grid", C.c_int32), ("learned", C.c_int32), ("n", C.c_int64), ("k", C.c_int64),
                ("finish_pop", C.c_int64), ("pops", C.c_int64 * 64), ("iterates", C.c_double * 64),
                ("t_ns", C.c_uint64 * 72), ("t_stream_ns", C.c_uint64 * 64), ("n_t", C.c_int32),
                ("pad", C.c_int32)]


class gbs_array_stats(C.Structure):
    _fields_ = [("n", C.c_int64), ("n_nan", C.c_int64), ("n_neginf", C.c_int64), ("n_posinf", C.c_int64),
                ("n_negzero", C.c_int64), ("n_finite", C.c_int64), ("min", C.c_double), ("max", C.c_double),
                ("c_le_min", C.c_int64), ("c_lt_max", C.c_int64), ("sum", C.c_double)]


class gbs_cost_eval(C.Structure):
    _fields_ = [("c_lt_t", C.c_int64), ("c_le_t", C.c_int64), ("c_le_a", C.c_int64), ("pad", C.c_int64),
                ("S", C.c_double), ("dphi", C.c_double)]


class gbs_shard_state(C.Structure):
    _fields_ = [("n", C.c_int64), ("k", C.c_int64), ("cap", C.c_int64), ("maxit", C.c_int32),
                ("elem_bytes", C.c_int32), ("phase", C.c_int32), ("how", C.c_int32), ("it", C.c_int32),
                ("use_bisect", C.c_int32), ("stalled", C.c_int32), ("dfv", C.c_int32), ("n_neginf", C.c_int64),
                ("n_negzero", C.c_int64), ("cle_a", C.c_int64), ("clt_b", C.c_int64), ("cle_b", C.c_int64),
                ("a", C.c_double), ("b", C.c_double), ("t", C.c_double), ("dF", C.c_double),
                ("result", C.c_double), ("driver", C.c_int32), ("pad2", C.c_int32), ("xmin", C.c_double),
                ("px", C.c_double), ("pg", C.c_double), ("step1", C.c_double), ("step2", C.c_double)]


class gbs_knn_stats(C.Structure):
    _fields_ = [("queries", C.c_int64), ("plain_queries", C.c_int64), ("passes", C.c_int32),
                ("pass_launches", C.c_int32), ("pass_ms", C.c_double)]


class gbs_lms_stats(C.Structure):
    _fields_ = [("passes", C.c_int32), ("pass_launches", C.c_int32), ("pass_ms", C.c_double),
                ("write_ms", C.c_double)]


GBS_SHARD_ITERATE, GBS_SHARD_DONE, GBS_SHARD_COMPACT, GBS_SHARD_NAN = range(4)
GBS_DRIVER_KELLEY, GBS_DRIVER_BISECT, GBS_DRIVER_BRENT, GBS_DRIVER_LOG = range(4)
DRIVERS = {"kelley": GBS_DRIVER_KELLEY, "bisect": GBS_DRIVER_BISECT, "brent": GBS_DRIVER_BRENT, "log": GBS_DRIVER_LOG}

_P = C.c_void_p
_I64 = C.c_int64
_SIGS = {
    "gbs_create": (C.c_int, [C.POINTER(_P), C.c_int]),
    "gbs_destroy": (None, [_P]),
    "gbs_reserve": (C.c_int, [_P, _I64, C.c_int32]),
    "gbs_set_config": (C.c_int, [_P, C.POINTER(gbs_config)]),
    "gbs_get_config": (C.c_int, [_P, C.POINTER(gbs_config)]),
    "gbs_select_kth_f32": (C.c_int, [_P, _P, _I64, _I64, _P, _P]),
    "gbs_select_kth_f64": (C.c_int, [_P, _P, _I64, _I64, _P, _P]),
    "gbs_median_f32": (C.c_int, [_P, _P, _I64, _P, _P]),
    "gbs_median_f64": (C.c_int, [_P, _P, _I64, _P, _P]),
    "gbs_array_stats_f32": (C.c_int, [_P, _P, _I64, _P, _P]),
    "gbs_array_stats_f64": (C.c_int, [_P, _P, _I64, _P, _P]),
    "gbs_cost_pass_f32": (C.c_int, [_P, _P, _I64, _I64, C.c_double, C.c_double, _P, _P]),
    "gbs_cost_pass_f64": (C.c_int, [_P, _P, _I64, _I64, C.c_double, C.c_double, _P, _P]),
    "gbs_last_stats": (C.c_int, [_P, C.POINTER(gbs_run_stats)]),
    "gbs_select_kth_f32_noalloc": (C.c_int, [_P, _I64, _I64, _P, _P]),
    "gbs_select_segmented_f32": (C.c_int, [_P, _P, _P, C.c_int32, _P, _P, _P]),
    "gbs_segmented_autotune_f32": (C.c_int, [_P, _P, _P, C.c_int32, _P, _P, _P, C.POINTER(C.c_int32),
                                             C.POINTER(C.c_float), C.c_int32]),
    "gbs_segmented_set_variant": (C.c_int, [_P, C.c_int32]),
    "gbs_segmented_get_variant": (C.c_int, [_P, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                            C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "gbs_segmented_passes": (C.c_int, [_P, C.POINTER(C.c_int32), C.c_int32]),
    "gbs_residual_sq_f32": (C.c_int, [_P, _P, _P, _I64, C.c_int32, _P, C.c_int32, _P, C.c_int32, _P]),
    "gbs_lms_lts_f32": (C.c_int, [_P, _P, _P, _I64, C.c_int32, _P, C.c_int32, _I64, _I64, _P, _P, C.c_int32,
                                  C.c_int32, _P]),
    "gbs_lms_lts_fused_f32": (C.c_int, [_P, _P, _P, _I64, C.c_int32, _P, C.c_int32, _I64, _I64, _P, _P,
                                        C.POINTER(C.c_int32), _P]),
    "gbs_lts_csteps_f32": (C.c_int, [_P, _P, _P, _I64, C.c_int32, _P, C.c_int32, _I64, C.c_int32, _P, _P, _P, _P]),
    "gbs_lms_lts_search_f32": (C.c_int, [_P, _P, _P, _I64, C.c_int32, _P, C.c_int32, _I64, _I64, C.c_int32, C.c_int32,
                                         _P, _P, _P, _P, _P, _P, _P]),
    "gbs_knn_regress_f32": (C.c_int, [_P, _P, _I64, C.c_int32, _P, _P, C.c_int32, _I64, C.c_int32, C.c_double, _P,
                                      _P, _P]),
    "gbs_knn_classify_f32": (C.c_int, [_P, _P, _I64, C.c_int32, _P, C.c_int32, _P, C.c_int32, _I64, _P, _P, _P,
                                       _P]),
    "gbs_knn_last_stats": (C.c_int, [_P, C.POINTER(gbs_knn_stats)]),
    "gbs_lms_last_stats": (C.c_int, [_P, C.POINTER(gbs_lms_stats)]),
    "gbs_bracket_model_set": (C.c_int, [_P, C.POINTER(C.c_float), C.c_int32]),
    "gbs_bracket_model_get": (C.c_int, [_P, C.POINTER(C.c_float), C.c_int32]),
    "gbs_bracket_model_save": (C.c_int, [_P, C.c_char_p]),
    "gbs_bracket_model_load": (C.c_int, [_P, C.c_char_p]),
    "gbs_bracket_features_f32": (C.c_int, [_P, _P, _I64, _P, _P, _P]),
    "gbs_bracket_propose_f32": (C.c_int, [_P, _P, _I64, _P, _P]),
    "gbs_bracket_forward": (C.c_int, [_P, _P, C.c_int32, _P, _P]),
    "gbs_bracket_grad": (C.c_int, [_P, _P, _P, C.c_int32, _P, _P, _P]),
    "gbs_bracket_train": (C.c_int, [_P, _P, _P, C.c_int32, C.c_int32, C.c_int32, C.c_float, C.c_uint64,
                                    C.POINTER(C.c_float), _P]),
    "gbs_generate_training_array_f32": (C.c_int, [_P, _P, _I64, C.c_int32, C.c_float, C.c_float, C.c_float,
                                                  C.c_float, C.c_float, C.c_uint64, _P]),
    "gbs_philox4x32_10": (C.c_int, [_P, _P, _P, _P, C.c_int32, _P]),
    "gbs_shard_begin": (C.c_int, [C.POINTER(gbs_shard_state), C.c_int32, _I64, _I64, C.POINTER(gbs_array_stats),
                                  _I64, C.c_int32]),
    "gbs_shard_next": (C.c_int, [C.POINTER(gbs_shard_state)]),
    "gbs_shard_update": (C.c_int, [C.POINTER(gbs_shard_state), C.POINTER(gbs_cost_eval)]),
    "gbs_shard_set_driver": (C.c_int, [C.POINTER(gbs_shard_state), C.c_int32]),
    "gbs_cost_pass_log_f32": (C.c_int, [_P, _P, _I64, _I64, C.c_double, C.c_double, C.c_double, _P, _P]),
    "gbs_cost_pass_log_f64": (C.c_int, [_P, _P, _I64, _I64, C.c_double, C.c_double, C.c_double, _P, _P]),
    "gbs_compact_f32": (C.c_int, [_P, _P, _I64, C.c_double, C.c_double, _P, _I64, C.POINTER(_I64), _P]),
    "gbs_compact_f64": (C.c_int, [_P, _P, _I64, C.c_double, C.c_double, _P, _I64, C.POINTER(_I64), _P]),
    "gbs_shard_pass_dev_f32": (C.c_int, [_P, _P, _I64, _P, _P, _P]),
    "gbs_shard_pass_dev_f64": (C.c_int, [_P, _P, _I64, _P, _P, _P]),
    "gbs_shard_step_dev": (C.c_int, [_P, _P, _P, _P]),
    "gbs_shard_passes_dev_f32": (C.c_int, [_P, C.POINTER(_P), C.POINTER(_I64), C.c_int32, _P, _P, C.c_int32, _P]),
    "gbs_shard_passes_dev_f64": (C.c_int, [_P, C.POINTER(_P), C.POINTER(_I64), C.c_int32, _P, _P, C.c_int32, _P]),
    "gbs_status_string": (C.c_char_p, [C.c_int]),
    "gbs_check_wait_timeout": (C.c_int, [_P, _I64, C.POINTER(C.c_int32), _P]),
}


def _bind(table):
    for name, (res, args) in table.items():
        try:
            fn = getattr(_lib, name)
        except AttributeError as e:
            raise ImportError(f"{LIB_PATH} lacks {name}: rebuild it with `python paper_1104_2732_gb300/build.py`") from e
        fn.restype = res
        fn.argtypes = args
        globals()[name] = fn


_bind(_SIGS)
EXPORTED = tuple(_SIGS)


def _check(status, what):
    if status != GBS_OK:
        raise GbsError(status, what)


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(int(stream.cuda_stream))


def _suffix(x):
    import torch
    if x.dtype == torch.float32:
        return "f32"
    if x.dtype == torch.float64:
        return "f64"
    raise TypeError(f"float32 or float64 expected, got {x.dtype}")


def _require(t, name, dtype=None, dim=None, cols=None, numel=None, min_numel=None, device=None):
    """Checks a tensor before its pointer crosses the ABI, where the kernels take sizes
    from the other arguments: element type, rank, row width and element count first (a
    short buffer would be read or written past its end), then that it is a contiguous
    CUDA tensor on the context's device."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name}: a torch tensor is required")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name}: {dtype} expected, got {t.dtype}")
    if dim is not None and t.dim() != dim:
        raise ValueError(f"{name}: {dim}-d expected, got shape {tuple(t.shape)}")
    if cols is not None and t.shape[-1] != cols:
        raise ValueError(f"{name}: rows of {cols} expected, got shape {tuple(t.shape)}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name}: {numel} elements expected, got {t.numel()}")
    if min_numel is not None and t.numel() < min_numel:
        raise ValueError(f"{name}: at least {min_numel} elements expected, got {t.numel()}")
    if not t.is_cuda:
        raise TypeError(f"{name}: a CUDA tensor is required")
    if not t.is_contiguous():
        raise ValueError(f"{name}: a contiguous tensor is required")
    if device is not None and t.device.index != device:
        raise ValueError(f"{name} is on cuda:{t.device.index}, the context on cuda:{device}")
    return t



class Context:
    """Owns a gbs_ctx (workspace, configuration) on one CUDA device."""

    def __init__(self, device=None):
        import torch
        if device is None:
            device = torch.cuda.current_device()
        self.device = int(device)
        h = _P()
        _check(gbs_create(C.byref(h), self.device), "gbs_create")
        self._h = h

    @property
    def torch_device(self):
        """The torch device of this context's GPU."""
        import torch
        return torch.device("cuda", self.device)

    def close(self):
        if getattr(self, "_h", None):
            gbs_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def _in(self, t, name, **kw):
        return _require(t, name, device=self.device, **kw)

    # -------------------------------------------------------------- configuration
    def set_config(self, **kw):
        known = {f for f, _ in gbs_config._fields_ if f != "reserved"}
        unknown = sorted(set(kw) - known)
        if unknown:
            raise TypeError(f"unknown configuration keys {unknown}; known: {sorted(known)}")
        cfg = gbs_config()
        _check(gbs_get_config(self._h, C.byref(cfg)), "gbs_get_config")
        for key, val in kw.items():
            setattr(cfg, key, int(val))
        _check(gbs_set_config(self._h, C.byref(cfg)), "gbs_set_config")

    def get_config(self):
        cfg = gbs_config()
        _check(gbs_get_config(self._h, C.byref(cfg)), "gbs_get_config")
        return {"cap": cfg.cap, "maxit": cfg.maxit, "blocks_per_sm": cfg.blocks_per_sm,
                "use_learned": cfg.use_learned, "lms_start": cfg.lms_start, "knn_start": cfg.knn_start}

    def reserve(self, n, elem_bytes=4):
        _check(gbs_reserve(self._h, int(n), int(elem_bytes)), "gbs_reserve")

    # -------------------------------------------------------------- selection
    def select_kth(self, x, k, out=None, stream=None):
        """x_(k) of a contiguous CUDA tensor (1-based k); returns a 1-element device tensor."""
        import torch
        x = self._in(x, "x")
        if out is None:
            out = torch.empty(1, dtype=x.dtype, device=x.device)
        self._in(out, "out", dtype=x.dtype, min_numel=1)
        fn = globals()["gbs_select_kth_" + _suffix(x)]
        _check(fn(self._h, C.c_void_p(x.data_ptr()), x.numel(), int(k), C.c_void_p(out.data_ptr()),
                  _stream_ptr(stream)), "gbs_select_kth")
        return out

    def median(self, x, out=None, stream=None):
        import torch
        x = self._in(x, "x")
        if out is None:
            out = torch.empty(1, dtype=x.dtype, device=x.device)
        self._in(out, "out", dtype=x.dtype, min_numel=1)
        fn = globals()["gbs_median_" + _suffix(x)]
        _check(fn(self._h, C.c_void_p(x.data_ptr()), x.numel(), C.c_void_p(out.data_ptr()),
                  _stream_ptr(stream)), "gbs_median")
        return out

    def array_stats(self, x, stream=None):
        import torch
        x = self._in(x, "x")
        buf = torch.empty(C.sizeof(gbs_array_stats), dtype=torch.uint8, device=x.device)
        fn = globals()["gbs_array_stats_" + _suffix(x)]
        _check(fn(self._h, C.c_void_p(x.data_ptr()), x.numel(), C.c_void_p(buf.data_ptr()),
                  _stream_ptr(stream)), "gbs_array_stats")
        rec = gbs_array_stats.from_buffer_copy(bytes(buf.cpu().numpy()))
        return {f: getattr(rec, f) for f, _ in gbs_array_stats._fields_}

    def cost_pass(self, x, k, a, t, stream=None):
        import torch
        x = self._in(x, "x")
        buf = torch.empty(C.sizeof(gbs_cost_eval), dtype=torch.uint8, device=x.device)
        fn = globals()["gbs_cost_pass_" + _suffix(x)]
        _check(fn(self._h, C.c_void_p(x.data_ptr()), x.numel(), int(k), float(a), float(t),
                  C.c_void_p(buf.data_ptr()), _stream_ptr(stream)), "gbs_cost_pass")
        rec = gbs_cost_eval.from_buffer_copy(bytes(buf.cpu().numpy()))
        return {f: getattr(rec, f) for f, _ in gbs_cost_eval._fields_ if f != "pad"}

    def cost_pass_log(self, x, k, a, t, xmin, stream=None):
        """The pass of gbs_cost_pass_log_*: counts at a and t, and the cost sum in the
        coordinates u = log1p(x - xmin)."""
        import torch
        x = self._in(x, "x")
        buf = torch.empty(C.sizeof(gbs_cost_eval), dtype=torch.uint8, device=x.device)
        fn = globals()["gbs_cost_pass_log_" + _suffix(x)]
        _check(fn(self._h, C.c_void_p(x.data_ptr()), x.numel(), int(k), float(a), float(t), float(xmin),
                  C.c_void_p(buf.data_ptr()), _stream_ptr(stream)), "gbs_cost_pass_log")
        rec = gbs_cost_eval.from_buffer_copy(bytes(buf.cpu().numpy()))
        return {f: getattr(rec, f) for f, _ in gbs_cost_eval._fields_ if f != "pad"}

    def shard_pass_dev(self, x, d_state, d_acc, stream=None):
        """gbs_shard_pass_dev_*: the shard's pass at the device state's (a, t), added into
        d_acc (device int64[8]); d_state is a device uint8 tensor holding one
        gbs_shard_state."""
        import torch
        x = self._in(x, "x")
        self._in(d_state, "d_state", dtype=torch.uint8, numel=C.sizeof(gbs_shard_state))
        self._in(d_acc, "d_acc", dtype=torch.int64, numel=8)
        fn = globals()["gbs_shard_pass_dev_" + _suffix(x)]
        _check(fn(self._h, C.c_void_p(x.data_ptr()), x.numel(), C.c_void_p(d_state.data_ptr()),
                  C.c_void_p(d_acc.data_ptr()), _stream_ptr(stream)), "gbs_shard_pass_dev")

    def shard_passes_dev(self, shards, d_state, d_acc, step=False):
        """A callable that runs one pass over all the shards (gbs_shard_passes_dev_*), then,
        with step, the device step: the tensors are checked and their pointers marshalled
        once, so each call costs one ABI call.  The call runs on the current stream."""
        import torch
        if not shards:
            raise ValueError("shards: at least one shard expected")
        dt = shards[0].dtype
        for i, x in enumerate(shards):
            self._in(x, f"shards[{i}]", dtype=dt)
        self._in(d_state, "d_state", dtype=torch.uint8, numel=C.sizeof(gbs_shard_state))
        self._in(d_acc, "d_acc", dtype=torch.int64, numel=8)
        m = len(shards)
        ptrs = (_P * m)(*[C.c_void_p(x.data_ptr()) for x in shards])
        lens = (_I64 * m)(*[x.numel() for x in shards])
        fn = globals()["gbs_shard_passes_dev_" + _suffix(shards[0])]
        h, sp, ap, st = self._h, C.c_void_p(d_state.data_ptr()), C.c_void_p(d_acc.data_ptr()), int(bool(step))
        keep = (shards, d_state, d_acc)   # the tensors outlive the callable

        def run():
            _check(fn(h, ptrs, lens, m, sp, ap, st, _stream_ptr(None)), "gbs_shard_passes_dev")
        run.keep = keep
        return run

    def shard_step_dev(self, d_state, d_acc, stream=None):
        """gbs_shard_step_dev: bracket update and next point on the device state."""
        import torch
        self._in(d_state, "d_state", dtype=torch.uint8, numel=C.sizeof(gbs_shard_state))
        self._in(d_acc, "d_acc", dtype=torch.int64, numel=8)
        _check(gbs_shard_step_dev(self._h, C.c_void_p(d_state.data_ptr()), C.c_void_p(d_acc.data_ptr()),
                                  _stream_ptr(stream)), "gbs_shard_step_dev")

    def compact(self, x, a, b, z=None, stream=None):
        """The elements of x in (a, b] (any order), as a view of z (allocated with room
        for all of x when None)."""
        import torch
        x = self._in(x, "x")
        if z is None:
            z = torch.empty(x.numel(), dtype=x.dtype, device=x.device)
        self._in(z, "z", dtype=x.dtype)
        cnt = _I64(0)
        fn = globals()["gbs_compact_" + _suffix(x)]
        _check(fn(self._h, C.c_void_p(x.data_ptr()), x.numel(), float(a), float(b), C.c_void_p(z.data_ptr()),
                  z.numel(), C.byref(cnt), _stream_ptr(stream)), "gbs_compact")
        return z[:cnt.value]

    # -------------------------------------------------------------- segmented
    def _seg_args(self, x, offsets, k, out):
        import torch
        x = self._in(x, "x", dtype=torch.float32)
        offsets = self._in(offsets, "offsets", dtype=torch.int64, min_numel=1)
        S = offsets.numel() - 1
        if k is not None:
            k = self._in(k, "k", dtype=torch.int64, numel=S)
        if out is None:
            out = torch.empty(S, dtype=torch.float32, device=x.device)
        self._in(out, "out", dtype=torch.float32, min_numel=S)
        kp = C.c_void_p(k.data_ptr()) if k is not None else None
        return x, offsets, S, kp, out

    def select_segmented(self, x, offsets, k=None, out=None, stream=None):
        """out[s] = x_(k[s]) of x[offsets[s]:offsets[s+1]] (medians when k is None)."""
        x, offsets, S, kp, out = self._seg_args(x, offsets, k, out)
        _check(gbs_select_segmented_f32(self._h, C.c_void_p(x.data_ptr()), C.c_void_p(offsets.data_ptr()), S, kp,
                                        C.c_void_p(out.data_ptr()), _stream_ptr(stream)), "gbs_select_segmented")
        return out

    def autotune_segmented(self, x, offsets, k=None, out=None, stream=None):
        """Times every launch variant on this batch; returns (chosen, ms per variant)."""
        x, offsets, S, kp, out = self._seg_args(x, offsets, k, out)
        nv = C.c_int32()
        _check(gbs_segmented_get_variant(self._h, None, None, None, C.byref(nv)), "gbs_segmented_get_variant")
        ms = (C.c_float * nv.value)()
        chosen = C.c_int32()
        _check(gbs_segmented_autotune_f32(self._h, C.c_void_p(x.data_ptr()), C.c_void_p(offsets.data_ptr()), S, kp,
                                          C.c_void_p(out.data_ptr()), _stream_ptr(stream), C.byref(chosen), ms,
                                          nv.value), "gbs_segmented_autotune")
        return chosen.value, list(ms)

    def segmented_variant(self):
        v, t, c, nv = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
        _check(gbs_segmented_get_variant(self._h, C.byref(v), C.byref(t), C.byref(c), C.byref(nv)),
               "gbs_segmented_get_variant")
        return {"variant": v.value, "threads": t.value, "smem_cap": c.value, "n_variants": nv.value}

    def set_segmented_variant(self, v):
        _check(gbs_segmented_set_variant(self._h, int(v)), "gbs_segmented_set_variant")

    def segmented_passes(self, S):
        buf = (C.c_int32 * int(S))()
        _check(gbs_segmented_passes(self._h, buf, int(S)), "gbs_segmented_passes")
        return list(buf)

    # -------------------------------------------------------------- robust regression
    def _reg_args(self, X, y, theta):
        import torch
        X = self._in(X, "X", dtype=torch.float32, dim=2)
        n, p = X.shape
        y = self._in(y, "y", dtype=torch.float32, numel=n)
        theta = self._in(theta, "theta (C, p): one row of p coefficients per candidate", dtype=torch.float32,
                         dim=2, cols=p)
        return X, y, theta, n, p, theta.shape[0]

    def residual_sq(self, X, y, theta, precision=1, out=None, stream=None):
        """(C, n) float32 squared residuals (y - X theta_c)^2; theta is (C, p)."""
        import torch
        X, y, theta, n, p, Cn = self._reg_args(X, y, theta)
        if out is None:
            out = torch.empty(Cn, n, dtype=torch.float32, device=X.device)
        self._in(out, "out", dtype=torch.float32, min_numel=Cn * n)
        _check(gbs_residual_sq_f32(self._h, C.c_void_p(X.data_ptr()), C.c_void_p(y.data_ptr()), n, p,
                                   C.c_void_p(theta.data_ptr()), Cn, C.c_void_p(out.data_ptr()), int(precision),
                                   _stream_ptr(stream)), "gbs_residual_sq")
        return out

    def lms_lts(self, X, y, theta, k=None, h=None, precision=1, batched=True, stream=None):
        """(LMS, LTS) per candidate: s_(k) and the sum of the h smallest s (float64)."""
        import torch
        X, y, theta, n, p, Cn = self._reg_args(X, y, theta)
        k = (n + 1) // 2 if k is None else int(k)
        h = (n + p + 1) // 2 if h is None else int(h)
        lms = torch.empty(Cn, dtype=torch.float32, device=X.device)
        lts = torch.empty(Cn, dtype=torch.float64, device=X.device)
        _check(gbs_lms_lts_f32(self._h, C.c_void_p(X.data_ptr()), C.c_void_p(y.data_ptr()), n, p,
                               C.c_void_p(theta.data_ptr()), Cn, k, h, C.c_void_p(lms.data_ptr()),
                               C.c_void_p(lts.data_ptr()), int(precision), int(bool(batched)), _stream_ptr(stream)),
               "gbs_lms_lts")
        return lms, lts

    def lms_lts_fused(self, X, y, theta, k=None, h=None, stream=None):
        """(LMS, LTS, passes): the same objectives with the residuals recomputed in every
        pass and never written (gbs_lms_lts_fused_f32)."""
        import torch
        X, y, theta, n, p, Cn = self._reg_args(X, y, theta)
        k = (n + 1) // 2 if k is None else int(k)
        h = (n + p + 1) // 2 if h is None else int(h)
        lms = torch.empty(Cn, dtype=torch.float32, device=X.device)
        lts = torch.empty(Cn, dtype=torch.float64, device=X.device)
        npass = C.c_int32(0)
        _check(gbs_lms_lts_fused_f32(self._h, C.c_void_p(X.data_ptr()), C.c_void_p(y.data_ptr()), n, p,
                                     C.c_void_p(theta.data_ptr()), Cn, k, h, C.c_void_p(lms.data_ptr()),
                                     C.c_void_p(lts.data_ptr()), C.byref(npass), _stream_ptr(stream)),
               "gbs_lms_lts_fused")
        return lms, lts, npass.value

    def lms_last_stats(self):
        """Record of the last gbs_lms_lts_fused_f32 call (synchronises its stream)."""
        rec = gbs_lms_stats()
        _check(gbs_lms_last_stats(self._h, C.byref(rec)), "gbs_lms_last_stats")
        return {f: getattr(rec, f) for f, _ in gbs_lms_stats._fields_}

    def lts_csteps(self, X, y, theta, h=None, max_steps=20, stream=None):
        """(theta_out (C, p) float32, objective (C,) float64, refits (C,) int32): C-steps of
        the LTS objective from every candidate row of theta (gbs_lts_csteps_f32)."""
        import torch
        X, y, theta, n, p, Cn = self._reg_args(X, y, theta)
        h = (n + p + 1) // 2 if h is None else int(h)
        th_out = torch.empty(Cn, p, dtype=torch.float32, device=X.device)
        obj = torch.empty(Cn, dtype=torch.float64, device=X.device)
        ref = torch.empty(Cn, dtype=torch.int32, device=X.device)
        _check(gbs_lts_csteps_f32(self._h, C.c_void_p(X.data_ptr()), C.c_void_p(y.data_ptr()), n, p,
                                  C.c_void_p(theta.data_ptr()), Cn, h, int(max_steps), C.c_void_p(th_out.data_ptr()),
                                  C.c_void_p(obj.data_ptr()), C.c_void_p(ref.data_ptr()), _stream_ptr(stream)),
               "gbs_lts_csteps")
        return th_out, obj, ref

    def lms_lts_search(self, X, y, theta, k=None, h=None, n_refine=10, max_steps=20, stream=None):
        """The LMS and LTS estimates over the candidate rows of theta: a dict of device
        tensors lms_theta, lms_value, lms_index, lts_theta, lts_value, lts_index."""
        import torch
        X, y, theta, n, p, Cn = self._reg_args(X, y, theta)
        k = (n + 1) // 2 if k is None else int(k)
        h = (n + p + 1) // 2 if h is None else int(h)
        dev = X.device
        out = {"lms_theta": torch.empty(p, dtype=torch.float32, device=dev),
               "lms_value": torch.empty(1, dtype=torch.float32, device=dev),
               "lms_index": torch.empty(1, dtype=torch.int32, device=dev),
               "lts_theta": torch.empty(p, dtype=torch.float32, device=dev),
               "lts_value": torch.empty(1, dtype=torch.float64, device=dev),
               "lts_index": torch.empty(1, dtype=torch.int32, device=dev)}
        ptr = {kk: C.c_void_p(v.data_ptr()) for kk, v in out.items()}
        _check(gbs_lms_lts_search_f32(self._h, C.c_void_p(X.data_ptr()), C.c_void_p(y.data_ptr()), n, p,
                                      C.c_void_p(theta.data_ptr()), Cn, k, h, int(n_refine), int(max_steps),
                                      ptr["lms_theta"], ptr["lms_value"], ptr["lms_index"], ptr["lts_theta"],
                                      ptr["lts_value"], ptr["lts_index"], _stream_ptr(stream)), "gbs_lms_lts_search")
        return out

    # -------------------------------------------------------------- kNN
    def _knn_args(self, X, Q, k):
        import torch
        X = self._in(X, "X (n, p points)", dtype=torch.float32, dim=2)
        n, p = X.shape
        Q = self._in(Q, "Q (m, p queries)", dtype=torch.float32, dim=2, cols=p)
        if not 1 <= int(k) <= n:
            raise ValueError(f"k = {k} outside [1, {n}]")
        return X, Q, n, p, Q.shape[0]

    def knn_regress(self, X, f, Q, k, weight="uniform", eps=1e-6, stream=None):
        """(pred, kth_d2): kNN regression of f at every query row of Q (float64) and the
        k-th smallest squared distance per query (float32)."""
        import torch
        X, Q, n, p, m = self._knn_args(X, Q, k)
        f = self._in(f, "f", dtype=torch.float32, numel=n)
        w = {"uniform": 0, "inverse": 1}[weight]
        pred = torch.empty(m, dtype=torch.float64, device=X.device)
        kth = torch.empty(m, dtype=torch.float32, device=X.device)
        _check(gbs_knn_regress_f32(self._h, C.c_void_p(X.data_ptr()), n, p, C.c_void_p(f.data_ptr()),
                                   C.c_void_p(Q.data_ptr()), m, int(k), w, float(eps), C.c_void_p(pred.data_ptr()),
                                   C.c_void_p(kth.data_ptr()), _stream_ptr(stream)), "gbs_knn_regress")
        return pred, kth

    def knn_classify(self, X, labels, n_classes, Q, k, votes=True, stream=None):
        """(cls, votes, kth_d2): the majority class among the k nearest points of every
        query (int32), the vote totals (float64, m x n_classes, or None) and the k-th
        smallest squared distance (float32)."""
        import torch
        X, Q, n, p, m = self._knn_args(X, Q, k)
        labels = self._in(labels, "labels", dtype=torch.int32, numel=n)
        cls = torch.empty(m, dtype=torch.int32, device=X.device)
        v = torch.empty(m, int(n_classes), dtype=torch.float64, device=X.device) if votes else None
        kth = torch.empty(m, dtype=torch.float32, device=X.device)
        _check(gbs_knn_classify_f32(self._h, C.c_void_p(X.data_ptr()), n, p, C.c_void_p(labels.data_ptr()),
                                    int(n_classes), C.c_void_p(Q.data_ptr()), m, int(k), C.c_void_p(cls.data_ptr()),
                                    C.c_void_p(v.data_ptr()) if v is not None else None, C.c_void_p(kth.data_ptr()),
                                    _stream_ptr(stream)), "gbs_knn_classify")
        return cls, v, kth

    def knn_last_stats(self):
        """Record of the last kNN call (synchronises its stream)."""
        rec = gbs_knn_stats()
        _check(gbs_knn_last_stats(self._h, C.byref(rec)), "gbs_knn_last_stats")
        return {f: getattr(rec, f) for f, _ in gbs_knn_stats._fields_}

    # -------------------------------------------------------------- learned bracket
    N_PARAMS = 6658
    N_FEATURES = 36

    def _train_args(self, F, Z):
        import torch
        F = self._in(F, "F (B, 36 features)", dtype=torch.float32, dim=2, cols=self.N_FEATURES)
        Z = self._in(Z, "Z (B standardised medians)", dtype=torch.float32, numel=F.shape[0])
        return F, Z

    def set_bracket_model(self, weights):
        import numpy as np
        w = np.ascontiguousarray(np.asarray(weights, dtype=np.float32).ravel())
        _check(gbs_bracket_model_set(self._h, w.ctypes.data_as(C.POINTER(C.c_float)), w.size), "gbs_bracket_model_set")

    def get_bracket_model(self):
        import numpy as np
        w = np.empty(self.N_PARAMS, dtype=np.float32)
        _check(gbs_bracket_model_get(self._h, w.ctypes.data_as(C.POINTER(C.c_float)), w.size), "gbs_bracket_model_get")
        return w

    def save_bracket_model(self, path):
        _check(gbs_bracket_model_save(self._h, os.fsencode(path)), "gbs_bracket_model_save")

    def load_bracket_model(self, path):
        _check(gbs_bracket_model_load(self._h, os.fsencode(path)), "gbs_bracket_model_load")

    def bracket_features(self, x, stream=None):
        import torch
        x = self._in(x, "x", dtype=torch.float32)
        feat = torch.empty(36, dtype=torch.float32, device=x.device)
        musd = torch.empty(2, dtype=torch.float64, device=x.device)
        _check(gbs_bracket_features_f32(self._h, C.c_void_p(x.data_ptr()), x.numel(), C.c_void_p(feat.data_ptr()),
                                        C.c_void_p(musd.data_ptr()), _stream_ptr(stream)), "gbs_bracket_features")
        return feat, musd

    def bracket_propose(self, x, stream=None):
        import torch
        x = self._in(x, "x", dtype=torch.float32)
        out = torch.empty(3, dtype=torch.float64, device=x.device)
        _check(gbs_bracket_propose_f32(self._h, C.c_void_p(x.data_ptr()), x.numel(), C.c_void_p(out.data_ptr()),
                                       _stream_ptr(stream)), "gbs_bracket_propose")
        return out

    def bracket_forward(self, F, stream=None):
        import torch
        F = self._in(F, "F (B, 36 features)", dtype=torch.float32, dim=2, cols=self.N_FEATURES)
        out = torch.empty(F.shape[0], 2, dtype=torch.float32, device=F.device)
        _check(gbs_bracket_forward(self._h, C.c_void_p(F.data_ptr()), F.shape[0], C.c_void_p(out.data_ptr()),
                                   _stream_ptr(stream)), "gbs_bracket_forward")
        return out

    def bracket_grad(self, F, Z, stream=None):
        import torch
        F, Z = self._train_args(F, Z)
        grad = torch.empty(self.N_PARAMS, dtype=torch.float32, device=F.device)
        loss = torch.empty(1, dtype=torch.float64, device=F.device)
        _check(gbs_bracket_grad(self._h, C.c_void_p(F.data_ptr()), C.c_void_p(Z.data_ptr()), F.shape[0],
                                C.c_void_p(grad.data_ptr()), C.c_void_p(loss.data_ptr()), _stream_ptr(stream)),
               "gbs_bracket_grad")
        return grad, loss

    def bracket_train(self, F, Z, batch, steps, lr=1e-3, seed=0, stream=None):
        F, Z = self._train_args(F, Z)
        hist = (C.c_float * int(steps))()
        _check(gbs_bracket_train(self._h, C.c_void_p(F.data_ptr()), C.c_void_p(Z.data_ptr()), F.shape[0], int(batch),
                                 int(steps), float(lr), int(seed), hist, _stream_ptr(stream)), "gbs_bracket_train")
        return list(hist)

    def generate_training_array(self, out, family, p0=0.0, p1=0.0, p2=1.0, loc=0.0, scale=1.0, seed=0, stream=None):
        import torch
        out = self._in(out, "out", dtype=torch.float32)
        _check(gbs_generate_training_array_f32(self._h, C.c_void_p(out.data_ptr()), out.numel(), int(family),
                                               float(p0), float(p1), float(p2), float(loc), float(scale), int(seed),
                                               _stream_ptr(stream)), "gbs_generate_training_array")
        return out

    def philox(self, counters, keys, stream=None):
        import torch
        if isinstance(counters, torch.Tensor) and counters.numel() % 4:
            raise ValueError("counters: a multiple of 4 words expected")
        counters = self._in(counters, "counters (m x 4 words)", dtype=torch.int32)
        m = counters.numel() // 4
        keys = self._in(keys, "keys (m x 2 words)", dtype=torch.int32, numel=2 * m)
        out = torch.empty(4 * m, dtype=torch.int32, device=counters.device)
        _check(gbs_philox4x32_10(self._h, C.c_void_p(counters.data_ptr()), C.c_void_p(keys.data_ptr()),
                                 C.c_void_p(out.data_ptr()), m, _stream_ptr(stream)), "gbs_philox4x32_10")
        return out

    def check_wait_timeout(self, limit_ns, stream=None):
        """Runs one device-side wait that cannot complete with a bound of limit_ns
        nanoseconds and returns the device status it recorded (GBS_ETIMEOUT)."""
        st = C.c_int32(0)
        _check(gbs_check_wait_timeout(self._h, int(limit_ns), C.byref(st), _stream_ptr(stream)),
               "gbs_check_wait_timeout")
        return st.value

    def last_stats(self, raise_on_error=True):
        """Synchronises the last call's stream and returns its record as a dict."""
        rs = gbs_run_stats()
        _check(gbs_last_stats(self._h, C.byref(rs)), "gbs_last_stats")
        if raise_on_error and rs.status != GBS_OK:
            raise GbsError(rs.status, "device")
        d = {f: getattr(rs, f) for f in ("status", "how", "passes", "kelley_steps", "bisect_steps",
                                           "finish_rounds", "grid", "learned", "n", "k", "finish_pop", "n_t")}
        npass = max(0, rs.passes - 1)
        d["how"] = HOW.get(rs.how, str(rs.how))
        d["pops"] = list(rs.pops[:min(npass, 64)])
        d["iterates"] = list(rs.iterates[:min(npass, 64)])
        d["t_ns"] = list(rs.t_ns[:rs.n_t])
        d["t_stream_ns"] = list(rs.t_stream_ns[:min(npass, 64)])
        return d


_default = {}


def default_context(device=None):
    import torch
    dev = torch.cuda.current_device() if device is None else int(device)
    if dev not in _default:
        _default[dev] = Context(dev)
    return _default[dev]


def select_kth(x, k, out=None, stream=None):
    return default_context(x.device.index).select_kth(x, k, out, stream)


def median(x, out=None, stream=None):
    return default_context(x.device.index).median(x, out, stream)
