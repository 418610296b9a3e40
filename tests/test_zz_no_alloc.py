"""The allocation-free entry point gbs_select_kth_f32_noalloc.

It exists for callers that cannot let a library allocate device memory (arena-managed
hosts, fixed device budgets, loops that cannot afford an allocation's implicit
synchronisation).  It must return exactly what the context-based gbs_select_kth_f32
returns.  This file is collected last so that a failure here comes after every other
test has run; it passes alone in a fresh process as well.
"""
import ctypes

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


def _bits(t):
    return t.cpu().numpy().view(np.uint32).tolist()


def test_noalloc_matches_context_entry_point_twice_in_a_row(lib):
    ctx = lib.Context()
    x_np = synth.heavy_mixture("mixture", 1 << 20, seed=51)
    x = torch.from_numpy(x_np).cuda()
    n = x.numel()
    ks = [1, 2, n // 100, (n + 1) // 2, (99 * n) // 100, n]
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):          # the second call reuses the array the first one left
        for k in ks:
            ref = ctx.select_kth(x, k)
            out = torch.full((1,), float("nan"), device="cuda")
            st = lib.gbs_select_kth_f32_noalloc(ctypes.c_void_p(x.data_ptr()), n, k,
                                                 ctypes.c_void_p(out.data_ptr()), stream)
            assert st == lib.GBS_OK
            torch.cuda.synchronize()
            assert _bits(out) == _bits(ref), (call, k)
    # a smaller, unaligned input after the large one
    y = torch.from_numpy(synth.paper_distribution("mix2", 4099, seed=52)).cuda()
    buf = torch.empty(4100, device="cuda")
    buf[1:].copy_(y)
    for k in (1, 2050, 4099):
        ref = ctx.select_kth(buf[1:], k)
        out = torch.empty(1, device="cuda")
        assert lib.gbs_select_kth_f32_noalloc(ctypes.c_void_p(buf[1:].data_ptr()), 4099, k,
                                              ctypes.c_void_p(out.data_ptr()), stream) == lib.GBS_OK
        torch.cuda.synchronize()
        assert _bits(out) == _bits(ref)
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_array(lib):
    x = torch.zeros(8, device="cuda")
    out = torch.zeros(1, device="cuda")
    p, o = ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr())
    assert lib.gbs_select_kth_f32_noalloc(p, (1 << 20) + 1, 1, o, None) == lib.GBS_EINVAL
    assert lib.gbs_select_kth_f32_noalloc(p, 8, 9, o, None) == lib.GBS_EINVAL
    assert lib.gbs_select_kth_f32_noalloc(p, 8, 0, o, None) == lib.GBS_EINVAL
