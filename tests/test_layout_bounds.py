"""CPU check of the single-array select kernel's index arithmetic (no GPU involved).

The streaming passes read x as a scalar head up to the first 16-byte boundary, a body of
16-byte vectors cut into chunks, and a scalar tail.  Chunk c belongs to CTA c mod G, and
thread t of a CTA loads vectors t + u * kThreads (u < kChunkVecs / kThreads) of each of
its chunks.  CTA 0's low threads also take the head and tail elements.  A compacting
pass appends what a CTA keeps to that CTA's region of the compaction area.

This test restates that assignment from the kernel's definitions, with the constants
read from the headers themselves.  For many sizes, alignments and grid sizes it checks:
- every element of x is read exactly once, and every vector load lies inside the body;
- the most a CTA can keep fits in its region [region_start(g), region_start(g+1));
- the per-thread term bound covers what a thread reads;
- the area allocated for n elements (any alignment) holds every region;
- the allocation-free entry point's static area holds the largest n it accepts.
The 32-bit chunk indices and per-CTA counters stay below 2^32 up to 2^36 elements.
"""
import os
import re

import numpy as np
import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1104_2732_gb300", "csrc")


def _const(name, fname):
    with open(os.path.join(CSRC, fname)) as f:
        src = f.read()
    m = re.search(r"constexpr\s+(?:int|long long)\s+" + name + r"\s*=\s*([^;]+);", src)
    assert m, (name, fname)
    return m.group(1).strip()


K_THREADS = int(_const("kThreads", "common.cuh"))
K_CHUNK_BYTES = int(_const("kChunkBytes", "layout.cuh"))
K_CHUNK_VECS = K_CHUNK_BYTES // 16
K_VPT = K_CHUNK_VECS // K_THREADS
NOALLOC_MAX_N = 1 << 20
NOALLOC_MAX_GRID = int(_const("kNoAllocMaxGrid", "noalloc.cu"))


def geometry(addr, n, esize):
    """(head, nv, tail0) of an element-aligned array at byte address addr."""
    vec = 16 // esize
    head = min(((16 - addr % 16) % 16) // esize, n)
    nv = (n - head) // vec
    return head, nv, head + nv * vec


def chunk_count(nv):
    return (nv + K_CHUNK_VECS - 1) // K_CHUNK_VECS


def region_start(g, nch, G, vec):
    q, r = nch // G, nch % G
    return (g * q + min(g, r)) * K_CHUNK_VECS * vec + (2 * vec if g > 0 else 0)


def per_thread_bound(nch, G, vec):
    return ((nch + G - 1) // G) * ((K_CHUNK_VECS + K_THREADS - 1) // K_THREADS) * vec + 2 * vec


def z_elems_for(n, G, vec):
    return region_start(G, chunk_count(n // vec + 1), G, vec)


def check_layout(n, addr, esize, G):
    vec = 16 // esize
    head, nv, tail0 = geometry(addr, n, esize)
    assert 0 <= head < vec or head == n
    assert 0 <= n - tail0 < vec
    nch = chunk_count(nv)
    assert nch < 2 ** 32
    # chunks of each CTA: c = bid + j * G, j < my(bid)
    bid = np.arange(G, dtype=np.int64)
    my = np.where(bid < nch, (nch - 1 - bid) // G + 1, 0)
    seen = np.zeros(nch, dtype=np.int64)
    for b in range(G):
        c = b + np.arange(my[b], dtype=np.int64) * G
        assert np.all(c < nch)
        np.add.at(seen, c, 1)
    assert np.all(seen == 1)
    # vectors of one chunk: thread t, slot u -> t + u * kThreads covers [0, kChunkVecs) once
    t, u = np.meshgrid(np.arange(K_THREADS), np.arange(K_VPT), indexing="ij")
    local = (t + u * K_THREADS).ravel()
    assert np.array_equal(np.sort(local), np.arange(K_CHUNK_VECS))
    # only the last chunk is partial; its loads are limited to the body
    if nch:
        assert (nch - 1) * K_CHUNK_VECS < nv <= nch * K_CHUNK_VECS
    # edges: threads gtid < head and gtid < n - tail0 exist (all in CTA 0)
    assert head <= K_THREADS and n - tail0 <= K_THREADS
    # elements per CTA (body vectors of its chunks, CTA 0 also the edges) fit its region
    last_owner = (nch - 1) % G if nch else -1
    for b in range(G):
        vecs = my[b] * K_CHUNK_VECS
        if b == last_owner:
            vecs -= nch * K_CHUNK_VECS - nv
        kept_max = vecs * vec + (head + (n - tail0) if b == 0 else 0)
        room = region_start(b + 1, nch, G, vec) - region_start(b, nch, G, vec)
        assert kept_max <= room, (n, addr, esize, G, b)
        assert kept_max < 2 ** 32      # per-CTA compaction counter
    # per-thread terms: every chunk of the CTA contributes at most K_VPT vectors
    assert int(my.max(initial=0)) * K_VPT * vec + 2 <= per_thread_bound(nch, G, vec)
    # the allocated area holds every region, whatever the alignment
    assert region_start(G, nch, G, vec) <= z_elems_for(n, G, vec)
    # body + edges cover [0, n) exactly
    assert head + nv * vec + (n - tail0) == n


def _sizes():
    cv = K_CHUNK_VECS
    out = set(range(1, 40))
    for vec in (2, 4):
        for m in (1, 2, 3, 151, 152, 153, 303, 304, 305, 1000):
            for d in (-5, -4, -3, -1, 0, 1, 2, 3, 4, 5):
                out.add(m * cv * vec + d)
    out.update({4099, 65537, 300007, (1 << 20) + 5, 1 << 20, 5_000_011})
    return sorted(s for s in out if s >= 1)


@pytest.mark.parametrize("esize", [4, 8])
def test_select_layout_covers_each_element_once_and_fits_regions(esize):
    for G in (1, 2, 7, 152, 304):
        for n in _sizes():
            for addr in range(0, 16, esize):
                check_layout(n, 4096 + addr, esize, G)


def test_select_layout_at_the_largest_sizes():
    """2^31 + 5 and 2^36 elements on the grids of this GPU (152 SMs, one or two CTAs
    each): chunk indices and per-CTA counters stay within 32 bits."""
    for esize in (4, 8):
        for n in (2 ** 31 + 5, 2 ** 36):
            for G in (152, 304):
                check_layout(n, 4100 if esize == 4 else 4104, esize, G)


def test_noalloc_area_holds_the_largest_input():
    """The allocation-free entry point's static compaction area (elements) covers
    z_elems_for(n, G) for every n it accepts and every grid up to its cap."""
    cap = ((NOALLOC_MAX_N // 4 + 1 + K_CHUNK_VECS - 1) // K_CHUNK_VECS) * K_CHUNK_VECS * 4 + 8
    src = _const("kNoAllocZ", "noalloc.cu")
    assert src.replace(" ", "") == "((kNoAllocMaxN/4+1+kChunkVecs-1)/kChunkVecs)*kChunkVecs*4+8"
    for G in (1, 152, 304, NOALLOC_MAX_GRID):
        for n in (1, 4099, NOALLOC_MAX_N - 1, NOALLOC_MAX_N):
            assert z_elems_for(n, G, 4) <= cap
