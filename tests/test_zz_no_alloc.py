"""pll_bp_labels_noalloc: bit-parallel labels computed without allocation.

The entry point is for callers that cannot call cudaMalloc (their device
memory belongs to another allocator, or they forbid allocation once running):
it keeps its scratch in a fixed device array inside the library. This test
calls it through the C ABI twice in a row (the scratch array keeps the last
call's contents, so the second call checks that what must start at zero is
cleared) and compares every value with the bit-parallel labels that the
allocating entry point pll_build exports for the same order and t. The
second call runs with the library's allocation-failure hook set so that any
allocation it made would fail, and the library's live-allocation count and
torch's allocated bytes must be the same after each call as before. The file
is collected after the others but the directed-graph tests, so that a run
stopping at its first failure has already run the tests before it; it passes
alone and after the others.
"""
import ctypes as C
import gc

import numpy as np
import pytest

from paper_1304_4661_gb300 import graphgen as gg
from paper_1304_4661_gb300 import pll

from .gpu_util import dev_u32, gpu_build

pytestmark = pytest.mark.gpu


def rank_space_csr(g, order):
    """The graph relabelled so that vertex id == rank (host side)."""
    n = g.n
    rank = np.empty(n, dtype=np.int64)
    rank[order] = np.arange(n)
    deg = np.diff(g.offsets.astype(np.int64))
    roff = np.zeros(n + 1, dtype=np.int64)
    roff[1:] = np.cumsum(deg[order])
    rcol = np.empty(g.nnz, dtype=np.int64)
    for r in range(n):
        v = order[r]
        nb = rank[g.cols[g.offsets[v]:g.offsets[v + 1]]]
        rcol[roff[r]:roff[r + 1]] = np.sort(nb)
    return roff.astype(np.uint32), rcol.astype(np.uint32), rank


@pytest.mark.parametrize("make,t", [(lambda: gg.rmat(13, 16, seed=3), 64),
                                    (lambda: gg.ba(3000, 3, 5), 16),
                                    (lambda: gg.ws(2000, 6, 0.1, 7), 5)])
def test_noalloc_matches_pll_build_twice(make, t):
    import torch
    g = make()
    ix = gpu_build(g, t)
    order = ix.order()
    d_ref, m1_ref, m0_ref = ix.bp()
    roots_ref, cnt_ref, S_ref = ix.bp_roots()
    roff, rcol, rank = rank_space_csr(g, order)
    n, tp = g.n, (t + 15) // 16 * 16
    droff, drcol = dev_u32(roff), dev_u32(rcol)
    lib = pll.load()
    for call in range(2):
        d = torch.full((n * tp,), 7, dtype=torch.uint8, device="cuda")
        masks = torch.full((n * t * 2,), 3, dtype=torch.int64, device="cuda")
        roots = torch.zeros(t, dtype=torch.int32, device="cuda")
        cnt = torch.zeros(t, dtype=torch.int32, device="cuda")
        S = torch.zeros(t * 64, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        # indices left by earlier tests are freed by the garbage collector,
        # which would move the counts in the middle of the measurement
        gc.collect()
        gc.disable()
        try:
            live, held = lib.pll_test_live_allocs(), torch.cuda.memory_allocated()
            if call == 1:
                # the second call runs with every allocation of the library set
                # to fail: it must still succeed, since it allocates nothing
                lib.pll_test_fail_alloc(0)
            try:
                pll.bp_labels_noalloc(droff, drcol, t, d, masks, roots, cnt, S)
                torch.cuda.synchronize()
            finally:
                lib.pll_test_fail_alloc(-1)
            assert lib.pll_test_live_allocs() == live, call
            assert torch.cuda.memory_allocated() == held, call
        finally:
            gc.enable()
        hd = d.cpu().numpy().reshape(n, tp)
        hm = masks.cpu().numpy().view(np.uint64).reshape(n, t, 2)
        assert (hd[:, t:] == 255).all(), call
        # rows are in rank space; the reference is by vertex id
        assert np.array_equal(hd[rank, :t], d_ref), call
        assert np.array_equal(hm[rank, :, 0], m1_ref), call
        assert np.array_equal(hm[rank, :, 1], m0_ref), call
        r = roots.cpu().numpy().view(np.uint32)
        c = cnt.cpu().numpy().view(np.uint32)
        s = S.cpu().numpy().view(np.uint32).reshape(t, 64)
        assert np.array_equal(c, cnt_ref), call
        assert np.array_equal(np.where(r == pll.NONE, pll.NONE, order[np.minimum(r, n - 1)]), roots_ref), call
        for i in range(t):
            assert np.array_equal(order[s[i, :c[i]]], S_ref[i, :cnt_ref[i]]), (call, i)


def test_noalloc_rejects_graphs_beyond_its_scratch():
    lib = pll.load()
    # 2^24 - 1 vertices need about 13 bytes each: more than 64 MiB. The size
    # check comes before any device access, so dummy pointers are never used.
    dummy = C.c_void_p(16)
    rc = lib.pll_bp_labels_noalloc(dummy, dummy, (1 << 24) - 1, 1 << 20, 16, dummy, dummy, dummy,
                                   dummy, dummy, None)
    assert rc == pll.PLL_E_RANGE
    assert lib.pll_bp_labels_noalloc(dummy, dummy, 100, 10, 65, dummy, dummy, dummy, dummy, dummy,
                                     None) == pll.PLL_E_RANGE
