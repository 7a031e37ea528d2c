"""Allocation failures during a build: every allocation of the build is made
to fail in turn; each time the build returns PLL_E_NOMEM and leaves no
allocation behind, and a build after that succeeds with exact labels."""
import numpy as np
import pytest

import oracle
from paper_1304_4661_gb300 import graphgen as gg
from paper_1304_4661_gb300 import pll

from .gpu_util import dev_u32, same_labels

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("t", [0, 8])
def test_every_allocation_failure_is_clean(t):
    lib = pll.load()
    g = gg.ba(1500, 3, 11)
    off, col = dev_u32(g.offsets), dev_u32(g.cols)
    base = lib.pll_test_live_allocs()
    failures = 0
    try:
        for k in range(400):
            lib.pll_test_fail_alloc(k)
            try:
                ix = pll.Index.build(off, col, t=t, root_batch=256)
            except pll.PLLError as e:
                assert e.code == pll.PLL_E_NOMEM, (k, e)
                assert lib.pll_test_live_allocs() == base, f"leak after failure {k}"
                failures += 1
                continue
            break  # k passed every allocation of the build
        else:
            pytest.fail("the build never completed")
    finally:
        lib.pll_test_fail_alloc(-1)
    assert failures > 10  # the build allocates at many places
    assert lib.pll_test_live_allocs() > base  # the index holds its arrays
    ref = oracle.Index(g.offsets, g.cols, t)
    assert same_labels(ix.labels(), ref.labels())
    ix.close()
    assert lib.pll_test_live_allocs() == base


def test_release_cached_scratch_then_build_again():
    """Scratch comes from the library's pool, which keeps freed memory mapped
    between builds; pll_release_cached hands it back. Builds before and after
    give the oracle's labels, and no allocation is left behind."""
    import torch
    lib = pll.load()
    g = gg.ba(3000, 3, 5)
    off, col = dev_u32(g.offsets), dev_u32(g.cols)
    ref = oracle.Index(g.offsets, g.cols, 16).labels()
    base = lib.pll_test_live_allocs()
    for _ in range(2):
        ix = pll.Index.build(off, col, t=16)
        assert same_labels(ix.labels(), ref)
        ix.close()
        assert lib.pll_test_live_allocs() == base
        pll.release_cached()
    torch.cuda.synchronize()
