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
