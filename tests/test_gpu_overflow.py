"""GPU parity on the paths a build takes only when its buffers run short, and
on the query's range error.

The pruned stage sizes its buffers for large graphs, so a small graph never
overflows one. pll_test_capacities shrinks the initial sizes (candidate and
tuple buffers, label pool, root-table pool) so that every growth path runs
on graphs the oracle builds in seconds:

  * a batch that overflows the candidate or tuple buffer is run again with a
    larger one (its visited rows are cleared whole first);
  * the label pool is moved to a larger one between batches;
  * roots whose label tables do not fit the table pool have their labels
    binary-searched by the prune test (the pool is kept small all build).

Each must give the oracle's labels exactly, and the build statistics must
show that the path was taken. The hook changes sizes on the host only; no
GPU fault is involved.

The range error: distances are 8-bit with 255 = unreachable (Sec. 4.5.1), so
a pair whose finite distance is 255 or more is answered 255 and counted as an
error (pll_query returns PLL_E_RANGE).
"""
import numpy as np
import pytest

import oracle
from paper_1304_4661_gb300 import graphgen as gg
from paper_1304_4661_gb300 import pll

from . import brute, graphs
from .gpu_util import dev_u32, first_label_diff, gpu_build, gpu_query, same_labels
from .test_oracle_pins import centroid_order

pytestmark = pytest.mark.gpu


@pytest.fixture
def small_capacities():
    lib = pll.load()
    lib.pll_test_capacities(256, 64, 256, 64)
    try:
        yield
    finally:
        lib.pll_test_capacities(0, 0, 0, 0)


def check(g, t, **kw):
    ref = oracle.Index(g.offsets, g.cols, t)
    ix = gpu_build(g, t, **kw)
    La, Lb = ix.labels(), ref.labels()
    assert same_labels(La, Lb), first_label_diff(La, Lb, g.n)
    if t:
        for a, b in zip(ix.bp(), ref.bp()):
            assert np.array_equal(a, b)
    s, u = gg.pairs(g.n, 20_000, 5)
    assert np.array_equal(gpu_query(ix, s, u), ref.query_batch(s, u))
    return ix.stats()


@pytest.mark.parametrize("t", [0, 16])
@pytest.mark.parametrize("g", graphs.small_family(), ids=lambda g: g.name)
def test_small_family_under_small_capacities(small_capacities, g, t):
    check(g, t)


@pytest.mark.parametrize("make,t,root_batch", [
    (lambda: gg.ba(10_000, 4, 1), 16, 0),
    (lambda: gg.ba(10_000, 4, 1), 0, 4096),
    (lambda: gg.rmat(14, 16, seed=3), 64, 0),
    (lambda: gg.ws(5000, 6, 0.1, 5), 16, 0),
])
def test_every_growth_path_is_taken_and_exact(small_capacities, make, t, root_batch):
    st = check(make(), t, root_batch=root_batch)
    assert st["redone_batches"] > 0
    assert st["pool_regrows"] > 0
    assert st["table_fallbacks"] > 0


def test_capacities_restore_the_default_sizing():
    g = gg.ba(3000, 3, 2)
    st = check(g, 16)
    assert st["redone_batches"] == 0 and st["pool_regrows"] == 0 and st["table_fallbacks"] == 0


@pytest.mark.parametrize("t", [0, 1])
def test_finite_distance_beyond_255_is_a_range_error(t):
    """A 400-vertex path, centroid order, one root per batch (so each BFS is
    pruned by every earlier hub, as in Alg. 2): the build succeeds and every
    pair at distance >= 255 is answered 255 with one error counted; all other
    pairs are exact. The oracle is pinned to the same rule on the CPU."""
    import torch
    g = graphs.path(400)
    order = centroid_order(g)
    ix = gpu_build(g, t, order=order, root_batch=1)
    ref = oracle.Index(g.offsets, g.cols, t, order=order)
    assert same_labels(ix.labels(), ref.labels())
    D = brute.apsp(g.offsets, g.cols)
    s, u = np.meshgrid(np.arange(g.n), np.arange(g.n), indexing="ij")
    s, u = s.ravel().astype(np.uint32), u.ravel().astype(np.uint32)
    out = torch.empty(len(s), dtype=torch.uint8, device="cuda")
    ix.query_async(dev_u32(s), dev_u32(u), out)
    got = out.cpu().numpy().astype(np.int64)
    far = D.ravel() >= 255
    assert far.sum() > 0
    assert ix.query_errors() == int(far.sum())
    assert (got[far] == 255).all()
    assert np.array_equal(got[~far], D.ravel()[~far])
    # the synchronous call reports the pair as PLL_E_RANGE
    with pytest.raises(pll.PLLError) as e:
        ix.query(dev_u32(np.array([0], np.uint32)), dev_u32(np.array([399], np.uint32)))
    assert e.value.code == pll.PLL_E_RANGE
    assert gpu_query(ix, np.array([0, 3], np.uint32), np.array([254, 257], np.uint32)).tolist() == [254, 254]


# ---- the device-side level loop (one cooperative launch per root batch)

@pytest.mark.parametrize("make,t,root_batch", [
    (lambda: gg.ba(3000, 3, 17), 16, 0),
    (lambda: gg.ba(3000, 3, 17), 16, 7),
    (lambda: gg.ws(4000, 6, 0.1, 5), 0, 0),
    (lambda: gg.rmat(13, 16, seed=3), 64, 100),
    (lambda: graphs.path(255), 2, 0),
])
def test_host_and_device_level_loops_give_the_oracle_labels(make, t, root_batch):
    """The three ways of running a batch's levels (default: one CUDA graph
    launch per batch whose while node runs the sweeps; PLL_BUILD_HOST_LEVELS:
    separate launches enqueued by the host; PLL_BUILD_COOP_LEVELS: one
    cooperative launch per batch) give the oracle's labels; the device-side
    ones really ran."""
    g = make()
    ref = oracle.Index(g.offsets, g.cols, t)
    Lref = ref.labels()
    for flags in (0, pll.PLL_BUILD_HOST_LEVELS, pll.PLL_BUILD_COOP_LEVELS):
        ix = gpu_build(g, t, root_batch=root_batch, flags=flags)
        La = ix.labels()
        assert same_labels(La, Lref), (flags, first_label_diff(La, Lref, g.n))
        st = ix.stats()
        if flags == pll.PLL_BUILD_HOST_LEVELS:
            assert st["levels_launches"] == 0
        elif g.nnz:
            assert st["levels_launches"] == st["batches"] > 0


def test_barrier_wait_that_runs_out_returns_timeout_and_the_gpu_stays_usable():
    """A grid barrier of the cooperative level loop that waits past its limit
    makes the build return PLL_E_TIMEOUT: the limit is set to 1 ns, so every CTA but the
    last to arrive gives up at the first barrier and leaves the kernel. No
    allocation leaks, and the next build (default limit) is exact."""
    import gc
    lib = pll.load()
    g = gg.ba(3000, 3, 2)
    gc.collect()
    gc.disable()  # indices of earlier tests must not be freed mid-count
    try:
        live = lib.pll_test_live_allocs()
        lib.pll_test_barrier_timeout(1)
        try:
            with pytest.raises(pll.PLLError) as e:
                gpu_build(g, 16, flags=pll.PLL_BUILD_COOP_LEVELS)
            assert e.value.code == pll.PLL_E_TIMEOUT
        finally:
            lib.pll_test_barrier_timeout(0)
        assert lib.pll_test_live_allocs() == live
    finally:
        gc.enable()
    ix = gpu_build(g, 16, flags=pll.PLL_BUILD_COOP_LEVELS)
    assert same_labels(ix.labels(), oracle.Index(g.offsets, g.cols, 16).labels())
