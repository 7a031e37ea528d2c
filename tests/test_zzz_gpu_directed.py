"""Directed graphs (Sec. 6) on the GPU: pll_build_directed and pll_dquery
against the directed oracle, exactly: order, every L_IN and L_OUT entry, every
distance (all pairs on small digraphs, 20011 sampled pairs on larger ones),
for the Degree order and an explicit one and for root batches from 1 to the
default; a digraph with every arc both ways against the undirected build;
the error codes.

The file is collected last (after tests/test_zz_no_alloc.py): a run that
stops at its first failure has run every other test before these.
"""
import numpy as np
import pytest

import oracle
from paper_1304_4661_gb300 import graphgen as gg
from paper_1304_4661_gb300 import pll

from . import graphs
from .gpu_util import dev_u32, first_label_diff, gpu_build, same_labels

pytestmark = pytest.mark.gpu

INF = 255


def small_digraphs():
    gs = [gg.digraph(9, [(i, (i + 1) % 9) for i in range(9)], "dcycle9"),
          gg.digraph(12, [(i, i + 1) for i in range(11)], "dpath12"),
          gg.digraph(10, [(i, j) for i in range(10) for j in range(i + 1, 10) if (i * 7 + j) % 3 == 0], "dag"),
          gg.digraph(8, [(0, i) for i in range(1, 8)], "out_star"),
          gg.digraph(8, [(i, 0) for i in range(1, 8)], "in_star"),
          gg.digraph(6, [], "empty6"), gg.digraph(1, [], "single")]
    for n, m, sd in ((20, 30, 1), (40, 160, 3), (80, 260, 5), (150, 600, 6)):
        gs.append(gg.random_digraph(n, m, sd))
    gs += [gg.oriented(gg.ba(120, 3, 3), 4), gg.oriented(gg.rmat(7, 8, seed=5), 6, both=0.1),
           gg.oriented(gg.ws(100, 6, 0.1, 2), 8, both=0.5)]
    return gs


def build(d, order=None, root_batch=0):
    return pll.DirectedIndex(dev_u32(d.offsets), dev_u32(d.cols),
                             order=None if order is None else dev_u32(order), root_batch=root_batch)


def gpu_dquery(ix, s, t):
    return ix.query(dev_u32(s), dev_u32(t)).cpu().numpy()


@pytest.mark.parametrize("root_batch", [0, 1, 7, 64])
@pytest.mark.parametrize("d", small_digraphs(), ids=lambda d: d.name)
def test_small_digraphs_exact(d, root_batch):
    n = d.n
    for order in (None, np.random.default_rng(n).permutation(n).astype(np.uint32)):
        ix = build(d, order, root_batch)
        ref = oracle.DirectedIndex(d.offsets, d.cols, order=order)
        assert np.array_equal(ix.order(), ref.order())
        gi, ri, go, ro = ix.labels_in(), ref.labels_in(), ix.labels_out(), ref.labels_out()
        assert same_labels(gi, ri), ("L_IN", first_label_diff(gi, ri, n))
        assert same_labels(go, ro), ("L_OUT", first_label_diff(go, ro, n))
        assert ix.entries() == (len(ri.hubs), len(ro.hubs))
        s = np.repeat(np.arange(n, dtype=np.uint32), n)
        t = np.tile(np.arange(n, dtype=np.uint32), n)
        assert np.array_equal(gpu_dquery(ix, s, t), ref.query_batch(s, t))
        ix.close()


@pytest.mark.parametrize("d", [gg.oriented(gg.ba(5000, 4, 1), 2), gg.oriented(gg.rmat(13, 16, seed=4), 3, both=0.2),
                               gg.random_digraph(3000, 12000, 9), gg.oriented(gg.ws(4000, 6, 0.1, 5), 6)],
                         ids=lambda d: d.name)
def test_larger_digraphs(d):
    ix = build(d)
    ref = oracle.DirectedIndex(d.offsets, d.cols)
    assert np.array_equal(ix.order(), ref.order())
    gi, ri, go, ro = ix.labels_in(), ref.labels_in(), ix.labels_out(), ref.labels_out()
    assert same_labels(gi, ri), ("L_IN", first_label_diff(gi, ri, d.n))
    assert same_labels(go, ro), ("L_OUT", first_label_diff(go, ro, d.n))
    s, t = gg.pairs(d.n, 20011, 5)
    assert np.array_equal(gpu_dquery(ix, s, t), ref.query_batch(s, t))


@pytest.mark.parametrize("g", [graphs.grid(6, 7), gg.ba(800, 3, 12), gg.rmat(10, 8, seed=33)],
                         ids=lambda g: g.name)
def test_both_ways_equals_undirected(g):
    d = gg.Digraph(g.n, g.offsets, g.cols, g.name)
    ix = build(d)
    u = gpu_build(g, 0).labels()
    assert same_labels(ix.labels_in(), u) and same_labels(ix.labels_out(), u)


def test_errors():
    d = gg.digraph(5, [(0, 1), (1, 2), (2, 3), (3, 4)])
    off, col = dev_u32(d.offsets), dev_u32(d.cols)
    with pytest.raises(pll.PLLError) as e:  # t must be 0
        lib = pll.load()
        import ctypes as C
        h = C.c_void_p()
        opts = pll.BuildOpts(1, 0, 0, 0, 0)
        pll._check(lib.pll_build_directed(off.data_ptr(), col.data_ptr(), 5, 4, None, C.byref(opts), None,
                                          C.byref(h)), "pll_build_directed")
    assert e.value.code == pll.PLL_E_INVAL
    for bad_col in ([1, 1, 3, 4], [1, 2, 2, 4], [1, 2, 3, 9]):  # self-loop, self-loop, id >= n
        with pytest.raises(pll.PLLError) as e:
            pll.DirectedIndex(off, dev_u32(np.array(bad_col, np.uint32)))
        assert e.value.code == pll.PLL_E_INVAL
    unsorted = gg.digraph(4, [(0, 1), (0, 2)])
    with pytest.raises(pll.PLLError) as e:
        pll.DirectedIndex(dev_u32(unsorted.offsets), dev_u32(unsorted.cols[::-1].copy()))
    assert e.value.code == pll.PLL_E_INVAL
    bad_off = d.offsets.copy()
    bad_off[2] = 7  # past nnz
    with pytest.raises(pll.PLLError) as e:
        pll.DirectedIndex(dev_u32(bad_off), col)
    assert e.value.code == pll.PLL_E_INVAL
    with pytest.raises(pll.PLLError) as e:
        pll.DirectedIndex(off, col, order=dev_u32(np.array([0, 1, 1, 3, 4], np.uint32)))
    assert e.value.code == pll.PLL_E_ORDER
    longp = gg.digraph(300, [(i, i + 1) for i in range(299)])
    with pytest.raises(pll.PLLError) as e:
        pll.DirectedIndex(dev_u32(longp.offsets), dev_u32(longp.cols))
    assert e.value.code == pll.PLL_E_RANGE
    okp = gg.digraph(255, [(i, i + 1) for i in range(254)])
    ix = pll.DirectedIndex(dev_u32(okp.offsets), dev_u32(okp.cols))
    assert gpu_dquery(ix, np.array([0, 254], np.uint32), np.array([254, 0], np.uint32)).tolist() == [254, INF]
    with pytest.raises(pll.PLLError) as e:
        ix.query(dev_u32(np.array([0, 255], np.uint32)), dev_u32(np.array([1, 1], np.uint32)))
    assert e.value.code == pll.PLL_E_INVAL
    assert gpu_dquery(ix, np.array([3], np.uint32), np.array([10], np.uint32)).tolist() == [7]  # still answers


def test_edgeless_and_no_leaks():
    import gc
    gc.collect()
    base = pll.load().pll_test_live_allocs()
    d = gg.digraph(7, [], "empty7")
    ix = build(d)
    assert ix.entries() == (7, 7)
    v = np.arange(7, dtype=np.uint32)
    assert gpu_dquery(ix, v, v).tolist() == [0] * 7
    assert gpu_dquery(ix, v, (v + 1) % 7).tolist() == [INF] * 7
    ix.close()
    d = gg.oriented(gg.ba(300, 2, 5), 1)
    ix = build(d, root_batch=16)
    ix.close()
    assert pll.load().pll_test_live_allocs() == base
