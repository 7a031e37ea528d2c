"""pll_build_batch: several graphs in one build, each exactly as built alone.

Every graph of the batch is checked against the oracle built on that graph
alone: its order, its bit-parallel roots and labels, every label entry (hub
ranks mapped from the union's interleaved order back to the graph's own
ranks) and all-pairs / sampled distances; pairs across graphs answer 255.
"""
import numpy as np
import pytest

import oracle
from paper_1304_4661_gb300 import graphgen as gg
from paper_1304_4661_gb300 import pll

from . import graphs
from .gpu_util import dev_u32, gpu_query

pytestmark = pytest.mark.gpu


def check_batch(gl, t, sample_pairs=2000, oracle_graphs=None, **kw):
    off, col, start = gg.union(gl)
    ix = pll.Index.build_batch(dev_u32(off), dev_u32(col), start, t=t, **kw)
    order = ix.order()
    L = ix.labels()
    bp = ix.bp() if t else None
    roots, cnt, S = ix.bp_roots() if t else (None, None, None)
    owner = np.searchsorted(start, order, side="right") - 1
    for gi, g in enumerate(gl):
        if oracle_graphs is not None and gi not in oracle_graphs:
            continue
        ref = oracle.Index(g.offsets, g.cols, t)
        b = int(start[gi])
        mine = order[owner == gi]                    # this graph's vertices, in union order
        assert np.array_equal(mine - b, ref.order()), gi
        local = np.full(len(order), -1, dtype=np.int64)
        local[np.flatnonzero(owner == gi)] = np.arange(len(mine))   # union rank -> own rank
        rl = ref.labels()
        for v in range(g.n):
            a0, a1 = int(L.offsets[b + v]), int(L.offsets[b + v + 1])
            hubs = local[L.hubs[a0:a1].astype(np.int64)]
            r0, r1 = int(rl.offsets[v]), int(rl.offsets[v + 1])
            assert np.array_equal(hubs, rl.hubs[r0:r1].astype(np.int64)), (gi, v)
            assert np.array_equal(L.dists[a0:a1], rl.dists[r0:r1]), (gi, v)
        if t:
            r_roots, r_cnt, r_S = ref.bp_roots()
            q = slice(gi * t, (gi + 1) * t)
            rr = roots[q].astype(np.int64)
            assert np.array_equal(np.where(rr == pll.NONE, pll.NONE, rr - b), r_roots), gi
            assert np.array_equal(cnt[q], r_cnt), gi
            for i in range(t):
                assert np.array_equal(S[gi * t + i, : cnt[gi * t + i]] - b, r_S[i, : r_cnt[i]])
            for a, r in zip(bp, ref.bp()):
                assert np.array_equal(a[b:b + g.n], r), gi
        if g.n:
            s, u = gg.pairs(g.n, sample_pairs, 7 + gi)
            got = gpu_query(ix, s + np.uint32(b), u + np.uint32(b))
            assert np.array_equal(got, ref.query_batch(s, u)), gi
    # pairs across graphs are unreachable
    if len(gl) > 1 and start[-1] > 0:
        rng = np.random.default_rng(1)
        s = rng.integers(0, int(start[-1]), 5000).astype(np.uint32)
        u = rng.integers(0, int(start[-1]), 5000).astype(np.uint32)
        og = np.searchsorted(start, s, side="right") - 1
        ug = np.searchsorted(start, u, side="right") - 1
        got = gpu_query(ix, s, u)
        assert (got[og != ug] == 255).all()
        # small launches take the several-warps-per-pair path
        for q in (1, 9, 300):
            assert np.array_equal(gpu_query(ix, s[:q], u[:q]), got[:q]), q
    return ix


@pytest.mark.parametrize("t", [0, 4, 16])
def test_mixed_small_batch(t):
    gl = [gg.ba(300, 3, 1), gg.ws(200, 6, 0.1, 2), graphs.complete(1), graphs.star(7),
          gg.from_edges(5, [], []), gg.rmat(9, 8, seed=3), graphs.path(40), gg.ba(1000, 2, 4),
          graphs.disjoint(graphs.cycle(9), graphs.complete(4)), gg.ws(500, 4, 0.3, 5)]
    check_batch(gl, t)


@pytest.mark.parametrize("root_batch,block", [(64, 256), (4096, 128), (1024, 512)])
def test_batch_options_do_not_change_labels(root_batch, block):
    gl = [gg.ba(2000, 4, 11), gg.ws(3000, 6, 0.1, 12), gg.rmat(11, 16, seed=13)]
    check_batch(gl, 16, root_batch=root_batch, block=block)


def test_uneven_batch_of_64_sampled_against_oracle():
    specs = gg.batch_specs(64, seed=9, n_lo=500, n_hi=8000)
    gl = [gg.make(sp) for sp in specs]
    check_batch(gl, 16, oracle_graphs=set(range(0, 64, 7)))


def test_batch_rejects_arcs_between_graphs():
    g1, g2 = gg.ba(50, 2, 1), gg.ba(60, 2, 2)
    # the union plus one arc joining vertex 0 (graph 0) and vertex 100 (graph 1)
    j = graphs.disjoint(g1, g2)
    rows = np.repeat(np.arange(j.n), np.diff(j.offsets.astype(np.int64)))
    joined = gg.union([gg.from_edges(j.n, np.r_[rows, [0]], np.r_[j.cols, [100]])])
    with pytest.raises(pll.PLLError) as e:
        pll.Index.build_batch(dev_u32(joined[0]), dev_u32(joined[1]), np.array([0, 50, 110]), t=2)
    ok = pll.Index.build_batch(dev_u32(joined[0]), dev_u32(joined[1]), np.array([0, 110]), t=2)
    assert e.value.code == pll.PLL_E_INVAL and ok.label_entries() > 0


def test_autotune_returns_a_valid_choice():
    g = gg.rmat(12, 16, seed=3)
    rb, block, ms = pll.autotune(dev_u32(g.offsets), dev_u32(g.cols), 16)
    assert rb in (1024, 2048, 4096, 8192, 16384) and block in (128, 256, 512) and ms > 0
    ix = pll.Index.build(dev_u32(g.offsets), dev_u32(g.cols), t=16, root_batch=rb, block=block)
    ref = oracle.Index(g.offsets, g.cols, 16)
    a, b = ix.labels(), ref.labels()
    assert np.array_equal(a.hubs, b.hubs) and np.array_equal(a.dists, b.dists)
