"""Parity at the benchmark's full size: R-MAT-20, t = 64, default launch
configuration (the one bench.py times).

The oracle's whole pruned stage would take ~15 minutes here, so the check is
split into what the oracle can compute one piece at a time:
  * the vertex order, the bit-parallel roots and S_r, and every bit-parallel
    distance and mask (the oracle's Alg. 3 over the whole graph);
  * full labels L(u) of sampled vertices (the oracle's closed form, one BFS per
    vertex), plus the first non-X vertex, an isolated vertex and the vertex
    with the longest GPU label;
  * every distance from sampled sources to all vertices (plain BFS);
  * d(s, t) = d(t, s) over the benchmark's 10M pairs.
"""
import numpy as np
import pytest

import oracle
from paper_1304_4661_gb300 import graphgen as gg

from .gpu_util import dev_u32, gpu_build, gpu_query

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rmat20():
    g = gg.rmat(20, 16, seed=1)
    ix = gpu_build(g, 64)
    ref = oracle.Index(g.offsets, g.cols, 64, with_pruned=False)
    return g, ix, ref


def test_order_and_bit_parallel_labels(rmat20):
    g, ix, ref = rmat20
    assert np.array_equal(ix.order(), ref.order())
    r_roots, r_cnt, r_S = ref.bp_roots()
    roots, cnt, S = ix.bp_roots()
    assert np.array_equal(roots, r_roots) and np.array_equal(cnt, r_cnt)
    for i in range(64):
        assert np.array_equal(S[i, : cnt[i]], r_S[i, : r_cnt[i]])
    for a, b in zip(ix.bp(), ref.bp()):
        assert np.array_equal(a, b)


def test_sampled_labels_match_closed_form(rmat20):
    g, ix, ref = rmat20
    rank, inX = ref.rank_inX()
    L = ix.labels()
    sizes = np.diff(L.offsets.astype(np.int64))
    order = ref.order()
    rng = np.random.default_rng(20)
    sample = list(rng.choice(g.n, size=48, replace=False))
    first_non_x = int(order[np.flatnonzero(inX[order] == 0)[0]])
    isolated = int(np.flatnonzero(g.degrees == 0)[0])
    sample += [first_non_x, isolated, int(np.argmax(sizes))]
    for u in sample:
        h, d = oracle.label_of(g.offsets, g.cols, rank, inX, int(u))
        a, b = int(L.offsets[u]), int(L.offsets[u + 1])
        assert np.array_equal(L.hubs[a:b], h), u
        assert np.array_equal(L.dists[a:b], d), u
    assert int(sizes.sum()) == ix.label_entries()


def test_sampled_sources_all_targets(rmat20):
    g, ix, _ = rmat20
    rng = np.random.default_rng(21)
    srcs = list(rng.choice(g.n, size=12, replace=False)) + [int(np.argmax(g.degrees))]
    t = np.arange(g.n, dtype=np.uint32)
    for s in srcs:
        got = gpu_query(ix, np.full(g.n, s, dtype=np.uint32), t)
        assert np.array_equal(got, oracle.bfs(g.offsets, g.cols, int(s))), s


def test_bench_pairs_symmetric_and_bounded(rmat20):
    g, ix, _ = rmat20
    s, u = gg.pairs(g.n, 10_000_000, 3)
    a = ix.query(dev_u32(s), dev_u32(u)).cpu().numpy()
    b = ix.query(dev_u32(u), dev_u32(s)).cpu().numpy()
    assert np.array_equal(a, b)
    iso = g.degrees == 0
    # isolated endpoints are unreachable unless s == t
    mask = (iso[s] | iso[u]) & (s != u)
    assert (a[mask] == 255).all()
    assert (a[s == u] == 0).all()
