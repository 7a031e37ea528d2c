"""Shortest-path queries (Sec. 6) on the GPU: pll_paths_create,
pll_paths_parents, pll_path_offsets and pll_path_query.

Many paths and parents are correct for one pair or one entry, so the tests
compare what is unique and check that the rest is valid:
  * unique: every path's vertex count is d(s, t) + 1 with the oracle's
    distance (0 when unreachable), and so is every slot of pll_path_offsets;
    on trees the whole path is unique and equals the oracle's path exactly;
  * valid: a path starts at s, ends at t and follows edges; a parent is a
    neighbour whose label holds the hub one hop lower (labels equal the
    oracle's, so that neighbour is one hop nearer to the hub).
"""
import numpy as np
import pytest

import oracle
from paper_1304_4661_gb300 import graphgen as gg
from paper_1304_4661_gb300 import pll

from . import brute, graphs
from .gpu_util import dev_u32, gpu_build, same_labels
from .paths_util import adjacency_sets, check_parents, check_path

pytestmark = pytest.mark.gpu

INF = 255


def make_paths(g, ix):
    return pll.Paths(ix, dev_u32(g.offsets), dev_u32(g.cols))


def host_paths(P, s, u):
    return P.paths(dev_u32(s), dev_u32(u))


def expected_offsets(d):
    lens = np.where(d == INF, 0, d.astype(np.int64) + 1)
    return np.concatenate([[0], np.cumsum(lens)])


@pytest.mark.parametrize("t", [0, 1, 16, 64])
@pytest.mark.parametrize("g", graphs.small_family(), ids=lambda g: g.name)
def test_every_pair_small_graphs(g, t):
    ix = gpu_build(g, t)
    ref = oracle.Index(g.offsets, g.cols, t)
    L = ix.labels()
    assert same_labels(L, ref.labels())
    with make_paths(g, ix) as P:
        D = brute.apsp(g.offsets, g.cols)
        check_parents(g, L, P.parents(), ix.order(), D)
        s = np.repeat(np.arange(g.n, dtype=np.uint32), g.n)
        u = np.tile(np.arange(g.n, dtype=np.uint32), g.n)
        off, tot = P.offsets(dev_u32(s), dev_u32(u))
        d = ref.query_batch(s, u)
        assert np.array_equal(off.cpu().numpy(), expected_offsets(d)) and tot == int(expected_offsets(d)[-1])
        adj = adjacency_sets(g)
        for a, b, p in zip(s.tolist(), u.tolist(), host_paths(P, s, u)):
            check_path(p, a, b, D, adj)


def random_tree(n, seed):
    rng = np.random.default_rng(seed)
    par = np.array([rng.integers(0, v) for v in range(1, n)], dtype=np.int64)
    perm = rng.permutation(n)
    return gg.from_edges(n, perm[np.arange(1, n)], perm[par], f"tree{n}_{seed}")


@pytest.mark.parametrize("t", [0, 3, 16])
def test_trees_equal_oracle_exactly(t):
    g = random_tree(300, 5)
    ix = gpu_build(g, t)
    ref = oracle.Index(g.offsets, g.cols, t)
    with make_paths(g, ix) as P:
        assert np.array_equal(P.parents(), ref.parents())  # one parent per entry on a tree
        s, u = gg.pairs(g.n, 4000, 6)
        for a, b, p in zip(s.tolist(), u.tolist(), host_paths(P, s, u)):
            assert p.tolist() == ref.path(a, b).tolist(), (a, b)


@pytest.mark.parametrize("g,t", [(gg.ba(10000, 4, 1), 16), (gg.ws(5000, 6, 0.1, 2), 16),
                                 (gg.rmat(13, 16, seed=4), 64), (gg.rmat(12, 8, seed=7), 0)],
                         ids=lambda x: getattr(x, "name", str(x)))
def test_sampled_pairs_larger_graphs(g, t):
    """Several tiles of pairs and a ragged tail (20011 pairs)."""
    ix = gpu_build(g, t)
    ref = oracle.Index(g.offsets, g.cols, t)
    L = ix.labels()
    assert same_labels(L, ref.labels())
    adj = adjacency_sets(g)
    with make_paths(g, ix) as P:
        check_parents(g, L, P.parents(), ix.order())
        s, u = gg.pairs(g.n, 20011, 8)
        d = ref.query_batch(s, u)
        off, _ = P.offsets(dev_u32(s), dev_u32(u))
        assert np.array_equal(off.cpu().numpy(), expected_offsets(d))
        paths = host_paths(P, s, u)
        for a, b, dd, p in zip(s.tolist(), u.tolist(), d.tolist(), paths):
            if dd == INF:
                assert len(p) == 0
                continue
            assert len(p) == dd + 1 and p[0] == a and p[-1] == b, (a, b, dd, p)
            assert all(int(y) in adj[int(x)] for x, y in zip(p[:-1], p[1:])), (a, b, p)


def test_fullsize_rmat20_sources():
    """R-MAT-20, t = 64 (the benchmark's index): paths from 6 sources (among
    them the highest-degree vertex) to 2000 targets each, against plain BFS."""
    g = gg.rmat(20, 16, seed=1)
    ix = gpu_build(g, 64)
    rng = np.random.default_rng(20)
    with make_paths(g, ix) as P:
        off = g.offsets.astype(np.int64)
        for src in list(rng.choice(g.n, 5, replace=False)) + [int(np.argmax(g.degrees))]:
            dist = oracle.bfs(g.offsets, g.cols, int(src))
            tg = rng.integers(0, g.n, 2000).astype(np.uint32)
            s = np.full(len(tg), src, dtype=np.uint32)
            for b, p in zip(tg.tolist(), host_paths(P, s, tg)):
                if dist[b] == INF:
                    assert len(p) == 0
                    continue
                assert len(p) == dist[b] + 1 and p[0] == src and p[-1] == b
                for x, y in zip(p[:-1].tolist(), p[1:].tolist()):
                    row = g.cols[off[x]:off[x + 1]]
                    k = np.searchsorted(row, y)
                    assert k < len(row) and row[k] == y, (src, b, p)


def test_batch_index_paths():
    gl = [gg.ba(300, 3, 2), graphs.path(40), gg.ws(200, 4, 0.2, 3), graphs.star(30)]
    off, col, start = gg.union(gl)
    ix = pll.Index.build_batch(dev_u32(off), dev_u32(col), start, t=4)
    adj = [set(col[off[v]:off[v + 1]].tolist()) for v in range(len(off) - 1)]
    with pll.Paths(ix, dev_u32(off), dev_u32(col)) as P:
        s, u = gg.pairs(int(start[-1]), 6000, 3)
        d = ix.query(dev_u32(s), dev_u32(u)).cpu().numpy()
        same = np.searchsorted(start, s, side="right") == np.searchsorted(start, u, side="right")
        assert (d[~same] == INF).all()
        for a, b, dd, p in zip(s.tolist(), u.tolist(), d.tolist(), host_paths(P, s, u)):
            gi = int(np.searchsorted(start, a, side="right") - 1)
            base = int(start[gi])
            if dd == INF:
                assert len(p) == 0
                continue
            ref = oracle.bfs(gl[gi].offsets, gl[gi].cols, a - base)
            assert dd == ref[b - base]
            assert len(p) == dd + 1 and p[0] == a and p[-1] == b
            assert all(int(y) in adj[int(x)] for x, y in zip(p[:-1], p[1:]))


def test_self_pairs_empty_batch_and_slot_fill():
    import torch
    g = gg.ba(500, 3, 4)
    ix = gpu_build(g, 16)
    with make_paths(g, ix) as P:
        off, path = P.query(dev_u32(np.zeros(0, np.uint32)), dev_u32(np.zeros(0, np.uint32)))
        assert off.cpu().tolist() == [0] and path.numel() == 0
        v = np.arange(50, dtype=np.uint32)
        for a, p in zip(v.tolist(), host_paths(P, v, v)):
            assert p.tolist() == [a]
        # slots larger than the paths: the rest is 0xffffffff
        s, u = gg.pairs(g.n, 100, 5)
        d = ix.query(dev_u32(s), dev_u32(u)).cpu().numpy()
        big = torch.arange(0, 101 * 300, 300, dtype=torch.int64, device="cuda")
        _, path = P.query(dev_u32(s), dev_u32(u), path_off=big, cap=100 * 300)
        h = path.cpu().numpy().view(np.uint32).reshape(100, 300)
        for i in range(100):
            k = int(d[i]) + 1 if d[i] != INF else 0
            if k:
                assert h[i, 0] == s[i] and h[i, k - 1] == u[i]
            assert (h[i, k:] == 0xFFFFFFFF).all()


def test_rejections():
    import torch
    g = gg.ba(400, 3, 6)
    ix = gpu_build(g, 8)
    with make_paths(g, ix) as P:
        s = np.array([1, 2, 400], dtype=np.uint32)  # 400 >= n
        u = np.array([5, 6, 7], dtype=np.uint32)
        with pytest.raises(pll.PLLError) as e:
            P.offsets(dev_u32(s), dev_u32(u))
        assert e.value.code == pll.PLL_E_INVAL
        with pytest.raises(pll.PLLError):
            P.query(dev_u32(s), dev_u32(u), path_off=torch.zeros(4, dtype=torch.int64, device="cuda"), cap=0)
        s, u = gg.pairs(g.n, 64, 7)
        d = ix.query(dev_u32(s), dev_u32(u)).cpu().numpy()
        i = int(np.argmax(d))
        assert 1 <= d[i] < INF
        good, tot = P.offsets(dev_u32(s), dev_u32(u))
        short = good.clone()
        short[i + 1:] -= 1  # pair i's slot one vertex short
        with pytest.raises(pll.PLLError) as e:
            P.query(dev_u32(s), dev_u32(u), path_off=short, cap=tot)
        assert e.value.code == pll.PLL_E_INVAL
        with pytest.raises(pll.PLLError):  # offsets past cap
            P.query(dev_u32(s), dev_u32(u), path_off=good, cap=tot - 1)
        dec = good.clone()
        dec[10] = dec[11] + 1  # decreasing offsets
        with pytest.raises(pll.PLLError):
            P.query(dev_u32(s), dev_u32(u), path_off=dec, cap=tot + 1)
        # the object still answers afterwards
        _, tot2 = P.offsets(dev_u32(s), dev_u32(u))
        assert tot2 == tot


def test_create_checks_the_graph():
    g = graphs.path(8)
    ix = gpu_build(g, 0)
    with pytest.raises(pll.PLLError):  # another vertex count
        pll.Paths(ix, dev_u32(graphs.path(9).offsets), dev_u32(graphs.path(9).cols))
    # same n and nnz, other edges: vertex 0 holds the first hub (vertex 1) at
    # distance 1, but its only neighbour here (2) holds that hub at 1, not 0
    h = gg.from_edges(8, [0, 1, 2, 3, 4, 5, 6], [2, 3, 1, 4, 5, 6, 7], "other")
    assert h.offsets[-1] == g.offsets[-1]
    with pytest.raises(pll.PLLError) as e:
        pll.Paths(ix, dev_u32(h.offsets), dev_u32(h.cols))
    assert e.value.code == pll.PLL_E_INVAL
    bad = g.cols.copy()
    bad[0] = 3  # asymmetric
    with pytest.raises(pll.PLLError):
        pll.Paths(ix, dev_u32(g.offsets), dev_u32(bad))


def test_empty_graph_and_no_leaks():
    import gc
    gc.collect()
    base = pll.load().pll_test_live_allocs()
    g = gg.from_edges(5, [], [], "empty5")
    ix = gpu_build(g, 2)
    with make_paths(g, ix) as P:
        s = np.array([0, 1, 4], dtype=np.uint32)
        u = np.array([0, 2, 4], dtype=np.uint32)
        assert [p.tolist() for p in host_paths(P, s, u)] == [[0], [], [4]]
    ix.close()
    assert pll.load().pll_test_live_allocs() == base
