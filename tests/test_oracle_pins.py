"""Pins of the CPU oracle to things other than itself (no GPU needed).

Each test checks the oracle against a fact that the paper or mathematics
fixes independently of the oracle's own code: a library BFS, the definitions
of Sec. 3 and Sec. 5.1, the closed form that Thm 4.1 / Thm 4.2 give for the
label set, a hand-worked example (tests/golden), closed forms on special
graphs (complete graph, star, path/tree with a centroid order, Thm 4.4),
minimality (Thm 4.2), and the bit-parallel bound of Sec. 5.3.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_1304_4661_gb300 import graphgen as gg

from . import brute, graphs

INF = 255
HERE = os.path.dirname(os.path.abspath(__file__))


def labels_dict(ix):
    L = ix.labels()
    out = {}
    for v in range(ix.n):
        a, b = int(L.offsets[v]), int(L.offsets[v + 1])
        out[v] = list(zip(L.hubs[a:b].tolist(), L.dists[a:b].tolist()))
    return out


def all_pairs(n):
    s, t = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    return s.ravel().astype(np.uint32), t.ravel().astype(np.uint32)


# ---------------------------------------------------------------- BFS & order
@pytest.mark.parametrize("g", graphs.small_family(), ids=lambda g: g.name)
def test_bfs_matches_library_apsp(g):
    D = brute.apsp(g.offsets, g.cols)
    for s in range(g.n):
        assert np.array_equal(oracle.bfs(g.offsets, g.cols, s), D[s].astype(np.uint8))


@pytest.mark.parametrize("g", graphs.small_family() + [gg.rmat(12, 16, seed=5)], ids=lambda g: g.name)
def test_degree_order_is_lexsort(g):
    """Sec. 4.4.2 Degree: descending degree; ties by ascending id (numpy lexsort)."""
    deg = g.degrees
    expect = np.lexsort((np.arange(g.n), -deg))
    assert np.array_equal(oracle.degree_order(g.offsets, g.cols), expect)


# ------------------------------------------------------ exact distances (Cor.)
@pytest.mark.parametrize("t", [0, 1, 2, 16, 64])
@pytest.mark.parametrize("g", graphs.small_family(), ids=lambda g: g.name)
def test_queries_equal_bfs_distance(g, t):
    """Corollary of Thm 4.1: Query(s, t, L'_n) = d_G(s, t) for every pair."""
    D = brute.apsp(g.offsets, g.cols)
    ix = oracle.Index(g.offsets, g.cols, t)
    s, u = all_pairs(g.n)
    got = ix.query_batch(s, u).reshape(g.n, g.n)
    assert np.array_equal(got.astype(np.int64), D)


@pytest.mark.parametrize("t", [0, 1, 2])
def test_exhaustive_5_vertices(t):
    """Every simple graph on 5 vertices: distances and the canonical label set."""
    for g in graphs.all_graphs(5):
        D = brute.apsp(g.offsets, g.cols)
        ix = oracle.Index(g.offsets, g.cols, t)
        s, u = all_pairs(g.n)
        assert np.array_equal(ix.query_batch(s, u).reshape(5, 5).astype(np.int64), D), g.name
        rank, inX = ix.rank_inX()
        assert labels_dict(ix) == brute.canonical(D, ix.order(), inX), g.name


@pytest.mark.parametrize("t", [0, 1, 3])
def test_every_graph_up_to_7_vertices(t):
    """Every graph on at most 7 vertices up to isomorphism (the 1,253 graphs of
    the graph atlas, in its labelling): distances and the canonical label set,
    with the bit-parallel stage taking up to t roots."""
    nx = pytest.importorskip("networkx")
    for G in nx.graph_atlas_g():
        n = G.number_of_nodes()
        e = np.asarray(list(G.edges()), dtype=np.int64).reshape(-1, 2)
        g = gg.from_edges(n, e[:, 0], e[:, 1], f"atlas{n}")
        D = brute.apsp(g.offsets, g.cols)
        ix = oracle.Index(g.offsets, g.cols, t)
        s, u = all_pairs(n)
        assert np.array_equal(ix.query_batch(s, u).reshape(n, n).astype(np.int64), D), G.edges()
        _, inX = ix.rank_inX()
        assert labels_dict(ix) == brute.canonical(D, ix.order(), inX), G.edges()


# -------------------------------------------------- canonical label set (O1)
@pytest.mark.parametrize("t", [0, 1, 3, 16])
@pytest.mark.parametrize("g", graphs.small_family(), ids=lambda g: g.name)
def test_labels_equal_closed_form(g, t):
    """The label set of Alg. 1/2 + Sec. 5.4 equals its closed form (Thm 4.1/4.2)."""
    D = brute.apsp(g.offsets, g.cols)
    ix = oracle.Index(g.offsets, g.cols, t)
    _, inX = ix.rank_inX()
    assert labels_dict(ix) == brute.canonical(D, ix.order(), inX)


@pytest.mark.parametrize("t", [0, 2, 16])
@pytest.mark.parametrize("g", graphs.small_family(), ids=lambda g: g.name)
def test_label_of_equals_closed_form(g, t):
    """orc_label_of (one BFS + predecessor DP) equals the set-based closed form."""
    D = brute.apsp(g.offsets, g.cols)
    ix = oracle.Index(g.offsets, g.cols, t)
    rank, inX = ix.rank_inX()
    canon = brute.canonical(D, ix.order(), inX)
    for u in range(g.n):
        h, d = oracle.label_of(g.offsets, g.cols, rank, inX, u)
        assert list(zip(h.tolist(), d.tolist())) == canon[u], u


def test_labels_independent_of_order_argument_identity():
    """Passing the Degree order explicitly gives the same index as NULL."""
    g = gg.ba(300, 3, 7)
    a = oracle.Index(g.offsets, g.cols, 16)
    b = oracle.Index(g.offsets, g.cols, 16, order=oracle.degree_order(g.offsets, g.cols))
    assert labels_dict(a) == labels_dict(b)


def test_random_order_still_exact():
    """Distances are exact under any order (Cor. of Thm 4.1); labels follow the
    closed form for that order."""
    g = gg.ba(150, 3, 8)
    rng = np.random.default_rng(0)
    order = rng.permutation(g.n).astype(np.uint32)
    D = brute.apsp(g.offsets, g.cols)
    for t in (0, 4):
        ix = oracle.Index(g.offsets, g.cols, t, order=order)
        s, u = all_pairs(g.n)
        assert np.array_equal(ix.query_batch(s, u).reshape(g.n, g.n).astype(np.int64), D)
        _, inX = ix.rank_inX()
        assert labels_dict(ix) == brute.canonical(D, order, inX)


# --------------------------------------------------------- hand-worked example
def test_hand_worked_example():
    fx = json.load(open(os.path.join(HERE, "golden", "hand_example_6v.json")))
    e = np.array(fx["edges"])
    g = gg.from_edges(fx["n"], e[:, 0], e[:, 1])
    assert oracle.degree_order(g.offsets, g.cols).tolist() == fx["degree_order"]
    ix0 = oracle.Index(g.offsets, g.cols, 0)
    L0 = labels_dict(ix0)
    for v, ent in fx["t0"]["labels"].items():
        assert L0[int(v)] == [tuple(x) for x in ent]
    assert oracle.Index(g.offsets, g.cols, 0).labels().hubs.shape[0] == fx["t0"]["total"]
    ix1 = oracle.Index(g.offsets, g.cols, 1)
    roots, cnt, S = ix1.bp_roots()
    assert int(roots[0]) == fx["t1"]["bp_root"]
    assert S[0, : cnt[0]].tolist() == fx["t1"]["bp_S"]
    d, m1, m0 = ix1.bp()
    assert d[:, 0].tolist() == fx["t1"]["bp"]["d"]
    assert m1[:, 0].tolist() == fx["t1"]["bp"]["m1"]
    assert m0[:, 0].tolist() == fx["t1"]["bp"]["m0"]
    L1 = labels_dict(ix1)
    for v, ent in fx["t1"]["labels"].items():
        assert L1[int(v)] == [tuple(x) for x in ent]


# ---------------------------------------------------- bit-parallel labels (O1)
@pytest.mark.parametrize("t", [1, 2, 5, 16, 64])
@pytest.mark.parametrize("g", graphs.small_family(), ids=lambda g: g.name)
def test_bp_labels_pointwise(g, t):
    """Alg. 3's DP equals the pointwise definition of S^{-1}, S^0 (Sec. 5.1)."""
    D = brute.apsp(g.offsets, g.cols)
    ix = oracle.Index(g.offsets, g.cols, t)
    roots, cnt, S = ix.bp_roots()
    d, m1, m0 = ix.bp()
    ed, e1, e0 = brute.bp_pointwise(D, roots, cnt, S)
    assert np.array_equal(d, ed)
    assert np.array_equal(m1, e1)
    assert np.array_equal(m0, e0)


@pytest.mark.parametrize("t", [1, 4, 16, 64])
@pytest.mark.parametrize("g", graphs.small_family() + [gg.rmat(10, 16, seed=9)], ids=lambda g: g.name)
def test_bp_root_selection_rule(g, t):
    """Sec. 5.4: r = highest-priority (lowest-rank) remaining vertex; S_r = up
    to 64 highest-priority remaining neighbours, bit j = j-th in rank order."""
    ix = oracle.Index(g.offsets, g.cols, t)
    order = ix.order()
    rank = np.empty(g.n, dtype=np.int64)
    rank[order] = np.arange(g.n)
    roots, cnt, S = ix.bp_roots()
    used = np.zeros(g.n, dtype=bool)
    for i in range(t):
        free = [v for v in order if not used[v]]
        if not free:
            assert roots[i] == 0xFFFFFFFF and cnt[i] == 0
            continue
        r = int(roots[i])
        assert r == free[0]
        used[r] = True
        nb = g.cols[g.offsets[r]:g.offsets[r + 1]]
        cand = sorted((int(w) for w in nb if not used[w]), key=lambda w: rank[w])
        assert S[i, : cnt[i]].tolist() == cand[:64]
        used[cand[:64]] = True
    _, inX = ix.rank_inX()
    assert np.array_equal(inX.astype(bool), used)


@pytest.mark.parametrize("g", [gg.ba(200, 4, 3), gg.ws(150, 6, 0.1, 4), gg.rmat(8, 8, seed=5)],
                         ids=lambda g: g.name)
def test_bp_query_bound(g):
    """Sec. 5.3: with d~ = d(s,r) + d(r,t), the distance via {r} U S_r is in
    [d~ - 2, d~], and the mask rule returns exactly min over {r} U S_r."""
    D = brute.apsp(g.offsets, g.cols)
    ix = oracle.Index(g.offsets, g.cols, 16)
    roots, cnt, S = ix.bp_roots()
    d, m1, m0 = ix.bp()
    for i in range(16):
        if roots[i] == 0xFFFFFFFF:
            continue
        via = [int(roots[i])] + [int(x) for x in S[i, : cnt[i]]]
        for s in range(0, g.n, 3):
            for u in range(0, g.n, 5):
                if d[s, i] == INF or d[u, i] == INF:
                    continue
                td = int(d[s, i]) + int(d[u, i])
                true_via = min(D[s, x] + D[x, u] for x in via)
                assert td - 2 <= true_via <= td
                rule = td - (2 if m1[s, i] & m1[u, i] else
                             1 if (m0[s, i] & m1[u, i]) | (m1[s, i] & m0[u, i]) else 0)
                assert rule == true_via


# ------------------------------------------------------------ closed forms
@pytest.mark.parametrize("n", [1, 2, 5, 17])
def test_complete_graph(n):
    """K_n, t = 0: root k reaches everyone at distance 1 but is pruned at all
    earlier roots, so L(v_k) = {(i, 1) : i < k} U {(k, 0)}: n(n+1)/2 entries."""
    g = graphs.complete(n)
    ix = oracle.Index(g.offsets, g.cols, 0)
    L = labels_dict(ix)
    order = ix.order()
    for k in range(n):
        assert L[int(order[k])] == [(i, 1) for i in range(k)] + [(k, 0)]
    assert sum(len(x) for x in L.values()) == n * (n + 1) // 2


def test_star():
    """Star, t = 0: the centre has the highest degree and goes first; every leaf
    gets (centre, 1) and itself; the centre gets only itself."""
    g = graphs.star(12)
    ix = oracle.Index(g.offsets, g.cols, 0)
    L = labels_dict(ix)
    assert L[0] == [(0, 0)]
    rank = {int(v): r for r, v in enumerate(ix.order())}
    for leaf in range(1, 12):
        assert L[leaf] == [(0, 1), (rank[leaf], 0)]


def centroid_order(g):
    """Centroid-decomposition order of a tree (Thm 4.4 for tree-width 1)."""
    n = g.n
    adj = [g.cols[g.offsets[v]:g.offsets[v + 1]].tolist() for v in range(n)]
    removed = [False] * n
    order = []

    def comp(v):
        seen, st = {v}, [v]
        while st:
            x = st.pop()
            for y in adj[x]:
                if not removed[y] and y not in seen:
                    seen.add(y)
                    st.append(y)
        return seen

    def centroid(c):
        size = len(c)
        for v in c:
            parts = []
            removed[v] = True
            for y in adj[v]:
                if not removed[y]:
                    parts.append(len(comp(y)))
            removed[v] = False
            if all(p <= size // 2 for p in parts):
                return v

    stack = [0] if n else []
    while stack:
        v0 = stack.pop()
        c = comp(v0)
        v = centroid(c)
        order.append(v)
        removed[v] = True
        for y in adj[v]:
            if not removed[y]:
                stack.append(y)
    return np.array(order, dtype=np.uint32)


@pytest.mark.parametrize("g", [graphs.path(100), graphs.binary_tree(127), graphs.path(255)],
                         ids=lambda g: g.name)
def test_tree_centroid_order_label_bound(g):
    """Thm 4.4 with tree-width 1: with a centroid-decomposition order every label
    of an n-vertex tree has at most floor(log2 n) + 1 entries."""
    order = centroid_order(g)
    assert sorted(order.tolist()) == list(range(g.n))
    ix = oracle.Index(g.offsets, g.cols, 0, order=order)
    L = labels_dict(ix)
    assert max(len(x) for x in L.values()) <= math.floor(math.log2(g.n)) + 1
    D = brute.apsp(g.offsets, g.cols)
    s, u = all_pairs(g.n)
    assert np.array_equal(ix.query_batch(s, u).reshape(g.n, g.n).astype(np.int64), D)


def test_finite_distance_beyond_255_is_a_range_error():
    """Distances are 8-bit with 255 = unreachable (Sec. 4.5.1, "Arrays"), so a
    finite distance of 255 or more cannot be answered: Query reports E_RANGE
    for that pair (reading 10). A 400-vertex path with a centroid order keeps
    every pruned BFS below depth 255 (the first root's reaches depth 200 and
    later BFSs stop at earlier hubs), so the index builds, yet its ends are
    399 apart. Every pair is checked against library APSP: exact below 255,
    E_RANGE from 255 up. With two bit-parallel roots the second root's
    unpruned BFS (Sec. 5.2) runs the whole path and the build is E_RANGE."""
    g = graphs.path(400)
    order = centroid_order(g)
    D = brute.apsp(g.offsets, g.cols)
    assert D.max() == 399 and (D >= 255).sum() > 0
    for t in (0, 1):
        ix = oracle.Index(g.offsets, g.cols, t, order=order)
        far = 0
        for s in range(g.n):
            for u in range(g.n):
                if D[s, u] < 255:
                    assert ix.query(s, u) == D[s, u], (t, s, u)
                else:
                    far += 1
                    with pytest.raises(oracle.OracleError) as e:
                        ix.query(s, u)
                    assert e.value.code == oracle.E_RANGE, (t, s, u)
        assert far == int((D >= 255).sum())
    with pytest.raises(oracle.OracleError) as e:
        oracle.Index(g.offsets, g.cols, 2, order=order)
    assert e.value.code == oracle.E_RANGE


def test_disconnected_and_isolated():
    g = graphs.disjoint(graphs.complete(4), graphs.path(3), graphs.complete(1))
    for t in (0, 2):
        ix = oracle.Index(g.offsets, g.cols, t)
        assert ix.query(0, 5) == INF and ix.query(4, 7) == INF and ix.query(7, 7) == 0
    ix = oracle.Index(g.offsets, g.cols, 0)
    L = labels_dict(ix)
    rank = {int(v): r for r, v in enumerate(ix.order())}
    assert L[7] == [(rank[7], 0)]  # isolated vertex: only itself


def test_self_distance_zero():
    for g in graphs.small_family():
        for t in (0, 1, 16):
            ix = oracle.Index(g.offsets, g.cols, t)
            v = np.arange(g.n, dtype=np.uint32)
            assert (ix.query_batch(v, v) == 0).all()


# --------------------------------------------------------- minimality (Thm 4.2)
@pytest.mark.parametrize("t", [0, 2])
@pytest.mark.parametrize("g", [gg.ba(30, 2, 1), gg.ws(24, 4, 0.3, 2), graphs.grid(4, 5),
                               graphs.disjoint(graphs.cycle(7), graphs.star(5))],
                         ids=lambda g: g.name)
def test_minimality_drop_one(g, t):
    """Thm 4.2: removing any single entry breaks the distance of some pair."""
    D = brute.apsp(g.offsets, g.cols)
    ix = oracle.Index(g.offsets, g.cols, t)
    L = labels_dict(ix)
    d, m1, m0 = ix.bp() if t else (None, None, None)

    def bpq(s, u):
        best = INF
        for i in range(t):
            if d[s, i] == INF or d[u, i] == INF:
                continue
            td = int(d[s, i]) + int(d[u, i])
            td -= 2 if m1[s, i] & m1[u, i] else 1 if (m0[s, i] & m1[u, i]) | (m1[s, i] & m0[u, i]) else 0
            best = min(best, td)
        return best

    BP = np.array([[bpq(s, u) for u in range(g.n)] for s in range(g.n)])
    for v in range(g.n):
        for x in range(len(L[v])):
            L2 = dict(L)
            L2[v] = L[v][:x] + L[v][x + 1:]
            broken = any(min(BP[s, u], brute.label_query(L2[s], L2[u])) != D[s, u]
                         for s in range(g.n) for u in range(g.n))
            assert broken, (v, L[v][x])


# ----------------------------------------------------------------- errors
def test_order_not_permutation():
    g = gg.ba(20, 2, 1)
    bad = np.arange(20, dtype=np.uint32)
    bad[3] = 4
    with pytest.raises(oracle.OracleError) as e:
        oracle.Index(g.offsets, g.cols, 0, order=bad)
    assert e.value.code == oracle.E_ORDER


def test_depth_range_error():
    """8-bit distances: a BFS depth of 255 or more is a range error."""
    g = graphs.path(300)
    with pytest.raises(oracle.OracleError) as e:
        oracle.Index(g.offsets, g.cols, 0)
    assert e.value.code == oracle.E_RANGE


def test_threaded_batch_query_equals_the_plain_one():
    """orc_query_batch_mt (a timing aid for the all-core query rate) answers
    exactly as the single-threaded batch query, for any thread count."""
    g = gg.rmat(12, 16, seed=4)
    ix = oracle.Index(g.offsets, g.cols, 16)
    s, u = gg.pairs(g.n, 30_001, 9)
    ref = ix.query_batch(s, u)
    for th in (1, 3, 8, 64):
        assert np.array_equal(ix.query_batch_mt(s, u, th), ref)
    assert ix.query_batch_mt(s[:2], u[:2], 16).tolist() == ref[:2].tolist()
