"""Pins of the oracle's directed labels (Sec. 6, "Directed Graphs"): L_IN and
L_OUT from a forward and a reverse pruned BFS per root.

Pinned to things other than the oracle:
  * a 4-vertex digraph worked by hand (tests/golden);
  * every distance against a library directed all-pairs BFS (scipy);
  * every label against its closed form (tests/brute.py): (v_j, d) is in
    L_IN(u) iff no earlier vertex lies on a shortest v_j -> u path, and in
    L_OUT(u) iff none lies on a shortest u -> v_j path;
  * a digraph with every arc in both directions is an undirected graph: both
    label sets equal the undirected oracle's labels (t = 0, same order);
  * minimality: dropping any entry breaks some distance (Thm 4.2 along arcs);
  * the Degree order counts in- plus out-arcs, ties by ascending id.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1304_4661_gb300 import graphgen as gg

from . import brute, graphs

HERE = os.path.dirname(os.path.abspath(__file__))
INF = 255


def family():
    """(name, offsets, cols) of small digraphs: cycle, path, DAG, stars,
    empty, single vertex, uniform random arcs, oriented power-law graphs."""
    gs = [gg.digraph(9, [(i, (i + 1) % 9) for i in range(9)], "dcycle9"),
          gg.digraph(12, [(i, i + 1) for i in range(11)], "dpath12"),
          gg.digraph(10, [(i, j) for i in range(10) for j in range(i + 1, 10) if (i * 7 + j) % 3 == 0], "dag"),
          gg.digraph(8, [(0, i) for i in range(1, 8)], "out_star"),
          gg.digraph(8, [(i, 0) for i in range(1, 8)], "in_star"),
          gg.digraph(6, [], "empty6"), gg.digraph(1, [], "single")]
    for n, m, sd in ((20, 30, 1), (30, 45, 2), (40, 160, 3), (60, 110, 4), (80, 260, 5)):
        gs.append(gg.random_digraph(n, m, sd))
    gs += [gg.oriented(gg.ba(70, 2, 3), 4), gg.oriented(gg.rmat(6, 4, seed=5), 6, both=0.1)]
    return [(d.name, (d.offsets, d.cols)) for d in gs]


def as_dict(L, n):
    return {u: list(zip(L.hubs[L.offsets[u]:L.offsets[u + 1]].tolist(),
                        L.dists[L.offsets[u]:L.offsets[u + 1]].tolist())) for u in range(n)}


def test_hand_worked_example():
    fx = json.load(open(os.path.join(HERE, "golden", "hand_example_directed_4v.json")))
    d = gg.digraph(fx["n"], fx["arcs"])
    off, col = d.offsets, d.cols
    ix = oracle.DirectedIndex(off, col)
    assert ix.order().tolist() == fx["degree_order"]
    Lin, Lout = as_dict(ix.labels_in(), 4), as_dict(ix.labels_out(), 4)
    for u in range(4):
        assert [list(e) for e in Lin[u]] == fx["labels_in"][str(u)], u
        assert [list(e) for e in Lout[u]] == fx["labels_out"][str(u)], u
    for s in range(4):
        for t in range(4):
            assert ix.query(s, t) == fx["distances"][s][t], (s, t)


@pytest.mark.parametrize("name,g", family(), ids=lambda x: x if isinstance(x, str) else "")
def test_distances_and_closed_form(name, g):
    off, col = g
    n = len(off) - 1
    D = brute.apsp_directed(off, col)
    for order in (None, np.random.default_rng(n).permutation(n).astype(np.uint32)):
        ix = oracle.DirectedIndex(off, col, order=order)
        s = np.repeat(np.arange(n, dtype=np.uint32), n)
        t = np.tile(np.arange(n, dtype=np.uint32), n)
        assert np.array_equal(ix.query_batch(s, t).astype(np.int64), D.reshape(-1)), name
        Lin, Lout = brute.canonical_directed(D, ix.order())
        assert as_dict(ix.labels_in(), n) == Lin, name
        assert as_dict(ix.labels_out(), n) == Lout, name


@pytest.mark.parametrize("n", [2, 3, 4])
def test_every_digraph_up_to_4_vertices(n):
    """Every labelled digraph without self-loops on n vertices (2^(n(n-1))
    of them): distances and both label sets against their closed forms."""
    pairs = [(a, b) for a in range(n) for b in range(n) if a != b]
    s = np.repeat(np.arange(n, dtype=np.uint32), n)
    t = np.tile(np.arange(n, dtype=np.uint32), n)
    for mask in range(1 << len(pairs)):
        d = gg.digraph(n, [pairs[i] for i in range(len(pairs)) if mask >> i & 1])
        D = brute.apsp_directed(d.offsets, d.cols)
        ix = oracle.DirectedIndex(d.offsets, d.cols)
        assert np.array_equal(ix.query_batch(s, t).astype(np.int64), D.reshape(-1)), mask
        Lin, Lout = brute.canonical_directed(D, ix.order())
        assert as_dict(ix.labels_in(), n) == Lin and as_dict(ix.labels_out(), n) == Lout, mask


def test_degree_order_counts_in_and_out_arcs():
    d = gg.random_digraph(70, 240, 9)
    off, col, n = d.offsets, d.cols, 70
    indeg = np.bincount(col.astype(np.int64), minlength=n)
    deg = np.diff(off.astype(np.int64)) + indeg
    expect = np.lexsort((np.arange(n), -deg))
    assert np.array_equal(oracle.DirectedIndex(off, col).order(), expect)


@pytest.mark.parametrize("g", [graphs.path(10), graphs.cycle(9), graphs.grid(4, 5), gg.ba(120, 3, 12),
                               gg.ws(100, 4, 0.2, 22), gg.rmat(8, 4, seed=33),
                               graphs.disjoint(graphs.star(6), graphs.path(5))],
                         ids=lambda g: g.name)
def test_symmetric_digraph_is_the_undirected_method(g):
    d = oracle.DirectedIndex(g.offsets, g.cols)
    u = oracle.Index(g.offsets, g.cols, 0)
    assert np.array_equal(d.order(), u.order())
    Lu = u.labels()
    for L in (d.labels_in(), d.labels_out()):
        assert np.array_equal(L.offsets, Lu.offsets)
        assert np.array_equal(L.hubs, Lu.hubs) and np.array_equal(L.dists, Lu.dists)


@pytest.mark.parametrize("seed", [11, 12, 13])
def test_minimality_drop_one(seed):
    """Thm 4.2 along arcs: every entry is needed by some pair."""
    d = gg.random_digraph(18, 40, seed)
    off, col, n = d.offsets, d.cols, 18
    D = brute.apsp_directed(off, col)
    ix = oracle.DirectedIndex(off, col)
    Lin, Lout = as_dict(ix.labels_in(), n), as_dict(ix.labels_out(), n)

    def dist(Lo, Li, s, t):
        a = dict(Lo[s])
        return min([a[h] + x for h, x in Li[t] if h in a], default=INF)

    for side in ("in", "out"):
        L = Lin if side == "in" else Lout
        for u in range(n):
            for k in range(len(L[u])):
                cut = dict(L)
                cut[u] = L[u][:k] + L[u][k + 1:]
                Li, Lo = (cut, Lout) if side == "in" else (Lin, cut)
                broken = any(dist(Lo, Li, s, t) != D[s, t] for s in range(n) for t in range(n)
                             if D[s, t] < INF)
                assert broken, (side, u, L[u][k])


def test_bad_inputs_and_range():
    d = gg.digraph(4, [(0, 1), (1, 2)])
    off, col = d.offsets, d.cols
    with pytest.raises(oracle.OracleError) as e:
        oracle.DirectedIndex(off, col, order=np.array([0, 1, 1, 3], dtype=np.uint32))
    assert e.value.code == oracle.E_ORDER
    bad = col.copy()
    bad[0] = 7
    with pytest.raises(oracle.OracleError) as e:
        oracle.DirectedIndex(off, bad)
    assert e.value.code == oracle.E_INVAL
    d = gg.digraph(300, [(i, i + 1) for i in range(299)])
    off, col = d.offsets, d.cols
    with pytest.raises(oracle.OracleError) as e:
        oracle.DirectedIndex(off, col)
    assert e.value.code == oracle.E_RANGE
    d = gg.digraph(255, [(i, i + 1) for i in range(254)])
    off, col = d.offsets, d.cols
    ix = oracle.DirectedIndex(off, col)
    assert ix.query(0, 254) == 254 and ix.query(254, 0) == INF
