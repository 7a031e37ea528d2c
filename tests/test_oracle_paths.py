"""Pins of the oracle's shortest-path queries (Sec. 6, "Shortest-Path
Queries"): the parent kept with each label entry and the paths restored from
them, checked against things other than the oracle itself:

  * a 6-vertex example worked by hand (tests/golden), parents and paths;
  * every parent against a library all-pairs BFS (scipy): the hub's own entry
    names the hub, any other names a neighbour one hop nearer to the hub, and
    that neighbour holds the hub one hop lower (so the tree can be climbed);
  * on trees, where shortest paths are unique, parents and paths equal the
    library's predecessor matrix exactly;
  * on every pair of a family of small graphs and on sampled pairs of larger
    ones, a path is a walk along edges from s to t with d_G(s, t) + 1
    vertices, i.e. a shortest path, and is empty exactly when t is
    unreachable.
"""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import shortest_path

import oracle
from paper_1304_4661_gb300 import graphgen as gg

from . import brute, graphs
from .paths_util import adjacency_sets, check_parents, check_path

HERE = os.path.dirname(os.path.abspath(__file__))
INF = 255


def test_hand_worked_parents_and_paths():
    fx = json.load(open(os.path.join(HERE, "golden", "hand_example_6v.json")))
    e = np.asarray(fx["edges"])
    g = gg.from_edges(fx["n"], e[:, 0], e[:, 1], "hand6")
    for key, t in (("t0", 0), ("t1", 1)):
        ix = oracle.Index(g.offsets, g.cols, t)
        L, P = ix.labels(), ix.parents()
        for v in range(g.n):
            got = P[L.offsets[v]:L.offsets[v + 1]].tolist()
            assert got == fx[key]["parents"][str(v)], (key, v)
        for s, u, expect in fx[key]["paths"]:
            assert ix.path(s, u).tolist() == expect, (key, s, u)


@pytest.mark.parametrize("t", [0, 1, 4, 16])
@pytest.mark.parametrize("g", graphs.small_family(), ids=lambda g: g.name)
def test_parents_and_every_path(g, t):
    D = brute.apsp(g.offsets, g.cols)
    ix = oracle.Index(g.offsets, g.cols, t)
    check_parents(g, ix.labels(), ix.parents(), ix.order(), D)
    adj = adjacency_sets(g)
    for s in range(g.n):
        for u in range(g.n):
            check_path(ix.path(s, u), s, u, D, adj)


def random_tree(n, seed):
    rng = np.random.default_rng(seed)
    par = np.array([rng.integers(0, v) for v in range(1, n)], dtype=np.int64)
    perm = rng.permutation(n)
    return gg.from_edges(n, perm[np.arange(1, n)], perm[par], f"tree{n}_{seed}")


def tree_path(pred, s, u):
    """The unique s-u path of a tree from the library's predecessor matrix:
    pred[u, v] is the vertex before v on the path from u."""
    out = [s]
    while out[-1] != u:
        out.append(int(pred[u, out[-1]]))
    return out


@pytest.mark.parametrize("t", [0, 3, 16])
@pytest.mark.parametrize("n,seed", [(2, 1), (40, 2), (150, 3)])
def test_trees_parents_and_paths_are_unique(n, seed, t):
    g = random_tree(n, seed)
    rows = np.repeat(np.arange(n), np.diff(g.offsets.astype(np.int64)))
    A = sp.csr_matrix((np.ones(len(g.cols)), (rows, g.cols.astype(np.int64))), shape=(n, n))
    _, pred = shortest_path(A, unweighted=True, directed=False, return_predecessors=True)
    ix = oracle.Index(g.offsets, g.cols, t)
    L, P, order = ix.labels(), ix.parents(), ix.order()
    for v in range(n):
        for x in range(int(L.offsets[v]), int(L.offsets[v + 1])):
            hv = int(order[int(L.hubs[x])])
            assert int(P[x]) == (v if hv == v else int(pred[hv, v])), (v, hv)
    for s in range(n):
        for u in range(n):
            assert ix.path(s, u).tolist() == tree_path(pred, s, u), (s, u)


@pytest.mark.parametrize("g,t", [(gg.ba(2000, 3, 1), 16), (gg.ws(1500, 6, 0.1, 2), 16),
                                 (gg.rmat(11, 8, seed=4), 64), (gg.rmat(11, 8, seed=4), 0)],
                         ids=lambda x: getattr(x, "name", str(x)))
def test_sampled_paths_larger_graphs(g, t):
    D = brute.apsp(g.offsets, g.cols)
    ix = oracle.Index(g.offsets, g.cols, t)
    check_parents(g, ix.labels(), ix.parents(), ix.order(), D)
    adj = adjacency_sets(g)
    s, u = gg.pairs(g.n, 3000, 9)
    for a, b in zip(s.tolist(), u.tolist()):
        check_path(ix.path(a, b), a, b, D, adj)


def test_path_bad_id():
    g = graphs.path(4)
    ix = oracle.Index(g.offsets, g.cols, 0)
    with pytest.raises(oracle.OracleError):
        ix.path(0, 4)
