"""Checks shared by the oracle's and the GPU's shortest-path tests (Sec. 6):
a path is a shortest walk, a parent is a neighbour one hop nearer to the hub
that holds the hub one hop lower."""
from __future__ import annotations

import numpy as np

INF = 255


def adjacency_sets(g):
    off = g.offsets.astype(np.int64)
    return [set(g.cols[off[v]:off[v + 1]].tolist()) for v in range(g.n)]


def check_path(p, s, u, D, adj):
    d = int(D[s, u])
    if d >= INF:
        assert len(p) == 0, (s, u, p)
        return
    assert len(p) == d + 1, (s, u, d, p)
    assert p[0] == s and p[-1] == u, (s, u, p)
    for a, b in zip(p[:-1], p[1:]):
        assert b in adj[a], (s, u, p)


def check_parents(g, L, P, order, D=None):
    """Every parent of the exported labels L (P in their layout, caller ids),
    against the graph and, when D (all-pairs distances) is given, against it."""
    adj = adjacency_sets(g)
    where = {}
    for v in range(g.n):
        for x in range(int(L.offsets[v]), int(L.offsets[v + 1])):
            where[(v, int(L.hubs[x]))] = int(L.dists[x])
    for v in range(g.n):
        for x in range(int(L.offsets[v]), int(L.offsets[v + 1])):
            h, d, p = int(L.hubs[x]), int(L.dists[x]), int(P[x])
            hv = int(order[h])
            if d == 0:
                assert p == v == hv, (v, h, p)
                continue
            assert p in adj[v], (v, h, p)
            if D is not None:
                assert D[hv, p] == d - 1, (v, h, p)
            assert where.get((p, h)) == d - 1, (v, h, p)
