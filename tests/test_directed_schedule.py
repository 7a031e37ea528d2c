"""The root-batch schedule of the directed build, restated on the CPU.

The GPU builds directed labels (Sec. 6) in root batches [k0, k1). For each
direction, all BFSs of a batch advance together and prune only with hubs
below k0. Then each direction's tuples are cleaned against the other's
pre-cleanup tuples. This file restates that schedule in plain Python and
checks the claim it rests on: for every batch size, and for any order in
which the frontier is processed, it yields exactly the labels of the
sequential method (the oracle, pinned in tests/test_oracle_directed.py).
The schedule is what csrc/pll_directed.cu implements; this file is a check
of the design on the CPU, not a test of the CUDA code, whose parity tests
are in tests/test_zzz_gpu_directed.py.
"""
import bisect
import random

import numpy as np
import pytest

import oracle
from paper_1304_4661_gb300 import graphgen as gg


def degree_order(d):
    indeg = np.bincount(d.cols.astype(np.int64), minlength=d.n)
    deg = np.diff(d.offsets.astype(np.int64)) + indeg
    return np.lexsort((np.arange(d.n), -deg)).tolist()


def schedule(d, order, bmax, rng):
    """Labels (rank space) L[0] = L_IN, L[1] = L_OUT, built batch by batch."""
    n = d.n
    rank = [0] * n
    for r, v in enumerate(order):
        rank[v] = r
    out_adj = [[] for _ in range(n)]
    in_adj = [[] for _ in range(n)]
    for v in range(n):
        for w in d.cols[d.offsets[v]:d.offsets[v + 1]].tolist():
            out_adj[rank[v]].append(rank[w])
            in_adj[rank[w]].append(rank[v])
    adj = (out_adj, in_adj)
    L = ([[] for _ in range(n)], [[] for _ in range(n)])  # (hub, dist), hubs ascending
    B, k0 = min(64, bmax), 0
    while k0 < n:
        k1 = min(k0 + B, n)
        T = ([], [])
        for dr in (0, 1):  # forward fills L_IN from L_OUT(root); reverse the other way
            frm, to = L[1 - dr], L[dr]
            seen = set((k, k) for k in range(k0, k1))
            frontier = [(k, k) for k in range(k0, k1)]
            level = 0
            while frontier:
                assert level < 255
                rng.shuffle(frontier)
                alive = []
                for u, k in frontier:
                    a = dict(frm[k])
                    if any(h in a and a[h] + x <= level for h, x in to[u]):
                        continue
                    T[dr].append((u, k, level))
                    alive.append((u, k))
                nxt = []
                for u, k in alive:
                    for w in adj[dr][u]:
                        if (w, k) not in seen:
                            seen.add((w, k))
                            nxt.append((w, k))
                frontier, level = nxt, level + 1
        S = (sorted(T[0]), sorted(T[1]))
        for dr in (0, 1):
            own, other = S[dr], S[1 - dr]
            for x, (u, k, dist) in enumerate(own):
                lo_u = bisect.bisect_left(own, (u, -1, -1), 0, x)
                lo_k = bisect.bisect_left(other, (k, -1, -1))
                hi_k = bisect.bisect_left(other, (k, k, -1), lo_k)
                mine = {h: a for _, h, a in own[lo_u:x]}
                if any(h in mine and mine[h] + b <= dist for _, h, b in other[lo_k:hi_k]):
                    continue
                L[dr][u].append((k, dist))
        k0, B = k1, min(2 * B, bmax)
    return L


def exported(L, order):
    rank = {v: r for r, v in enumerate(order)}
    return [L[rank[v]] for v in range(len(order))]


def as_lists(Lx, n):
    return [list(zip(Lx.hubs[Lx.offsets[v]:Lx.offsets[v + 1]].tolist(),
                     Lx.dists[Lx.offsets[v]:Lx.offsets[v + 1]].tolist())) for v in range(n)]


@pytest.mark.parametrize("bmax", [1, 3, 64, 1024])
@pytest.mark.parametrize("d", [gg.digraph(9, [(i, (i + 1) % 9) for i in range(9)], "dcycle9"),
                               gg.random_digraph(60, 200, 5), gg.random_digraph(150, 500, 7),
                               gg.oriented(gg.ba(200, 3, 3), 4), gg.oriented(gg.rmat(7, 8, seed=5), 6, both=0.1),
                               gg.oriented(gg.ws(150, 6, 0.1, 2), 8, both=0.5)],
                         ids=lambda d: d.name)
def test_batches_give_the_sequential_labels(d, bmax):
    rng = random.Random(bmax)
    for order in (degree_order(d), np.random.default_rng(d.n).permutation(d.n).tolist()):
        ref = oracle.DirectedIndex(d.offsets, d.cols, order=np.asarray(order, dtype=np.uint32))
        L = schedule(d, order, bmax, rng)
        assert exported(L[0], order) == as_lists(ref.labels_in(), d.n)
        assert exported(L[1], order) == as_lists(ref.labels_out(), d.n)
