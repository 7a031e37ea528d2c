"""Small named graphs for tests, all built through the seeded input generators."""
from __future__ import annotations

import itertools

import numpy as np

from paper_1304_4661_gb300 import graphgen as gg


def complete(n):
    e = list(itertools.combinations(range(n), 2))
    return _edges(n, e, f"K{n}")


def star(n):
    return _edges(n, [(0, i) for i in range(1, n)], f"star{n}")


def path(n):
    return _edges(n, [(i, i + 1) for i in range(n - 1)], f"path{n}")


def cycle(n):
    return _edges(n, [(i, (i + 1) % n) for i in range(n)], f"cycle{n}")


def binary_tree(n):
    return _edges(n, [((i - 1) // 2, i) for i in range(1, n)], f"bintree{n}")


def grid(a, b):
    e = []
    for i in range(a):
        for j in range(b):
            v = i * b + j
            if j + 1 < b:
                e.append((v, v + 1))
            if i + 1 < a:
                e.append((v, v + b))
    return _edges(a * b, e, f"grid{a}x{b}")


def disjoint(*gs):
    n = sum(g.n for g in gs)
    us, vs, base = [], [], 0
    for g in gs:
        rows = np.repeat(np.arange(g.n), np.diff(g.offsets.astype(np.int64)))
        us.append(rows + base)
        vs.append(g.cols.astype(np.int64) + base)
        base += g.n
    u = np.concatenate(us) if us else np.zeros(0)
    v = np.concatenate(vs) if vs else np.zeros(0)
    return gg.from_edges(n, u, v, "+".join(g.name for g in gs))


def _edges(n, e, name):
    e = np.asarray(e, dtype=np.int64).reshape(-1, 2)
    return gg.from_edges(n, e[:, 0], e[:, 1], name)


def small_family():
    """A mix of structures: power-law, small-world, grids, trees, disconnected."""
    gs = [
        complete(1), complete(2), complete(6), star(9), path(12), cycle(11), binary_tree(31),
        grid(5, 7),
        gg.ba(60, 2, 11), gg.ba(120, 3, 12), gg.ba(200, 4, 13),
        gg.ws(60, 4, 0.2, 21), gg.ws(150, 6, 0.1, 22),
        gg.rmat(6, 8, seed=31), gg.rmat(7, 8, seed=32), gg.rmat(8, 4, seed=33),
        disjoint(gg.ba(40, 2, 41), path(7), complete(1), star(5)),
        gg.from_edges(10, [], [], "empty10"),
    ]
    return gs


def all_graphs(n):
    """Every labelled simple graph on n vertices (2^(n choose 2) of them)."""
    pairs = list(itertools.combinations(range(n), 2))
    for mask in range(1 << len(pairs)):
        e = [pairs[i] for i in range(len(pairs)) if mask >> i & 1]
        yield _edges(n, e, f"g{n}_{mask}")
