"""Input generators: CSR invariants, determinism, family shapes (no GPU)."""
import numpy as np
import pytest

from paper_1304_4661_gb300 import graphgen as gg


def check_csr(g):
    off = g.offsets.astype(np.int64)
    assert off[0] == 0 and (np.diff(off) >= 0).all() and off[-1] == g.nnz
    rows = np.repeat(np.arange(g.n), np.diff(off))
    cols = g.cols.astype(np.int64)
    assert (cols < g.n).all()
    assert (rows != cols).all(), "self-loop"
    # strictly ascending within each list
    same = rows[1:] == rows[:-1]
    assert (cols[1:][same] > cols[:-1][same]).all(), "unsorted or duplicate"
    # symmetric
    fwd = np.sort(rows * g.n + cols)
    bwd = np.sort(cols * g.n + rows)
    assert np.array_equal(fwd, bwd), "asymmetric"


@pytest.mark.parametrize("make", [
    lambda: gg.ba(10_000, 4, 1),
    lambda: gg.ws(5_000, 6, 0.1, 2),
    lambda: gg.rmat(14, 16, seed=3),
    lambda: gg.ba(3, 4, 1),
    lambda: gg.from_edges(5, [0, 1, 1, 3], [1, 0, 1, 4]),
])
def test_csr_invariants(make):
    check_csr(make())


def test_ba_shape():
    g = gg.ba(10_000, 4, 1)
    # (m+1)-clique plus m edges per new vertex, all distinct
    assert g.nnz == 2 * (10 + (10_000 - 5) * 4)
    assert g.degrees.min() >= 4


def test_ws_shape():
    g = gg.ws(1000, 6, 0.1, 5)
    assert g.nnz == 2 * 1000 * 3  # rewiring keeps the edge count
    assert g.degrees.min() >= 1


def test_rmat_shape():
    g = gg.rmat(12, 16, seed=1)
    assert g.n == 4096
    assert g.nnz <= 2 * 16 * 4096
    # power-law-ish: max degree far above the mean; many isolated vertices
    d = g.degrees
    assert d.max() > 20 * d.mean()
    assert (d == 0).sum() > 0


def test_determinism():
    a, b = gg.rmat(11, 8, seed=7), gg.rmat(11, 8, seed=7)
    assert np.array_equal(a.offsets, b.offsets) and np.array_equal(a.cols, b.cols)
    c = gg.rmat(11, 8, seed=8)
    assert not np.array_equal(a.cols[: min(a.nnz, c.nnz)], c.cols[: min(a.nnz, c.nnz)])
    s1, t1 = gg.pairs(1000, 100, 2)
    s2, t2 = gg.pairs(1000, 100, 2)
    assert np.array_equal(s1, s2) and np.array_equal(t1, t2)
    assert s1.max() < 1000 and t1.max() < 1000


def test_batch_specs():
    specs = gg.batch_specs()
    assert len(specs) == 256
    assert sum(1 for s in specs if s[0] == "ba") == 128
    assert all(1000 <= s[1] <= 50000 for s in specs)
    assert all(2 <= s[2] <= 8 for s in specs if s[0] == "ba")


def test_serve_request_mix():
    n = 5000
    s, t, off, many = gg.serve_requests(n, 2000, 11)
    sizes = np.diff(off.astype(np.int64))
    assert sizes.min() >= 1 and sizes.max() <= 4096
    assert (sizes[many] == 1000).all()
    assert 0.06 < many.mean() < 0.14
    normal = sizes[~many]
    # log-uniform on [1, 4096]: about half the requests below sqrt(4097) ~ 64
    assert 0.4 < (normal < 64).mean() < 0.6
    assert s.max() < n and t.max() < n and len(s) == len(t) == int(off[-1])
    for i in np.flatnonzero(many)[:20]:
        a, b = int(off[i]), int(off[i + 1])
        assert (s[a:b] == s[a]).all()
    s2, t2, off2, _ = gg.serve_requests(n, 2000, 11)
    assert np.array_equal(s, s2) and np.array_equal(t, t2) and np.array_equal(off, off2)


def test_poisson_arrivals():
    a = gg.poisson_arrivals(20000, 1000.0, 5)
    gaps = np.diff(a)
    assert a[0] == 0 and (gaps >= 0).all()
    # exponential gaps of mean 1 ms: mean and coefficient of variation near 1
    assert abs(gaps.mean() - 1000.0) < 30
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.05


def _arcs(d):
    rows = np.repeat(np.arange(d.n), np.diff(d.offsets.astype(np.int64)))
    return set(zip(rows.tolist(), d.cols.tolist()))


def test_digraph_csr_shape():
    d = gg.digraph(5, [(0, 1), (0, 1), (2, 2), (3, 0), (0, 4), (4, 3)])
    assert d.offsets.tolist() == [0, 2, 2, 2, 3, 4]
    assert d.cols.tolist() == [1, 4, 0, 3]  # repeats and the self-loop dropped, rows ascending
    e = gg.digraph(3, [])
    assert e.offsets.tolist() == [0, 0, 0, 0] and e.nnz == 0


def test_random_digraph_seeded():
    a, b, c = gg.random_digraph(200, 1000, 3), gg.random_digraph(200, 1000, 3), gg.random_digraph(200, 1000, 4)
    assert np.array_equal(a.cols, b.cols) and np.array_equal(a.offsets, b.offsets)
    assert not np.array_equal(a.cols, c.cols)
    arcs = _arcs(a)
    assert all(u != v for u, v in arcs) and 900 < len(arcs) <= 1000
    for v in range(a.n):
        row = a.cols[a.offsets[v]:a.offsets[v + 1]]
        assert (np.diff(row.astype(np.int64)) > 0).all()


def test_oriented_keeps_every_edge_once_or_both_ways():
    g = gg.ba(2000, 3, 5)
    d = gg.oriented(g, 7, both=0.3)
    arcs = _arcs(d)
    und = _arcs(gg.Digraph(g.n, g.offsets, g.cols))
    assert arcs <= und
    edges = {(u, v) for u, v in und if u < v}
    two = sum(1 for u, v in edges if (u, v) in arcs and (v, u) in arcs)
    assert all((u, v) in arcs or (v, u) in arcs for u, v in edges)
    assert abs(two / len(edges) - 0.3) < 0.03
    one_fwd = sum(1 for u, v in edges if (u, v) in arcs and (v, u) not in arcs)
    one_rev = sum(1 for u, v in edges if (v, u) in arcs and (u, v) not in arcs)
    assert abs(one_fwd - one_rev) < 0.1 * (one_fwd + one_rev)
    assert np.array_equal(gg.oriented(g, 7, both=0.3).cols, d.cols)
