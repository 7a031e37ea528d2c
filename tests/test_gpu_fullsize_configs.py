"""Parity at the full sizes of the batch, serving and learned-order
configurations, in the launch configuration bench.py times (default build
options), checked on what the oracle can compute piece by piece:

  * 256 uneven graphs in one batch build: six graphs (among them the smallest
    and the largest Barabasi-Albert graphs and the smallest and a mid-size
    Watts-Strogatz one) against the oracle built on each alone:
    order, bit-parallel roots and sampled pairs; pairs across graphs answer
    255;
  * R-MAT-22 (t = 64) behind the serving loop: every answer of a stream of
    requests from the benchmark's mix equals the direct query path, and the
    direct path equals plain BFS from sampled sources;
  * R-MAT-21 (t = 64) ordered by a network trained on R-MAT graphs: distances
    from sampled sources equal plain BFS (the labels are exact for any order).
"""
import numpy as np
import pytest

import oracle
from paper_1304_4661_gb300 import graphgen as gg
from paper_1304_4661_gb300 import learned as L
from paper_1304_4661_gb300 import pll

from .gpu_util import dev_u32, gpu_build, gpu_query

pytestmark = pytest.mark.gpu


def test_batch_of_256_uneven_graphs():
    """Every label of a batch build is compared at smaller batch sizes
    (test_gpu_batch.py); at the full size, each selected graph's order,
    bit-parallel roots and sampled distances are compared with the oracle
    built on that graph alone."""
    specs = gg.batch_specs(256, seed=4)
    gl = [gg.make(sp) for sp in specs]
    off, col, start = gg.union(gl)
    t = 16
    ix = pll.Index.build_batch(dev_u32(off), dev_u32(col), start, t=t)
    order = ix.order()
    roots, cnt, S = ix.bp_roots()
    owner = np.searchsorted(start, order, side="right") - 1
    # the smallest and largest Barabasi-Albert graphs, the smallest and a
    # mid-size Watts-Strogatz graph (the oracle needs minutes for the largest
    # ones, whose labels are long), and two more
    for gi in (83, 111, 136, 254, 0, 200):
        g, b = gl[gi], int(start[gi])
        ref = oracle.Index(g.offsets, g.cols, t)
        assert np.array_equal(order[owner == gi] - b, ref.order()), gi
        r_roots, r_cnt, _ = ref.bp_roots()
        rr = roots[gi * t:(gi + 1) * t].astype(np.int64)
        assert np.array_equal(np.where(rr == pll.NONE, pll.NONE, rr - b), r_roots), gi
        assert np.array_equal(cnt[gi * t:(gi + 1) * t], r_cnt), gi
        s, u = gg.pairs(g.n, 5000, 40 + gi)
        assert np.array_equal(gpu_query(ix, s + np.uint32(b), u + np.uint32(b)), ref.query_batch(s, u)), gi
    # pairs across graphs are unreachable
    rng = np.random.default_rng(2)
    s = rng.integers(0, int(start[-1]), 20000).astype(np.uint32)
    u = rng.integers(0, int(start[-1]), 20000).astype(np.uint32)
    cross = (np.searchsorted(start, s, side="right") != np.searchsorted(start, u, side="right"))
    assert (gpu_query(ix, s, u)[cross] == 255).all()


def bfs_check(g, ix, sources):
    t = np.arange(g.n, dtype=np.uint32)
    for s in sources:
        got = gpu_query(ix, np.full(g.n, s, dtype=np.uint32), t)
        assert np.array_equal(got, oracle.bfs(g.offsets, g.cols, int(s))), s


def test_serving_rmat22():
    g = gg.rmat(22, 16, seed=6)
    ix = gpu_build(g, 64)
    rng = np.random.default_rng(22)
    srcs = list(rng.choice(g.n, size=4, replace=False)) + [int(np.argmax(g.degrees))]
    bfs_check(g, ix, srcs)
    s, u, off, _ = gg.serve_requests(g.n, 20000, seed=8)
    off = off.astype(np.int64)
    direct = ix.query(s, u)
    with pll.Server(ix) as sv:
        out, lat, _ = sv.replay(s, u, off, np.zeros(len(off) - 1))
        st = sv.stats()
    assert np.array_equal(out, direct)
    assert st["batches"] < len(off) - 1 and (lat > 0).all()


def test_learned_order_rmat21():
    specs = gg.learned_training_specs(40, scales=(12, 13, 14))
    X, y, rows, _ = L.harvest([gg.rmat(sc, 16, seed=sd) for sc, sd in specs], t=64)
    mlp, _ = L.train(X, y, rows, epochs=2, batch=16384, lr=2e-3)
    g = gg.rmat(21, 16, seed=5)
    order = L.learned_order(mlp, g, t=64).cpu().numpy().astype(np.uint32)
    assert np.array_equal(np.sort(order), np.arange(g.n, dtype=np.uint32))
    ix = gpu_build(g, 64, order=order)
    assert np.array_equal(ix.order(), order)
    rng = np.random.default_rng(21)
    bfs_check(g, ix, list(rng.choice(g.n, size=4, replace=False)) + [int(order[0])])
