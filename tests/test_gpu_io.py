"""pll_save / pll_load: a loaded index is the saved one, and a damaged file
is refused before anything reaches the device."""
import os

import numpy as np
import pytest

from paper_1304_4661_gb300 import graphgen as gg
from paper_1304_4661_gb300 import pll

from .gpu_util import dev_u32, gpu_build, gpu_query, same_labels

pytestmark = pytest.mark.gpu


def same_index(a, b, g):
    assert np.array_equal(a.order(), b.order())
    assert same_labels(a.labels(), b.labels())
    if a.t:
        for x, y in zip(a.bp(), b.bp()):
            assert np.array_equal(x, y)
        for x, y in zip(a.bp_roots(), b.bp_roots()):
            assert np.array_equal(x, y)
    s, u = gg.pairs(g.n, 20000, 5)
    assert np.array_equal(gpu_query(a, s, u), gpu_query(b, s, u))


@pytest.mark.parametrize("t", [0, 16])
def test_round_trip(tmp_path, t):
    g = gg.rmat(13, 16, seed=4)
    ix = gpu_build(g, t)
    p = tmp_path / "ix.pll"
    ix.save(p)
    assert os.path.getsize(p) == 48 + g.n * 8 + g.n * ((t + 15) // 16 * 16) + g.n * t * 16 \
        + t * (2 + 64) * 4 + (g.n + 1) * 8 + ix.label_entries() * 4
    jx = pll.Index.load(p)
    same_index(ix, jx, g)
    assert jx.stats()["label_entries"] == ix.label_entries()


def test_round_trip_batch_index(tmp_path):
    gl = [gg.ba(700, 3, 1), gg.ws(500, 6, 0.1, 2), gg.rmat(9, 8, seed=3)]
    off, col, start = gg.union(gl)
    ix = pll.Index.build_batch(dev_u32(off), dev_u32(col), start, t=4)
    p = tmp_path / "batch.pll"
    ix.save(p)
    jx = pll.Index.load(p)
    assert jx.graphs == 3
    g = gg.Graph(int(start[-1]), off, col)
    same_index(ix, jx, g)
    # pairs across graphs still answer 255 after the reload
    s = np.array([0, 1], dtype=np.uint32)
    u = np.array([int(start[1]), int(start[2]) + 1], dtype=np.uint32)
    assert (gpu_query(jx, s, u) == 255).all()


def test_empty_graph(tmp_path):
    g = gg.from_edges(5, [], [])
    ix = gpu_build(g, 2)
    p = tmp_path / "e.pll"
    ix.save(p)
    jx = pll.Index.load(p)
    same_index(ix, jx, g)


def test_damaged_files_are_refused(tmp_path):
    g = gg.ba(400, 2, 7)
    ix = gpu_build(g, 4)
    p = tmp_path / "ok.pll"
    ix.save(p)
    raw = bytearray(open(p, "rb").read())
    n = g.n

    def refused(data, name):
        q = tmp_path / name
        open(q, "wb").write(bytes(data))
        with pytest.raises(pll.PLLError) as e:
            pll.Index.load(q)
        assert e.value.code == pll.PLL_E_INVAL

    bad = bytearray(raw)
    bad[0:8] = b"NOTINDEX"
    refused(bad, "magic.pll")
    # order no longer the inverse of inv: vertex 0's rank points past n
    bad = bytearray(raw)
    inv0 = 48 + 4 * n
    bad[inv0:inv0 + 4] = (n + 5).to_bytes(4, "little")
    refused(bad, "perm.pll")
    # a decreasing label offset
    tp = 16
    off0 = 48 + 8 * n + n * tp + n * 4 * 16 + 4 * (2 + 64) * 4
    bad = bytearray(raw)
    bad[off0 + 8 * 3:off0 + 8 * 4] = (2 ** 40).to_bytes(8, "little")
    refused(bad, "offsets.pll")
    refused(raw[: len(raw) - 7], "short.pll")
    with pytest.raises(pll.PLLError):
        pll.Index.load(tmp_path / "missing.pll")
    # the good file still loads
    same_index(ix, pll.Index.load(p), g)
