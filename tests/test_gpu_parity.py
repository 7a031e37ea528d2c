"""GPU parity: the CUDA build and queries against the CPU oracle.

Integer work throughout, so every comparison is exact: order, bit-parallel
roots and masks, every label entry (hub rank and distance), every distance.
Sizes run from single vertices through several root batches with ragged
tails (n not a multiple of the batch or warp size) up to 10k-vertex graphs.
"""
import numpy as np
import pytest

import oracle
from paper_1304_4661_gb300 import graphgen as gg

from . import graphs
from .gpu_util import dev_u32, first_label_diff, gpu_build, gpu_query, same_labels

pytestmark = pytest.mark.gpu


def check_index(g, t, **kw):
    ref = oracle.Index(g.offsets, g.cols, t, order=kw.get("order"))
    ix = gpu_build(g, t, **kw)
    assert np.array_equal(ix.order(), ref.order())
    if t:
        r_roots, r_cnt, r_S = ref.bp_roots()
        roots, cnt, S = ix.bp_roots()
        assert np.array_equal(roots, r_roots) and np.array_equal(cnt, r_cnt)
        for i in range(t):
            assert np.array_equal(S[i, : cnt[i]], r_S[i, : r_cnt[i]])
        for a, b in zip(ix.bp(), ref.bp()):
            assert np.array_equal(a, b)
    La, Lb = ix.labels(), ref.labels()
    assert same_labels(La, Lb), first_label_diff(La, Lb, g.n)
    return ix, ref


@pytest.mark.parametrize("t", [0, 1, 2, 16, 64])
@pytest.mark.parametrize("g", graphs.small_family(), ids=lambda g: g.name)
def test_small_graphs_labels_and_all_pairs(g, t):
    ix, ref = check_index(g, t)
    s, u = np.meshgrid(np.arange(g.n), np.arange(g.n), indexing="ij")
    s, u = s.ravel().astype(np.uint32), u.ravel().astype(np.uint32)
    if g.n:
        assert np.array_equal(gpu_query(ix, s, u), ref.query_batch(s, u))


@pytest.mark.parametrize("root_batch,block", [(1, 256), (7, 128), (32, 512), (100, 256), (4096, 256)])
def test_batch_size_and_block_shape_do_not_change_labels(root_batch, block):
    g = gg.ba(3000, 3, 17)
    check_index(g, 16, root_batch=root_batch, block=block)


@pytest.mark.parametrize("t", [0, 16])
def test_ba_10k_config(t):
    """Barabasi-Albert n=10,000, m=4, Degree order; 100k uniform pairs checked
    against per-source BFS."""
    g = gg.ba(10_000, 4, 1)
    ix, ref = check_index(g, t)
    s, u = gg.pairs(g.n, 100_000, 2)
    got = gpu_query(ix, s, u)
    order = np.argsort(s, kind="stable")
    expect = np.empty_like(got)
    srt = s[order]
    starts = np.flatnonzero(np.r_[True, srt[1:] != srt[:-1]])
    ends = np.r_[starts[1:], len(srt)]
    for a, b in zip(starts, ends):
        dist = oracle.bfs(g.offsets, g.cols, int(srt[a]))
        expect[order[a:b]] = dist[u[order[a:b]]]
    assert np.array_equal(got, expect)


@pytest.mark.parametrize("make,t", [
    (lambda: gg.rmat(14, 16, seed=3), 64),
    (lambda: gg.rmat(15, 8, seed=4), 16),
    (lambda: gg.ws(5000, 6, 0.1, 5), 16),
    (lambda: gg.ws(3001, 4, 0.05, 6), 0),
    (lambda: graphs.disjoint(gg.ba(2000, 2, 7), gg.ws(1500, 6, 0.2, 8), graphs.complete(1)), 64),
])
def test_mid_size_graphs(make, t):
    g = make()
    ix, ref = check_index(g, t)
    s, u = gg.pairs(g.n, 20_000, 11)
    assert np.array_equal(gpu_query(ix, s, u), ref.query_batch(s, u))


def test_explicit_order():
    g = gg.ba(2000, 3, 9)
    order = np.random.default_rng(3).permutation(g.n).astype(np.uint32)
    check_index(g, 8, order=order)


def test_host_entry_points_match_device():
    from paper_1304_4661_gb300 import pll
    g = gg.rmat(12, 16, seed=2)
    a = gpu_build(g, 16)
    b = pll.Index.build(g.offsets, g.cols, t=16)  # numpy -> pll_build_host
    assert same_labels(a.labels(), b.labels())
    s, u = gg.pairs(g.n, 5000, 3)
    assert np.array_equal(b.query(s, u), gpu_query(a, s, u))


def test_query_async_and_error_counts():
    import torch
    g = gg.ba(500, 2, 1)
    ix = gpu_build(g, 4)
    s, u = gg.pairs(g.n, 1000, 5)
    out = torch.empty(1000, dtype=torch.uint8, device="cuda")
    ix.query_async(dev_u32(s), dev_u32(u), out)
    assert ix.query_errors() == 0
    assert np.array_equal(out.cpu().numpy(), oracle.Index(g.offsets, g.cols, 4).query_batch(s, u))
    bad = s.copy()
    bad[7] = g.n + 3
    from paper_1304_4661_gb300 import pll
    with pytest.raises(pll.PLLError) as e:
        ix.query(dev_u32(bad), dev_u32(u))
    assert e.value.code == pll.PLL_E_INVAL


def test_errors():
    from paper_1304_4661_gb300 import pll
    g = gg.ba(50, 2, 1)

    def code(off, col, **kw):
        with pytest.raises(pll.PLLError) as e:
            pll.Index.build(dev_u32(off), dev_u32(col), **kw)
        return e.value.code

    # asymmetric: drop one arc of an edge
    off = g.offsets.copy().astype(np.int64)
    col = g.cols.copy()
    bad_col = col.copy()
    bad_col[0] = (bad_col[0] + 1) % g.n if (bad_col[0] + 1) % g.n != 0 else 2
    assert code(g.offsets, bad_col, t=2) == pll.PLL_E_INVAL
    # self-loop
    sl = col.copy()
    sl[0] = 0
    assert code(g.offsets, sl, t=2) == pll.PLL_E_INVAL
    # id out of range
    oor = col.copy()
    oor[-1] = g.n + 5
    assert code(g.offsets, oor) == pll.PLL_E_INVAL
    # unsorted neighbour list
    uns = col.copy()
    a, b = int(off[3]), int(off[4])
    if b - a >= 2:
        uns[a], uns[a + 1] = uns[a + 1], uns[a]
        assert code(g.offsets, uns) == pll.PLL_E_INVAL
    # order not a permutation
    bad_order = np.arange(g.n, dtype=np.uint32)
    bad_order[5] = 6
    assert code(g.offsets, g.cols, order=dev_u32(bad_order)) == pll.PLL_E_ORDER
    # too many bit-parallel roots
    assert code(g.offsets, g.cols, t=65) == pll.PLL_E_RANGE
    # BFS depth of 255 or more
    p = graphs.path(300)
    assert code(p.offsets, p.cols) == pll.PLL_E_RANGE
    assert code(p.offsets, p.cols, t=1) == pll.PLL_E_RANGE


def test_empty_and_tiny():
    from paper_1304_4661_gb300 import pll
    e = gg.from_edges(0, [], [])
    ix = pll.Index.build(np.zeros(1, np.uint32), np.zeros(0, np.uint32), t=4)
    assert ix.label_entries() == 0
    for g in (graphs.complete(1), gg.from_edges(10, [], []), graphs.complete(2)):
        for t in (0, 1, 64):
            check_index(g, t)


@pytest.mark.parametrize("t", [0, 64])
def test_query_launch_sizes(t):
    """Launches of every size class: a few pairs (8 warps per pair), up to
    one, two and four pairs per resident block (8, 4, 2 warps per pair), and
    large launches (one warp per pair); each also with a bad id, which must
    answer 255 and be counted."""
    import torch
    from paper_1304_4661_gb300 import pll
    g = gg.rmat(13, 16, seed=3)
    ix, ref = check_index(g, t)
    props = torch.cuda.get_device_properties(0)
    res = props.multi_processor_count * 8  # resident 256-thread blocks, upper bound
    sizes = sorted({1, 2, 7, 33, res // 2, res, res + 1, 2 * res - 1, 2 * res + 3, 4 * res - 5,
                    4 * res + 7, 10 * res, 200_000})
    for q in sizes:
        s, u = gg.pairs(g.n, q, 100 + q)
        expect = ref.query_batch(s, u)
        assert np.array_equal(gpu_query(ix, s, u), expect), q
        bad = s.copy()
        bad[q // 2] = g.n
        out = torch.empty(q, dtype=torch.uint8, device="cuda")
        ix.query_async(dev_u32(bad), dev_u32(u), out)
        assert ix.query_errors() == 1, q
        got = out.cpu().numpy()
        assert got[q // 2] == 255
        keep = np.arange(q) != q // 2
        assert np.array_equal(got[keep], expect[keep]), q


def test_size_and_distance_limits():
    """n must stay below 2^24 (hub ranks are packed into 24 bits): n = 2^24 is
    PLL_E_RANGE before any memory is read. A path of 255 vertices has the
    largest finite 8-bit distance, 254, between its ends; it is answered
    exactly (255 vertices is the longest path the labels can hold)."""
    import torch
    from paper_1304_4661_gb300 import pll
    off = torch.zeros((1 << 24) + 1, dtype=torch.int32, device="cuda")
    col = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(pll.PLLError) as e:
        pll.Index.build(off, col[:0], t=0)
    assert e.value.code == pll.PLL_E_RANGE
    del off
    p = graphs.path(255)
    for t in (0, 2):
        ix, ref = check_index(p, t)
        s = np.array([0, 254, 0, 127], dtype=np.uint32)
        u = np.array([254, 0, 127, 254], dtype=np.uint32)
        got = gpu_query(ix, s, u)
        assert got.tolist() == [254, 254, 127, 127]
        assert np.array_equal(got, ref.query_batch(s, u))
