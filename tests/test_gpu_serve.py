"""The serving loop (pll_server_*): continuous batching over a resident index.

Each request's answer is compared with the same pairs answered alone (one
pll_query call per request) and with the oracle; a request stream replayed
fast enough to be batched must give every request the same bytes. Memory
admission is checked with a pool far smaller than the offered work.
"""
import numpy as np
import pytest

import oracle
from paper_1304_4661_gb300 import graphgen as gg
from paper_1304_4661_gb300 import pll

from .gpu_util import gpu_build, gpu_query

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def served():
    g = gg.rmat(14, 16, seed=7)
    ix = gpu_build(g, 16)
    ref = oracle.Index(g.offsets, g.cols, 16)
    return g, ix, ref


def requests(g, count, seed):
    s, t, off, many = gg.serve_requests(g.n, count, seed)
    return s, t, off.astype(np.int64), many


def test_each_request_same_alone_and_mixed(served):
    g, ix, ref = served
    s, t, off, _ = requests(g, 150, 12)
    expect = ref.query_batch(s, t)
    alone = np.concatenate([gpu_query(ix, s[a:b], t[a:b]) for a, b in zip(off[:-1], off[1:])])
    assert np.array_equal(alone, expect)
    with pll.Server(ix) as sv:
        # one at a time: submit, wait
        one = []
        for a, b in zip(off[:-1], off[1:]):
            d, lat = sv.wait(sv.submit(s[a:b], t[a:b]))
            assert lat > 0
            one.append(d)
        assert np.array_equal(np.concatenate(one), expect)
        # all at once: the dispatcher packs many requests into each launch
        n0 = sv.stats()["batches"]
        arr = np.zeros(len(off) - 1)
        mixed, lat, el = sv.replay(s, t, off, arr)
        st = sv.stats()
    assert np.array_equal(mixed, expect)
    assert (lat > 0).all() and el > 0
    assert st["batches"] - n0 < len(off) - 1, "burst was not batched"
    assert st["requests"] == 2 * (len(off) - 1)


def test_poisson_replay_matches(served):
    g, ix, ref = served
    s, t, off, _ = requests(g, 300, 13)
    arr = gg.poisson_arrivals(len(off) - 1, 20000.0, 14)
    with pll.Server(ix, streams=2) as sv:
        out, lat, el = sv.replay(s, t, off, arr)
    assert np.array_equal(out, ref.query_batch(s, t))
    assert el >= arr[-1]
    assert (lat > 0).all()


def test_admission_with_small_pool(served):
    g, ix, ref = served
    s, t, off, _ = requests(g, 200, 15)
    pool = 64 << 10  # holds ~7,000 pairs; the stream offers ~100x that
    with pll.Server(ix, pool_bytes=pool, streams=4) as sv:
        st0 = sv.stats()
        assert st0["max_request_pairs"] < 8000
        keep = np.diff(off) <= st0["max_request_pairs"]
        idx = np.flatnonzero(keep)
        s2 = np.concatenate([s[off[i]:off[i + 1]] for i in idx])
        t2 = np.concatenate([t[off[i]:off[i + 1]] for i in idx])
        off2 = np.zeros(len(idx) + 1, dtype=np.int64)
        off2[1:] = np.cumsum(np.diff(off)[idx])
        out, lat, _ = sv.replay(s2, t2, off2, np.zeros(len(idx)))
        st = sv.stats()
    assert np.array_equal(out, ref.query_batch(s2, t2))
    assert st["max_inflight_bytes"] <= pool
    assert st["batches"] > 1
    assert st["max_batch_pairs"] <= st["max_request_pairs"]


def test_rejections(served):
    g, ix, _ = served
    with pll.Server(ix, pool_bytes=1 << 20) as sv:
        big = sv.stats()["max_request_pairs"] + 1
        z = np.zeros(big, dtype=np.uint32)
        with pytest.raises(pll.PLLError) as e:
            sv.submit(z, z)
        assert e.value.args[0].endswith(f"(status {pll.PLL_E_RANGE})")
        with pytest.raises(pll.PLLError):
            sv.submit(np.array([0, g.n], dtype=np.uint32), np.array([1, 2], dtype=np.uint32))
        # the server keeps working after rejected requests
        d, _ = sv.wait(sv.submit(np.array([0], dtype=np.uint32), np.array([0], dtype=np.uint32)))
        assert d.tolist() == [0]
    with pytest.raises(pll.PLLError):
        pll.Server(ix, streams=65)


def test_concurrent_clients(served):
    """Several client threads submit and wait at once (the binding releases
    the GIL inside each call); every answer still matches the oracle."""
    import threading
    g, ix, ref = served
    s, t, off, _ = requests(g, 240, 16)
    expect = ref.query_batch(s, t)
    got = [None] * (len(off) - 1)
    errors = []
    with pll.Server(ix, pool_bytes=1 << 20, streams=3) as sv:
        def client(k):
            try:
                for i in range(k, len(off) - 1, 4):
                    a, b = off[i], off[i + 1]
                    got[i] = sv.wait(sv.submit(s[a:b], t[a:b]))[0]
            except Exception as e:  # surfaced below
                errors.append(e)
        th = [threading.Thread(target=client, args=(k,)) for k in range(4)]
        for x in th:
            x.start()
        for x in th:
            x.join()
        st = sv.stats()
    assert not errors, errors
    assert np.array_equal(np.concatenate(got), expect)
    assert st["requests"] == len(off) - 1


def test_wait_timeout_keeps_the_ticket(served):
    """A wait that runs out returns PLL_E_TIMEOUT and leaves the ticket valid;
    the next wait delivers the answer."""
    g, ix, ref = served
    s, t = gg.pairs(g.n, 1_000_000, 31)
    with pll.Server(ix) as sv:
        tk = sv.submit(s, t)
        with pytest.raises(TimeoutError):
            sv.wait(tk, timeout_us=0)
        d, lat = sv.wait(tk)
    assert lat > 0
    sample = np.arange(0, len(s), 997)
    assert np.array_equal(d[sample], ref.query_batch(s[sample], t[sample]))
