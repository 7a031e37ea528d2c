"""The multi-rank path of bench.py on CPU: two gloo ranks (world size 2)
run the same setup, barrier and timing reductions as the GPU ranks do under
torchrun (replicas: no data-path collective, only timings are reduced)."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(ws),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    import bench
    import torch.distributed as dist
    try:
        w, r, local = bench.dist_setup(backend="gloo")
        assert (w, r, local) == (ws, rank, rank)
        bench.barrier(w)
        # rank r "took" 1 + r seconds for 100 * (r + 1) units
        t = 1.0 + r
        q.put((r, bench.max_over_ranks(w, t), bench.sum_over_ranks(w, t),
               bench.job_rate(w, 100.0 * (r + 1), t)))
        bench.barrier(w)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_timings():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for r, mx, sm, rate in got:
        assert mx == 2.0 and sm == 3.0
        assert rate == pytest.approx(300.0 / 2.0)  # all units over the slowest rank's time


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(1, 3.5) == 3.5
    assert bench.sum_over_ranks(1, 3.5) == 3.5
    assert bench.job_rate(1, 10.0, 2.0) == 5.0
