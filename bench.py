#!/usr/bin/env python3
"""Benchmark of the PLL hot path on one GB300: index build + batched queries.

One step = the whole path over one synthetic graph: pll_build (CSR checks,
Degree order, relabel, bit-parallel stage, batched pruned BFS + cleanup,
compaction) followed by pll_query over the workload's uniform pairs. Inputs
are resident in HBM before the timed region; every step builds a fresh index.

Prints ONE JSON line (rank 0). `value` is the index build time in seconds of
the named workload (lower is better); queries/s and the query p99 latency sit
beside it. `e2e` repeats the step through the host-pointer entry points
(pll_build_host, pll_query_host) with the host<->device copies inside the
timed region. `--impl reference` times the CPU oracle instead (a bounded
sample of the same workload; see its `sample` field).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PLL build s + queries/s, p99 us on R-MAT-20; learned/served vs plain GPU"

WORKLOADS = {
    # R-MAT scale 20, edge factor 16, (a,b,c,d) = (.57,.19,.19,.05), graph seed 1,
    # Degree order, t = 64, 10M uniform pairs (seed 3)
    "rmat20": dict(kind="rmat", scale=20, ef=16, t=64, queries=10_000_000, graph_seed=1, pair_seed=3),
    # Barabasi-Albert n = 10,000, m = 4, seed 1, t = 16, 100k pairs (seed 2)
    "ba10k": dict(kind="ba", n=10_000, m=4, t=16, queries=100_000, graph_seed=1, pair_seed=2),
    # smaller R-MATs of the same family (profiling, quick runs)
    "rmat19": dict(kind="rmat", scale=19, ef=16, t=64, queries=1_000_000, graph_seed=1, pair_seed=3),
    "rmat18": dict(kind="rmat", scale=18, ef=16, t=64, queries=1_000_000, graph_seed=1, pair_seed=3),
    "rmat17": dict(kind="rmat", scale=17, ef=16, t=64, queries=1_000_000, graph_seed=1, pair_seed=3),
    "rmat16": dict(kind="rmat", scale=16, ef=16, t=64, queries=1_000_000, graph_seed=1, pair_seed=3),
}

# DRAM bytes per algorithmic byte of a kernel, measured by ncu over every
# launch of one build of a smaller R-MAT (dram__bytes_read.sum +
# dram__bytes_write.sum, one pass), valid only for the kernel source with this
# hash (else traffic is reported as null). The level-loop graph's figure is
# ncu's per-graph-launch count (--graph-profiling graph) on R-MAT scale 18:
# 24 launches, 4.955 GB of DRAM against 6.953 GB of algorithmic bytes.
PROFILED = {
    "level-loop graph (k_batch_expand_g + k_batch_test_g)": {
        "src_sha": "f86b4bd6dc924da0", "dram_per_alg_byte": 0.713},
}


def make_graph(w):
    from paper_1304_4661_gb300 import graphgen as gg
    if w["kind"] == "rmat":
        return gg.rmat(w["scale"], w["ef"], seed=w["graph_seed"])
    return gg.ba(w["n"], w["m"], w["graph_seed"])


def _workload_name(w):
    if w["kind"] == "rmat":
        return f"R-MAT scale {w['scale']} ef {w['ef']} (a,b,c,d)=(.57,.19,.19,.05) seed {w['graph_seed']}"
    return f"Barabasi-Albert n={w['n']} m={w['m']} seed {w['graph_seed']}"


def describe(w, g):
    return {"workload": _workload_name(w), "n": g.n, "arcs": g.nnz, "t": w["t"], "order": "degree (ties by id)",
            "queries": w["queries"], "pair_seed": w["pair_seed"],
            "l2": "L2 flushed (512 MiB write) between timed steps"}


def sequential_work(w, g):
    """Work counts of the oracle's sequential build of this workload's graph
    (vertices dequeued, labelled, label entries scanned, arcs of labelled
    vertices), from its stored digest; None if there is none for it."""
    if w.get("kind") != "rmat":
        return None
    path = os.path.join(ROOT, "tests", "golden", f"rmat{w['scale']}_t{w['t']}_digest.json")
    try:
        d = json.load(open(path))
    except OSError:
        return None
    gr = d["graph"]
    if (gr["seed"], gr["n"], gr["nnz"], gr["edge_factor"]) != (w["graph_seed"], g.n, g.nnz, w["ef"]):
        return None
    return d.get("sequential_work")


def file_sha(path):
    return hashlib.sha256(open(path, "rb").read()).hexdigest()[:16]


class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.lines = []
        self.proc = None

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.uuid:
            cmd += ["-i", self.uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def dist_setup(backend=None):
    """One process per GPU, launched by torchrun (RANK / WORLD_SIZE /
    MASTER_* from the environment). Every rank runs an independent replica
    of the workload; ranks meet only in barriers and in the reduction of
    their timings. NCCL with GPUs, gloo without (the CPU tests)."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        if backend is None:
            backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)  # each rank's communicator on its own GPU
        dist.init_process_group(backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def _reduce(ws, x, op):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(ws, x):
    import torch.distributed as dist
    return _reduce(ws, x, dist.ReduceOp.MAX) if ws > 1 else x


def sum_over_ranks(ws, x):
    import torch.distributed as dist
    return _reduce(ws, x, dist.ReduceOp.SUM) if ws > 1 else x


def job_rate(ws, units, seconds):
    """Whole-job throughput: the units every rank processed over the time
    of the slowest rank."""
    return sum_over_ranks(ws, units) / max_over_ranks(ws, seconds)


# ---------------------------------------------------------------- our arm
def run_ours(args, w, ws, rank, local):
    import numpy as np
    import torch

    from paper_1304_4661_gb300 import graphgen as gg
    from paper_1304_4661_gb300 import pll

    torch.cuda.set_device(local)
    pll.load()
    g = make_graph(w)
    s, u = gg.pairs(g.n, w["queries"], w["pair_seed"])
    t = w["t"]

    def dev(a):
        return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()

    off_d, col_d, s_d, u_d = dev(g.offsets), dev(g.cols), dev(s), dev(u)
    out_d = torch.empty(w["queries"], dtype=torch.uint8, device="cuda")
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def step(record):
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        ix = pll.Index.build(off_d, col_d, t=t, root_batch=args.root_batch, block=args.block,
                             flags=args.flags)
        e1.record(stream)
        ix.query(s_d, u_d, out_d)
        e2.record(stream)
        e2.synchronize()
        st = ix.stats()
        ix.close()
        if record is not None:
            record.append((e0.elapsed_time(e1), e1.elapsed_time(e2), st))

    for _ in range(args.warmup):
        flush.fill_(1)
        step(None)
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        pass
    clocks = ClockSampler(uuid)
    recs = []
    clocks.start()
    barrier(ws)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        flush.fill_(1)
        step(recs)
    torch.cuda.synchronize()
    barrier(ws)
    wall = time.perf_counter() - t0
    clk = clocks.stop()

    build_ms = statistics.mean(r[0] for r in recs)
    query_ms = statistics.mean(r[1] for r in recs)
    step_ms = build_ms + query_ms
    queries_per_s = job_rate(ws, w["queries"], query_ms * 1e-3)
    build_ms = max_over_ranks(ws, build_ms)
    step_ms = max_over_ranks(ws, step_ms)
    st = recs[-1][2]

    # per-pair latency through the synchronous C-ABI query (host wall clock)
    ix = pll.Index.build(off_d, col_d, t=t)
    lat = []
    one_out = torch.empty(1, dtype=torch.uint8, device="cuda")
    for i in range(args.latency_samples):
        a, b = s_d[i:i + 1], u_d[i:i + 1]
        torch.cuda.synchronize()
        tq = time.perf_counter()
        ix.query(a, b, one_out)
        lat.append((time.perf_counter() - tq) * 1e6)
    lat.sort()
    p50 = lat[len(lat) // 2]
    p99 = lat[min(len(lat) - 1, int(0.99 * len(lat)))]

    # query kernel alone: one launch, CUDA events on the launching stream
    qk = []
    for _ in range(3):
        flush.fill_(1)
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        ix.query_async(s_d, u_d, out_d)
        a1.record(stream)
        a1.synchronize()
        qk.append(a0.elapsed_time(a1))
    assert ix.query_errors() == 0
    qk_ms = statistics.mean(qk)
    lab = ix.labels()
    Lsz = np.diff(lab.offsets.astype(np.int64))
    ix.close()

    # ---- e2e through the host-pointer entry points
    e2e = None
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).pin_memory()
        off_h, col_h, s_h, u_h = pin(g.offsets), pin(g.cols), pin(s), pin(u)
        res_h = torch.empty(w["queries"], dtype=torch.uint8).pin_memory()
        off_n, col_n = off_h.numpy().view(np.uint32), col_h.numpy().view(np.uint32)
        s_n, u_n, res_n = s_h.numpy().view(np.uint32), u_h.numpy().view(np.uint32), res_h.numpy()
        lib = pll.load()
        import ctypes as C
        times_b, times_q = [], []
        for it in range(args.warmup + args.steps):
            torch.cuda.synchronize()
            tb = time.perf_counter()
            opts = pll.BuildOpts(t, args.root_batch, args.block, args.flags, 0)
            h = C.c_void_p()
            rc = lib.pll_build_host(off_n.ctypes.data, col_n.ctypes.data, g.n, g.nnz, None,
                                    C.byref(opts), None, C.byref(h))
            assert rc == 0, pll.status_str(rc)
            tm = time.perf_counter()
            rc = lib.pll_query_host(h.value, s_n.ctypes.data, u_n.ctypes.data, w["queries"],
                                    res_n.ctypes.data, None)
            assert rc == 0, pll.status_str(rc)
            te = time.perf_counter()
            lib.pll_free(h.value)
            if it >= args.warmup:
                times_b.append(tm - tb)
                times_q.append(te - tm)
        assert np.array_equal(res_n, out_d.cpu().numpy())
        e2e = {"value": round(statistics.mean(times_b), 6), "unit": "s",
               "queries_per_s": round(w["queries"] / statistics.mean(times_q), 1),
               "step_s": round(statistics.mean(times_b) + statistics.mean(times_q), 6),
               "h2d_bytes_per_step": int(4 * (g.n + 1) + 4 * g.nnz + 8 * w["queries"]),
               "d2h_bytes_per_step": int(w["queries"])}

    # ---- roofline of the dominant kernel (algorithmic bytes / event time)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm = peaks.get("hbm_gbs")
    peak_src = "measured" if hbm else "fallback"
    hbm = hbm or 6800.0
    q = w["queries"]
    # algorithmic bytes of each kernel over one build: the per-unit figures of
    # the method's pruned stage times the units of work the method does. The
    # units are the counts of the oracle's sequential run (Alg. 1 for every
    # root, in rank order) where the workload has a stored oracle digest:
    # vertices dequeued, vertices labelled, label entries scanned by prune
    # tests, arcs of labelled vertices. Otherwise the GPU's own counters stand
    # in (they include the root batches' surplus work).
    seq = sequential_work(w, g)
    if seq:
        units, unit_src = seq, "oracle sequential counts (tests/golden digest)"
    else:
        units = {"visited": st["visited"], "labeled": st["pre_cleanup"],
                 "scanned": st["pruned_scanned"], "labeled_deg": st["pruned_expanded"]}
        unit_src = "GPU counters"
    # expand: a labelled vertex's neighbour ids (4 per arc) and its entry (4 + 1);
    # a dequeued vertex's offsets (8) and bit-parallel distance row (t bytes)
    def expand_bytes(u):
        return 4 * u["labeled_deg"] + 5 * u["labeled"] + (8 + t) * u["visited"]

    # test: the label entries its prune tests scan (4 bytes each); mask bytes
    # are not counted (the distance filter of Sec. 5.3 leaves most unread)
    def test_bytes_of(u):
        return 4 * u["scanned"]

    exp_bytes = expand_bytes(units)
    test_bytes = test_bytes_of(units)
    # the same per-unit bytes over the GPU's own work counts (its root batches'
    # surplus included; a vertex that the bit-parallel bound prunes is counted
    # each time it is reached), for comparison with the sequential-count figure
    gpu_units = {"visited": st["visited"], "labeled": st["pre_cleanup"],
                 "scanned": st["pruned_scanned"], "labeled_deg": st["pruned_expanded"]}
    # per pair: ids (8), ranks (8), 2 x t distance bytes, 4 label offsets (32),
    # the result byte, and both labels (4 bytes per entry; Lsz is by vertex id)
    q_bytes = q * (8 + 8 + 2 * t + 32 + 1) + 4 * int(Lsz[s].sum() + Lsz[u].sum())
    if st["levels_launches"]:
        # one launch per root batch (a CUDA graph whose while node runs both
        # sweeps of every level, or one cooperative kernel) covers every level;
        # its phases' wall times split the time between the sweeps
        loop_name = ("k_batch_levels" if args.flags & 4
                     else "level-loop graph (k_batch_expand_g + k_batch_test_g)")
        kern = {
            loop_name: {"ms_per_step": st["ms_levels"], "launches": st["levels_launches"],
                        "bytes": exp_bytes + test_bytes},
            "k_query": {"ms_per_step": qk_ms, "launches": 1, "bytes": q_bytes},
        }
        phases = {"expand": {"ms_per_step": st["ms_expand"], "bytes": exp_bytes},
                  "test": {"ms_per_step": st["ms_test"], "bytes": test_bytes}}
    else:
        kern = {
            "k_batch_test": {"ms_per_step": st["ms_test"], "launches": st["test_launches"],
                             "bytes": test_bytes},
            "k_batch_expand": {"ms_per_step": st["ms_expand"], "launches": st["expand_launches"],
                               "bytes": exp_bytes},
            "k_query": {"ms_per_step": qk_ms, "launches": 1, "bytes": q_bytes},
        }
        phases = {}
    for v in kern.values():
        v["launches"] = max(v["launches"], 1)
        v["bytes_per_launch"] = v["bytes"] / v["launches"]
        v["ms_per_launch"] = v["ms_per_step"] / v["launches"]
        v["achieved_gbs"] = v["bytes"] / max(v["ms_per_step"], 1e-9) / 1e6
    dom = max(kern, key=lambda k: kern[k]["ms_per_step"])
    kd = kern[dom]
    achieved = kd["achieved_gbs"]
    src = os.path.join(ROOT, "paper_1304_4661_gb300", "csrc",
                       "k_query.cu" if dom == "k_query" else "k_pruned.cu")
    prof = PROFILED.get(dom)
    # DRAM bytes per algorithmic byte, measured by ncu on a smaller graph of the
    # same family with this kernel source, scaled to this launch's bytes
    traffic = (round(prof["dram_per_alg_byte"] * kd["bytes_per_launch"])
               if prof and prof["src_sha"] == file_sha(src) else None)
    roofline = {"kernel": dom, "bound": "hbm", "achieved": round(achieved, 1), "peak": hbm,
                "peak_source": peak_src, "unit": "GB/s", "frac": round(achieved / hbm, 4),
                "traffic": traffic,
                "algorithmic_bytes_per_launch": round(kd["bytes_per_launch"]),
                "units": unit_src,
                "launch_ms": round(kd["ms_per_launch"], 4),
                "others": {k: {"achieved_gbs": round(v["achieved_gbs"], 1),
                               "ms_per_step": round(v["ms_per_step"], 3), "launches": v["launches"]}
                           for k, v in kern.items()},
                "phases": {k: {"ms_per_step": round(v["ms_per_step"], 3),
                               "achieved_gbs": round(v["bytes"] / max(v["ms_per_step"], 1e-9) / 1e6, 1)}
                           for k, v in phases.items()}}
    if st["levels_launches"] and dom != "k_query" and seq:
        gb = expand_bytes(gpu_units) + test_bytes_of(gpu_units)
        ga = gb / max(kd["ms_per_step"], 1e-9) / 1e6
        roofline["with_gpu_counts"] = {"achieved": round(ga, 1), "frac": round(ga / hbm, 4),
                                       "algorithmic_bytes_per_launch": round(gb / kd["launches"])}

    out = {
        "metric": METRIC, "value": round(build_ms / 1e3, 6), "unit": "s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(step_ms, 3),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic", "config": describe(w, g),
        "build_s": round(build_ms / 1e3, 6),
        "queries_per_s": round(queries_per_s, 1),
        "query_kernel_ms": round(qk_ms, 3),
        "query_p50_us": round(p50, 2), "query_p99_us": round(p99, 2),
        "latency_note": "per single-pair synchronous pll_query call, host wall clock",
        "label_entries": st["label_entries"],
        "label_entries_per_s": round(st["label_entries"] / (build_ms * 1e-3), 1),
        "avg_label": round(st["label_entries"] / max(g.n, 1), 2),
        "phases_ms": {"prep": round(st["ms_prep"], 3), "bp": round(st["ms_bp"], 3),
                      "pruned": round(st["ms_pruned"], 3), "pruned_bfs": round(st["ms_pruned_kernel"], 3),
                      "expand_sweeps": round(st["ms_expand"], 3), "test_sweeps": round(st["ms_test"], 3),
                      "level_loop": round(st["ms_levels"], 3),
                      "post": round(st["ms_post"], 3),
                      "host_gaps": round(st["ms_pruned"] - st["ms_pruned_kernel"] - st["ms_post"]
                                         - st["ms_finalize"], 3),
                      "finalize": round(st["ms_finalize"], 3)},
        "batches": st["batches"], "pre_cleanup": st["pre_cleanup"], "visited": st["visited"],
        "memory_gb": {"index": round(st["index_bytes"] / 1e9, 3),
                      "build_scratch_peak": round(st["scratch_peak_bytes"] / 1e9, 3)},
        "prune_work": {"label_entries_scanned": st["pruned_scanned"], "mask_pairs": st["pruned_masks"],
                       "arcs_expanded": st["pruned_expanded"], "candidates": st["candidates"]},
        "wall_s_timed_region": round(wall, 3),
        "clocks": clk, "e2e": e2e, "roofline": roofline,
        "gpu_launches": int(args.steps * (st["launches"] + 1)),
        "cub_calls_per_step": st["cub_calls"],
    }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args, with_gpu=True)
    if rank == 0:
        print(json.dumps(out), flush=True)


# ------------------------------------------------------- multi-graph batch
def run_batch(args, ws, rank, local):
    """256 uneven graphs (half Barabasi-Albert n log-uniform 1k-50k, m 2-8;
    half Watts-Strogatz n log-uniform 1k-50k, k = 6, p = 0.1), t = 16:
    one pll_build per graph vs one pll_build_batch over their union, with the
    library defaults and with the autotuner's choice."""
    import numpy as np
    import torch

    from paper_1304_4661_gb300 import graphgen as gg
    from paper_1304_4661_gb300 import pll

    torch.cuda.set_device(local)
    pll.load()
    t = 16
    specs = gg.batch_specs(256, seed=4)
    gl = [gg.make(sp) for sp in specs]
    off, col, start = gg.union(gl)

    def dev(a):
        return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()

    d_off, d_col = dev(off), dev(col)
    per = [(dev(g.offsets), dev(g.cols)) for g in gl]
    stream = torch.cuda.current_stream()

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        r = fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1), r

    def sequential():
        total = 0
        for o, c in per:
            ix = pll.Index.build(o, c, t=t, flags=args.flags)
            total += ix.label_entries()
            ix.close()
        return total

    def batched(rb=0, bl=0):
        ix = pll.Index.build_batch(d_off, d_col, start, t=t, root_batch=rb, block=bl, flags=args.flags)
        e = ix.label_entries()
        ix.close()
        return e

    for _ in range(args.warmup):
        sequential()
        batched()
    seq = [timed(sequential) for _ in range(args.steps)]
    bat = [timed(batched) for _ in range(args.steps)]
    tune_ms_wall = time.perf_counter()
    rb, bl, tuned_trial_ms = pll.autotune(d_off, d_col, t, graph_start=start)
    tune_ms_wall = (time.perf_counter() - tune_ms_wall) * 1e3
    tun = [timed(lambda: batched(rb, bl)) for _ in range(args.steps)]
    assert seq[0][1] == bat[0][1] == tun[0][1], "label counts differ between builds"
    seq_ms = statistics.mean(x[0] for x in seq)
    bat_ms = statistics.mean(x[0] for x in bat)
    tun_ms = statistics.mean(x[0] for x in tun)
    out = {"metric": "C3 batched build of 256 uneven graphs (t=16): total build s",
           "value": round(tun_ms / 1e3, 6), "unit": "s", "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(tun_ms, 3), "higher_is_better": False,
           "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
           "config": {"workload": "256 graphs: 128 Barabasi-Albert (n log-uniform 1k-50k, m 2-8), "
                                  "128 Watts-Strogatz (n log-uniform 1k-50k, k=6, p=0.1), seed 4",
                      "vertices": int(start[-1]), "arcs": int(col.shape[0]), "t": t},
           "plain_sequential_s": round(seq_ms / 1e3, 6),
           "batched_default_s": round(bat_ms / 1e3, 6),
           "batched_tuned_s": round(tun_ms / 1e3, 6),
           "speedup_vs_sequential": round(seq_ms / tun_ms, 2),
           "autotune": {"root_batch": rb, "block": bl, "wall_ms": round(tune_ms_wall, 1)},
           "label_entries": int(seq[0][1])}
    if rank == 0:
        print(json.dumps(out), flush=True)


# ------------------------------------------------------------ serving loop
def run_serve(args, ws, rank, local):
    """R-MAT-22 (ef 16, seed 6), t = 64, index resident in HBM, served by the
    continuous-batching loop (pll_server_*). Requests: 90 % hold a log-uniform
    1-4096 number of uniform pairs, 10 % are one source with 1,000 uniform
    targets. Saturation = the whole request stream offered at once; then
    open-loop Poisson arrivals at 0.25 / 0.5 / 0.75 / 0.9 x saturation. The
    plain form answers the same requests one synchronous pll_query_host call
    at a time."""
    import numpy as np
    import torch

    from paper_1304_4661_gb300 import graphgen as gg
    from paper_1304_4661_gb300 import pll

    torch.cuda.set_device(local)
    pll.load()
    g = gg.rmat(22, 16, seed=6)

    def dev(a):
        return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()

    d_off, d_col = dev(g.offsets), dev(g.cols)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ix = pll.Index.build(d_off, d_col, t=64)
    build_s = time.perf_counter() - t0
    del d_off, d_col
    count = args.serve_requests
    s, u, off, many = gg.serve_requests(g.n, count, seed=8)
    off = off.astype(np.int64)
    total = int(off[-1])
    mean_pairs = total / count
    # the query kernel alone over the whole request stream, device-resident pairs
    d_s, d_u = dev(s), dev(u)
    d_o = torch.empty(total, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    kern = []
    for it in range(args.warmup + args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ix.query_async(d_s, d_u, d_o)
        e1.record(stream)
        e1.synchronize()
        if it >= args.warmup:
            kern.append(e0.elapsed_time(e1))
    assert ix.query_errors() == 0
    kernel_qps = total / (statistics.median(kern) * 1e-3)
    del d_s, d_u, d_o
    sv = pll.Server(ix, streams=args.serve_streams)
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        pass
    clocks = ClockSampler(uuid)

    def replay(k, arrivals):
        return sv.replay(s[: off[k]], u[: off[k]], off[: k + 1], arrivals, threads=args.serve_clients)

    for _ in range(args.warmup):
        replay(min(count, 2000), np.zeros(min(count, 2000)))
    clocks.start()
    sat = []
    ss0 = sv.stats()
    for _ in range(args.steps):
        out, lat, el = replay(count, np.zeros(count))
        sat.append(total / (el * 1e-6))
    ss1 = sv.stats()
    sat_detail = {k: round((ss1[k] - ss0[k]) / args.steps / 1e3, 2)
                  for k in ("pack_us", "unpack_us", "device_us")}
    sat_detail["batches_per_step"] = (ss1["batches"] - ss0["batches"]) / args.steps
    sat_detail["p50_us"] = round(float(np.percentile(lat, 50)), 1)
    sat_detail["p99_us"] = round(float(np.percentile(lat, 99)), 1)
    qps_sat = statistics.median(sat)
    served_out = out.copy()
    loads = []
    for i, frac in enumerate((0.25, 0.5, 0.75, 0.9)):
        rate = frac * qps_sat / mean_pairs  # requests per second
        k = min(count, max(2000, int(rate * args.serve_seconds)))
        arr = gg.poisson_arrivals(k, rate, 9 + i)
        st0 = sv.stats()
        _, lat, el = replay(k, arr)
        st1 = sv.stats()
        nb = st1["batches"] - st0["batches"]
        loads.append({"load": frac, "offered_req_per_s": round(rate, 1), "requests": k,
                      "queries_per_s": round(int(off[k]) / (el * 1e-6), 1),
                      "p50_us": round(float(np.percentile(lat, 50)), 1),
                      "p99_us": round(float(np.percentile(lat, 99)), 1),
                      "mean_pairs_per_batch": round(int(off[k]) / max(nb, 1), 1),
                      "host_pack_unpack_ms": round((st1["pack_us"] + st1["unpack_us"]
                                                    - st0["pack_us"] - st0["unpack_us"]) / 1e3, 2),
                      "device_stream_ms": round((st1["device_us"] - st0["device_us"]) / 1e3, 2),
                      "wall_ms": round(el / 1e3, 2)})
    clk = clocks.stop()
    st = sv.stats()
    sv.stop()
    # plain form: one synchronous host-pointer query call per request
    kp = min(count, args.serve_plain)
    plain_lat = []
    plain_out = np.empty(int(off[kp]), dtype=np.uint8)
    tp0 = time.perf_counter()
    for i in range(kp):
        a, b = int(off[i]), int(off[i + 1])
        c0 = time.perf_counter()
        plain_out[a:b] = ix.query(s[a:b], u[a:b])
        plain_lat.append((time.perf_counter() - c0) * 1e6)
    plain_el = time.perf_counter() - tp0
    assert np.array_equal(plain_out, served_out[: int(off[kp])]), "served != plain answers"
    entries = ix.label_entries()
    ix.close()
    out = {"metric": "C5 served queries/s at saturation (R-MAT-22, t=64), p50/p99 request latency "
                     "at 0.25-0.9x load",
           "value": round(qps_sat, 1), "unit": "queries/s", "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(total / qps_sat * 1e3, 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
           "data": "synthetic",
           "config": {"workload": "R-MAT-22 (ef 16, seed 6), t=64; requests: 90% log-uniform "
                                  "1-4096 uniform pairs, 10% one-to-1000 (seed 8)",
                      "vertices": g.n, "arcs": g.nnz, "requests": count, "pairs": total,
                      "server": {"pool_bytes": st["pool_bytes"], "streams": args.serve_streams, "client_threads": args.serve_clients,
                                 "max_batch_pairs": st["max_request_pairs"]},
                      "l2": "request pairs are copied fresh from host memory every request"},
           "build_s": round(build_s, 3), "label_entries": entries,
           "kernel_only_queries_per_s": round(kernel_qps, 1),
           "saturation_queries_per_s": [round(x, 1) for x in sat],
           "saturation_step_ms": sat_detail,
           "loads": loads,
           "plain": {"form": "one synchronous pll_query_host call per request", "requests": kp,
                     "queries_per_s": round(int(off[kp]) / plain_el, 1),
                     "p50_us": round(float(np.percentile(plain_lat, 50)), 1),
                     "p99_us": round(float(np.percentile(plain_lat, 99)), 1)},
           "server_stats": st,
           "clocks": clk,
           "e2e": {"value": round(qps_sat, 1), "unit": "queries/s",
                   "h2d_bytes_per_step": 8 * total, "d2h_bytes_per_step": total},
           "gpu_launches": st["batches"]}
    if rank == 0:
        print(json.dumps(out), flush=True)


# ------------------------------------------------------------ learned order
def run_learned(args, ws, rank, local):
    """Learned order: features, targets and training on 200 R-MAT graphs
    (scale uniform in 14-16, ef 16, seeds 1000-1199, t = 64, Degree-order
    builds); evaluation on R-MAT-21 (seed 5), t = 64: index size and build
    time with the network's order against the Degree order."""
    import numpy as np
    import torch

    from paper_1304_4661_gb300 import graphgen as gg
    from paper_1304_4661_gb300 import learned as L
    from paper_1304_4661_gb300 import pll

    torch.cuda.set_device(local)
    pll.load()
    t = 64
    specs = gg.learned_training_specs(args.learned_graphs)
    tg = [gg.rmat(sc, 16, seed=sd) for sc, sd in specs]
    X, y, rows, hs = L.harvest(tg, t=t)
    mlp, th = L.train(X, y, rows, epochs=args.learned_epochs, batch=16384, lr=2e-3)
    del X, y, rows
    g = gg.rmat(21, 16, seed=5)
    d_off, d_col = L._dev(g.offsets), L._dev(g.cols)
    stream = torch.cuda.current_stream()

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        r = fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1), r

    def build(order=None):
        ix = pll.Index.build(d_off, d_col, t=t, order=order)
        e = ix.label_entries()
        ix.close()
        return e

    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        pass
    clocks = ClockSampler(uuid)
    order = mlp.order(d_off, d_col, t)
    for _ in range(args.warmup):
        build()
        build(order)
    clocks.start()
    deg = [timed(build) for _ in range(args.steps)]
    ords = [timed(lambda: mlp.order(d_off, d_col, t)) for _ in range(args.steps)]
    lrn = [timed(lambda: build(ords[-1][1])) for _ in range(args.steps)]
    clk = clocks.stop()
    assert len({e for _, e in deg}) == 1 and len({e for _, e in lrn}) == 1
    deg_ms = statistics.mean(x[0] for x in deg)
    ord_ms = statistics.mean(x[0] for x in ords)
    lrn_ms = statistics.mean(x[0] for x in lrn)
    deg_e, lrn_e = deg[0][1], lrn[0][1]
    out = {"metric": "C4 learned order, R-MAT-21 (t=64): build s with the network's order "
                     "(order + build) vs Degree order",
           "value": round((ord_ms + lrn_ms) / 1e3, 6), "unit": "s", "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(ord_ms + lrn_ms, 3), "higher_is_better": False,
           "scaling": "weak", "vs_baseline": None, "dtype": "u8 labels, bf16/f32 network",
           "data": "synthetic",
           "config": {"workload": "train: 200 R-MAT (scale 14-16, ef 16, seeds 1000-1199), t=64; "
                                  "eval: R-MAT-21 (ef 16, seed 5), t=64",
                      "vertices": g.n, "arcs": g.nnz, "training_graphs": len(tg),
                      "epochs": args.learned_epochs},
           "degree": {"build_s": round(deg_ms / 1e3, 6), "label_entries": int(deg_e)},
           "learned": {"order_s": round(ord_ms / 1e3, 6), "build_s": round(lrn_ms / 1e3, 6),
                       "label_entries": int(lrn_e)},
           "label_entries_ratio": round(lrn_e / deg_e, 4),
           "build_time_ratio": round(lrn_ms / deg_ms, 4),
           "harvest": {k: (round(v, 3) if isinstance(v, float) else v) for k, v in hs.items()},
           "training": {"steps": th["steps"], "seconds": round(th["seconds"], 3),
                        "loss_first_last": [round(th["loss"][0][1], 5), round(th["loss"][-1][1], 5)]},
           "clocks": clk}
    if rank == 0:
        print(json.dumps(out), flush=True)


# ------------------------------------------------------------ paper variants
def run_variants(args, ws, rank, local):
    """Analogues of the paper's parameter studies on synthetic graphs: the
    number of bit-parallel roots t (Fig. 6: index size, build and query time
    against t) on R-MAT-20, and the vertex order (Table 4: Random, Degree and
    Closeness label size; closeness estimated from the distances to 64
    sample vertices, the bit-parallel roots) on
    R-MAT-14 and R-MAT-16 (Random order grows the index by orders of
    magnitude, so the larger graphs are left out)."""
    import numpy as np
    import torch

    from paper_1304_4661_gb300 import graphgen as gg
    from paper_1304_4661_gb300 import pll

    torch.cuda.set_device(local)
    pll.load()

    def dev(a):
        return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()

    stream = torch.cuda.current_stream()

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        r = fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1), r

    g = gg.rmat(20, 16, seed=1)
    d_off, d_col = dev(g.offsets), dev(g.cols)
    s, u = gg.pairs(g.n, 10_000_000, 3)
    ds, du = dev(s), dev(u)
    out = torch.empty(len(s), dtype=torch.uint8, device="cuda")
    tsweep = []
    for t in (0, 4, 16, 32, 64):
        for _ in range(args.warmup):
            pll.Index.build(d_off, d_col, t=t).close()
        bt = []
        for _ in range(args.steps):
            ms, ix = timed(lambda: pll.Index.build(d_off, d_col, t=t))
            bt.append(ms)
            qms, _ = timed(lambda: ix.query_async(ds, du, out))
            st = ix.stats()
            ent = ix.label_entries()
            ix.close()
        tsweep.append({"t": t, "build_s": round(statistics.mean(bt) / 1e3, 4), "label_entries": ent,
                       "avg_normal_label": round(ent / g.n, 2),
                       "index_bytes": int(st["index_bytes"]),
                       "queries_per_s": round(len(s) / (qms * 1e-3), 1)})
    orders = []
    for scale in (14, 16):
        h = gg.rmat(scale, 16, seed=1)
        o_off, o_col = dev(h.offsets), dev(h.cols)
        rnd = pll.order_from_scores(torch.from_numpy(gg.uniform(21, h.n).astype(np.float32)).cuda())
        # closeness estimated from BFSs out of sample vertices: the 64
        # bit-parallel roots of the Degree order (feature column 3 is the mean
        # distance to them, capped at 32); smaller mean distance first
        feat = pll.features(o_off, o_col, 64)
        clo = pll.order_from_scores(-feat[:, 3].contiguous())
        row = {"graph": f"R-MAT-{scale}", "vertices": h.n}
        for name, order in (("degree", None), ("closeness", clo), ("random", rnd)):
            ms, ix = timed(lambda: pll.Index.build(o_off, o_col, t=0, order=order))
            row[name] = {"label_entries": ix.label_entries(), "build_s": round(ms / 1e3, 4)}
            ix.close()
        row["random_over_degree"] = round(row["random"]["label_entries"] / row["degree"]["label_entries"], 2)
        row["closeness_over_degree"] = round(row["closeness"]["label_entries"] / row["degree"]["label_entries"], 3)
        orders.append(row)
    outj = {"metric": "Paper variants: t sweep on R-MAT-20 (Fig. 6 analogue) and Random vs Degree "
                      "order without bit-parallel labels (Table 4 analogue)",
            "value": tsweep[-1]["build_s"], "unit": "s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(tsweep[-1]["build_s"] * 1e3, 3),
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic",
            "config": {"workload": "R-MAT-20 (seed 1), 10M pairs (seed 3), t in {0,4,16,32,64}; "
                                   "R-MAT-14/16 (seed 1), t = 0, Degree vs Closeness (distances to 64 samples) vs Random (scores seed 21)"},
            "t_sweep": tsweep, "orders": orders}
    if rank == 0:
        print(json.dumps(outj), flush=True)


def run_paths(args, ws, rank, local):
    """Shortest-path queries (Sec. 6) over the R-MAT-20 index (t = 64): the
    parent pass (pll_paths_create) once, then per step 1M uniform pairs through
    pll_path_offsets + pll_path_query, beside the distance-only query of the
    same pairs. The index (1.4 GB) and the paths (tens of MB) are larger than
    L2."""
    import numpy as np
    import torch

    from paper_1304_4661_gb300 import graphgen as gg
    from paper_1304_4661_gb300 import pll

    torch.cuda.set_device(local)
    pll.load()

    def dev(a):
        return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()

    stream = torch.cuda.current_stream()

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        r = fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1), r

    g = gg.rmat(20, 16, seed=1)
    d_off, d_col = dev(g.offsets), dev(g.cols)
    ix = pll.Index.build(d_off, d_col, t=64)
    pms, P = timed(lambda: pll.Paths(ix, d_off, d_col))
    q = 1_000_000
    s, u = gg.pairs(g.n, q, 3)
    ds, du = dev(s), dev(u)
    out = torch.empty(q, dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        P.query(ds, du)
        ix.query_async(ds, du, out)
    pt, qt = [], []
    verts = 0
    barrier(ws)
    for _ in range(args.steps):
        ms, (off, path) = timed(lambda: P.query(ds, du))
        pt.append(ms)
        verts = int(path.numel())
        qt.append(timed(lambda: ix.query_async(ds, du, out))[0])
    barrier(ws)
    mean_ms = max_over_ranks(ws, statistics.mean(pt))
    reach = int((out != 255).sum().item())
    outj = {"metric": "Shortest-path queries (Sec. 6) on R-MAT-20, t = 64: paths per second",
            "value": round(job_rate(ws, q * args.steps, mean_ms * 1e-3 * args.steps), 1),
            "unit": "paths/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(mean_ms, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": "R-MAT-20 (seed 1, ef 16), t = 64, 1M uniform pairs (seed 3); "
                                   "inputs larger than L2 (index 1.4 GB)"},
            "parents_ms": round(pms, 2), "label_entries": ix.label_entries(),
            "reachable_pairs": reach, "path_vertices_per_step": verts,
            "path_vertices_per_s": round(verts / (mean_ms * 1e-3), 1),
            "distance_query_ms": round(statistics.mean(qt), 3),
            "gpu_launches": 3 * args.steps}
    P.close()
    ix.close()
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        outj["cpu_baseline"] = cpu_paths_sample()
    if rank == 0:
        print(json.dumps(outj), flush=True)


def run_directed(args, ws, rank, local):
    """Directed graphs (Sec. 6): pll_build_directed on an R-MAT graph whose
    edges are oriented at random (30 % both ways), then 1M uniform pairs
    through pll_dquery."""
    import numpy as np
    import torch

    from paper_1304_4661_gb300 import graphgen as gg
    from paper_1304_4661_gb300 import pll

    torch.cuda.set_device(local)
    pll.load()

    def dev(a):
        return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()

    stream = torch.cuda.current_stream()

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        r = fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1), r

    scale = args.directed_scale
    d = gg.oriented(gg.rmat(scale, 16, seed=1), 2)
    d_off, d_col = dev(d.offsets), dev(d.cols)
    for _ in range(args.warmup):
        pll.DirectedIndex(d_off, d_col).close()
    bt = []
    barrier(ws)
    for i in range(args.steps):
        ms, ix = timed(lambda: pll.DirectedIndex(d_off, d_col))
        bt.append(ms)
        ent = ix.entries()
        if i < args.steps - 1:
            ix.close()  # the last one answers the queries
    barrier(ws)
    mean_ms = max_over_ranks(ws, statistics.mean(bt))
    q = 1_000_000
    s, u = gg.pairs(d.n, q, 3)
    ds, du = dev(s), dev(u)
    for _ in range(3):
        ix.query(ds, du)
    qms = statistics.mean(timed(lambda: ix.query(ds, du))[0] for _ in range(5))
    ix.close()
    outj = {"metric": f"Directed index build (Sec. 6) on oriented R-MAT-{scale}: seconds per build",
            "value": round(mean_ms / 1e3, 4), "unit": "s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(mean_ms, 3), "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": f"R-MAT-{scale} (seed 1, ef 16), each edge one way at random, 30 % both "
                                   f"ways (seed 2); {d.n} vertices, {d.nnz} arcs; 1M uniform pairs (seed 3)"},
            "label_entries_in": ent[0], "label_entries_out": ent[1],
            "queries_per_s": round(q / (qms * 1e-3), 1)}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        outj["cpu_baseline"] = cpu_directed_sample()
    if rank == 0:
        print(json.dumps(outj), flush=True)


# ------------------------------------------------------------ CPU oracle
def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def gpu_same_sample(g, s_host, u_host, t, steps=3):
    """The GPU path on the oracle's sample: pll_build (device-timed, mean of
    `steps` after one warm-up) and one pll_query launch over the same pairs."""
    import numpy as np
    import torch

    from paper_1304_4661_gb300 import pll

    def dev(a):
        return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()

    off, col, sd, ud = dev(g.offsets), dev(g.cols), dev(s_host), dev(u_host)
    out = torch.empty(len(s_host), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    bt, qt = [], []
    for it in range(steps + 1):
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        ix = pll.Index.build(off, col, t=t)
        e1.record(stream)
        ix.query_async(sd, ud, out)
        e2.record(stream)
        e2.synchronize()
        assert ix.query_errors() == 0
        ix.close()
        if it:
            bt.append(e0.elapsed_time(e1) * 1e-3)
            qt.append(e1.elapsed_time(e2) * 1e-3)
    return statistics.mean(bt), len(s_host) / statistics.mean(qt), out.cpu().numpy()


def cpu_baseline(args, scale=None, with_gpu=False):
    """The oracle as it stands on a bounded sample: a full index build of a
    smaller R-MAT of the same family (single thread, as the paper's build is
    sequential), plus 1M queries on one thread and on all host cores. With
    with_gpu, the GPU path is timed on the very same sample beside it."""
    import numpy as np

    import oracle
    from paper_1304_4661_gb300 import graphgen as gg
    scale = scale or args.cpu_scale
    g = gg.rmat(scale, 16, seed=1)
    t0 = time.perf_counter()
    ix = oracle.Index(g.offsets, g.cols, 64)
    tb = time.perf_counter() - t0
    s, u = gg.pairs(g.n, 1_000_000, 3)
    t1 = time.perf_counter()
    ref = ix.query_batch(s, u)
    tq = time.perf_counter() - t1
    cores = host_cores()
    t2 = time.perf_counter()
    ix.query_batch_mt(s, u, cores)
    tqa = time.perf_counter() - t2
    out = {"value": round(tb, 3), "unit": "s", "cores": 1, "kind": "oracle",
           "queries_per_s": round(1_000_000 / tq, 1),
           "queries_per_s_all_cores": round(1_000_000 / tqa, 1), "query_cores": cores,
           "sample": f"full oracle build of R-MAT scale {scale} (ef 16, seed 1, t=64, "
                     f"{g.n} vertices, {g.nnz} arcs; one thread), then 1M uniform queries "
                     f"(one thread, then {cores} threads)"}
    if with_gpu:
        gb, gq, ans = gpu_same_sample(g, s, u, 64)
        assert np.array_equal(ans, ref), "GPU answers differ from the oracle on the sample"
        out["gpu_same_sample"] = {
            "build_s": round(gb, 5), "queries_per_s": round(gq, 1),
            "build_speedup": round(tb / gb, 1),
            "query_speedup_vs_1_core": round(gq * tq / 1_000_000, 1),
            "query_speedup_vs_all_cores": round(gq * tqa / 1_000_000, 1),
            "note": "pll_build + one pll_query launch on the same graph and pairs, CUDA events; "
                    "answers checked equal to the oracle's"}
    return out


def cpu_paths_sample(scale: int = 16, q: int = 20000):
    """The oracle's path restoration (Sec. 6) as it stands, single-threaded,
    on a bounded sample: R-MAT at `scale` (t = 64), q uniform pairs."""
    import oracle
    from paper_1304_4661_gb300 import graphgen as gg
    g = gg.rmat(scale, 16, seed=1)
    ix = oracle.Index(g.offsets, g.cols, 64)
    s, u = gg.pairs(g.n, q, 3)
    t0 = time.perf_counter()
    verts = sum(len(ix.path(int(a), int(b))) for a, b in zip(s, u))
    dt = time.perf_counter() - t0
    return {"value": round(q / dt, 1), "unit": "paths/s", "cores": 1, "kind": "oracle",
            "path_vertices_per_s": round(verts / dt, 1),
            "sample": f"{q} uniform pairs on R-MAT scale {scale} (ef 16, seed 1, t = 64, oracle index "
                      f"built beforehand, not timed); one oracle call per pair; single thread"}


def cpu_directed_sample(scale: int = 14):
    """The oracle's directed build (Sec. 6) as it stands, single-threaded, on
    an oriented R-MAT of the given scale."""
    import oracle
    from paper_1304_4661_gb300 import graphgen as gg
    d = gg.oriented(gg.rmat(scale, 16, seed=1), 2)
    t0 = time.perf_counter()
    ix = oracle.DirectedIndex(d.offsets, d.cols)
    dt = time.perf_counter() - t0
    return {"value": round(dt, 3), "unit": "s", "cores": 1, "kind": "oracle",
            "label_entries": [len(ix.labels_in().hubs), len(ix.labels_out().hubs)],
            "sample": f"full oracle directed build of oriented R-MAT scale {scale} (ef 16, seed 1, "
                      f"orientation seed 2, 30 % both ways; {d.n} vertices, {d.nnz} arcs); single thread"}


def run_reference(args, w, ws, rank):
    """The CPU oracle as the reference arm, each step a bounded sample."""
    if rank != 0:
        return
    import oracle
    from paper_1304_4661_gb300 import graphgen as gg
    scale = args.ref_scale
    g = gg.rmat(scale, 16, seed=1)
    nq = 1_000_000
    s, u = gg.pairs(g.n, nq, 3)
    bt, qt = [], []
    for it in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        ix = oracle.Index(g.offsets, g.cols, 64)
        t1 = time.perf_counter()
        ix.query_batch(s, u)
        t2 = time.perf_counter()
        del ix
        if it >= args.warmup:
            bt.append(t1 - t0)
            qt.append(t2 - t1)
    v = statistics.mean(bt)
    sample = (f"oracle full build of R-MAT scale {scale} (ef 16, seed 1, t=64, {g.n} vertices, "
              f"{g.nnz} arcs) + 1M uniform queries per step; single thread; the same sample the "
              f"GPU line times beside its cpu_baseline (gpu_same_sample)")
    out = {"impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": "s", "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": round((v + statistics.mean(qt)) * 1e3, 3), "higher_is_better": False,
           "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
           "config": {"workload": _workload_name(w), "sample": sample,
                      "why_sample": "one oracle build of the full workload takes about 15 minutes on "
                                    "one core, too long for W + K steps; the sample is the same "
                                    "family at a smaller scale"},
           "queries_per_s": round(nq / statistics.mean(qt), 1),
           "cpu_baseline": {"value": round(v, 4), "unit": "s", "cores": 1, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": round(v, 4), "unit": "s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["batch256", "serve", "learned", "variants", "paths", "directed"], default="rmat20")
    ap.add_argument("--root-batch", type=int, default=0)
    ap.add_argument("--block", type=int, default=0)
    ap.add_argument("--latency-samples", type=int, default=2000)
    ap.add_argument("--cpu-scale", type=int, default=17)
    ap.add_argument("--ref-scale", type=int, default=17)
    ap.add_argument("--serve-requests", type=int, default=100_000)
    ap.add_argument("--serve-seconds", type=float, default=2.0)
    ap.add_argument("--serve-plain", type=int, default=5000)
    ap.add_argument("--serve-streams", type=int, default=4)
    ap.add_argument("--serve-clients", type=int, default=12)
    ap.add_argument("--learned-graphs", type=int, default=200)
    ap.add_argument("--learned-epochs", type=int, default=4)
    ap.add_argument("--directed-scale", type=int, default=16)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--host-levels", action="store_true",
                    help="run each root batch's levels as separate launches (PLL_BUILD_HOST_LEVELS)")
    ap.add_argument("--coop-levels", action="store_true",
                    help="run each root batch's levels as one cooperative launch (PLL_BUILD_COOP_LEVELS)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    args.flags = (1 if args.host_levels else 0) | (4 if args.coop_levels else 0)  # PLL_BUILD_*_LEVELS
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.workload in ("batch256", "serve", "learned", "variants", "paths", "directed"):
        ws, rank, local = dist_setup()
        {"batch256": run_batch, "serve": run_serve, "learned": run_learned,
         "variants": run_variants, "paths": run_paths,
         "directed": run_directed}[args.workload](args, ws, rank, local)
        return
    w = WORKLOADS[args.workload]
    ws, rank, local = dist_setup() if args.impl == "ours" else (
        int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), 0)
    if args.impl == "reference":
        run_reference(args, w, ws, rank)
        return
    run_ours(args, w, ws, rank, local)


if __name__ == "__main__":
    main()
