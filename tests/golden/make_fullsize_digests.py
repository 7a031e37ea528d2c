"""Write SHA-256 digests of the oracle's full index for the full-size graphs.

The oracle (plain single-threaded C, ``oracle/``) builds the whole index of
each graph below: the Degree order (Sec. 4.4.2), the bit-parallel roots and
labels (Sec. 5.4, Alg. 3), every normal label (Alg. 1/2 with bit-parallel
pruning) and the answers to a seeded set of uniform query pairs (Sec. 3.3,
Sec. 5.3). The digests go to ``tests/golden/<name>.json``; the GPU tests
compare the CUDA path's exports with them byte for byte.

Nothing here calls the CUDA library: the inputs come from the seeded
generators and every value from ``oracle/``. A build takes about 15 minutes
(R-MAT-20) to a few hours (R-MAT-22) on one CPU core.

    python tests/golden/make_fullsize_digests.py rmat20 [rmat21 rmat22 ...]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1304_4661_gb300 import graphgen as gg  # noqa: E402

# name -> (R-MAT scale, graph seed, t, query pairs, pair seed)
CONFIGS = {
    "rmat20": (20, 1, 64, 10_000_000, 3),   # the benchmark workload
    "rmat21": (21, 5, 64, 10_000_000, 3),   # the learned-order evaluation graph, Degree order
    "rmat22": (22, 6, 64, 10_000_000, 3),   # the served index
    "rmat16": (16, 1, 64, 1_000_000, 3),    # a small case of the same recipe (quick self-check)
    "rmat18": (18, 1, 64, 1_000_000, 3),    # the profiling cases of the sweeps
    "rmat19": (19, 1, 64, 1_000_000, 3),
}
BLOCK = 1 << 16  # vertices per label block digest


def sha(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def label_block_digests(off: np.ndarray, hubs: np.ndarray, dists: np.ndarray, n: int) -> list:
    """One digest per block of BLOCK vertex ids, so a mismatch names its block."""
    out = []
    for v0 in range(0, n, BLOCK):
        v1 = min(n, v0 + BLOCK)
        a, b = int(off[v0]), int(off[v1])
        h = hashlib.sha256()
        h.update(np.diff(off[v0:v1 + 1].astype(np.int64)).astype(np.uint32).tobytes())
        h.update(hubs[a:b].tobytes())
        h.update(dists[a:b].tobytes())
        out.append(h.hexdigest()[:32])
    return out


def digest(name: str) -> dict:
    scale, seed, t, q, pseed = CONFIGS[name]
    t0 = time.time()
    g = gg.rmat(scale, 16, seed=seed)
    ix = oracle.Index(g.offsets, g.cols, t)
    t_build = time.time() - t0
    roots, cnt, S = ix.bp_roots()
    d, m1, m0 = ix.bp()
    L = ix.labels()
    s, u = gg.pairs(g.n, q, pseed)
    t1 = time.time()
    ans = ix.query_batch(s, u)
    t_query = time.time() - t1
    hist = np.bincount(ans, minlength=256)
    return {
        "what": "SHA-256 digests of the CPU oracle's full index (Degree order, bit-parallel "
                "roots and labels, normal labels) and of its answers to seeded uniform pairs",
        "cite": "Sec. 4.4.2 (Degree order); Sec. 5.4 and Alg. 3 (bit-parallel labels); Alg. 1/2 "
                "(pruned labels); Sec. 3.3 and Sec. 5.3 (queries)",
        "writer": "tests/golden/make_fullsize_digests.py (calls only oracle/ and the seeded generators)",
        "graph": {"family": "rmat", "scale": scale, "edge_factor": 16, "abcd": [0.57, 0.19, 0.19, 0.05],
                  "seed": seed, "n": g.n, "nnz": g.nnz, "offsets": sha(g.offsets), "cols": sha(g.cols)},
        "t": t,
        "order": sha(ix.order()),
        "bp_roots": sha(roots), "bp_cnt": sha(cnt),
        "bp_S": sha(np.where(np.arange(64)[None, :] < cnt[:, None], S, np.uint32(0xffffffff)).astype(np.uint32)),
        "bp_d": sha(d), "bp_m1": sha(m1), "bp_m0": sha(m0),
        "label_entries": int(L.hubs.shape[0]),
        "label_offsets": sha(L.offsets.astype(np.uint64)),
        "label_hubs": sha(L.hubs.astype(np.uint32)),
        "label_dists": sha(L.dists.astype(np.uint8)),
        "label_block": BLOCK,
        "label_blocks": label_block_digests(L.offsets, L.hubs, L.dists, g.n),
        "pairs": {"count": q, "seed": pseed, "answers": sha(ans),
                  "histogram": {str(i): int(c) for i, c in enumerate(hist) if c}},
        # work of the sequential pruned BFSs (Alg. 1): vertices dequeued, vertices
        # labelled, label entries scanned by prune tests, arcs of labelled vertices
        "sequential_work": ix.counters(),
        "oracle_seconds": {"build": round(t_build, 1), "queries": round(t_query, 1)},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("names", nargs="+", choices=sorted(CONFIGS))
    args = ap.parse_args()
    here = os.path.dirname(os.path.abspath(__file__))
    for name in args.names:
        rec = digest(name)
        path = os.path.join(here, f"{name}_t{rec['t']}_digest.json")
        with open(path + ".tmp", "w") as f:
            json.dump(rec, f, indent=1)
            f.write("\n")
        os.replace(path + ".tmp", path)
        print(name, rec["label_entries"], rec["oracle_seconds"], flush=True)


if __name__ == "__main__":
    main()
