"""Full-size parity by digest: the CUDA build of each full-size R-MAT graph,
at the default options (the launch configuration bench.py times), against the
CPU oracle's whole index.

``tests/golden/<name>_t<t>_digest.json`` holds SHA-256 digests of the
oracle's Degree order, bit-parallel roots and labels, every normal label and
its answers to seeded uniform pairs, written by
``tests/golden/make_fullsize_digests.py`` (which calls only the oracle and the
seeded generators). The GPU exports are hashed the same way and must match
byte for byte; on a mismatch the per-block label digests name the first
block of 65,536 vertex ids that differs.
"""
import hashlib
import json
import os

import numpy as np
import pytest

from paper_1304_4661_gb300 import graphgen as gg

from .gpu_util import dev_u32, gpu_build

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
NAMES = ["rmat16_t64", "rmat18_t64", "rmat19_t64", "rmat20_t64", "rmat21_t64", "rmat22_t64"]


def sha(a):
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def load(name):
    path = os.path.join(GOLDEN, f"{name}_digest.json")
    if not os.path.exists(path):
        pytest.skip(f"{name}: no oracle digest written")
    return json.load(open(path))


def block_digests(off, hubs, dists, n, block):
    out = []
    for v0 in range(0, n, block):
        v1 = min(n, v0 + block)
        a, b = int(off[v0]), int(off[v1])
        h = hashlib.sha256()
        h.update(np.diff(off[v0:v1 + 1].astype(np.int64)).astype(np.uint32).tobytes())
        h.update(hubs[a:b].tobytes())
        h.update(dists[a:b].tobytes())
        out.append(h.hexdigest()[:32])
    return out


@pytest.mark.parametrize("name", NAMES)
def test_full_index_equals_the_oracle_digest(name):
    import torch
    ref = load(name)
    gr = ref["graph"]
    g = gg.rmat(gr["scale"], gr["edge_factor"], seed=gr["seed"])
    assert (g.n, g.nnz) == (gr["n"], gr["nnz"])
    assert sha(g.offsets) == gr["offsets"] and sha(g.cols) == gr["cols"]
    t = ref["t"]
    ix = gpu_build(g, t)
    assert sha(ix.order()) == ref["order"]
    roots, cnt, S = ix.bp_roots()
    assert sha(roots) == ref["bp_roots"] and sha(cnt) == ref["bp_cnt"]
    Sm = np.where(np.arange(64)[None, :] < cnt[:, None], S, np.uint32(0xffffffff)).astype(np.uint32)
    assert sha(Sm) == ref["bp_S"]
    d, m1, m0 = ix.bp()
    assert sha(d) == ref["bp_d"] and sha(m1) == ref["bp_m1"] and sha(m0) == ref["bp_m0"]
    L = ix.labels()
    assert int(L.hubs.shape[0]) == ref["label_entries"] == ix.label_entries()
    blocks = block_digests(L.offsets, L.hubs, L.dists, g.n, ref["label_block"])
    bad = [i for i, (a, b) in enumerate(zip(blocks, ref["label_blocks"])) if a != b]
    assert not bad, f"labels differ in vertex blocks {bad[:8]} (block = {ref['label_block']} ids)"
    assert sha(L.offsets.astype(np.uint64)) == ref["label_offsets"]
    assert sha(L.hubs.astype(np.uint32)) == ref["label_hubs"]
    assert sha(L.dists.astype(np.uint8)) == ref["label_dists"]
    del L
    p = ref["pairs"]
    s, u = gg.pairs(g.n, p["count"], p["seed"])
    out = torch.empty(p["count"], dtype=torch.uint8, device="cuda")
    ix.query_async(dev_u32(s), dev_u32(u), out)
    assert ix.query_errors() == 0
    ans = out.cpu().numpy()
    hist = np.bincount(ans, minlength=256)
    assert {str(i): int(c) for i, c in enumerate(hist) if c} == p["histogram"]
    assert sha(ans) == p["answers"]
