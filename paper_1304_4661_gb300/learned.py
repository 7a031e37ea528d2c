"""Training and use of the learned vertex order (host orchestration only).

Every arithmetic step runs in the library's kernels (pll_features,
pll_hub_counts, pll_mlp_*, pll_learned_order); this module moves tensors,
picks the training rows and schedules the minibatches.

  harvest(graphs, t)   features of every vertex and its target, log(1 + the
                       label entries it hubs in the Degree-order build); the
                       rows kept are the vertices that were pruned-BFS roots
                       (count > 0; bit-parallel vertices hub no entries)
  train(...)           Adam on the mean squared error, shuffled minibatches
  learned_order(...)   the order the trained network proposes for a graph
"""
from __future__ import annotations

import time

import numpy as np

from . import graphgen as gg
from . import pll


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()


def harvest(graphs, t: int = 64):
    """Returns (X float32 CUDA [N, 8], y float32 CUDA [N], rows int32 CUDA
    [M] indices of the kept rows, stats)."""
    import torch
    N = sum(g.n for g in graphs)
    X = torch.empty((N, 8), dtype=torch.float32, device="cuda")
    y = torch.empty(N, dtype=torch.float32, device="cuda")
    keep = []
    base = 0
    entries = 0
    t0 = time.perf_counter()
    for g in graphs:
        off, col = _dev(g.offsets), _dev(g.cols)
        pll.features(off, col, t, out=X[base:base + g.n])
        ix = pll.Index.build(off, col, t=t)
        c, f = ix.hub_counts()
        y[base:base + g.n] = f
        entries += ix.label_entries()
        ix.close()
        keep.append(np.flatnonzero(c.cpu().numpy() > 0) + base)
        base += g.n
    torch.cuda.synchronize()
    rows = torch.from_numpy(np.concatenate(keep).astype(np.int32)).cuda()
    return X, y, rows, {"graphs": len(graphs), "vertices": N, "rows": int(rows.shape[0]),
                        "label_entries": entries, "seconds": time.perf_counter() - t0}


def train(X, y, rows, epochs: int = 4, batch: int = 16384, lr: float = 2e-3, seed: int = 5,
          init_seed: int = 1, log_every: int = 0):
    """Adam over shuffled minibatches of `rows`; returns (MLP, history)."""
    import torch
    mlp = pll.MLP(max_batch=batch)
    mlp.set_params(gg.mlp_init(init_seed))
    rng = np.random.default_rng(seed)
    rows_h = rows.cpu().numpy()
    hist = []
    t0 = time.perf_counter()
    step = 0
    for ep in range(epochs):
        perm = torch.from_numpy(rows_h[rng.permutation(rows_h.shape[0])]).cuda()
        for b in range(0, perm.shape[0], batch):
            mlp.train_step(X, y, perm[b:b + batch], lr)
            step += 1
            if log_every and step % log_every == 0:
                hist.append((step, mlp.loss()))
        hist.append((step, mlp.loss()))
    torch.cuda.synchronize()
    return mlp, {"steps": step, "seconds": time.perf_counter() - t0, "loss": hist}


def learned_order(mlp, g, t: int = 64):
    off, col = _dev(g.offsets), _dev(g.cols)
    return mlp.order(off, col, t)
