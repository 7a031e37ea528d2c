"""Helpers shared by the GPU tests: device upload and label comparison."""
from __future__ import annotations

import numpy as np

INF = 255


def dev_u32(a):
    """numpy uint32 array -> contiguous CUDA tensor holding the same bits."""
    import torch
    a = np.ascontiguousarray(np.asarray(a, dtype=np.uint32))
    return torch.from_numpy(a.view(np.int32)).cuda()


def gpu_build(g, t, order=None, root_batch=0, block=0, flags=0):
    from paper_1304_4661_gb300 import pll
    return pll.Index.build(dev_u32(g.offsets), dev_u32(g.cols), t=t,
                           order=None if order is None else dev_u32(order),
                           root_batch=root_batch, block=block, flags=flags)


def gpu_query(ix, s, t):
    out = ix.query(dev_u32(s), dev_u32(t))
    return out.cpu().numpy()


def same_labels(a, b):
    """Exact equality of two exported label sets (offsets, hubs, dists)."""
    return (np.array_equal(a.offsets, b.offsets) and np.array_equal(a.hubs, b.hubs)
            and np.array_equal(a.dists, b.dists))


def first_label_diff(a, b, n):
    for v in range(n):
        la = list(zip(a.hubs[a.offsets[v]:a.offsets[v + 1]].tolist(),
                      a.dists[a.offsets[v]:a.offsets[v + 1]].tolist()))
        lb = list(zip(b.hubs[b.offsets[v]:b.offsets[v + 1]].tolist(),
                      b.dists[b.offsets[v]:b.offsets[v + 1]].tolist()))
        if la != lb:
            return v, la, lb
    return None
