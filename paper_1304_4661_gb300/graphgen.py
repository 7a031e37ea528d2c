"""Seeded synthetic inputs: graphs (uint32 CSR) and uniform query pairs.

Thin ctypes front end of ``csrc/graphgen.c``. The generators hold none of the
labelling method's arithmetic; both the CUDA library and the CPU oracle take
their output as plain arrays. Graph families stand in for the power-law,
small-world networks the paper evaluates on (Sec. 6.1, Table 3):
Barabasi-Albert, Watts-Strogatz (high diameter) and R-MAT.
"""
from __future__ import annotations

import ctypes as C
import math
from dataclasses import dataclass

import numpy as np

from . import _build

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build_graphgen()
        lib = C.CDLL(path)
        vp, u32, u64, dbl = C.c_void_p, C.c_uint32, C.c_uint64, C.c_double
        lib.gg_from_edges.restype = vp
        lib.gg_from_edges.argtypes = [u32, u64, vp, vp]
        lib.gg_ba.restype = vp
        lib.gg_ba.argtypes = [u32, u32, u64]
        lib.gg_ws.restype = vp
        lib.gg_ws.argtypes = [u32, u32, dbl, u64]
        lib.gg_rmat.restype = vp
        lib.gg_rmat.argtypes = [u32, u32, dbl, dbl, dbl, u64]
        lib.gg_n.restype = u32
        lib.gg_n.argtypes = [vp]
        lib.gg_nnz.restype = u64
        lib.gg_nnz.argtypes = [vp]
        lib.gg_copy.restype = None
        lib.gg_copy.argtypes = [vp, vp, vp]
        lib.gg_free.restype = None
        lib.gg_free.argtypes = [vp]
        lib.gg_pairs.restype = None
        lib.gg_pairs.argtypes = [u32, u64, u64, vp, vp]
        lib.gg_uniform.restype = None
        lib.gg_uniform.argtypes = [u64, u64, vp]
        lib.gg_below.restype = None
        lib.gg_below.argtypes = [u64, u64, u64, vp]
        _lib = lib
    return _lib


@dataclass
class Graph:
    """Undirected simple graph as a symmetric CSR (sorted neighbour lists)."""

    n: int
    offsets: np.ndarray  # uint32 [n + 1]
    cols: np.ndarray     # uint32 [nnz]
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.cols.shape[0])

    @property
    def degrees(self) -> np.ndarray:
        return np.diff(self.offsets.astype(np.int64))


def _take(handle, name) -> Graph:
    lib = _load()
    if not handle:
        raise MemoryError(f"graph generator failed for {name}")
    try:
        n = lib.gg_n(handle)
        nnz = lib.gg_nnz(handle)
        off = np.empty(n + 1, dtype=np.uint32)
        col = np.empty(max(nnz, 1), dtype=np.uint32)
        lib.gg_copy(handle, off.ctypes.data, col.ctypes.data)
    finally:
        lib.gg_free(handle)
    return Graph(n, off, col[:nnz].copy(), name)


def from_edges(n: int, u, v, name: str = "edges") -> Graph:
    """Symmetrised simple graph on n vertices from an edge list."""
    u = np.ascontiguousarray(np.asarray(u, dtype=np.uint32))
    v = np.ascontiguousarray(np.asarray(v, dtype=np.uint32))
    assert u.shape == v.shape
    h = _load().gg_from_edges(n, u.shape[0], u.ctypes.data, v.ctypes.data)
    return _take(h, name)


def ba(n: int, m: int, seed: int) -> Graph:
    return _take(_load().gg_ba(n, m, seed), f"ba(n={n},m={m},seed={seed})")


def ws(n: int, k: int, p: float, seed: int) -> Graph:
    return _take(_load().gg_ws(n, k, p, seed), f"ws(n={n},k={k},p={p},seed={seed})")


def rmat(scale: int, ef: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 1) -> Graph:
    return _take(_load().gg_rmat(scale, ef, a, b, c, seed),
                 f"rmat(scale={scale},ef={ef},seed={seed})")


def pairs(n: int, q: int, seed: int):
    """q uniform query pairs (s, t) in [0, n)^2 as two uint32 arrays."""
    s = np.empty(max(q, 1), dtype=np.uint32)
    t = np.empty(max(q, 1), dtype=np.uint32)
    if q:
        _load().gg_pairs(n, q, seed, s.ctypes.data, t.ctypes.data)
    return s[:q], t[:q]


def uniform(seed: int, count: int) -> np.ndarray:
    out = np.empty(max(count, 1), dtype=np.float64)
    if count:
        _load().gg_uniform(seed, count, out.ctypes.data)
    return out[:count]


def below(seed: int, count: int, bound: int) -> np.ndarray:
    out = np.empty(max(count, 1), dtype=np.uint64)
    if count:
        _load().gg_below(seed, count, bound, out.ctypes.data)
    return out[:count]


def batch_specs(count: int = 256, seed: int = 4, n_lo: int = 1000, n_hi: int = 50000):
    """The uneven multi-graph workload: half Barabasi-Albert (n log-uniform on
    [n_lo, n_hi], m uniform in 2..8), half Watts-Strogatz (n log-uniform on
    [n_lo, n_hi], k = 6, p = 0.1). Returns a list of (kind, n, param, seed)."""
    u = uniform(seed, 2 * count)
    ms = below(seed + 1, count, 7)
    specs = []
    lo, hi = math.log(n_lo), math.log(n_hi)
    for i in range(count):
        n = int(math.floor(math.exp(lo + (hi - lo) * float(u[i]))))
        n = max(n_lo, min(n_hi, n))
        if i < count // 2:
            specs.append(("ba", n, int(ms[i]) + 2, 10_000 + i))
        else:
            specs.append(("ws", n, 6, 20_000 + i))
    return specs


def make(spec) -> Graph:
    kind, n, param, seed = spec
    if kind == "ba":
        return ba(n, param, seed)
    if kind == "ws":
        return ws(n, param, 0.1, seed)
    raise ValueError(kind)


def union(graphs):
    """Disjoint union of graphs as one CSR: graph g gets the vertex ids
    [start[g], start[g+1]). Returns (offsets, cols, start) as uint32 arrays."""
    sizes = np.array([g.n for g in graphs], dtype=np.int64)
    start = np.zeros(len(graphs) + 1, dtype=np.int64)
    start[1:] = np.cumsum(sizes)
    n = int(start[-1])
    arcs = np.array([g.nnz for g in graphs], dtype=np.int64)
    astart = np.zeros(len(graphs) + 1, dtype=np.int64)
    astart[1:] = np.cumsum(arcs)
    off = np.zeros(n + 1, dtype=np.int64)
    col = np.empty(int(astart[-1]), dtype=np.uint32)
    for i, g in enumerate(graphs):
        off[start[i]:start[i + 1] + 1] = g.offsets.astype(np.int64) + astart[i]
        col[astart[i]:astart[i + 1]] = g.cols + np.uint32(start[i])
    return off.astype(np.uint32), col, start.astype(np.uint32)


def serve_requests(n: int, count: int, seed: int, one_to_many: float = 0.1, fan: int = 1000,
                   max_pairs: int = 4096):
    """A request mix for the serving loop: a fraction `one_to_many` of the
    requests are one source with `fan` uniform targets, the rest hold a
    log-uniform number of uniform pairs in [1, max_pairs]. Returns (src, dst,
    req_off, one_to_many_mask); request i is pairs req_off[i] .. req_off[i+1]."""
    u = uniform(seed, 2 * count)
    many = u[:count] < one_to_many
    sizes = np.floor(np.exp(u[count:] * math.log(max_pairs + 1))).astype(np.int64)
    sizes = np.clip(sizes, 1, max_pairs)
    sizes[many] = fan
    off = np.zeros(count + 1, dtype=np.uint64)
    off[1:] = np.cumsum(sizes)
    s, t = pairs(n, int(off[-1]), seed + 1)
    req = np.repeat(np.arange(count), sizes)
    first = s[off[:-1].astype(np.int64)]
    s = np.where(many[req], first[req], s).astype(np.uint32)
    return s, t, off, many


def poisson_arrivals(count: int, rate_per_s: float, seed: int) -> np.ndarray:
    """Arrival times in microseconds of an open-loop Poisson process of the
    given rate (exponential gaps from seeded uniforms), starting at 0."""
    u = uniform(seed, count)
    gaps = -np.log1p(-u) / rate_per_s * 1e6
    out = np.cumsum(gaps)
    return out - out[0] if count else out


MLP_NPARAM = 4801  # 8 -> 64 -> 64 -> 1: W1 [64][8], b1 [64], W2 [64][64], b2 [64], w3 [64], b3


def mlp_init(seed: int) -> np.ndarray:
    """Initial parameters of the vertex-scoring network, float32[4801] in the
    layout W1 [64][8], b1 [64], W2 [64][64], b2 [64], w3 [64], b3 [1]:
    weights He-uniform, U(-a, a) with a = sqrt(6 / fan_in), from the seeded
    uniform generator; biases zero."""
    u = uniform(seed, MLP_NPARAM)
    p = np.zeros(MLP_NPARAM)
    for lo, hi, fan in ((0, 512, 8), (576, 4672, 64), (4736, 4800, 64)):
        p[lo:hi] = (2 * u[lo:hi] - 1) * math.sqrt(6.0 / fan)
    return p.astype(np.float32)


def learned_training_specs(count: int = 200, seed: int = 11, scales=(14, 15, 16),
                           first_seed: int = 1000):
    """Training graphs of the learned order: R-MAT (ef 16, default a/b/c),
    scale drawn uniformly from `scales`, graph seeds first_seed, first_seed + 1,
    ... Returns a list of (scale, graph_seed)."""
    u = uniform(seed, count)
    k = len(scales)
    return [(scales[min(k - 1, int(u[i] * k))], first_seed + i) for i in range(count)]


# ------------------------------------------------------------ directed graphs
@dataclass
class Digraph:
    """Directed graph as an out-neighbour CSR: arcs u -> cols[e] for e in
    [offsets[u], offsets[u + 1]), ascending, no repeats, no self-loops."""

    n: int
    offsets: np.ndarray  # uint32 [n + 1]
    cols: np.ndarray     # uint32 [nnz]
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.cols.shape[0])


def digraph(n: int, arcs, name: str = "arcs") -> Digraph:
    """Digraph from (u, v) arcs; self-loops and repeats are dropped."""
    a = np.asarray(list(arcs), dtype=np.int64).reshape(-1, 2)
    a = a[a[:, 0] != a[:, 1]]
    if a.shape[0]:
        a = np.unique(a, axis=0)  # sorted by (u, v)
    off = np.zeros(n + 1, dtype=np.int64)
    np.add.at(off, a[:, 0] + 1, 1)
    return Digraph(n, np.cumsum(off).astype(np.uint32), a[:, 1].astype(np.uint32), name)


def random_digraph(n: int, m: int, seed: int) -> Digraph:
    """m arcs with both ends uniform on [0, n) (repeats and self-loops then
    dropped)."""
    if n == 0 or m == 0:
        return digraph(n, [], f"rand_digraph(n={n},m={m},seed={seed})")
    x = below(seed, 2 * m, n).astype(np.int64).reshape(m, 2)
    return digraph(n, x, f"rand_digraph(n={n},m={m},seed={seed})")


def oriented(g: Graph, seed: int, both: float = 0.3) -> Digraph:
    """A digraph from an undirected graph: each edge {u, v} becomes both arcs
    with probability `both`, else one arc in a uniformly chosen direction."""
    rows = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.offsets.astype(np.int64)))
    cols = g.cols.astype(np.int64)
    keep = rows < cols
    u, v = rows[keep], cols[keep]
    r = uniform(seed, 2 * len(u)).reshape(-1, 2) if len(u) else np.zeros((0, 2))
    two = r[:, 0] < both
    fwd = r[:, 1] < 0.5
    arcs = np.concatenate([np.stack([u[two | fwd], v[two | fwd]], 1),
                           np.stack([v[two | ~fwd], u[two | ~fwd]], 1)])
    return digraph(g.n, arcs, f"oriented({g.name},seed={seed},both={both})")
