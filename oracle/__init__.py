"""CPU oracle for Pruned Landmark Labeling -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package. The product
path (the CUDA library and its binding) never imports it, and it never
imports the product: the two meet only through the seeded inputs.

``oracle.c`` is a plain single-threaded C restatement of the paper:
the Degree order (Sec. 4.4.2), bit-parallel labels (Alg. 3, Sec. 5),
the pruned BFSs of Alg. 1/2 with bit-parallel pruning (Sec. 5.4), the
label query (Sec. 3.3, Sec. 5.3), plain BFS, the closed form of one
label derived from Thm 4.1 / Thm 4.2, the parents and path restoration of
the shortest-path queries of Sec. 6, and the directed-graph labels of Sec. 6
(see the header of oracle.c).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass
from pathlib import Path

import numpy as np

HERE = Path(__file__).resolve().parent
SRC = HERE / "oracle.c"
SO = HERE / "liboracle.so"

OK, E_INVAL, E_ORDER, E_RANGE, E_NOMEM = 0, 1, 2, 3, 4
INF = 255
BPW = 64


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (plain -O2; no vector intrinsics)."""
    if force or not SO.exists() or SO.stat().st_mtime < SRC.stat().st_mtime:
        tmp = SO.with_suffix(f".so.tmp{os.getpid()}")
        r = subprocess.run(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread", "-o", str(tmp),
                            str(SRC)],
                           capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("oracle build failed:\n" + r.stderr)
        os.replace(tmp, SO)
    return str(SO)


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        vp, u32, u64, i32, i64 = C.c_void_p, C.c_uint32, C.c_uint64, C.c_int, C.c_int64
        lib.orc_degree_order.restype = i32
        lib.orc_degree_order.argtypes = [u32, vp, vp, vp]
        lib.orc_bfs.restype = i32
        lib.orc_bfs.argtypes = [u32, vp, vp, u32, vp]
        lib.orc_build.restype = vp
        lib.orc_build.argtypes = [u32, vp, vp, vp, u32, C.POINTER(C.c_int)]
        lib.orc_build_ex.restype = vp
        lib.orc_build_ex.argtypes = [u32, vp, vp, vp, u32, i32, C.POINTER(C.c_int)]
        lib.orc_free.restype = None
        lib.orc_free.argtypes = [vp]
        lib.orc_query.restype = i32
        lib.orc_query.argtypes = [vp, u32, u32]
        lib.orc_query_batch.restype = i32
        lib.orc_query_batch.argtypes = [vp, u64, vp, vp, vp]
        lib.orc_query_batch_mt.restype = i32
        lib.orc_query_batch_mt.argtypes = [vp, u64, vp, vp, vp, u32]
        lib.orc_total_entries.restype = u64
        lib.orc_total_entries.argtypes = [vp]
        lib.orc_export_labels.restype = None
        lib.orc_export_labels.argtypes = [vp, vp, vp, vp]
        lib.orc_export_bp.restype = None
        lib.orc_export_bp.argtypes = [vp, vp, vp, vp]
        lib.orc_export_bp_roots.restype = None
        lib.orc_export_bp_roots.argtypes = [vp, vp, vp, vp]
        lib.orc_export_parents.restype = None
        lib.orc_export_parents.argtypes = [vp, vp]
        lib.orc_path.restype = C.c_long
        lib.orc_path.argtypes = [vp, vp, vp, u32, u32, vp]
        lib.orc_build_directed.restype = vp
        lib.orc_build_directed.argtypes = [u32, vp, vp, vp, C.POINTER(C.c_int)]
        lib.orc_dfree.restype = None
        lib.orc_dfree.argtypes = [vp]
        lib.orc_dquery.restype = i32
        lib.orc_dquery.argtypes = [vp, u32, u32]
        lib.orc_dquery_batch.restype = i32
        lib.orc_dquery_batch.argtypes = [vp, u64, vp, vp, vp]
        lib.orc_dtotal.restype = u64
        lib.orc_dtotal.argtypes = [vp, i32]
        lib.orc_dexport.restype = None
        lib.orc_dexport.argtypes = [vp, i32, vp, vp, vp]
        lib.orc_dexport_order.restype = None
        lib.orc_dexport_order.argtypes = [vp, vp]
        lib.orc_export_order.restype = None
        lib.orc_export_order.argtypes = [vp, vp]
        lib.orc_counters.restype = None
        lib.orc_counters.argtypes = [vp, vp]
        lib.orc_label_of.restype = i64
        lib.orc_label_of.argtypes = [u32, vp, vp, vp, vp, u32, vp, vp]
        lib.orc_core_numbers.restype = i32
        lib.orc_core_numbers.argtypes = [u32, vp, vp, vp]
        lib.orc_export_rank_inX.restype = None
        lib.orc_export_rank_inX.argtypes = [vp, vp, vp]
        _lib = lib
    return _lib


def _u32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint32))


class OracleError(RuntimeError):
    def __init__(self, code, what=""):
        super().__init__(f"oracle status {code} {what}")
        self.code = code


def degree_order(offsets, cols) -> np.ndarray:
    off, col = _u32(offsets), _u32(cols)
    n = off.shape[0] - 1
    out = np.empty(max(n, 1), dtype=np.uint32)
    st = _load().orc_degree_order(n, off.ctypes.data, col.ctypes.data, out.ctypes.data)
    if st:
        raise OracleError(st, "degree_order")
    return out[:n]


def core_numbers(offsets, cols) -> np.ndarray:
    """Core number of every vertex (bucket peeling, see oracle.c)."""
    off, col = _u32(offsets), _u32(cols)
    n = off.shape[0] - 1
    out = np.empty(max(n, 1), dtype=np.uint32)
    st = _load().orc_core_numbers(n, off.ctypes.data, col.ctypes.data, out.ctypes.data)
    if st:
        raise OracleError(st, "core_numbers")
    return out[:n]


def bfs(offsets, cols, src: int) -> np.ndarray:
    off, col = _u32(offsets), _u32(cols)
    n = off.shape[0] - 1
    out = np.empty(max(n, 1), dtype=np.uint8)
    st = _load().orc_bfs(n, off.ctypes.data, col.ctypes.data, src, out.ctypes.data)
    if st:
        raise OracleError(st, "bfs")
    return out[:n]


@dataclass
class Labels:
    offsets: np.ndarray  # uint64 [n + 1], by vertex id
    hubs: np.ndarray     # uint32 hub ranks, ascending within a vertex
    dists: np.ndarray    # uint8


class Index:
    """Index built by the oracle (Alg. 3 then Alg. 2/1)."""

    def __init__(self, offsets, cols, t: int, order=None, with_pruned: bool = True):
        self._off, self._col = _u32(offsets), _u32(cols)
        self.n = self._off.shape[0] - 1
        self.t = t
        lib = _load()
        st = C.c_int(0)
        ordp = None
        if order is not None:
            self._ord = _u32(order)
            ordp = self._ord.ctypes.data
        self._h = lib.orc_build_ex(self.n, self._off.ctypes.data, self._col.ctypes.data, ordp, t,
                                   1 if with_pruned else 0, C.byref(st))
        if not self._h:
            raise OracleError(st.value, "build")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            _load().orc_free(h)
            self._h = None

    def query(self, s: int, u: int) -> int:
        d = _load().orc_query(self._h, s, u)
        if d < 0:
            raise OracleError(-d, "query")
        return d

    def query_batch(self, s, u) -> np.ndarray:
        s, u = _u32(s), _u32(u)
        out = np.empty(max(s.shape[0], 1), dtype=np.uint8)
        st = _load().orc_query_batch(self._h, s.shape[0], s.ctypes.data, u.ctypes.data, out.ctypes.data)
        if st:
            raise OracleError(st, "query_batch")
        return out[: s.shape[0]]

    def query_batch_mt(self, s, u, threads: int) -> np.ndarray:
        """query_batch with the pairs split over `threads` host threads."""
        s, u = _u32(s), _u32(u)
        out = np.empty(max(s.shape[0], 1), dtype=np.uint8)
        st = _load().orc_query_batch_mt(self._h, s.shape[0], s.ctypes.data, u.ctypes.data,
                                        out.ctypes.data, threads)
        if st:
            raise OracleError(st, "query_batch_mt")
        return out[: s.shape[0]]

    def labels(self) -> Labels:
        lib = _load()
        tot = lib.orc_total_entries(self._h)
        off = np.empty(self.n + 1, dtype=np.uint64)
        hubs = np.empty(max(tot, 1), dtype=np.uint32)
        dists = np.empty(max(tot, 1), dtype=np.uint8)
        lib.orc_export_labels(self._h, off.ctypes.data, hubs.ctypes.data, dists.ctypes.data)
        return Labels(off, hubs[:tot], dists[:tot])

    def parents(self) -> np.ndarray:
        """Parent of each label entry in its hub's pruned BFS tree (Sec. 6),
        vertex ids, in the layout of labels()."""
        lib = _load()
        tot = lib.orc_total_entries(self._h)
        out = np.empty(max(tot, 1), dtype=np.uint32)
        lib.orc_export_parents(self._h, out.ctypes.data)
        return out[:tot]

    def path(self, s: int, u: int) -> np.ndarray:
        """One shortest s-u path (vertex ids, s first) restored from the
        labels and parents (Sec. 6); empty if u is unreachable."""
        out = np.empty(256, dtype=np.uint32)
        c = _load().orc_path(self._h, self._off.ctypes.data, self._col.ctypes.data, s, u,
                             out.ctypes.data)
        if c < 0:
            raise OracleError(-c, "path")
        return out[:c].copy()

    def bp(self):
        nt = max(self.n * self.t, 1)
        d = np.empty(nt, dtype=np.uint8)
        m1 = np.empty(nt, dtype=np.uint64)
        m0 = np.empty(nt, dtype=np.uint64)
        _load().orc_export_bp(self._h, d.ctypes.data, m1.ctypes.data, m0.ctypes.data)
        k = self.n * self.t
        shp = (self.n, self.t)
        return d[:k].reshape(shp), m1[:k].reshape(shp), m0[:k].reshape(shp)

    def bp_roots(self):
        t = max(self.t, 1)
        roots = np.empty(t, dtype=np.uint32)
        cnt = np.empty(t, dtype=np.uint32)
        S = np.empty(t * BPW, dtype=np.uint32)
        _load().orc_export_bp_roots(self._h, roots.ctypes.data, cnt.ctypes.data, S.ctypes.data)
        return roots[: self.t], cnt[: self.t], S[: self.t * BPW].reshape(self.t, BPW)

    def order(self) -> np.ndarray:
        out = np.empty(max(self.n, 1), dtype=np.uint32)
        _load().orc_export_order(self._h, out.ctypes.data)
        return out[: self.n]

    def rank_inX(self):
        rank = np.empty(max(self.n, 1), dtype=np.uint32)
        inX = np.empty(max(self.n, 1), dtype=np.uint8)
        _load().orc_export_rank_inX(self._h, rank.ctypes.data, inX.ctypes.data)
        return rank[: self.n], inX[: self.n]

    def counters(self) -> dict:
        out = np.zeros(4, dtype=np.uint64)
        _load().orc_counters(self._h, out.ctypes.data)
        return dict(visited=int(out[0]), labeled=int(out[1]), scanned=int(out[2]),
                    labeled_deg=int(out[3]))


class DirectedIndex:
    """Directed-graph index of Sec. 6: L_IN and L_OUT from a forward and a
    reverse pruned BFS per root, no bit-parallel labels. offsets/cols list
    the out-arcs of each vertex."""

    def __init__(self, offsets, cols, order=None):
        self._off, self._col = _u32(offsets), _u32(cols)
        self.n = self._off.shape[0] - 1
        lib = _load()
        st = C.c_int(0)
        ordp = None
        if order is not None:
            self._ord = _u32(order)
            ordp = self._ord.ctypes.data
        self._h = lib.orc_build_directed(self.n, self._off.ctypes.data, self._col.ctypes.data, ordp,
                                         C.byref(st))
        if not self._h:
            raise OracleError(st.value, "build_directed")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            _load().orc_dfree(h)
            self._h = None

    def query(self, s: int, t: int) -> int:
        d = _load().orc_dquery(self._h, s, t)
        if d < 0:
            raise OracleError(-d, "dquery")
        return d

    def query_batch(self, s, t) -> np.ndarray:
        s, t = _u32(s), _u32(t)
        out = np.empty(max(s.shape[0], 1), dtype=np.uint8)
        st = _load().orc_dquery_batch(self._h, s.shape[0], s.ctypes.data, t.ctypes.data, out.ctypes.data)
        if st:
            raise OracleError(st, "dquery_batch")
        return out[: s.shape[0]]

    def _labels(self, which: int) -> Labels:
        lib = _load()
        tot = lib.orc_dtotal(self._h, which)
        off = np.empty(self.n + 1, dtype=np.uint64)
        hubs = np.empty(max(tot, 1), dtype=np.uint32)
        dists = np.empty(max(tot, 1), dtype=np.uint8)
        lib.orc_dexport(self._h, which, off.ctypes.data, hubs.ctypes.data, dists.ctypes.data)
        return Labels(off, hubs[:tot], dists[:tot])

    def labels_in(self) -> Labels:
        """L_IN(v): (hub rank, d(hub, v))."""
        return self._labels(0)

    def labels_out(self) -> Labels:
        """L_OUT(v): (hub rank, d(v, hub))."""
        return self._labels(1)

    def order(self) -> np.ndarray:
        out = np.empty(max(self.n, 1), dtype=np.uint32)
        _load().orc_dexport_order(self._h, out.ctypes.data)
        return out[: self.n]


def label_of(offsets, cols, rank, inX, u: int):
    """Closed-form L(u) for the order given by `rank` and bit-parallel set `inX`:
    returns (hub ranks ascending, distances)."""
    off, col = _u32(offsets), _u32(cols)
    n = off.shape[0] - 1
    rank = _u32(rank)
    inX = np.ascontiguousarray(np.asarray(inX, dtype=np.uint8))
    hubs = np.empty(max(n, 1), dtype=np.uint32)
    dists = np.empty(max(n, 1), dtype=np.uint8)
    c = _load().orc_label_of(n, off.ctypes.data, col.ctypes.data, rank.ctypes.data, inX.ctypes.data,
                             u, hubs.ctypes.data, dists.ctypes.data)
    if c < 0:
        raise OracleError(-c, "label_of")
    return hubs[:c].copy(), dists[:c].copy()
