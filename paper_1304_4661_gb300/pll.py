"""ctypes binding of libpll.so (include/pll.h) -- argument marshalling only.

Every step of the index build and of the queries runs in the library's CUDA
kernels. Device arguments are torch CUDA tensors (their data pointers and
the current CUDA stream are passed through); host arguments are numpy arrays
and go to the ``*_host`` entry points, which copy inside the call. There is
no CPU fallback: if the library cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
import weakref
from dataclasses import dataclass

import numpy as np

from . import _build

PLL_OK, PLL_E_INVAL, PLL_E_ORDER, PLL_E_RANGE, PLL_E_NOMEM, PLL_E_TIMEOUT, PLL_E_CUDA = range(7)
PLL_MAX_T = 64
NONE = 0xFFFFFFFF

SYMBOLS = [
    "pll_build", "pll_build_host", "pll_query", "pll_query_async", "pll_query_errors",
    "pll_query_host", "pll_label_entries", "pll_export_labels", "pll_export_bp",
    "pll_export_bp_roots", "pll_export_order", "pll_get_stats", "pll_free", "pll_status_str",
    "pll_bp_labels_noalloc", "pll_build_batch", "pll_autotune",
    "pll_server_start", "pll_server_submit", "pll_server_wait", "pll_server_replay",
    "pll_server_get_stats", "pll_server_stop",
    "pll_features", "pll_hub_counts", "pll_order_from_scores", "pll_mlp_create", "pll_mlp_free",
    "pll_mlp_set_params", "pll_mlp_get_params", "pll_mlp_forward", "pll_mlp_grad",
    "pll_mlp_read_grad", "pll_mlp_adam", "pll_mlp_train_step", "pll_learned_order",
    "pll_save", "pll_load", "pll_test_fail_alloc", "pll_test_live_allocs", "pll_test_capacities",
    "pll_test_barrier_timeout", "pll_release_cached",
    "pll_paths_create", "pll_paths_parents", "pll_path_offsets", "pll_path_query",
    "pll_paths_free",
    "pll_build_directed", "pll_dquery", "pll_dlabel_entries", "pll_dexport_labels",
    "pll_dexport_order", "pll_dfree",
]
MLP_NPARAM = 4801
PLL_NOALLOC_SCRATCH_BYTES = 64 << 20


# pll_build_opts.flags: how each root batch's levels run
PLL_BUILD_HOST_LEVELS = 1   # separate launches enqueued by the host
PLL_BUILD_GRAPH_LEVELS = 2  # one CUDA graph launch with a while node (the default)
PLL_BUILD_COOP_LEVELS = 4   # one cooperative persistent launch


class BuildOpts(C.Structure):
    _fields_ = [("t", C.c_uint32), ("root_batch", C.c_uint32), ("block", C.c_uint32),
                ("flags", C.c_uint32), ("reserved", C.c_uint64)]


class Stats(C.Structure):
    _fields_ = [("n", C.c_uint32), ("t", C.c_uint32), ("nnz", C.c_uint64),
                ("label_entries", C.c_uint64), ("pre_cleanup", C.c_uint64),
                ("visited", C.c_uint64), ("batches", C.c_uint64), ("index_bytes", C.c_uint64),
                ("ms_prep", C.c_double), ("ms_bp", C.c_double), ("ms_pruned", C.c_double),
                ("ms_finalize", C.c_double), ("ms_pruned_kernel", C.c_double),
                ("pruned_launches", C.c_uint64), ("pruned_scanned", C.c_uint64),
                ("pruned_masks", C.c_uint64), ("pruned_expanded", C.c_uint64),
                ("launches", C.c_uint64), ("cub_calls", C.c_uint64),
                ("ms_expand", C.c_double), ("ms_test", C.c_double),
                ("expand_launches", C.c_uint64), ("test_launches", C.c_uint64),
                ("candidates", C.c_uint64), ("graphs", C.c_uint32), ("reserved32", C.c_uint32),
                ("redone_batches", C.c_uint64), ("pool_regrows", C.c_uint64),
                ("table_fallbacks", C.c_uint64), ("levels_launches", C.c_uint64),
                ("ms_levels", C.c_double), ("ms_post", C.c_double),
                ("scratch_peak_bytes", C.c_uint64)]


class ServerOpts(C.Structure):
    _fields_ = [("pool_bytes", C.c_uint64), ("max_batch_pairs", C.c_uint64),
                ("streams", C.c_uint32), ("reserved", C.c_uint32)]


class ServerStats(C.Structure):
    _fields_ = [("requests", C.c_uint64), ("pairs", C.c_uint64), ("batches", C.c_uint64),
                ("max_batch_pairs", C.c_uint64), ("max_inflight_bytes", C.c_uint64),
                ("pool_bytes", C.c_uint64), ("max_request_pairs", C.c_uint64),
                ("pack_us", C.c_double), ("unpack_us", C.c_double), ("device_us", C.c_double)]


class PLLError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {status_str(code)} (status {code})")
        self.code = code


_lib = None


def lib_path() -> str:
    return str(_build.OUT / "libpll.so")


def load(build_if_missing: bool = True):
    """Load libpll.so (building it in-tree with nvcc when absent or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if build_if_missing:
        path = _build.build_pll()
    if not os.path.exists(path):
        raise RuntimeError(f"libpll.so not found at {path}; run __graft_entry__.build()")
    lib = C.CDLL(path)
    vp, u32, u64, i32 = C.c_void_p, C.c_uint32, C.c_uint64, C.c_int
    pp = C.POINTER(C.c_void_p)
    for name in ("pll_build", "pll_build_host"):
        f = getattr(lib, name)
        f.restype = i32
        f.argtypes = [vp, vp, u32, u64, vp, C.POINTER(BuildOpts), vp, pp]
    for name in ("pll_query", "pll_query_async", "pll_query_host"):
        f = getattr(lib, name)
        f.restype = i32
        f.argtypes = [vp, vp, vp, u64, vp, vp]
    lib.pll_query_errors.restype = i32
    lib.pll_query_errors.argtypes = [vp, vp, C.POINTER(C.c_uint64)]
    lib.pll_label_entries.restype = i32
    lib.pll_label_entries.argtypes = [vp, C.POINTER(C.c_uint64)]
    lib.pll_export_labels.restype = i32
    lib.pll_export_labels.argtypes = [vp, vp, vp, vp]
    lib.pll_export_bp.restype = i32
    lib.pll_export_bp.argtypes = [vp, vp, vp, vp]
    lib.pll_export_bp_roots.restype = i32
    lib.pll_export_bp_roots.argtypes = [vp, vp, vp, vp]
    lib.pll_export_order.restype = i32
    lib.pll_export_order.argtypes = [vp, vp]
    lib.pll_get_stats.restype = i32
    lib.pll_get_stats.argtypes = [vp, C.POINTER(Stats)]
    lib.pll_free.restype = None
    lib.pll_free.argtypes = [vp]
    lib.pll_status_str.restype = C.c_char_p
    lib.pll_status_str.argtypes = [i32]
    lib.pll_autotune.restype = i32
    lib.pll_autotune.argtypes = [vp, vp, u32, u64, vp, u32, u32, vp, C.POINTER(BuildOpts),
                                 C.POINTER(C.c_double)]
    lib.pll_build_batch.restype = i32
    lib.pll_build_batch.argtypes = [vp, vp, u32, u64, vp, u32, C.POINTER(BuildOpts), vp, pp]
    lib.pll_bp_labels_noalloc.restype = i32
    lib.pll_bp_labels_noalloc.argtypes = [vp, vp, u32, u64, u32, vp, vp, vp, vp, vp, vp]
    dp = C.POINTER(C.c_double)
    lib.pll_server_start.restype = i32
    lib.pll_server_start.argtypes = [vp, C.POINTER(ServerOpts), pp]
    lib.pll_server_submit.restype = i32
    lib.pll_server_submit.argtypes = [vp, vp, vp, u64, vp, C.POINTER(C.c_uint64)]
    lib.pll_server_wait.restype = i32
    lib.pll_server_wait.argtypes = [vp, u64, C.c_int64, dp]
    lib.pll_server_replay.restype = i32
    lib.pll_server_replay.argtypes = [vp, vp, vp, vp, vp, u64, u32, vp, vp, dp]
    lib.pll_server_get_stats.restype = i32
    lib.pll_server_get_stats.argtypes = [vp, C.POINTER(ServerStats)]
    lib.pll_server_stop.restype = i32
    lib.pll_server_stop.argtypes = [vp]
    fp = C.c_float
    for name, args in (("pll_features", [vp, vp, u32, u64, u32, vp, vp, vp, vp]),
                       ("pll_hub_counts", [vp, vp, vp, vp]),
                       ("pll_order_from_scores", [vp, u32, vp, vp]),
                       ("pll_mlp_create", [u32, pp]),
                       ("pll_mlp_set_params", [vp, vp, vp]),
                       ("pll_mlp_get_params", [vp, vp, vp]),
                       ("pll_mlp_forward", [vp, vp, u64, vp, vp]),
                       ("pll_mlp_grad", [vp, vp, vp, vp, u32, vp]),
                       ("pll_mlp_read_grad", [vp, vp, vp, vp]),
                       ("pll_mlp_adam", [vp, fp, vp]),
                       ("pll_mlp_train_step", [vp, vp, vp, vp, u32, fp, vp]),
                       ("pll_learned_order", [vp, vp, u32, u64, u32, vp, vp, vp])):
        f = getattr(lib, name)
        f.restype = i32
        f.argtypes = args
    lib.pll_mlp_free.restype = None
    lib.pll_mlp_free.argtypes = [vp]
    lib.pll_save.restype = i32
    lib.pll_save.argtypes = [vp, C.c_char_p]
    lib.pll_load.restype = i32
    lib.pll_load.argtypes = [C.c_char_p, pp]
    lib.pll_paths_create.restype = i32
    lib.pll_paths_create.argtypes = [vp, vp, vp, u32, u64, vp, pp]
    lib.pll_paths_parents.restype = i32
    lib.pll_paths_parents.argtypes = [vp, vp]
    lib.pll_path_offsets.restype = i32
    lib.pll_path_offsets.argtypes = [vp, vp, vp, u64, vp, C.POINTER(C.c_uint64), vp]
    lib.pll_path_query.restype = i32
    lib.pll_path_query.argtypes = [vp, vp, vp, u64, vp, u64, vp, vp]
    lib.pll_paths_free.restype = None
    lib.pll_paths_free.argtypes = [vp]
    lib.pll_build_directed.restype = i32
    lib.pll_build_directed.argtypes = [vp, vp, u32, u64, vp, C.POINTER(BuildOpts), vp, pp]
    lib.pll_dquery.restype = i32
    lib.pll_dquery.argtypes = [vp, vp, vp, u64, vp, vp]
    lib.pll_dlabel_entries.restype = i32
    lib.pll_dlabel_entries.argtypes = [vp, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)]
    lib.pll_dexport_labels.restype = i32
    lib.pll_dexport_labels.argtypes = [vp, i32, vp, vp, vp]
    lib.pll_dexport_order.restype = i32
    lib.pll_dexport_order.argtypes = [vp, vp]
    lib.pll_dfree.restype = None
    lib.pll_dfree.argtypes = [vp]
    lib.pll_test_fail_alloc.restype = None
    lib.pll_test_fail_alloc.argtypes = [C.c_int64]
    lib.pll_test_live_allocs.restype = C.c_int64
    lib.pll_test_live_allocs.argtypes = []
    lib.pll_test_capacities.restype = None
    lib.pll_test_capacities.argtypes = [C.c_uint64] * 4
    lib.pll_test_barrier_timeout.restype = None
    lib.pll_test_barrier_timeout.argtypes = [C.c_uint64]
    lib.pll_release_cached.restype = i32
    lib.pll_release_cached.argtypes = []
    _lib = lib
    return lib


def release_cached():
    """pll_release_cached: hand the current context's cached scratch memory
    back to the driver (synchronises the current device)."""
    _check(load().pll_release_cached(), "pll_release_cached")


def status_str(code: int) -> str:
    return load().pll_status_str(code).decode()


def _check(code: int, where: str):
    if code != PLL_OK:
        raise PLLError(code, where)


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _stream_handle(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _dptr(x):
    assert x.is_cuda and x.is_contiguous(), "device arguments must be contiguous CUDA tensors"
    return x.data_ptr()


def _hptr(a, dtype):
    a = np.ascontiguousarray(np.asarray(a, dtype=dtype))
    return a, a.ctypes.data


def autotune(offsets, cols, t: int, graph_start=None, stream=None):
    """pll_autotune on CUDA tensors; returns (root_batch, block, build_ms)."""
    lib = load()
    n = int(offsets.shape[0]) - 1
    nnz = int(cols.shape[0])
    gp, G = None, 0
    if graph_start is not None:
        gs, gp = _hptr(graph_start, np.uint32)
        G = len(gs) - 1
    best = BuildOpts()
    ms = C.c_double(0)
    _check(lib.pll_autotune(_dptr(offsets), _dptr(cols) if nnz else None, n, nnz, gp, G, t,
                            _stream_handle(stream), C.byref(best), C.byref(ms)), "pll_autotune")
    return int(best.root_batch), int(best.block), float(ms.value)


def bp_labels_noalloc(rank_offsets, rank_cols, t: int, d, masks, roots, cnt, S, stream=None):
    """pll_bp_labels_noalloc on CUDA tensors (outputs preallocated by the caller):
    d uint8[n * tp] (tp = t rounded up to 16), masks uint64[n * t * 2],
    roots/cnt uint32[t], S uint32[t * 64]; ids are ranks."""
    import torch
    n = int(rank_offsets.shape[0]) - 1
    nnz = int(rank_cols.shape[0])
    tp = (t + 15) // 16 * 16
    # the library writes exactly these sizes: refuse anything else before the call
    want = [("rank_offsets", rank_offsets, (torch.int32, torch.uint32), n + 1),
            ("rank_cols", rank_cols, (torch.int32, torch.uint32), nnz),
            ("d", d, (torch.uint8,), n * tp),
            ("masks", masks, (torch.int64, torch.uint64), 2 * n * t),
            ("roots", roots, (torch.int32, torch.uint32), t),
            ("cnt", cnt, (torch.int32, torch.uint32), t),
            ("S", S, (torch.int32, torch.uint32), 64 * t)]
    for name, x, dtypes, numel in want:
        if not _is_torch(x):
            raise ValueError(f"{name}: a torch tensor is required")
        if x.dtype not in dtypes:
            raise ValueError(f"{name}: dtype {x.dtype}, expected one of {dtypes}")
        if x.numel() != numel:
            raise ValueError(f"{name}: {x.numel()} elements, expected {numel}")
    for name, x, _, _ in want:
        if not (x.is_cuda and x.is_contiguous()):
            raise ValueError(f"{name}: a contiguous CUDA tensor is required")
    dev = torch.cuda.current_device()
    for name, x, _, _ in want:
        if x.device.index != dev:
            raise ValueError(f"{name}: on cuda:{x.device.index}, the current device is cuda:{dev}")
    _check(load().pll_bp_labels_noalloc(_dptr(rank_offsets), _dptr(rank_cols) if nnz else None, n,
                                        nnz, t, _dptr(d), _dptr(masks), _dptr(roots), _dptr(cnt),
                                        _dptr(S), _stream_handle(stream)), "pll_bp_labels_noalloc")


@dataclass
class Labels:
    offsets: np.ndarray  # uint64 [n + 1], by vertex id
    hubs: np.ndarray     # uint32 hub ranks
    dists: np.ndarray    # uint8


class Index:
    """A PLL index resident on the current CUDA device."""

    def __init__(self, handle: int, n: int, t: int):
        self._h = handle
        self.n = n
        self.t = t
        self.graphs = 1
        self._users = weakref.WeakSet()  # Server / Paths objects that borrow the index

    def _lend(self, user):
        self._users.add(user)

    # ------------------------------------------------------------- build
    @classmethod
    def build(cls, offsets, cols, t: int = 0, order=None, root_batch: int = 0, block: int = 0,
              stream=None, flags: int = 0) -> "Index":
        """pll_build (CUDA tensors) or pll_build_host (numpy arrays)."""
        lib = load()
        opts = BuildOpts(t, root_batch, block, flags, 0)
        out = C.c_void_p()
        n = int(offsets.shape[0]) - 1
        nnz = int(cols.shape[0])
        if _is_torch(offsets):
            import torch
            assert offsets.dtype == torch.int32 or offsets.dtype == torch.uint32
            optr = _dptr(order) if order is not None else None
            st = lib.pll_build(_dptr(offsets), _dptr(cols) if nnz else None, n, nnz, optr,
                               C.byref(opts), _stream_handle(stream), C.byref(out))
        else:
            off, op = _hptr(offsets, np.uint32)
            col, cp = _hptr(cols, np.uint32)
            ordp = None
            if order is not None:
                order_a, ordp = _hptr(order, np.uint32)
            st = lib.pll_build_host(op, cp if nnz else None, n, nnz, ordp, C.byref(opts),
                                    _stream_handle(stream) if stream is not None else None,
                                    C.byref(out))
        _check(st, "pll_build")
        return cls(out.value, n, t)

    @classmethod
    def build_batch(cls, offsets, cols, graph_start, t: int = 0, root_batch: int = 0,
                    block: int = 0, stream=None, flags: int = 0) -> "Index":
        """pll_build_batch: CUDA tensors for the union CSR, graph_start as a
        host uint32 array of graphs + 1 vertex boundaries."""
        lib = load()
        opts = BuildOpts(t, root_batch, block, flags, 0)
        out = C.c_void_p()
        n = int(offsets.shape[0]) - 1
        nnz = int(cols.shape[0])
        gs, gp = _hptr(graph_start, np.uint32)
        st = lib.pll_build_batch(_dptr(offsets), _dptr(cols) if nnz else None, n, nnz, gp,
                                 len(gs) - 1, C.byref(opts), _stream_handle(stream), C.byref(out))
        _check(st, "pll_build_batch")
        ix = cls(out.value, n, t)
        ix.graphs = len(gs) - 1
        return ix

    def close(self):
        """pll_free. Refused while a Server or Paths object built on this
        index is still open (they borrow its device arrays)."""
        if getattr(self, "_h", None):
            if any(getattr(u, "_h", None) for u in getattr(self, "_users", ())):
                raise RuntimeError("stop the Server / close the Paths objects of this index first")
            load().pll_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------- query
    def query(self, src, dst, out=None, stream=None):
        """Distances for pairs (src[i], dst[i]); CUDA tensors in -> CUDA uint8
        tensor out (synchronous), numpy in -> numpy out (pll_query_host)."""
        lib = load()
        q = int(src.shape[0])
        if _is_torch(src):
            import torch
            if out is None:
                out = torch.empty(q, dtype=torch.uint8, device=src.device)
            if q:
                _check(lib.pll_query(self._h, _dptr(src), _dptr(dst), q, _dptr(out),
                                     _stream_handle(stream)), "pll_query")
            return out
        s, sp = _hptr(src, np.uint32)
        d, dp = _hptr(dst, np.uint32)
        res = np.empty(max(q, 1), dtype=np.uint8)
        if q:
            _check(lib.pll_query_host(self._h, sp, dp, q, res.ctypes.data,
                                      _stream_handle(stream) if stream is not None else None),
                   "pll_query_host")
        return res[:q]

    def query_async(self, src, dst, out, stream=None):
        q = int(src.shape[0])
        if q:
            _check(load().pll_query_async(self._h, _dptr(src), _dptr(dst), q, _dptr(out),
                                          _stream_handle(stream)), "pll_query_async")
        return out

    def query_errors(self, stream=None) -> int:
        c = C.c_uint64(0)
        _check(load().pll_query_errors(self._h, _stream_handle(stream), C.byref(c)), "pll_query_errors")
        return int(c.value)

    # ------------------------------------------------------------ exports
    def label_entries(self) -> int:
        c = C.c_uint64(0)
        _check(load().pll_label_entries(self._h, C.byref(c)), "pll_label_entries")
        return int(c.value)

    def save(self, path):
        """pll_save: write the index to a file."""
        _check(load().pll_save(self._h, os.fsencode(path)), "pll_save")

    @classmethod
    def load(cls, path):
        """pll_load: read an index written by save() onto the current device."""
        h = C.c_void_p()
        _check(load().pll_load(os.fsencode(path), C.byref(h)), "pll_load")
        st = Stats()
        _check(load().pll_get_stats(h.value, C.byref(st)), "pll_get_stats")
        ix = cls(h.value, int(st.n), int(st.t))
        ix.graphs = max(int(st.graphs), 1)
        return ix

    def hub_counts(self, stream=None):
        """pll_hub_counts: (counts int32 CUDA [n], log1p(counts) float32 CUDA [n])."""
        import torch
        n = max(self.n, 1)
        c = torch.empty(n, dtype=torch.int32, device="cuda")
        f = torch.empty(n, dtype=torch.float32, device="cuda")
        _check(load().pll_hub_counts(self._h, _dptr(c), _dptr(f), _stream_handle(stream)),
               "pll_hub_counts")
        return c[: self.n], f[: self.n]

    def labels(self) -> Labels:
        tot = self.label_entries()
        off = np.empty(self.n + 1, dtype=np.uint64)
        hubs = np.empty(max(tot, 1), dtype=np.uint32)
        dists = np.empty(max(tot, 1), dtype=np.uint8)
        _check(load().pll_export_labels(self._h, off.ctypes.data, hubs.ctypes.data, dists.ctypes.data),
               "pll_export_labels")
        return Labels(off, hubs[:tot], dists[:tot])

    def bp(self):
        nt = max(self.n * self.t, 1)
        d = np.empty(nt, dtype=np.uint8)
        m1 = np.empty(nt, dtype=np.uint64)
        m0 = np.empty(nt, dtype=np.uint64)
        _check(load().pll_export_bp(self._h, d.ctypes.data, m1.ctypes.data, m0.ctypes.data), "pll_export_bp")
        k, shp = self.n * self.t, (self.n, self.t)
        return d[:k].reshape(shp), m1[:k].reshape(shp), m0[:k].reshape(shp)

    def bp_roots(self):
        """roots, cnt [graphs * t] and S [graphs * t, 64] (graph-major)."""
        gt = self.graphs * self.t
        roots = np.empty(max(gt, 1), dtype=np.uint32)
        cnt = np.empty(max(gt, 1), dtype=np.uint32)
        S = np.empty(max(gt, 1) * 64, dtype=np.uint32)
        _check(load().pll_export_bp_roots(self._h, roots.ctypes.data, cnt.ctypes.data, S.ctypes.data),
               "pll_export_bp_roots")
        return roots[:gt], cnt[:gt], S[: gt * 64].reshape(gt, 64)

    def order(self) -> np.ndarray:
        out = np.empty(max(self.n, 1), dtype=np.uint32)
        _check(load().pll_export_order(self._h, out.ctypes.data), "pll_export_order")
        return out[: self.n]

    def stats(self) -> dict:
        s = Stats()
        _check(load().pll_get_stats(self._h, C.byref(s)), "pll_get_stats")
        return {f: getattr(s, f) for f, _ in Stats._fields_}


class DirectedIndex:
    """pll_build_directed / pll_dquery: a directed-graph index (Sec. 6) on
    the current CUDA device. offsets/cols are CUDA tensors of the
    out-neighbour CSR."""

    def __init__(self, offsets, cols, order=None, root_batch: int = 0, stream=None):
        self._lib = load()
        self.n = int(offsets.shape[0]) - 1
        nnz = int(cols.shape[0])
        opts = BuildOpts(0, root_batch, 0, 0, 0)
        h = C.c_void_p()
        _check(self._lib.pll_build_directed(_dptr(offsets), _dptr(cols) if nnz else None, self.n, nnz,
                                            _dptr(order) if order is not None else None, C.byref(opts),
                                            _stream_handle(stream), C.byref(h)), "pll_build_directed")
        self._h = h.value

    def query(self, src, dst, stream=None):
        """d(src[i], dst[i]) along arcs: CUDA uint8 tensor (synchronous)."""
        import torch
        q = int(src.shape[0])
        out = torch.empty(q, dtype=torch.uint8, device=src.device)
        if q:
            _check(self._lib.pll_dquery(self._h, _dptr(src), _dptr(dst), q, _dptr(out),
                                        _stream_handle(stream)), "pll_dquery")
        return out

    def entries(self):
        a, b = C.c_uint64(0), C.c_uint64(0)
        _check(self._lib.pll_dlabel_entries(self._h, C.byref(a), C.byref(b)), "pll_dlabel_entries")
        return int(a.value), int(b.value)

    def _labels(self, which: int) -> Labels:
        tot = self.entries()[which]
        off = np.empty(self.n + 1, dtype=np.uint64)
        hubs = np.empty(max(tot, 1), dtype=np.uint32)
        dists = np.empty(max(tot, 1), dtype=np.uint8)
        _check(self._lib.pll_dexport_labels(self._h, which, off.ctypes.data, hubs.ctypes.data,
                                            dists.ctypes.data), "pll_dexport_labels")
        return Labels(off, hubs[:tot], dists[:tot])

    def labels_in(self) -> Labels:
        return self._labels(0)

    def labels_out(self) -> Labels:
        return self._labels(1)

    def order(self) -> np.ndarray:
        out = np.empty(max(self.n, 1), dtype=np.uint32)
        _check(self._lib.pll_dexport_order(self._h, out.ctypes.data), "pll_dexport_order")
        return out[: self.n]

    def close(self):
        if getattr(self, "_h", None):
            self._lib.pll_dfree(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Paths:
    """pll_paths_*: shortest-path queries (Sec. 6) over an Index built from
    the graph given here (CUDA tensors, as for Index.build)."""

    def __init__(self, index: "Index", offsets, cols, stream=None):
        self._lib = load()
        self.index = index  # the paths object borrows the index
        n = int(offsets.shape[0]) - 1
        nnz = int(cols.shape[0])
        h = C.c_void_p()
        _check(self._lib.pll_paths_create(index._h, _dptr(offsets), _dptr(cols) if nnz else None, n,
                                          nnz, _stream_handle(stream), C.byref(h)), "pll_paths_create")
        self._h = h.value
        index._lend(self)

    def _live(self):
        # the C object borrows the index's device arrays
        if not getattr(self.index, "_h", None) or not getattr(self, "_h", None):
            raise RuntimeError("Paths used after its Index (or itself) was closed")

    def parents(self) -> np.ndarray:
        """Parent (caller id) of every label entry, in the layout of Index.labels()."""
        self._live()
        tot = self.index.label_entries()
        out = np.empty(max(tot, 1), dtype=np.uint32)
        _check(self._lib.pll_paths_parents(self._h, out.ctypes.data), "pll_paths_parents")
        return out[:tot]

    def offsets(self, src, dst, stream=None):
        """pll_path_offsets: (path_off int64 CUDA [q + 1], total)."""
        import torch
        self._live()
        q = int(src.shape[0])
        off = torch.empty(q + 1, dtype=torch.int64, device=src.device)
        tot = C.c_uint64(0)
        _check(self._lib.pll_path_offsets(self._h, _dptr(src) if q else None, _dptr(dst) if q else None,
                                          q, _dptr(off), C.byref(tot), _stream_handle(stream)),
               "pll_path_offsets")
        return off, int(tot.value)

    def query(self, src, dst, path_off=None, cap=None, stream=None):
        """pll_path_query on CUDA tensors: returns (path_off, path), pair i's
        path (caller ids) in path[path_off[i]:path_off[i + 1]]. Without
        path_off the slots come from offsets()."""
        import torch
        self._live()
        q = int(src.shape[0])
        if path_off is None:
            path_off, cap = self.offsets(src, dst, stream)
        elif cap is None:
            cap = int(path_off[-1].item()) if q else 0
        path = torch.empty(max(cap, 1), dtype=torch.int32, device=src.device)
        if q:
            _check(self._lib.pll_path_query(self._h, _dptr(src), _dptr(dst), q, _dptr(path_off), cap,
                                            _dptr(path), _stream_handle(stream)), "pll_path_query")
        return path_off, path[:cap]

    def paths(self, src, dst, stream=None):
        """Host list of numpy uint32 paths, one per pair."""
        off, path = self.query(src, dst, stream=stream)
        off = off.cpu().numpy()
        p = path.cpu().numpy().view(np.uint32)
        return [p[off[i]:off[i + 1]] for i in range(len(off) - 1)]

    def close(self):
        if getattr(self, "_h", None):
            self._lib.pll_paths_free(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """pll_server_*: continuous-batching query service over a resident Index.

    Requests are host numpy arrays; the server keeps references to them until
    they are waited for, so callers may drop their own."""

    def __init__(self, index: "Index", pool_bytes: int = 0, max_batch_pairs: int = 0,
                 streams: int = 0):
        self._lib = load()
        self.index = index  # keeps the index alive while the server runs
        o = ServerOpts(pool_bytes, max_batch_pairs, streams, 0)
        h = C.c_void_p()
        _check(self._lib.pll_server_start(index._h, C.byref(o), C.byref(h)), "pll_server_start")
        self._h = h.value
        self._live = {}
        index._lend(self)

    def submit(self, src, dst) -> int:
        s, sp = _hptr(src, np.uint32)
        d, dp = _hptr(dst, np.uint32)
        assert s.shape == d.shape and s.ndim == 1
        out = np.empty(max(len(s), 1), dtype=np.uint8)
        tk = C.c_uint64(0)
        _check(self._lib.pll_server_submit(self._h, sp, dp, len(s), out.ctypes.data,
                                           C.byref(tk)), "pll_server_submit")
        self._live[tk.value] = (s, out)  # the server writes `out` until waited for
        return tk.value

    def wait(self, ticket: int, timeout_us: int = -1):
        """Returns (distances, latency_us) of a submitted request."""
        lat = C.c_double(0)
        code = self._lib.pll_server_wait(self._h, ticket, timeout_us, C.byref(lat))
        if code == PLL_E_TIMEOUT:
            raise TimeoutError(f"request {ticket} not done after {timeout_us} us")
        s, out = self._live.pop(ticket)
        _check(code, "pll_server_wait")
        return out[: len(s)], float(lat.value)

    def replay(self, src, dst, req_off, arrival_us, threads: int = 4):
        """Open-loop replay by `threads` client threads; returns
        (out uint8[total], latency_us[count], elapsed_us)."""
        s, sp = _hptr(src, np.uint32)
        d, dp = _hptr(dst, np.uint32)
        off, op = _hptr(req_off, np.uint64)
        arr, ap = _hptr(arrival_us, np.float64)
        count = len(off) - 1
        assert len(arr) == count and int(off[-1]) == len(s) == len(d)
        out = np.empty(max(len(s), 1), dtype=np.uint8)
        lat = np.empty(max(count, 1), dtype=np.float64)
        el = C.c_double(0)
        _check(self._lib.pll_server_replay(self._h, sp, dp, op, ap, count, threads, out.ctypes.data,
                                           lat.ctypes.data, C.byref(el)), "pll_server_replay")
        return out[: len(s)], lat[:count], float(el.value)

    def stats(self) -> dict:
        st = ServerStats()
        _check(self._lib.pll_server_get_stats(self._h, C.byref(st)), "pll_server_get_stats")
        return {f: (round(getattr(st, f), 1) if t is C.c_double else int(getattr(st, f)))
                for f, t in ServerStats._fields_}

    def stop(self):
        if getattr(self, "_h", None):
            h, self._h = self._h, None
            code = self._lib.pll_server_stop(h)
            self._live.clear()
            _check(code, "pll_server_stop")

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.stop()

    def __del__(self):
        try:
            self.stop()
        except Exception:
            pass


# ------------------------------------------------------------ learned order
def features(offsets, cols, t: int, out=None, raw: bool = False, stream=None):
    """pll_features on CUDA tensors: float32 [n, 8] standardised features
    (written into `out` if given); with raw=True also (core uint32, two_hop
    uint64) as int tensors."""
    import torch
    n = int(offsets.shape[0]) - 1
    nnz = int(cols.shape[0])
    if out is None:
        out = torch.empty((max(n, 0), 8), dtype=torch.float32, device=offsets.device)
    core = two = None
    if raw:
        core = torch.empty(max(n, 1), dtype=torch.int32, device=offsets.device)
        two = torch.empty(max(n, 1), dtype=torch.int64, device=offsets.device)
    _check(load().pll_features(_dptr(offsets), _dptr(cols) if nnz else None, n, nnz, t,
                               _stream_handle(stream), _dptr(out) if n else None,
                               _dptr(core) if raw else None, _dptr(two) if raw else None),
           "pll_features")
    return (out, core[:n], two[:n]) if raw else out


def order_from_scores(scores, stream=None):
    """pll_order_from_scores: CUDA float32 scores -> CUDA int32 order."""
    import torch
    n = int(scores.shape[0])
    order = torch.empty(max(n, 1), dtype=torch.int32, device=scores.device)
    _check(load().pll_order_from_scores(_dptr(scores) if n else None, n, _dptr(order),
                                        _stream_handle(stream)), "pll_order_from_scores")
    return order[:n]


class MLP:
    """pll_mlp: the vertex-scoring network (bf16 parameters, float32 master
    copy and Adam state on the device)."""

    def __init__(self, max_batch: int = 16384):
        self._lib = load()
        h = C.c_void_p()
        _check(self._lib.pll_mlp_create(max_batch, C.byref(h)), "pll_mlp_create")
        self._h = h.value
        self.max_batch = max_batch

    def set_params(self, params, stream=None):
        p, pp = _hptr(params, np.float32)
        assert p.shape == (MLP_NPARAM,)
        _check(self._lib.pll_mlp_set_params(self._h, pp, _stream_handle(stream)), "pll_mlp_set_params")

    def params(self):
        """(float32 master [4801], bfloat16 bit patterns uint16 [4801])."""
        m = np.empty(MLP_NPARAM, dtype=np.float32)
        b = np.empty(MLP_NPARAM, dtype=np.uint16)
        _check(self._lib.pll_mlp_get_params(self._h, m.ctypes.data, b.ctypes.data), "pll_mlp_get_params")
        return m, b

    def forward(self, x, out=None, stream=None):
        import torch
        n = int(x.shape[0])
        if out is None:
            out = torch.empty(max(n, 1), dtype=torch.float32, device=x.device)
        _check(self._lib.pll_mlp_forward(self._h, _dptr(x) if n else None, n, _dptr(out),
                                         _stream_handle(stream)), "pll_mlp_forward")
        return out[:n]

    def grad(self, x, target, idx=None, batch=None, stream=None):
        """Gradient and loss of the mean squared error (host float32 [4801], float)."""
        b = int(idx.shape[0]) if idx is not None else (batch or int(x.shape[0]))
        sh = _stream_handle(stream)
        _check(self._lib.pll_mlp_grad(self._h, _dptr(x), _dptr(target),
                                      _dptr(idx) if idx is not None else None, b, sh), "pll_mlp_grad")
        g = np.empty(MLP_NPARAM, dtype=np.float32)
        loss = C.c_float(0)
        _check(self._lib.pll_mlp_read_grad(self._h, g.ctypes.data, C.byref(loss), sh), "pll_mlp_read_grad")
        return g, float(loss.value)

    def adam(self, lr: float, stream=None):
        _check(self._lib.pll_mlp_adam(self._h, lr, _stream_handle(stream)), "pll_mlp_adam")

    def train_step(self, x, target, idx, lr: float, stream=None):
        _check(self._lib.pll_mlp_train_step(self._h, _dptr(x), _dptr(target), _dptr(idx),
                                            int(idx.shape[0]), lr, _stream_handle(stream)),
               "pll_mlp_train_step")

    def loss(self, stream=None) -> float:
        v = C.c_float(0)
        _check(self._lib.pll_mlp_read_grad(self._h, None, C.byref(v), _stream_handle(stream)),
               "pll_mlp_read_grad")
        return float(v.value)

    def order(self, offsets, cols, t: int, stream=None):
        """pll_learned_order: CUDA int32 order of the graph's vertices."""
        import torch
        n = int(offsets.shape[0]) - 1
        nnz = int(cols.shape[0])
        order = torch.empty(max(n, 1), dtype=torch.int32, device=offsets.device)
        _check(self._lib.pll_learned_order(_dptr(offsets), _dptr(cols) if nnz else None, n, nnz, t,
                                           self._h, _dptr(order), _stream_handle(stream)),
               "pll_learned_order")
        return order[:n]

    def close(self):
        if getattr(self, "_h", None):
            self._lib.pll_mlp_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
