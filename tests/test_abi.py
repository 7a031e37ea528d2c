"""The C-ABI library builds, loads and exports every symbol of include/pll.h
(CPU only: no call here touches a GPU)."""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_1304_4661_gb300 import _build, pll

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "pll.h")).read()
    return sorted(set(re.findall(r"PLL_API\s+[\w\s\*]+?\b(pll_\w+)\s*\(", text)))


def test_header_declares_the_binding_symbols():
    assert declared_symbols() == sorted(pll.SYMBOLS)


def test_library_exports_every_declared_symbol():
    path = _build.build_pll()
    lib = C.CDLL(path)
    for name in declared_symbols():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (pll_\w+)", out))
    assert set(declared_symbols()) <= exported
    # nothing else of ours leaks out of the shared object
    assert all(not s.startswith("_ZN3pll") for s in re.findall(r"\bT (\S+)", out))


def test_status_strings():
    lib = pll.load()
    for code in range(7):
        assert lib.pll_status_str(code)
    assert pll.status_str(pll.PLL_E_RANGE) == "size or distance out of range"


def test_header_compiles_as_c():
    src = '#include "pll.h"\nint main(void){ pll_build_opts o = {0}; (void)o; return PLL_OK; }\n'
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                        "-x", "c", "-", "-o", "/dev/null"], input=src, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_null_arguments_are_rejected_without_a_gpu():
    lib = pll.load()
    assert lib.pll_query(None, None, None, 1, None, None) == pll.PLL_E_INVAL
    assert lib.pll_label_entries(None, None) == pll.PLL_E_INVAL
    assert lib.pll_get_stats(None, None) == pll.PLL_E_INVAL
    lib.pll_free(None)


def test_path_and_directed_argument_checks_without_a_gpu():
    """The host-side checks of the shortest-path and directed entry points
    return before any CUDA call."""
    lib = pll.load()
    out = C.c_void_p()
    assert lib.pll_paths_create(None, None, None, 0, 0, None, C.byref(out)) == pll.PLL_E_INVAL
    assert lib.pll_paths_create(None, None, None, 0, 0, None, None) == pll.PLL_E_INVAL
    assert lib.pll_paths_parents(None, None) == pll.PLL_E_INVAL
    tot = C.c_uint64(0)
    assert lib.pll_path_offsets(None, None, None, 1, None, C.byref(tot), None) == pll.PLL_E_INVAL
    assert lib.pll_path_query(None, None, None, 1, None, 0, None, None) == pll.PLL_E_INVAL
    lib.pll_paths_free(None)
    opts = pll.BuildOpts(0, 0, 0, 0, 0)
    assert lib.pll_build_directed(None, None, 0, 0, None, C.byref(opts), None, None) == pll.PLL_E_INVAL
    assert lib.pll_build_directed(None, None, 1 << 24, 0, None, C.byref(opts), None,
                                  C.byref(out)) == pll.PLL_E_RANGE
    assert lib.pll_build_directed(None, None, 0, 1, None, C.byref(opts), None, C.byref(out)) == pll.PLL_E_INVAL
    assert lib.pll_build_directed(None, None, 5, 0, None, C.byref(opts), None, C.byref(out)) == pll.PLL_E_INVAL
    for bad in (pll.BuildOpts(1, 0, 0, 0, 0), pll.BuildOpts(0, 0, 0, 1, 0), pll.BuildOpts(0, 0, 0, 0, 1)):
        assert lib.pll_build_directed(None, None, 0, 0, None, C.byref(bad), None, C.byref(out)) == pll.PLL_E_INVAL
    assert out.value is None
    assert lib.pll_dquery(None, None, None, 1, None, None) == pll.PLL_E_INVAL
    a, b = C.c_uint64(0), C.c_uint64(0)
    assert lib.pll_dlabel_entries(None, C.byref(a), C.byref(b)) == pll.PLL_E_INVAL
    assert lib.pll_dexport_labels(None, 0, None, None, None) == pll.PLL_E_INVAL
    assert lib.pll_dexport_order(None, None) == pll.PLL_E_INVAL
    lib.pll_dfree(None)


def test_noalloc_binding_refuses_wrong_outputs_without_a_gpu():
    """bp_labels_noalloc checks every tensor's dtype and exact size before the
    call: an undersized output would otherwise be written past its end."""
    import torch
    n, nnz, t = 10, 18, 16
    tp = 16

    def args(**over):
        a = dict(rank_offsets=torch.zeros(n + 1, dtype=torch.int32),
                 rank_cols=torch.zeros(nnz, dtype=torch.int32),
                 d=torch.zeros(n * tp, dtype=torch.uint8),
                 masks=torch.zeros(2 * n * t, dtype=torch.int64),
                 roots=torch.zeros(t, dtype=torch.int32),
                 cnt=torch.zeros(t, dtype=torch.int32),
                 S=torch.zeros(64 * t, dtype=torch.int32))
        a.update(over)
        return a

    def call(a):
        pll.bp_labels_noalloc(a["rank_offsets"], a["rank_cols"], t, a["d"], a["masks"], a["roots"],
                              a["cnt"], a["S"])

    bad = [dict(d=torch.zeros(n * tp - 1, dtype=torch.uint8)),
           dict(d=torch.zeros(n * t, dtype=torch.int32)),
           dict(masks=torch.zeros(2 * n * t - 2, dtype=torch.int64)),
           dict(masks=torch.zeros(2 * n * t, dtype=torch.float64)),
           dict(roots=torch.zeros(t - 1, dtype=torch.int32)),
           dict(cnt=torch.zeros(t, dtype=torch.int64)),
           dict(S=torch.zeros(64 * t - 64, dtype=torch.int32)),
           dict(rank_cols=torch.zeros(nnz, dtype=torch.int64))]
    for over in bad:
        with pytest.raises(ValueError, match="dtype|elements"):
            call(args(**over))
    # right sizes on the host are refused too: the outputs must be CUDA tensors
    with pytest.raises(ValueError, match="CUDA tensor"):
        call(args())
