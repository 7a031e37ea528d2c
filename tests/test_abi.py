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
