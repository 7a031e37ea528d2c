"""In-tree build of the native libraries (no setuptools, no cmake).

``build_graphgen()`` compiles the seeded input generators with gcc;
``build_pll()`` compiles the CUDA library ``libpll.so`` for sm_103a with nvcc,
one translation unit per process so the whole build takes well under a minute.
A library is rebuilt only when one of its sources is newer than it.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
from pathlib import Path

PKG = Path(__file__).resolve().parent
CSRC = PKG / "csrc"
OUT = PKG / "_lib"
INCLUDE = PKG.parent / "include"

ARCH = "-gencode=arch=compute_103a,code=sm_103a"

CU_SOURCES = [
    "pll_abi.cu",
    "k_prep.cu",
    "k_bp.cu",
    "k_pruned.cu",
    "k_labels.cu",
    "k_query.cu",
    "pll_noalloc.cu",
    "pll_serve.cu",
    "k_learned.cu",
    "pll_io.cu",
    "pll_paths.cu",
    "pll_directed.cu",
]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not Path(cand).exists():
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpll.so")
    return cand


def _stale(target: Path, sources) -> bool:
    if not target.exists():
        return True
    t = target.stat().st_mtime
    return any(Path(s).stat().st_mtime > t for s in sources)


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed:\n" + " ".join(map(str, cmd)) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def build_graphgen(force: bool = False) -> str:
    OUT.mkdir(exist_ok=True)
    src = CSRC / "graphgen.c"
    so = OUT / "libpllgen.so"
    if force or _stale(so, [src]):
        tmp = so.with_suffix(f".so.tmp{os.getpid()}")
        _run(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", str(tmp), str(src)])
        os.replace(tmp, so)
    return str(so)


def pll_sources():
    hdrs = sorted(CSRC.glob("*.cuh")) + sorted(CSRC.glob("*.h")) + sorted(INCLUDE.glob("*.h"))
    return [CSRC / s for s in CU_SOURCES], hdrs


def build_pll(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    """Compile every CUDA translation unit for sm_103a and link libpll.so."""
    OUT.mkdir(exist_ok=True)
    so = OUT / "libpll.so"
    srcs, hdrs = pll_sources()
    if not force and not _stale(so, srcs + hdrs + [Path(__file__)]):
        return str(so)
    nvcc = _nvcc()
    objdir = OUT / "obj"
    objdir.mkdir(exist_ok=True)
    common = [nvcc, ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
              "-Xcompiler", "-fvisibility=hidden", f"-I{INCLUDE}", f"-I{CSRC}",
              "--expt-relaxed-constexpr", *extra_flags]
    if verbose:
        common += ["-Xptxas", "-v"]

    def one(src: Path):
        obj = objdir / (src.stem + ".o")
        return _run(common + ["-c", str(src), "-o", str(obj)]), obj

    workers = min(len(srcs), os.cpu_count() or 4)
    with cf.ThreadPoolExecutor(workers) as ex:
        results = list(ex.map(one, srcs))
    logs = "".join(r[0] for r in results)
    tmp = so.with_suffix(f".so.tmp{os.getpid()}")
    _run([nvcc, ARCH, "-shared", "-o", str(tmp), *[str(r[1]) for r in results], "-lcudart"])
    os.replace(tmp, so)
    if verbose:
        print(logs)
    return str(so)


def build_all(force: bool = False, verbose: bool = False):
    return build_graphgen(force), build_pll(force, verbose)
