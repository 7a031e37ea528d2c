"""The serving ring's slot placement (csrc/serve_ring.h, host code) under
random admit / retire sequences, compiled here with g++ and checked against a
model of the live blocks (tests/serve_ring_check.cpp)."""
import shutil
import subprocess
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]


def test_ring_placement(tmp_path):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not available")
    exe = tmp_path / "serve_ring_check"
    subprocess.run([gxx, "-O2", "-std=c++17", f"-I{ROOT / 'paper_1304_4661_gb300' / 'csrc'}",
                    str(ROOT / "tests" / "serve_ring_check.cpp"), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.startswith("ok ") and int(r.stdout.split()[1]) > 100000
