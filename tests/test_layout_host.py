"""The run-major shared-memory layout of the slab (csrc/slab.cuh), checked on
the host: every cell a window pass may touch has its own slot inside the
extent the launch sizes, a warp's interleaved writes are free of bank
conflicts, and the window reads of consecutive lanes are consecutive words
(tests/layout_check.cu, compiled with nvcc and run on the CPU)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_run_major_layout():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    out = os.path.join(ROOT, "tests", "_build")   # git-ignored
    os.makedirs(out, exist_ok=True)
    exe = os.path.join(out, "layout_check.%d" % os.getpid())
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-O1", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "layout_check.cu"), "-o", exe],
                   check=True, capture_output=True, text=True, timeout=600)
    try:
        r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    finally:
        os.remove(exe)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "0 failures" in r.stdout
