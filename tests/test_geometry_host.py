"""The kernels' index arithmetic (parity-split site index, coordinates and the
neighbour shifts) checked exhaustively on the host for ragged and degenerate
extents: every neighbour index in range and pointing at x +- mu-hat.  This
stands in for a device-side bounds checker, which these tests do not run.
The same program checks the C++ rolling-band order of the streaming launches
(a permutation, dependencies first) for every valid stagger and shift."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_index_arithmetic_on_the_host(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = tmp_path / "geometry_check"
    subprocess.check_call([nvcc, "-std=c++17", "-O1", "-I", os.path.join(ROOT, "paper_1305_3440_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "geometry_check.cu"), "-o", str(exe)])
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.strip().endswith("ok"), out.stdout + out.stderr
