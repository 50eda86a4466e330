"""Host check (no GPU) of the shared-memory layout the tcgen05 field kernel stages its bf16
operand tiles in: each (row, feature) pair has its own slot, the slots tile the 128-row A and
64-row B tiles exactly, and every element sits where the K-major core-matrix layout that the
MMA descriptors describe (leading byte offset 128 along K, stride byte offset 256 along the
rows) puts it."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1607_03252_gb300", "csrc")


def test_tile_layout_matches_core_matrix_layout(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = tmp_path / "umma_layout_check"
    res = subprocess.run([gxx, "-std=c++17", "-O1", "-Wall", "-I", CSRC,
                          os.path.join(HERE, "host_emu", "umma_layout_check.cpp"), "-o", str(exe)],
                         capture_output=True, text=True)
    assert res.returncode == 0, res.stderr[-2000:]
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout + out.stderr
