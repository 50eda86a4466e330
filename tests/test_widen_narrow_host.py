"""Host check (no GPU) of the FP32 <-> FP64 conversions on the integer pipe in
paper_1607_03252_gb300/csrc/widen.cuh: the functions' own text, compiled with g++ next to
shims of the CUDA bit-cast intrinsics, must agree bit for bit with the C conversions
(round to nearest even) on random values and on the tie, carry, overflow, zero and
subnormal cases (subnormals flush to zero by design)."""
import os
import re
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_widen_and_narrow_round_like_ieee(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    src = open(os.path.join(ROOT, "paper_1607_03252_gb300", "csrc", "widen.cuh")).read()
    body = src[src.index("__device__ __forceinline__ double widen(float f) {"):src.index("}  // namespace mlmc")]
    body = body.replace("__device__ __forceinline__", "static inline")
    assert "narrow(double d)" in body
    (tmp_path / "widen_narrow.inc").write_text(body)
    exe = tmp_path / "emu"
    res = subprocess.run([gxx, "-std=c++17", "-O2", "-ffp-contract=off", "-I", str(tmp_path),
                          os.path.join(HERE, "host_emu", "widen_narrow_emu.cpp"), "-o", str(exe)],
                         capture_output=True, text=True)
    assert res.returncode == 0, res.stderr[-3000:]
    run = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert run.returncode == 0, run.stdout[-3000:]
    assert re.search(r"^0 mismatches", run.stdout, re.M)
