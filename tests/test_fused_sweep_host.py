"""Host emulation of the fused red-black sweep kernel (no GPU): the kernel body from
paper_1607_03252_gb300/csrc/smooth.cu, compiled with g++ and AddressSanitizer, one OS
thread per CUDA thread and a barrier for __syncthreads; 16-byte copies assert the
alignment cp.async needs. Every tile shape, FP32 and FP64, n = 5 .. 33, several samples
(every sample start modulo 16 bytes), one inactive sample: the sweep must equal the
sequential red-then-black sweep bit for bit, with no out-of-bounds or misaligned access.
The index arithmetic of the kernel is therefore checked before any GPU run."""
import os
import shutil
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def emu_binary(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("fused_emu")
    inc = d / "fused_sweep.inc"
    subprocess.run([sys.executable, os.path.join(HERE, "host_emu", "extract.py"),
                    os.path.join(ROOT, "paper_1607_03252_gb300", "csrc", "smooth.cu"), str(inc)], check=True)
    exe = d / "fused_sweep_emu"
    cmd = [gxx, "-std=c++20", "-O1", "-g", "-fsanitize=address", "-fno-omit-frame-pointer", "-ffp-contract=off",
           "-pthread", "-I", str(d), os.path.join(HERE, "host_emu", "fused_sweep_emu.cpp"), "-o", str(exe)]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0 and "sanitize" in res.stderr:
        pytest.skip("AddressSanitizer not available: " + res.stderr[-200:])
    assert res.returncode == 0, res.stderr[-4000:]
    return str(exe)


def test_fused_sweep_equals_sequential_sweep_on_host(emu_binary):
    res = subprocess.run([emu_binary], capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stdout[-3000:] + res.stderr[-3000:]
    assert "all ok" in res.stdout
