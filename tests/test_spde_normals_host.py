"""The SPDE sampler's normals (polar method, FP32, correctly rounded steps and the series
logarithm) are the same bits on the device and in the oracle: the device functions' own
text (paper_1607_03252_gb300/csrc/spde.cu, philox.cuh), built for the host with the _rn
intrinsics as the IEEE operations they denote, against orc_octant_normal. No GPU."""
import os
import shutil
import struct
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_1607_03252_gb300", "csrc")


def _extract():
    spde = open(os.path.join(CSRC, "spde.cu")).read()
    philox = open(os.path.join(CSRC, "philox.cuh")).read()
    a = philox.index("__device__ __forceinline__ void philox10(")
    b = philox.index("}  // namespace mlmc", a)
    c = spde.index("__device__ __forceinline__ float log_series(float s) {")
    d = spde.index("// g = W(cell) / h for every cell of B samples")
    text = philox[a:b] + "\n" + spde[c:d]
    return text.replace("__device__ __forceinline__", "static inline").replace("__device__", "static")


def test_device_normals_equal_oracle_bits(tmp_path, orc):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    (tmp_path / "spde_normals.inc").write_text(_extract())
    exe = tmp_path / "emu"
    res = subprocess.run([gxx, "-std=c++17", "-O2", "-ffp-contract=off", "-Wno-unknown-pragmas", "-I", str(tmp_path),
                          os.path.join(HERE, "host_emu", "spde_normals_emu.cpp"), "-o", str(exe)],
                         capture_output=True, text=True)
    assert res.returncode == 0, res.stderr[-3000:]
    cases = [(1607032520, 12345, 0, 4000), (1, (3 << 48) | 7, 1 << 33, 2000), ((1 << 40) + 3, 99, 10 ** 9, 2000)]
    for seed, sid, first, count in cases:
        out = subprocess.run([str(exe), str(seed), str(sid), str(first), str(count)], capture_output=True,
                             text=True, check=True).stdout.split()
        for i, word in enumerate(out):
            want = struct.unpack("<I", struct.pack("<f", orc.octant_normal(seed, sid, first + i)))[0]
            assert int(word, 16) == want, (seed, sid, first + i)
