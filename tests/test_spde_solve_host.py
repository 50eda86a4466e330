"""Host run of a whole SPDE field (Sec. 3.2) from the kernels' own text: the FP64
refinement around FP32 cell-centred V-cycles (sweep, residuals, restriction, prolongation
with the zero-flux clamp, exact 2^3 solve, update, convergence test) must reach the
oracle's exact solve (eigenvectors of the zero-flux second difference). No GPU."""
import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

from paper_1607_03252_gb300.workloads import RUN_SEED, sample_id

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_1607_03252_gb300", "csrc")


def _cut(text, start, end):
    a = text.index(start)
    return text[a:text.index(end, a)]


def _drop(text, start, end_marker):
    a = text.index(start)
    b = text.index(end_marker, a) + len(end_marker)
    return text[:a] + text[b:]


def _host(text):
    text = text.replace("__device__ __forceinline__", "static inline").replace("__device__", "static")
    text = text.replace("__global__", "static").replace("__restrict__", "")
    while "__launch_bounds__(" in text:
        i = text.index("__launch_bounds__(")
        j, depth = i + len("__launch_bounds__("), 1
        while depth:
            depth += {"(": 1, ")": -1}.get(text[j], 0)
            j += 1
        text = text[:i] + text[j:]
    return text


@pytest.fixture(scope="module")
def emu(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    spde = open(os.path.join(CSRC, "spde.cu")).read()
    philox = open(os.path.join(CSRC, "philox.cuh")).read()
    widen = open(os.path.join(CSRC, "widen.cuh")).read()
    spdeh = open(os.path.join(CSRC, "spde.cuh")).read()
    body = _cut(spde, "constexpr int kT = 256;", "struct SpdeLevels {")
    body = _drop(body, "template <int THREADS>\n__device__ __forceinline__ double block_sum", "  return r;\n}\n")
    body = _drop(body, "__device__ __forceinline__ double warp_partial_sum(", "  return a;  // valid in lane 0\n}\n")
    tail = _cut(spde, "int log2i(int c) {", "// FP32 V(2,2) cycle on grid l")
    consts = _cut(spdeh, "constexpr double kSpdeRtol", "// Bytes of device scratch")
    text = "\n".join([consts,
                      _cut(philox, "__device__ __forceinline__ void philox10(", "}  // namespace mlmc"),
                      _cut(widen, "__device__ __forceinline__ double widen(float f) {", "}  // namespace mlmc"),
                      body, tail])
    d = tmp_path_factory.mktemp("spde_emu")
    (d / "spde_kernels.inc").write_text(_host(text))
    exe = d / "emu"
    res = subprocess.run([gxx, "-std=c++17", "-O2", "-ffp-contract=off", "-Wno-unknown-pragmas", "-I", str(d),
                          "-I", os.path.join(ROOT, "include"), os.path.join(HERE, "host_emu", "spde_solve_emu.cpp"),
                          "-o", str(exe)], capture_output=True, text=True)
    assert res.returncode == 0, res.stderr[-4000:]
    return str(exe)


@pytest.mark.parametrize("n,n_noise,sigma2,ell", [(5, 5, 1.0, 0.3), (9, 9, 1.0, 0.3), (9, 17, 2.0, 0.1),
                                                   (17, 17, 1.0, 0.05)])
def test_host_spde_field_matches_oracle(emu, orc, n, n_noise, sigma2, ell):
    sid = sample_id(4, 9)
    res = subprocess.run([emu, str(RUN_SEED), str(sid), str(n), str(n_noise), repr(sigma2), repr(ell)],
                         capture_output=True, text=True)
    assert res.returncode == 0, res.stderr[-2000:]
    k = np.array([struct.unpack("<d", bytes.fromhex(w)[::-1])[0] for w in res.stdout.split()]).reshape(n, n, n)
    ko = orc.spde_field(RUN_SEED, sid, sigma2, ell, n, n_noise)
    assert np.max(np.abs(k - ko) / ko) < 1e-9
