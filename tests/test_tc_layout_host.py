"""Host run (no GPU) of the warp-level tensor-core field's data path: the kernels' own text
for the feature draw, the phasor tables, the x- and y-phasor slice fragments (k_xslices), the
face factors (k_face_factors) and the staging of the line factors' slices (tc_stage, volume
and face), built with g++ and launched as loops, with the mma.sync products emulated from the
PTX fragment layout in exact arithmetic. The slice group sums must give the oracle's
log k / scale at every node x < n - 1 and on the face x = n - 1, y < n - 1 (1e-11 absolute,
plus the phase-rounding bound for Cauchy frequencies), with every staged slot written (the
staging buffer is NaN-filled first). This pins the fragment orders of both operands, the
block and warp tiling (16 to 64 x-values per block here) and the packing of samples into line
groups on the CPU."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle as orc
from paper_1607_03252_gb300.workloads import RUN_SEED, sample_ids

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1607_03252_gb300", "csrc")


def _cut(text, start, end):
    a = text.index(start)
    return text[a:text.index(end, a)]


def _host(text):
    text = text.replace("__host__ __device__ __forceinline__", "static inline")
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
    field = open(os.path.join(CSRC, "field.cu")).read()
    philox = open(os.path.join(CSRC, "philox.cuh")).read()
    widen = open(os.path.join(CSRC, "widen.cuh")).read()
    parts = [
        _cut(philox, "__device__ __forceinline__ void philox10(", "}  // namespace mlmc"),
        _cut(widen, "__device__ __forceinline__ double widen(float f) {", "}  // namespace mlmc"),
        _cut(field, "__device__ __forceinline__ double u53(", "constexpr int kFieldThreads = 256;"),
        _cut(field, "constexpr int kTcSlices = 7;", "__device__ __forceinline__ void mma_bf16_16816("),
        _cut(field, "size_t tc_xslice_bytes(int B, int M, int n) {", "// The edge x = y = n - 1 in FP64"),
        _cut(field, "template <int RX>\nstruct TcShape {",
             "template <typename TOut, int RX, bool FACE>\n__global__ void __launch_bounds__(kTcThreads, 1) k_field_tc("),
    ]
    d = tmp_path_factory.mktemp("tcemu")
    (d / "kernels.inc").write_text(_host("\n".join(parts)))
    exe = d / "tc_emu"
    res = subprocess.run([gxx, "-std=c++17", "-O2", "-ffp-contract=off", "-Wno-unknown-pragmas", "-I", str(d),
                          "-I", CSRC, os.path.join(HERE, "host_emu", "tc_emu.cpp"), "-o", str(exe)],
                         capture_output=True, text=True)
    assert res.returncode == 0, res.stderr[-4000:]
    return str(exe)


@pytest.mark.parametrize("n,B,M,ell,cov", [(17, 3, 40, 0.3, orc.COV_GAUSS), (33, 2, 100, 0.2, orc.COV_EXP),
                                           (65, 1, 24, 0.3, orc.COV_GAUSS)])
def test_tensor_core_data_path_matches_oracle(emu, tmp_path, n, B, M, ell, cov):
    ids = sample_ids(2, 5, B)
    out = tmp_path / "S.bin"
    res = subprocess.run([emu, str(RUN_SEED), str(M), str(n), repr(ell), str(cov), str(out)] + [str(int(i)) for i in ids],
                         capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stdout + res.stderr
    raw = np.fromfile(out, dtype=np.float64)
    S = raw[: B * n * n * (n - 1)].reshape(B, n, n, n - 1)  # [s][z][y][x < n - 1]
    Sf = raw[B * n * n * (n - 1):].reshape(B, n, n - 1)      # [s][z][y < n - 1] at x = n - 1
    assert np.all(np.isfinite(S)) and np.all(np.isfinite(Sf))
    x = np.arange(n) / (n - 1)
    for s in range(B):
        w, b = orc.features(RUN_SEED, int(ids[s]), M, ell, cov)
        # log k / scale = sum_m cos(w . x + b) at the nodes x < n - 1, [z][y][x]
        ph = (w[:, 0, None, None, None] * x[None, None, None, : n - 1] + w[:, 1, None, None, None] * x[None, None, :, None]
              + w[:, 2, None, None, None] * x[None, :, None, None] + b[:, None, None, None])
        So = np.cos(ph).sum(axis=0)
        phf = (w[:, 0, None, None] * 1.0 + w[:, 1, None, None] * x[None, None, : n - 1]
               + w[:, 2, None, None] * x[None, :, None] + b[:, None, None])
        Sfo = np.cos(phf).sum(axis=0)
        tol = 1e-11 + np.sum(4.0 * np.finfo(np.float64).eps * (np.abs(w).sum(axis=1) + 2.0 * np.pi))
        err = float(np.max(np.abs(S[s] - So)))
        errf = float(np.max(np.abs(Sf[s] - Sfo)))
        print("n %d M %d sample %d: max |S - S_oracle| %.3e, face %.3e (tol %.3e)" % (n, M, s, err, errf, tol))
        assert err <= tol and errf <= tol
