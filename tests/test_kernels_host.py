"""Host runs of CUDA kernels against the oracle (no GPU): the kernels' own text, with the
launch emulated as a loop over every block and thread, for the SPDE noise (bit for bit:
the same normals and the same summation order), the P1 finite-element faces (against the
oracle's element assembly), and the P1 transfers (against the oracle's interpolation
matrix). The index arithmetic of these kernels is thereby checked on the CPU."""
import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

from oracle import fe
from paper_1607_03252_gb300.workloads import RUN_SEED, sample_id

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_1607_03252_gb300", "csrc")


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
    spde = open(os.path.join(CSRC, "spde.cu")).read()
    mgcu = open(os.path.join(CSRC, "mg.cu")).read()
    philox = open(os.path.join(CSRC, "philox.cuh")).read()
    parts = [
        _cut(philox, "__device__ __forceinline__ void philox10(", "}  // namespace mlmc"),
        _cut(spde, "__device__ __forceinline__ float log_series(float s) {", "// One colour of red-black Gauss-Seidel"),
        _cut(mgcu, "__host__ __device__ __forceinline__ int split_pitch(int n)", "// Carves 256-byte"),
        _cut(mgcu, "template <typename T>\n__global__ void k_faces_fe(", "// Q[s] = u(1/4, 1/4, 1/4)"),
    ]
    d = tmp_path_factory.mktemp("kemu")
    (d / "kernels.inc").write_text(_host("\n".join(parts)))
    exe = d / "emu"
    res = subprocess.run([gxx, "-std=c++17", "-O2", "-ffp-contract=off", "-Wno-unknown-pragmas", "-I", str(d),
                          os.path.join(HERE, "host_emu", "kernels_emu.cpp"), "-o", str(exe)],
                         capture_output=True, text=True)
    assert res.returncode == 0, res.stderr[-4000:]
    return str(exe), d


@pytest.mark.parametrize("n,n_noise", [(5, 5), (9, 9), (5, 9), (9, 17)])
def test_spde_noise_kernel_equals_oracle_bits(emu, orc, n, n_noise):
    exe, _ = emu
    sid = sample_id(2, 31)
    out = subprocess.run([exe, "noise", str(RUN_SEED), str(sid), str(n), str(n_noise)], capture_output=True,
                         text=True, check=True).stdout.split()
    got = np.array([struct.unpack("<d", bytes.fromhex(w)[::-1])[0] for w in out])
    want = orc.spde_noise(RUN_SEED, sid, n, n_noise).ravel()
    assert np.array_equal(got, want)


def _run(emu, mode, n, arr, out_len):
    exe, d = emu
    src, dst = d / ("in_%s_%d.bin" % (mode, n)), d / ("out_%s_%d.bin" % (mode, n))
    np.ascontiguousarray(arr, dtype=np.float64).tofile(src)
    subprocess.run([exe, mode, str(n), str(src), str(dst)], check=True)
    return np.fromfile(dst, dtype=np.float64, count=out_len)


@pytest.mark.parametrize("n", [5, 9, 17])
def test_fe_faces_kernel_equals_element_assembly(emu, orc, n):
    k = orc.field(RUN_SEED, sample_id(1, 5), 32, 1.0, 0.3, n)
    out = _run(emu, "faces", n, k, 3 * n ** 3).reshape(3, n, n, n)
    A, _ = fe.assemble(n, k)
    h = 1.0 / (n - 1)
    for axis, step in ((0, 1), (1, n), (2, n * n)):
        for z in range(1, n - 1):
            for y in range(1, n - 1):
                for x in range(1, n - 1):
                    p = (z * n + y) * n + x
                    want = -A[p, p + step] / h
                    assert out[axis, z, y, x] == pytest.approx(want, rel=1e-13)
                    q = p - step  # the face to the lower neighbour lives at that neighbour
                    zz, yy, xx = np.unravel_index(q, (n, n, n))
                    assert out[axis, zz, yy, xx] == pytest.approx(-A[p, q] / h, rel=1e-13)


@pytest.mark.parametrize("nf", [5, 9, 17])
def test_p1_transfer_kernels_equal_interpolation_matrix(emu, nf):
    nc = (nf + 1) // 2
    rng = np.random.default_rng(nf)
    ec = np.zeros((nc, nc, nc))
    ec[1:-1, 1:-1, 1:-1] = rng.standard_normal((nc - 2,) * 3)
    P = fe.prolongation(nc)
    u = _run(emu, "prolong", nf, ec, nf ** 3)
    want = P @ ec.ravel()
    inner = fe.interior_mask(nf)
    assert np.allclose(u[inner], want[inner], rtol=0, atol=1e-15)
    assert np.all(u[~inner] == 0)
    r = np.zeros((nf, nf, nf))
    r[1:-1, 1:-1, 1:-1] = rng.standard_normal((nf - 2,) * 3)
    gc = _run(emu, "restrict", nf, r, nc ** 3)
    want_c = 0.5 * (P.T @ r.ravel())  # (h / h_c) P^T r for the h^2-scaled coarse system
    inner_c = fe.interior_mask(nc)
    assert np.allclose(gc[inner_c], want_c[inner_c], rtol=1e-14, atol=1e-14)
