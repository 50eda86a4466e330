"""Host runs of the colour-split kernels (MLMC_SMOOTH_SPLIT; FP32 nodal coefficient and
FP64 stored faces) against their plain-layout counterparts, no GPU: the kernels' own text
compiled with g++, the launch a loop over every block and thread. The split storage map is computed here from its
definition (per sample, colour c = (x + y + z) % 2 block of n x n rows of (n + 1) / 2
slots rounded up to a multiple of 4, node x at slot x // 2); slots that hold no node are NaN, so a kernel that read one
would poison its result. A red and a black pass, the residual, the trilinear correction,
full weighting into split coarse storage and the operator set-up (reciprocal coefficient;
faces, D and 1/D) must equal the plain kernels bit for bit."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_1607_03252_gb300.workloads import random_coefficient, random_rhs

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
    text = text.replace("template <>\nstatic inline", "template <>\ninline")  # no storage class on a specialisation
    while "__launch_bounds__(" in text:
        i = text.index("__launch_bounds__(")
        j, depth = i + len("__launch_bounds__("), 1
        while depth:
            depth += {"(": 1, ")": -1}.get(text[j], 0)
            j += 1
        text = text[:i] + text[j:]
    return text


def split_perm(n, B):
    """Plain index (s, z, y, x) -> colour-split index, from the definition (rows of
    (n + 1) / 2 slots padded to a multiple of 4)."""
    P = ((n + 1) // 2 + 3) // 4 * 4
    ns = 2 * n * n * P
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    c = (x + y + z) % 2
    within = c * (n * n * P) + (z * n + y) * P + x // 2
    return np.concatenate([s * ns + within.ravel() for s in range(B)]).astype(np.int64)


def test_split_map_is_a_bijection_onto_its_slots():
    for n in (5, 9, 17, 33):
        p = split_perm(n, 2)
        P = ((n + 1) // 2 + 3) // 4 * 4
        assert len(np.unique(p)) == len(p) and p.max() < 2 * (2 * n * n * P)  # two samples


@pytest.fixture(scope="module")
def emu(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    mgcu = open(os.path.join(CSRC, "mg.cu")).read()
    parts = [
        "namespace mlmc {",
        _cut(mgcu, "__host__ __device__ __forceinline__ int split_pitch(int n)", "// Carves 256-byte"),
        _cut(mgcu, "// x in the arithmetic type TD", "// Dense 27x27 scaled operator"),
        _cut(mgcu, "// One colour of a red-black sweep: threads enumerate", "// Reciprocal nodal coefficient rho"),
        _cut(mgcu, "template <typename T>\n__global__ void k_nodal_k(", "// Blocks per sample of the deterministic"),
        _cut(mgcu, "// r~ = g - D u + sum K u_q on interior nodes (0 on the boundary)", "inline dim3 zmarch_grid"),
        _cut(mgcu, "template <typename T, bool SPLIT = false>\n__global__ void k_prolong_p1(", "// Q[s] = u(1/4, 1/4, 1/4)"),
        _cut(mgcu, "template <typename T, bool SPLIT_OUT = false>\n__global__ void k_restrict(", "// g = h^2 f (f == NULL"),
        "}  // namespace mlmc",
    ]
    d = tmp_path_factory.mktemp("splitemu")
    (d / "split_kernels.inc").write_text(_host("\n".join(parts)))
    exe = d / "emu"
    res = subprocess.run([gxx, "-std=c++17", "-O2", "-ffp-contract=off", "-Wno-unknown-pragmas", "-I", str(d),
                          os.path.join(HERE, "host_emu", "split_emu.cpp"), "-o", str(exe)],
                         capture_output=True, text=True)
    assert res.returncode == 0, res.stderr[-4000:]
    return str(exe), d


@pytest.mark.parametrize("n,B", [(5, 2), (9, 2), (17, 3), (33, 2)])
def test_split_kernels_equal_plain_kernels_bitwise(emu, n, B):
    exe, d = emu
    nc = (n + 1) // 2
    rng = np.random.default_rng(n)
    k = np.stack([random_coefficient(n, 10 * n + s, 1.0) for s in range(B)])
    kn = (1.0 / k).astype(np.float32)
    g = np.stack([random_rhs(n, 20 * n + s) for s in range(B)]).astype(np.float32) * 1e-3
    u = np.zeros((B, n, n, n), dtype=np.float32)
    u[:, 1:-1, 1:-1, 1:-1] = rng.standard_normal((B, n - 2, n - 2, n - 2)).astype(np.float32)
    ec = np.zeros((B, nc, nc, nc), dtype=np.float32)
    ec[:, 1:-1, 1:-1, 1:-1] = rng.standard_normal((B, nc - 2, nc - 2, nc - 2)).astype(np.float32)
    r = np.zeros((B, n, n, n), dtype=np.float32)
    r[:, 1:-1, 1:-1, 1:-1] = rng.standard_normal((B, n - 2, n - 2, n - 2)).astype(np.float32)
    src, pm, dst = d / ("in_%d.bin" % n), d / ("perm_%d.bin" % n), d / ("out_%d.bin" % n)
    with open(src, "wb") as fh:
        for a in (kn, g, u):
            fh.write(np.ascontiguousarray(a, dtype=np.float32).tobytes())
        fh.write(np.ascontiguousarray(k, dtype=np.float64).tobytes())
        fh.write(ec.tobytes())
        fh.write(r.tobytes())
    with open(pm, "wb") as fh:
        fh.write(split_perm(n, B).tobytes())
        fh.write(split_perm(nc, B).tobytes())
    subprocess.run([exe, "split", str(n), str(B), str(src), str(pm), str(dst)], check=True)
    out = np.fromfile(dst, dtype=np.float32)
    n3, nc3 = B * n ** 3, B * nc ** 3
    sizes = [n3, n3, n3, n3, n3, n3, nc3, nc3, n3, n3]
    parts, off = [], 0
    for sz in sizes:
        parts.append(out[off:off + sz])
        off += sz
    assert off == out.size
    names = ["sweep", "residual", "prolongation", "restriction", "reciprocal k"]
    for i, name in enumerate(names):
        plain, split = parts[2 * i], parts[2 * i + 1]
        assert np.all(np.isfinite(plain)), name
        assert np.array_equal(plain.view(np.uint32), split.view(np.uint32)), name
    # the sweep changed the interior (the comparison is not of untouched arrays)
    assert not np.array_equal(parts[0].reshape(B, n, n, n), u)


@pytest.mark.parametrize("n,B", [(5, 2), (9, 2), (17, 3), (33, 2)])
def test_split64_kernels_equal_plain_kernels_bitwise(emu, n, B):
    exe, d = emu
    nc = (n + 1) // 2
    rng = np.random.default_rng(100 + n)
    k = np.stack([random_coefficient(n, 30 * n + s, 1.0) for s in range(B)])
    g = np.stack([random_rhs(n, 40 * n + s) for s in range(B)]) * 1e-3
    g[:, [0, -1], :, :] = 0.0
    g[:, :, [0, -1], :] = 0.0
    g[:, :, :, [0, -1]] = 0.0
    u = np.zeros((B, n, n, n))
    u[:, 1:-1, 1:-1, 1:-1] = rng.standard_normal((B, n - 2, n - 2, n - 2))
    ec = np.zeros((B, nc, nc, nc))
    ec[:, 1:-1, 1:-1, 1:-1] = rng.standard_normal((B, nc - 2, nc - 2, nc - 2))
    r = np.zeros((B, n, n, n))
    r[:, 1:-1, 1:-1, 1:-1] = rng.standard_normal((B, n - 2, n - 2, n - 2))
    src, pm, dst = d / ("in64_%d.bin" % n), d / ("perm64_%d.bin" % n), d / ("out64_%d.bin" % n)
    with open(src, "wb") as fh:
        for a in (k, g, u, ec, r):
            fh.write(np.ascontiguousarray(a, dtype=np.float64).tobytes())
    with open(pm, "wb") as fh:
        fh.write(split_perm(n, B).tobytes())
        fh.write(split_perm(nc, B).tobytes())
    subprocess.run([exe, "split64", str(n), str(B), str(src), str(pm), str(dst)], check=True)
    out = np.fromfile(dst, dtype=np.float64)
    n3, nc3 = B * n ** 3, B * nc ** 3
    names = ["Kx", "Ky", "Kz", "D", "1/D", "sweep", "residual", "block prolongation", "block prolongation, split",
             "block prolongation, FP32", "restriction", "copies", "P1 prolongation", "P1 restriction"]
    sizes = [nc3 if name in ("restriction", "P1 restriction") else n3 for name in names]
    off, got = 0, {}
    for name, sz in zip(names, sizes):
        got[name] = (out[off:off + sz], out[off + sz:off + 2 * sz])
        off += 2 * sz
    assert off == out.size
    for name in names:
        plain, split = got[name]
        assert np.all(np.isfinite(plain)), name
        assert np.array_equal(plain.view(np.uint64), split.view(np.uint64)), name
    assert not np.array_equal(got["sweep"][0].reshape(B, n, n, n), u)
