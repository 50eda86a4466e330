"""Pins for the oracle's Philox generator and its uniform / normal transforms.

Philox4x32-10 and Philox4x64-10 share one round structure (Salmon et al., SC'11):
the 64-bit variant is checked word for word against numpy's independent
implementation, which pins the round, the key schedule and the role of each counter
word. The 32-bit variant (its multipliers and Weyl constants included) is checked word
for word against PyTorch's independent host implementation (at::philox_engine, a
header of the installed torch, compiled here with g++), whose key is the 64-bit seed
and whose counter words are (offset low, offset high, subsequence low, subsequence
high): the method's counter (id low, id high, m, c) is offset = id, subsequence =
m + 2^32 c.
"""
import math
import os
import shutil
import subprocess

import numpy as np
import pytest
from scipy import stats as sst


@pytest.mark.parametrize("key", [(0, 0), (0x123456789ABCDEF0, 0x0FEDCBA987654321), (2**64 - 1, 7)])
@pytest.mark.parametrize("start", [(0, 0, 0, 0), (5, 7, 9, 11), (2**64 - 2, 3, 2**63, 1)])
def test_philox4x64_matches_numpy(orc, key, start):
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=np.array(start, dtype=np.uint64))
    raw = [int(x) for x in bg.random_raw(12)]
    ctr = list(start)
    for blk in range(3):
        # numpy advances the 256-bit counter (with carry) before each block
        for w in range(4):
            ctr[w] = (ctr[w] + 1) % 2**64
            if ctr[w] != 0:
                break
        assert orc.philox4x64(ctr, key) == raw[4 * blk: 4 * blk + 4]


_ATEN_PROBE = r"""
#include <ATen/core/PhiloxRNGEngine.h>
#include <cstdio>
#include <cstdlib>
int main(int argc, char** argv) {
  for (int a = 1; a + 2 < argc; a += 3) {
    at::philox_engine e(strtoull(argv[a], 0, 0), strtoull(argv[a + 1], 0, 0), strtoull(argv[a + 2], 0, 0));
    for (int i = 0; i < 4; ++i) printf("%u\n", e());
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def aten_philox(tmp_path_factory):
    """Runs PyTorch's host Philox4x32-10 for (seed, subsequence, offset) triples."""
    torch = pytest.importorskip("torch")
    inc = os.path.join(os.path.dirname(torch.__file__), "include")
    if not os.path.exists(os.path.join(inc, "ATen", "core", "PhiloxRNGEngine.h")) or not shutil.which("g++"):
        pytest.skip("no at::philox_engine header or no g++")
    d = tmp_path_factory.mktemp("aten_philox")
    src, exe = d / "probe.cpp", d / "probe"
    src.write_text(_ATEN_PROBE)
    subprocess.run(["g++", "-std=c++17", "-O1", "-I", inc, str(src), "-o", str(exe)], check=True,
                   capture_output=True)

    def run(triples):
        args = [str(x) for t in triples for x in t]
        out = subprocess.run([str(exe), *args], check=True, capture_output=True, text=True).stdout.split()
        words = [int(x) for x in out]
        return [words[4 * i: 4 * i + 4] for i in range(len(triples))]

    return run


def test_philox4x32_matches_aten_word_for_word(orc, aten_philox):
    seeds = [0, 1607032520, 0x123456789ABCDEF0, 2**64 - 1]
    ctrs = [(0, 0, 0, 0), (5, 0, 0, 0), ((1 << 48) | 77, 0, 3, 1), (2**64 - 1, 0, 255, 2), (12345, 0, 2**32 - 1,
                                                                                               2**32 - 1)]
    triples, expect = [], []
    for seed in seeds:
        for ident, _, m, c in ctrs:
            triples.append((seed, m | (c << 32), ident))
            expect.append(orc.philox4x32([ident & 0xFFFFFFFF, ident >> 32, m, c], [seed & 0xFFFFFFFF, seed >> 32]))
    assert aten_philox(triples) == expect


def test_philox4x32_bits_balanced(orc):
    words = []
    for i in range(8192):
        words.extend(orc.philox4x32([i, 17, 3, 0], [1607032520, 0]))
    w = np.array(words, dtype=np.uint64)
    bits = np.array([(w >> b) & 1 for b in range(32)], dtype=np.float64)
    frac = bits.mean(axis=1)
    # 32768 words: each bit fraction has std 1/(2 sqrt(32768)) ~ 0.0028
    assert np.all(np.abs(frac - 0.5) < 6 * 0.5 / math.sqrt(len(w)))
    # byte histogram chi^2 (255 dof)
    bytes_ = np.concatenate([(w >> s) & 0xFF for s in (0, 8, 16, 24)])
    counts = np.bincount(bytes_.astype(np.int64), minlength=256)
    expected = len(bytes_) / 256.0
    chi2 = ((counts - expected) ** 2 / expected).sum()
    assert sst.chi2.sf(chi2, 255) > 1e-4


def test_philox4x32_counter_and_key_sensitivity(orc):
    base = orc.philox4x32([1, 2, 3, 4], [5, 6])
    for pos in range(4):
        c = [1, 2, 3, 4]
        c[pos] ^= 1
        other = orc.philox4x32(c, [5, 6])
        flipped = sum(bin(a ^ b).count("1") for a, b in zip(base, other))
        assert 40 < flipped < 88  # about half of 128 bits change (avalanche)
    for pos in range(2):
        k = [5, 6]
        k[pos] ^= 1
        other = orc.philox4x32([1, 2, 3, 4], k)
        flipped = sum(bin(a ^ b).count("1") for a, b in zip(base, other))
        assert 40 < flipped < 88


def test_uniforms_open_interval_and_moments(orc):
    U = np.array([orc.uniforms(1607032520, (1 << 48) | i, m) for i in range(200) for m in range(50)]).ravel()
    assert U.min() > 0.0 and U.max() < 1.0
    assert abs(U.mean() - 0.5) < 5 * math.sqrt(1 / 12 / len(U))
    assert abs(U.var() - 1 / 12) < 0.005
    assert sst.kstest(U, "uniform").pvalue > 1e-4


def test_features_distribution(orc):
    ell = 0.1
    g, b = [], []
    for i in range(60):
        w, bb = orc.features(1607032520, (2 << 48) | i, 256, ell)
        g.append(w * ell)
        b.append(bb)
    g = np.concatenate(g).ravel()
    b = np.concatenate(b)
    assert sst.kstest(g, "norm").pvalue > 1e-4
    assert abs(g.mean()) < 5 / math.sqrt(len(g))
    assert abs(g.var() - 1.0) < 0.03
    assert b.min() >= 0.0 and b.max() < 2 * math.pi
    assert sst.kstest(b / (2 * math.pi), "uniform").pvalue > 1e-4
    # the three components of w are uncorrelated
    G = g.reshape(-1, 3)
    C = np.corrcoef(G.T)
    assert np.all(np.abs(C - np.eye(3)) < 0.03)


def test_features_depend_on_seed_and_id(orc):
    w0, b0 = orc.features(1, 10, 8, 0.3)
    w1, b1 = orc.features(1, 11, 8, 0.3)
    w2, b2 = orc.features(2, 10, 8, 0.3)
    w3, b3 = orc.features(1, 10 | (1 << 40), 8, 0.3)
    for w, b in ((w1, b1), (w2, b2), (w3, b3)):
        assert not np.any(w == w0) and not np.any(b == b0)
