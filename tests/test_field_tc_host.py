"""Host checks of the tensor-core field's arithmetic (no GPU): the double-float helpers of
dfloat.cuh built with g++ (-ffp-contract=off), their constants against high-precision values,
the seven-slice split (grids, bounds, bf16 exactness, remainder), Tang's double-float exp
against the C library's long-double exp, and a host model of the whole scheme (slices, the
28 exact slice-pair group sums, folds every 256 features, exp) against the oracle's field."""
import os
import re
import shutil
import struct
import subprocess
from decimal import Decimal, getcontext
from fractions import Fraction

import numpy as np
import pytest

import oracle as orc
from paper_1607_03252_gb300.workloads import RUN_SEED, sample_id

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_1607_03252_gb300", "csrc")
HDR = os.path.join(CSRC, "dfloat.cuh")


@pytest.fixture(scope="module")
def emu(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("dfemu")
    exe = d / "dfloat_emu"
    res = subprocess.run([gxx, "-std=c++17", "-O2", "-ffp-contract=off", "-Wall", "-Wno-unknown-pragmas", "-I", CSRC,
                          os.path.join(HERE, "host_emu", "dfloat_emu.cpp"), "-o", str(exe)],
                         capture_output=True, text=True)
    assert res.returncode == 0, res.stderr[-3000:]
    return str(exe)


def _run(exe, *args):
    res = subprocess.run([exe, *map(str, args)], capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stdout + res.stderr
    return res.stdout


def _const(name):
    src = open(HDR).read()
    m = re.search(r"const float %s = ([0-9.eE+-]+)f;" % name, src)
    assert m, name
    return Fraction(float(np.float32(float(m.group(1)))))


def _sig_bits(fr):
    if fr == 0:
        return 0
    num, den = abs(fr.numerator), fr.denominator
    while num % 2 == 0:
        num //= 2
    return num.bit_length()


def test_constants_against_high_precision():
    getcontext().prec = 60
    ln2 = Fraction(Decimal(2).ln())
    L1, L2, L3 = _const("L1"), _const("L2"), _const("L3")
    assert _sig_bits(L1) <= 12                  # N * L1 exact for |N| < 2^12
    assert abs(L1 + L2 + L3 - ln2 / 32) < Fraction(1, 10 ** 21)
    assert abs(_const("kInvL") - 32 / ln2) < Fraction(1, 10 ** 5)
    # the slice grids: C_i = 1.5 * 2^(23 - 7 (i + 1))
    for i in range(7):
        assert _const("C%d" % i) == Fraction(3, 2) * Fraction(2) ** (23 - 7 * (i + 1))


def test_slices_on_grid_bounded_and_exact(emu):
    out = _run(emu, "slices", 300000, 11)
    m = re.search(r"worst_abs_err (\S+) bad (\d+)", out)
    worst, bad = float(m.group(1)), int(m.group(2))
    print(out.strip())
    assert bad == 0
    assert worst <= 2.0 ** -50 + 2.0 ** -60


def test_exp_double_float_against_long_double(emu):
    out = _run(emu, "exp", 300000, 5)
    worst = float(re.search(r"worst_rel_err (\S+)", out).group(1))
    print(out.strip())
    assert worst <= 2e-14


@pytest.mark.parametrize("n,M,ell,cov", [(17, 256, 0.3, orc.COV_GAUSS), (17, 300, 0.1, orc.COV_GAUSS),
                                         (33, 256, 0.15, orc.COV_EXP)])
def test_field_model_matches_oracle(emu, tmp_path, n, M, ell, cov):
    """The scheme the tensor-core kernel runs, modelled on the host, gives the oracle's field to
    1e-12 relative (M = 300 folds the group sums twice)."""
    sid = sample_id(2, 3)
    w, b = orc.features(RUN_SEED, sid, M, ell, cov)
    sigma2 = 1.0
    scale = np.sqrt(sigma2) * np.sqrt(2.0 / M)
    inp = tmp_path / "in.bin"
    with open(inp, "wb") as f:
        f.write(struct.pack("<iid", M, n, scale))
        f.write(np.ascontiguousarray(w, dtype=np.float64).tobytes())
        f.write(np.ascontiguousarray(b, dtype=np.float64).tobytes())
    outp = tmp_path / "out.bin"
    _run(emu, "field", inp, outp)
    k = np.fromfile(outp, dtype=np.float64).reshape(n, n, n)
    ko = orc.field(RUN_SEED, sid, M, sigma2, ell, n, cov)
    rel = float(np.max(np.abs(k - ko) / np.abs(ko)))
    print("n %d M %d max rel err %.3e" % (n, M, rel))
    assert rel <= 1e-12
