"""The field's arithmetic variants (MLMC_FIELD_ARITH, read once per process, so each runs
in a child process): double-float per line, FP64, double-float with flattened outputs,
bf16 slices on the tensor cores (3, the default: tcgen05 for the volume from 65^3, the
warp-level mma.sync below; 4: mma.sync everywhere). Each must give the oracle's field to
1e-12 relative, and its FP32 output must be its FP64 output rounded. The tensor-core form
also runs every block shape (16 to 128 x-values per block, 17^3 to 257^3), a feature count
that is not a multiple of the 8 features of a k-step, the fold of its group sums every 256
features (M = 1024, both forms), a last chunk of one k-step on tcgen05 (M = 100), the
exponential covariance, and a batch whose samples differ."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import numpy as np, torch
import oracle as orc
import paper_1607_03252_gb300 as mg
from paper_1607_03252_gb300.workloads import RUN_SEED, sample_ids
orc.lib()
import os, sys
worst = 0.0
cases = [(33, 3, 256, 0.3, 0), (17, 2, 100, 0.1, 0)]
if len(sys.argv) > 1:
    cases = [(65, 2, 256, 0.3, 0), (129, 1, 256, 0.15, 1), (33, 2, 1024, 0.3, 0), (65, 1, 1024, 0.3, 0),
             (65, 1, 100, 0.2, 0), (257, 1, 64, 0.2, 0), (17, 40, 256, 0.3, 1)]
for n, B, M, ell, cov in cases:
    ids = sample_ids(2, 7, B)
    fc = mg.field_cfg(RUN_SEED, 1.0, ell, M, cov)
    k = torch.empty((B, n, n, n), dtype=torch.float64, device="cuda")
    k32 = torch.empty((B, n, n, n), dtype=torch.float32, device="cuda")
    mg.mlmc_field_eval(fc, ids, k)
    mg.mlmc_field_eval(fc, ids, k32)
    kh = k.cpu().numpy()
    assert np.array_equal(k32.cpu().numpy(), kh.astype(np.float32))
    for s in range(B):
        if B > 4 and s % 8:
            continue
        ko = orc.field(RUN_SEED, int(ids[s]), M, 1.0, ell, n, cov)
        tol = 1e-12
        if cov:  # the GPU rounds the three axis phases separately (bound as in the parity tests)
            w, _ = orc.features(RUN_SEED, int(ids[s]), M, ell, cov)
            tol += np.sqrt(2.0 / M) * np.sum(4.0 * np.finfo(np.float64).eps * (np.abs(w).sum(axis=1) + 2.0 * np.pi))
        err = float(np.max(np.abs(kh[s] - ko) / np.abs(ko)))
        print("n %d M %d ell %g cov %d sample %d: rel err %.3e, / tolerance %.3e" % (n, M, ell, cov, s, err, err / tol))
        worst = max(worst, err / tol)
print("max rel err / tolerance %.3e" % worst)
assert worst <= 1.0
"""


@pytest.mark.parametrize("arith", [0, 1, 2, 3, 4])
def test_field_arithmetic_variant_matches_oracle(arith):
    env = dict(os.environ, MLMC_FIELD_ARITH=str(arith))
    res = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stdout[-2000:] + res.stderr[-4000:]
    print(arith, res.stdout.strip())


@pytest.mark.parametrize("arith", [3, 4])
def test_field_tensor_core_shapes_match_oracle(arith):
    """3: tcgen05 for the 65^3-257^3 volumes, 4: the warp-level mma.sync everywhere."""
    env = dict(os.environ, MLMC_FIELD_ARITH=str(arith))
    res = subprocess.run([sys.executable, "-c", CHILD, "tc"], cwd=ROOT, env=env, capture_output=True, text=True,
                         timeout=900)
    assert res.returncode == 0, res.stdout[-2000:] + res.stderr[-4000:]
    print(res.stdout.strip())


DUMP = r"""
import sys, numpy as np, torch
import paper_1607_03252_gb300 as mg
from paper_1607_03252_gb300.workloads import RUN_SEED, sample_ids
out = {}
for n, B, M in ((65, 3, 256), (129, 1, 256), (65, 1, 1024)):
    k = torch.empty((B, n, n, n), dtype=torch.float64, device="cuda")
    mg.mlmc_field_eval(mg.field_cfg(RUN_SEED, 1.0, 0.3, M), sample_ids(3, 2, B), k)
    out["%d_%d" % (n, M)] = k.cpu().numpy()
np.savez(sys.argv[1], **out)
"""


def test_field_tcgen05_matches_warp_mma_bitwise(tmp_path):
    """The tcgen05 volume and the mma.sync volume form the same slices and exact group sums,
    so the whole field is bitwise the same (65^3 and 129^3, one and four folds)."""
    res = {}
    for arith in (3, 4):
        f = tmp_path / ("k%d.npz" % arith)
        env = dict(os.environ, MLMC_FIELD_ARITH=str(arith))
        r = subprocess.run([sys.executable, "-c", DUMP, str(f)], cwd=ROOT, env=env, capture_output=True, text=True,
                           timeout=600)
        assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
        res[arith] = dict(np.load(f))
    for key in res[3]:
        assert np.array_equal(res[3][key], res[4][key]), key
