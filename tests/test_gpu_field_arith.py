"""The field's arithmetic variants (MLMC_FIELD_ARITH, read once per process, so each runs
in a child process): double-float per line (the default), FP64, double-float with
flattened outputs. Each must give the oracle's field to 1e-12 relative, and its FP32 output
must be its FP64 output rounded."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import numpy as np, torch
import oracle as orc
import paper_1607_03252_gb300 as mg
from paper_1607_03252_gb300.workloads import RUN_SEED, sample_ids
orc.lib()
worst = 0.0
for n, B, M, ell in ((33, 3, 256, 0.3), (17, 2, 100, 0.1)):
    ids = sample_ids(2, 7, B)
    fc = mg.field_cfg(RUN_SEED, 1.0, ell, M)
    k = torch.empty((B, n, n, n), dtype=torch.float64, device="cuda")
    k32 = torch.empty((B, n, n, n), dtype=torch.float32, device="cuda")
    mg.mlmc_field_eval(fc, ids, k)
    mg.mlmc_field_eval(fc, ids, k32)
    kh = k.cpu().numpy()
    assert np.array_equal(k32.cpu().numpy(), kh.astype(np.float32))
    for s in range(B):
        ko = orc.field(RUN_SEED, int(ids[s]), M, 1.0, ell, n)
        worst = max(worst, float(np.max(np.abs(kh[s] - ko) / np.abs(ko))))
print("max rel err %.3e" % worst)
assert worst <= 1e-12
"""


@pytest.mark.parametrize("arith", [0, 1, 2])
def test_field_arithmetic_variant_matches_oracle(arith):
    env = dict(os.environ, MLMC_FIELD_ARITH=str(arith))
    res = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stdout[-2000:] + res.stderr[-4000:]
    print(arith, res.stdout.strip())
