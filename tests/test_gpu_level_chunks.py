"""A level batch split into sample chunks whose fields run on a side stream while the
previous chunks solve (MLMC_LEVEL_CHUNKS, read once per process, so the chunked run is a
child process): Y, Q_f, Q_c and the level record equal the one-batch run's bit for bit."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys
import numpy as np
import paper_1607_03252_gb300 as mg
from paper_1607_03252_gb300.workloads import RUN_SEED, sample_ids
out = {}
for name, level, kw in CASES:
    base = dict(n0=17, rtol=1e-10, max_cycles=300)
    base.update(kw)
    cfg = mg.make_mlmc_cfg(RUN_SEED, 1.0, 0.3, 64, **base)
    st, Y, Qf, Qc = mg.mlmc_level_estimate(cfg, level, int(sample_ids(level, 5, 1)[0]), 10)
    out[name] = np.concatenate([Y, Qf, Qc, [st.N, st.mean, st.M2, st.sum, st.mean_cycles_fine]])
np.savez(sys.argv[1], **out)
"""

CASES = """CASES = [
    ("f64_level2", 2, {}),
    ("f64_level0", 0, {}),
    ("mixed_cg_level1", 1, dict(precision=mg.MLMC_PREC_MIXED, accel=mg.MLMC_ACCEL_CG)),
    ("fe_fmg_level1", 1, dict(disc=mg.MLMC_DISC_FE, accel=mg.MLMC_ACCEL_FMG, qoi=mg.MLMC_QOI_POINT, nu1=4, nu2=4,
                              rtol=0.0, max_cycles=2)),
]
"""


def _run(tmp_path, chunks):
    path = tmp_path / ("chunks%d.npz" % chunks)
    env = dict(os.environ, MLMC_LEVEL_CHUNKS=str(chunks))
    code = CHILD.replace("out = {}", CASES + "out = {}")
    res = subprocess.run([sys.executable, "-c", code, str(path)], cwd=ROOT, env=env, capture_output=True, text=True,
                         timeout=900)
    assert res.returncode == 0, res.stdout[-2000:] + res.stderr[-4000:]
    return dict(np.load(path))


def test_chunked_level_batch_equals_one_batch(tmp_path):
    one = _run(tmp_path, 1)
    for chunks in (2, 3):
        got = _run(tmp_path, chunks)
        for name, ref in one.items():
            assert np.array_equal(got[name].view(np.uint64), ref.view(np.uint64)), (chunks, name)
