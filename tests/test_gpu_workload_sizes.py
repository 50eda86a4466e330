"""GPU parity at the largest sizes the workloads run, against values the FP64 oracle
computed for the same realisations (tests/golden/workload_sizes.json, written by
tests/golden/make_workload_golden.py, which calls only the oracle):

  - the mixed-precision 5-level workload's finest level: 257^3 fine / 129^3 coarse,
    sigma^2 = 2, ell = 0.1, M = 256;
  - the large adaptive workload's finest level: 513^3 fine / 257^3 coarse, sigma^2 = 1,
    ell = 0.05, M = 1024;

each solved as the benchmark solves it -- mixed precision, flexible CG around the FP32
V-cycle, the smoother and sweep count chosen by the autotuner for that level, a batch of
two realisations -- to the relative residual the oracle's values were computed with
(1e-11 at 257^3, 1e-10 at 513^3: just above the FP64 rounding floor of those grids). Bar:
Qf, Qc within 1e-9 relative and |dY| <= 1e-9 max(|Qf|, |Qc|) of the oracle, with the error
printed ("mixed vs FP64").
"""
import json
import os

import numpy as np
import pytest

import paper_1607_03252_gb300 as mg
from paper_1607_03252_gb300.workloads import RUN_SEED

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "workload_sizes.json")


def _cases():
    with open(GOLDEN) as fh:
        g = json.load(fh)
    assert g["run_seed"] == RUN_SEED
    return g["cases"]


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c["name"])
def test_largest_levels_match_oracle(case):
    level, sid = case["level"], int(case["sample_id"])
    cfg = mg.make_mlmc_cfg(RUN_SEED, case["sigma2"], case["ell"], case["M"], n0=17, nu1=0, nu2=0, rtol=case["rtol"],
                           max_cycles=300, precision=mg.MLMC_PREC_MIXED, accel=mg.MLMC_ACCEL_CG, max_batch=2)
    # the benchmark's plan: smoother and nu tuned for this level on tuning-only ids
    rows, best, nu = mg.mlmc_autotune(cfg, level, sid + (1 << 40), 2)
    stats, Y, Qf, Qc = mg.mlmc_level_estimate(cfg, level, sid, 2)
    err_y = abs(Y[0] - case["Y"]) / max(abs(case["Qf"]), abs(case["Qc"]))
    err_qf = abs(Qf[0] - case["Qf"]) / abs(case["Qf"])
    err_qc = abs(Qc[0] - case["Qc"]) / abs(case["Qc"])
    print("mixed vs FP64 (%s, %d^3/%d^3, smoother %s nu %d, cycles %.0f/%.0f): |dY|/max|Q| %.1e, dQf %.1e, dQc %.1e"
          % (case["name"], case["n_fine"], case["n_coarse"], mg._capi.SMOOTHER_NAMES.get(best, best), nu,
             stats.mean_cycles_fine, stats.mean_cycles_coarse, err_y, err_qf, err_qc))
    assert err_qf <= 1e-9 and err_qc <= 1e-9
    assert err_y <= 1e-9
    assert np.isfinite(Y[1]) and abs(Y[1]) < 10 * max(abs(case["Qf"]), abs(case["Qc"]))
