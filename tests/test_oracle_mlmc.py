"""Pins for the oracle's MLMC sample pipeline and estimator statistics.

  - telescoping E[Q_L] = E[Q_0] + sum_l E[Y_l] (Sec. 2.2) holds sample by sample when
    the coarse solve of each pair uses the same realisation as the fine solve;
  - sigma = 0 makes every sample equal, so V[Y_l] = 0 and Q_l is the deterministic solve;
  - V[Y_l] decays with l (Sec. 2.2, below Eq. 10);
  - Eq. 11 on a hand-evaluated case (tests/golden/optimal_nl.json).
"""
import json
import math
import os

import numpy as np
import pytest

from paper_1607_03252_gb300.workloads import RUN_SEED, level_n, sample_ids

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_telescoping_per_sample(orc):
    cfg = orc.make_cfg(RUN_SEED, 1.0, 0.3, 64, rtol=1e-12)
    for i in range(3):
        sid = int(sample_ids(9, i, 1)[0])
        st0, Q0, _, _, _ = orc.sample(cfg, 17, 0, sid)
        st1, Q1f, Q1c, _, _ = orc.sample(cfg, 33, 17, sid)
        st2, Q2f, Q2c, _, _ = orc.sample(cfg, 65, 33, sid)
        assert st0 == st1 == st2 == 0
        # the pair's coarse solve is the previous level's fine solve on the same realisation
        assert Q1c == Q0 and Q2c == Q1f
        Y1, Y2 = Q1f - Q1c, Q2f - Q2c
        assert Q0 + Y1 + Y2 == pytest.approx(Q2f, rel=1e-14)


def test_estimator_telescopes_on_common_seeds(orc):
    cfg = orc.make_cfg(RUN_SEED, 1.0, 0.3, 64, rtol=1e-12)
    ids = sample_ids(9, 100, 16)
    Y0, *_ = orc.level_batch(cfg, 17, 0, ids)
    Y1, *_ = orc.level_batch(cfg, 33, 17, ids)
    Q1, *_ = orc.level_batch(cfg, 33, 0, ids)
    est = orc.stats.mlmc_estimate([orc.stats.level_mean(Y0), orc.stats.level_mean(Y1)])
    assert est == pytest.approx(orc.stats.level_mean(Q1), rel=1e-13)


def test_sigma_zero_all_samples_equal(orc):
    cfg = orc.make_cfg(RUN_SEED, 0.0, 0.3, 32, rtol=1e-12)
    ids = sample_ids(1, 0, 6)
    Y, Qf, Qc, cf, cc, st = orc.level_batch(cfg, 33, 17, ids)
    assert st == 0
    assert np.all(Qf == Qf[0]) and np.all(Qc == Qc[0])
    assert orc.stats.level_var_biased(list(Y)) == 0.0
    u, _, _, _, _ = orc.mg_solve(np.ones((33, 33, 33)), None, rtol=1e-12)
    assert Qf[0] == orc.qoi(u)


def test_level_variance_decays(orc):
    cfg = orc.make_cfg(RUN_SEED, 1.0, 0.3, 256, rtol=1e-10)
    var = []
    for level, n in ((0, 17), (1, 33), (2, 65)):
        nc = level_n(level - 1) if level > 0 else 0
        Y, Qf, Qc, cf, cc, st = orc.level_batch(cfg, n, nc, sample_ids(level, 0, 24))
        assert st == 0
        var.append(orc.stats.level_var_unbiased(list(Y)))
    assert var[1] < var[0] / 4 and var[2] < var[1] / 2, var


def test_optimal_nl_hand_case(orc):
    with open(os.path.join(GOLDEN, "optimal_nl.json")) as fh:
        g = json.load(fh)
    assert orc.stats.optimal_N(g["V"], g["C"], g["eps_s"]) == g["N"]
    # the choice meets the sampling tolerance (Eq. 10 with the equality constraint of Sec. 2.2)
    assert orc.stats.sampling_variance(g["V"], g["N"]) <= g["eps_s"] ** 2


def test_eps_split_and_bias_bound(orc):
    es, eb = orc.stats.eps_split(1e-3, 0.5)
    assert es * es + eb * eb == pytest.approx(1e-6, rel=1e-14)
    assert orc.stats.bias_bound(-0.7, 1.0 / 3.0) == pytest.approx(0.7, rel=1e-14)


def test_statistics_definitions(orc):
    rng = np.random.default_rng(1)
    Y = list(rng.standard_normal(1001) * 1e-3 + 5.0)
    m = orc.stats.level_mean(Y)
    assert m == math.fsum(Y) / len(Y)
    vb = orc.stats.level_var_biased(Y)
    vu = orc.stats.level_var_unbiased(Y)
    assert vu == pytest.approx(vb * len(Y) / (len(Y) - 1), rel=1e-14)
    assert vb == pytest.approx(np.var(np.array(Y)), rel=1e-9)
