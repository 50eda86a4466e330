"""Adaptive estimator on the GPU: checkpoint / resume reproduces an uninterrupted run."""
import json

import pytest

import paper_1607_03252_gb300 as mg
from paper_1607_03252_gb300.estimator import MLMCEstimator
from paper_1607_03252_gb300.workloads import RUN_SEED

pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _est():
    # the node-count cost model makes the N_l sequence deterministic (measured wall times vary)
    return MLMCEstimator(RUN_SEED, 1.0, 0.3, 32, levels=[0, 1, 2], N_init=[32, 8, 4], eps=2e-3, n0=9, rtol=1e-10,
                         cost_model="nodes")


def test_resume_equals_uninterrupted(tmp_path):
    full = _est()
    full.run()
    part = _est()
    part.step()
    path = tmp_path / "ckpt.json"
    part.checkpoint(path)
    resumed = MLMCEstimator.restore(path)
    # continue where the checkpoint left off: the same ids and the same records
    while not resumed.step():
        pass
    assert resumed.have == full.have
    assert resumed.records == full.records
    res = resumed.result()
    assert res["sampling_var"] <= res["eps_s2"] * 1.0000001
    json.dumps(resumed.state())  # JSON-serialisable


def test_estimator_level_records_match_batch_call():
    est = _est()
    est.step()  # the pilot round: 8 samples of level 1, ids (1 << 48) + 0 .. 7
    cfg = mg.make_mlmc_cfg(RUN_SEED, 1.0, 0.3, 32, n0=9, rtol=1e-10)
    st, Y, _, _ = mg.mlmc_level_estimate(cfg, 1, (1 << 48), 8)
    n, mean, m2 = est.records[1]
    assert n == 8 and mean == st.mean and m2 == st.M2


def test_concurrent_level_lanes_give_the_same_records():
    """Levels of a round on two streams from two host threads: the same ids, records and
    sample counts as the levels in sequence."""
    import torch

    seq = _est()
    seq.run()
    s0, s1 = torch.cuda.Stream(), torch.cuda.Stream()
    par = MLMCEstimator(RUN_SEED, 1.0, 0.3, 32, levels=[0, 1, 2], N_init=[32, 8, 4], eps=2e-3, n0=9, rtol=1e-10,
                        cost_model="nodes", stream=s0, streams=[s0, s1])
    par.run()
    assert par.have == seq.have
    assert par.records == seq.records


def test_level_growth_matches_oracle_algorithm(orc):
    """Algorithm 2 with level growth on real samples (17^3 .. 65^3 hierarchy from n0 = 9,
    sigma^2 = 1, ell = 0.3): the same levels, counts, fitted alpha and estimate as the
    oracle's Algorithm 2 over the oracle's samples with the same ids. eps = 2e-4 makes the
    bias test add level 2 (|Y_1| ~ 6.5e-4 > 3 eps_b) and stop there (|Y_2| ~ 1.7e-4)."""
    import numpy as np

    from oracle import adaptive
    from paper_1607_03252_gb300.workloads import sample_id

    kw = dict(eps=2e-4, N_init=64, max_level=4)
    e = MLMCEstimator(RUN_SEED, 1.0, 0.3, 32, levels=[0, 1], n0=9, rtol=1e-12, cost_model="nodes", **kw)
    res = e.run()
    ocfg = orc.make_cfg(RUN_SEED, 1.0, 0.3, 32, rtol=1e-12)

    def n_of(l):
        return 8 * 2 ** l + 1

    def sample_Y(l, first, count):
        ids = np.array([sample_id(l, first + i) for i in range(count)], dtype=np.uint64)
        Y, *_, st = orc.level_batch(ocfg, n_of(l), n_of(l - 1) if l > 0 else 0, ids)
        assert st == 0
        return list(Y)

    ref = adaptive.adaptive_mlmc(sample_Y, lambda l: float(n_of(l) ** 3 + (n_of(l - 1) ** 3 if l > 0 else 0)), **kw)
    assert res["L"] == ref["L"] == 2
    assert res["N"] == ref["N"]
    assert res["rounds"] == ref["rounds"]
    assert res["alpha"] == pytest.approx(ref["alpha"], rel=1e-6)
    assert res["bias_ok"] and ref["bias_ok"]
    # Y_l agree to 1e-9 of Q per sample, so the means and the estimate do too
    assert res["Q_hat"] == pytest.approx(ref["Q_hat"], abs=1e-9 * 0.05)
    for a, b in zip(res["level_vars"], ref["level_vars"]):
        assert a == pytest.approx(b, rel=1e-6)
