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
    est.add_samples(1, 8)
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
