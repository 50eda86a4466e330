"""Host logic of the adaptive estimator (Algorithm 2 with level growth, in the library's
mlmc_adaptive_* calls), on the CPU.

The GPU level pipeline is replaced, through the C ABI's sampler hook, by a synthetic
sampler (level l: mean 0.1 * 8^-l, values alternating around it), and the estimator's
decisions -- the number of levels, the sample counts of every round, alpha -- must be
those of the oracle's Algorithm 2 on the same sampler.
"""
import math

import pytest

from oracle import adaptive as oracle_adaptive
from paper_1607_03252_gb300.estimator import MLMCEstimator


def _values(l, first, count):
    m = 0.1 * 8.0 ** (-l)
    s = 0.05 * m if l > 0 else 0.02
    return [m + (s if (first + i) % 2 == 0 else -s) for i in range(count)]


def _sampler(level, first, count):
    y = _values(level, first, count)
    mean = math.fsum(y) / count
    m2 = math.fsum((v - mean) ** 2 for v in y)
    return count, mean, m2


def _est(**kw):
    args = dict(levels=[0, 1], N_init=8, eps=2.5e-4, n0=9, cost_model="nodes", sampler=_sampler)
    args.update(kw)
    return MLMCEstimator(1, 1.0, 0.3, 8, **args)


def _node_cost(n0):
    def cost(l):
        nf = (n0 - 1) * 2 ** l + 1
        nc = (n0 - 1) * 2 ** (l - 1) + 1 if l > 0 else 0
        return float(nf ** 3 + nc ** 3)
    return cost


@pytest.mark.parametrize("alpha,eps", [(None, 2.5e-4), (1.0, 2.5e-4), (1.0 / 3.0, 2.5e-4), (None, 1e-4)])
def test_level_growth_matches_oracle_algorithm(alpha, eps):
    e = _est(eps=eps, max_level=6, alpha=alpha)
    res = e.run(max_rounds=100)
    ref = oracle_adaptive.adaptive_mlmc(_values, _node_cost(9), eps=eps, N_init=8, max_level=6, alpha=alpha)
    assert res["L"] == ref["L"]
    assert res["N"] == ref["N"]
    assert res["rounds"] == ref["rounds"]
    assert res["alpha"] == pytest.approx(ref["alpha"], rel=1e-9)
    assert res["bias_ok"] == ref["bias_ok"]
    assert res["Q_hat"] == pytest.approx(ref["Q_hat"], rel=1e-12)
    assert [entry["levels"][-1] for entry in e.log] == [entry["L"] for entry in ref["log"]]


def test_max_level_cap_and_reported_rates():
    e = _est(max_level=2, alpha=1.0)
    res = e.run()
    assert res["L"] == 2 and not res["bias_ok"]
    alpha, beta, gamma = e.rates()
    assert alpha == 1.0
    # the synthetic variances decay like the means squared (beta = 2 alpha, up to the
    # N / (N - 1) of small counts) and the node costs grow like 8^l (gamma near 1)
    assert beta == pytest.approx(2.0, abs=0.1)
    assert gamma == pytest.approx(1.0, abs=0.1)


def test_fixed_levels_unchanged_without_max_level():
    e = _est(levels=[0, 1, 2], N_init=[8, 8, 8])
    res = e.run()
    assert res["levels"] == [0, 1, 2]


def test_checkpoint_resume_after_growth(tmp_path):
    full = _est(max_level=6)
    full.run()
    part = _est(max_level=6)
    part.step()
    part.step()
    path = tmp_path / "ck.json"
    part.checkpoint(path)
    resumed = MLMCEstimator.restore(path, sampler=_sampler)
    while not resumed.step():
        pass
    assert resumed.levels == full.levels
    assert resumed.have == full.have
    assert resumed.records == full.records


def test_level_growth_arguments_validated():
    with pytest.raises(ValueError):
        MLMCEstimator(1, 1.0, 0.3, 8, levels=[1, 2], N_init=8, eps=1e-3, max_level=4)
    with pytest.raises(ValueError):
        MLMCEstimator(1, 1.0, 0.3, 8, levels=[0, 1, 2], N_init=[8, 8], eps=1e-3)
    import paper_1607_03252_gb300 as mg

    for bad in (dict(eps=-1.0), dict(theta=1.0), dict(alpha0=0.0)):
        with pytest.raises(mg.MlmcError):
            _est(**bad)


def test_state_rejected_by_another_configuration(tmp_path):
    import paper_1607_03252_gb300 as mg

    e = _est(max_level=6)
    e.step()
    e.step()
    st = e.state()
    st["params"]["max_level"] = None  # a fixed-level run cannot take a grown state
    with pytest.raises(mg.MlmcError):
        MLMCEstimator.from_state(st, sampler=_sampler)


def test_sampler_error_is_reported():
    import paper_1607_03252_gb300 as mg

    def broken(level, first, count):
        raise RuntimeError("no samples")

    e = _est(sampler=broken)
    with pytest.raises(mg.MlmcError) as ex:
        e.step()
    assert ex.value.status == mg.MLMC_ERR_INVALID
