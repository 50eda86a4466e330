"""Pins for the oracle's rate fit and its Algorithm 2 (adaptive MLMC with level growth).

The samplers here are synthetic: level l has mean m_l = 0.1 * 8^-l (so the bias ratio per
level is 8, alpha = 1) and the values m_l + s_l, m_l - s_l, m_l + s_l, ... The level counts
L that Algorithm 2 must reach are worked out by hand below; each of the plausible slips
(eps instead of eps_b, a wrong alpha, no absolute value) changes one of them.
"""
import math

import numpy as np
import pytest

from oracle import adaptive, stats


def test_fit_rate_exact_geometric():
    for a, c in ((1.0, 0.1), (2.0 / 3.0, -3e-2), (1.5, 7.0), (0.25, 1e-6)):
        ls = [1, 2, 3, 4]
        assert stats.fit_rate(ls, [c * 8.0 ** (-a * l) for l in ls]) == pytest.approx(a, abs=1e-12)


def test_fit_rate_matches_polyfit_on_noisy_data():
    rng = np.random.default_rng(5)
    ls = [1, 2, 3, 5]
    v = [0.3 * 8.0 ** (-0.7 * l) * math.exp(0.3 * rng.standard_normal()) for l in ls]
    slope = np.polyfit(ls, np.log(np.abs(v)) / np.log(8.0), 1)[0]
    assert stats.fit_rate(ls, v) == pytest.approx(-slope, abs=1e-12)


def test_fit_rate_needs_two_levels():
    with pytest.raises(ValueError):
        stats.fit_rate([2], [1.0])
    with pytest.raises(ValueError):
        stats.fit_rate([2, 2], [1.0, 0.5])


def _sampler(sign=1.0, s_rel=0.05):
    calls = []

    def sample_Y(l, first, count):
        calls.append((l, first, count))
        m = sign * 0.1 * 8.0 ** (-l)
        s = s_rel * abs(m) if l > 0 else 0.02
        return [m + (s if (first + i) % 2 == 0 else -s) for i in range(count)]

    return sample_Y, calls


def _cost(l):
    return 8.0 ** l


def test_level_growth_hand_worked():
    """eps = 2.5e-4, theta = 1/2: eps_b = 1.7678e-4, and with alpha = 1 the test bound is
    (8 - 1) eps_b = 1.2374e-3. |Y_1| = 1.25e-2 and |Y_2| = 1.5625e-3 exceed it, |Y_3| =
    1.953e-4 does not: L = 3. Against eps itself (7 eps = 1.75e-3) the run would stop at
    L = 2."""
    sample_Y, _ = _sampler()
    res = adaptive.adaptive_mlmc(sample_Y, _cost, eps=2.5e-4, N_init=8, max_level=6, alpha=1.0)
    assert res["L"] == 3
    assert res["bias_ok"]
    assert [e["L"] for e in res["log"]][:3] == [1, 2, 3]


def test_level_growth_depends_on_alpha():
    """alpha = 1/3: the bound is (8^(1/3) - 1) eps_b = eps_b = 1.7678e-4, which |Y_3| =
    1.953e-4 still exceeds: L = 4 (|Y_4| = 2.44e-5)."""
    sample_Y, _ = _sampler()
    res = adaptive.adaptive_mlmc(sample_Y, _cost, eps=2.5e-4, N_init=8, max_level=6, alpha=1.0 / 3.0)
    assert res["L"] == 4


def test_level_growth_with_fitted_alpha_and_negative_means():
    """The fit over l >= 1 recovers alpha = 1 from the means (to the sampling noise), and
    the test uses |Y_L|: negative means give the same levels."""
    for sign in (1.0, -1.0):
        sample_Y, _ = _sampler(sign=sign)
        res = adaptive.adaptive_mlmc(sample_Y, _cost, eps=2.5e-4, N_init=8, max_level=6)
        assert res["L"] == 3
        assert res["alpha"] == pytest.approx(1.0, abs=0.01)


def test_max_level_caps_growth():
    sample_Y, _ = _sampler()
    res = adaptive.adaptive_mlmc(sample_Y, _cost, eps=2.5e-4, N_init=8, max_level=2, alpha=1.0)
    assert res["L"] == 2 and not res["bias_ok"]


def test_stopping_invariants_and_lagrange_conditions():
    """At the stop the sampling variance of Eq. 10 is within eps_s^2, and the counts are
    the constrained minimisers of Eq. 9: N_l sqrt(C_l / V_l) is the same on every level
    (the Lagrange condition), up to the rounding up of each N_l."""
    sample_Y, calls = _sampler()
    eps = 2.5e-4
    res = adaptive.adaptive_mlmc(sample_Y, _cost, eps=eps, N_init=8, max_level=6, alpha=1.0)
    V, N = res["level_vars"], res["N"]
    assert res["sampling_var"] <= res["eps_s2"]
    assert res["sampling_var"] >= 0.8 * res["eps_s2"]
    ratios = [n * math.sqrt(_cost(l) / v) for l, (n, v) in enumerate(zip(N, V)) if n > 8]
    assert len(ratios) >= 2
    assert max(ratios) / min(ratios) < 1.05
    # samples are never recomputed: each level's calls tile 0 .. N_l - 1 in order
    for l in range(res["L"] + 1):
        starts = [(f, c) for (ll, f, c) in calls if ll == l]
        pos = 0
        for f, c in starts:
            assert f == pos
            pos += c
        assert pos == N[l]
    assert res["Q_hat"] == pytest.approx(sum(0.1 * 8.0 ** (-l) for l in range(res["L"] + 1)), rel=1e-6)


def test_small_eps_stops_with_fixed_point():
    """The loop ends on a round that changes neither N nor L: its log entry proposes
    exactly the counts the run holds."""
    sample_Y, _ = _sampler()
    res = adaptive.adaptive_mlmc(sample_Y, _cost, eps=1e-4, N_init=16, max_level=8)
    last = res["log"][-1]
    assert last["N_next"] == res["N"]
    assert res["bias_ok"]
