"""Adaptive multilevel Monte Carlo, Algorithm 2 of Sec. 2.4 (test infrastructure only).

A plain restatement of the algorithm's steps in the paper's order, on top of any sampler
of the level differences:

  1. L = 1, N_0 = N_1 = N_init;
  2. on every level l = 0..L compute new samples of Y_l until there are N_l, then the
     sample mean Y-hat_l, the sample variance s_l^2 and the cost per sample C_l;
  3. re-estimate N_l by Eq. 15 for eps_s^2 = theta eps^2 (Eq. 6), and if the bias estimate
     of Eq. 14 says the bias is above eps_b, i.e. |Y-hat_L| > (8^alpha - 1) eps_b, add a
     level with N_L = N_init;
  4. stop when no N_l and not L changed, else return to 2;
  5. Q-hat = sum of the level means (Eq. 8).

Readings (the paper leaves them open): samples already computed are kept, so N_l never
decreases, and N_l is at least 2; the bias test takes |Y-hat_L| (the paper's inequality
has no absolute value); s_l^2 uses the 1/(N-1) normaliser; alpha is either given or fitted
online by `stats.fit_rate` over the levels l >= 1 that have samples (with fewer than two
such levels, `alpha0`), and never taken below `alpha_floor`; a level beyond `max_level`
is never added (the result then says that the bias test failed).
"""
from __future__ import annotations

import math
from typing import Callable, List, Optional

from . import stats


def adaptive_mlmc(sample_Y: Callable[[int, int, int], List[float]], cost: Callable[[int], float], eps: float,
                  N_init: int, max_level: int, theta: float = 0.5, alpha: Optional[float] = None,
                  alpha0: float = 2.0 / 3.0, alpha_floor: float = 0.1, max_rounds: int = 100) -> dict:
    """sample_Y(l, first, count) returns Y_l for the sample indices first .. first+count-1
    of level l; cost(l) is C_l. Returns the estimate and the run's decisions."""
    eps_s, eps_b = stats.eps_split(eps, theta)
    L = 1
    N = [N_init, N_init]
    Y: List[List[float]] = [[], []]
    log = []
    for rnd in range(1, max_rounds + 1):
        # step 2
        for l in range(L + 1):
            if len(Y[l]) < N[l]:
                Y[l] = Y[l] + list(sample_Y(l, len(Y[l]), N[l] - len(Y[l])))
        means = [stats.level_mean(Y[l]) for l in range(L + 1)]
        s2 = [stats.level_var_unbiased(Y[l]) for l in range(L + 1)]
        C = [float(cost(l)) for l in range(L + 1)]
        # new sample sizes by Eq. 15, then the bias test of Eq. 14
        N_opt = stats.optimal_N([max(v, 1e-30) for v in s2], C, eps_s)
        N_new = [max(N[l], max(2, N_opt[l])) for l in range(L + 1)]
        a = _alpha(alpha, alpha0, alpha_floor, means)
        bias = abs(means[L]) / (8.0 ** a - 1.0)
        grow = bias > eps_b and L < max_level
        log.append({"round": rnd, "L": L, "N": list(N), "N_next": list(N_new), "alpha": a, "bias": bias})
        if grow:
            L += 1
            N_new.append(N_init)
            Y.append([])
        # stop when nothing changes
        if not grow and N_new == N:
            break
        N = N_new
    means = [stats.level_mean(Y[l]) for l in range(L + 1)]
    s2 = [stats.level_var_unbiased(Y[l]) for l in range(L + 1)]
    a = _alpha(alpha, alpha0, alpha_floor, means)
    return {
        "Q_hat": stats.mlmc_estimate(means),  # step 5, Eq. 8
        "L": L,
        "N": [len(y) for y in Y],
        "level_means": means,
        "level_vars": s2,
        "sampling_var": stats.sampling_variance(s2, [len(y) for y in Y]),
        "eps_s2": eps_s * eps_s,
        "alpha": a,
        "bias": abs(means[L]) / (8.0 ** a - 1.0),
        "bias_ok": abs(means[L]) / (8.0 ** a - 1.0) <= eps_b,
        "rounds": len(log),
        "log": log,
    }


def _alpha(alpha, alpha0, alpha_floor, means):
    if alpha is not None:
        return float(alpha)
    ls = list(range(1, len(means)))
    if len(ls) < 2:
        return max(alpha0, alpha_floor)
    return max(stats.fit_rate(ls, [means[l] for l in ls]), alpha_floor)
