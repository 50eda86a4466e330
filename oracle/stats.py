"""MLMC estimator statistics from their plain definitions (test infrastructure only).

Sums are exactly rounded (math.fsum), so these are the definitions themselves, not a
compensated approximation of them.
"""
from __future__ import annotations

import math
from typing import Sequence


def level_mean(Y: Sequence[float]) -> float:
    """Y-hat_l = (1/N) sum_i Y_l^i (Sec. 2.2, Algorithm 1's level mean; Eq. 3 on one level)."""
    return math.fsum(Y) / len(Y)


def level_var_biased(Y: Sequence[float]) -> float:
    """s_l^2 = (1/N) sum_i (Y_l^i - Y-hat_l)^2, the normaliser of Sec. 2.3."""
    m = level_mean(Y)
    return math.fsum((y - m) ** 2 for y in Y) / len(Y)


def level_var_unbiased(Y: Sequence[float]) -> float:
    """(1/(N-1)) sum_i (Y_l^i - Y-hat_l)^2."""
    m = level_mean(Y)
    return math.fsum((y - m) ** 2 for y in Y) / (len(Y) - 1)


def mlmc_estimate(level_means: Sequence[float]) -> float:
    """Q-hat_L^ML = sum_l Y-hat_l (Eq. 8)."""
    return math.fsum(level_means)


def eps_split(eps: float, theta: float):
    """eps_s^2 = theta eps^2 and eps_b^2 = (1 - theta) eps^2 (Eq. 6); returns (eps_s, eps_b)."""
    return math.sqrt(theta) * eps, math.sqrt(1.0 - theta) * eps


def optimal_N(V: Sequence[float], C: Sequence[float], eps_s: float) -> list:
    """N_l = eps_s^-2 (sum_k sqrt(V_k C_k)) sqrt(V_l / C_l) (Eq. 11; Eq. 15 with s_l^2 for V_l),
    rounded up to an integer."""
    total = math.fsum(math.sqrt(v * c) for v, c in zip(V, C))
    return [int(math.ceil(total * math.sqrt(v / c) / (eps_s * eps_s))) for v, c in zip(V, C)]


def mlmc_cost(N: Sequence[float], C: Sequence[float]) -> float:
    """Cost = sum_l N_l C_l (Eq. 9)."""
    return math.fsum(n * c for n, c in zip(N, C))


def sampling_variance(V: Sequence[float], N: Sequence[float]) -> float:
    """sum_l V[Y_l] / N_l, the sampling part of the MLMC mean square error (Eq. 10)."""
    return math.fsum(v / n for v, n in zip(V, N))


def bias_bound(Y_hat_L: float, alpha: float) -> float:
    """|E[Q_L - Q]| <= |Y-hat_L| / (8^alpha - 1) (Eq. 14, absolute value taken)."""
    return abs(Y_hat_L) / (8.0 ** alpha - 1.0)


def fit_rate(levels: Sequence[int], values: Sequence[float]) -> float:
    """Rate a of values ~ c 8^(-a l) on a uniformly refined hierarchy (M_l ~ 8^l M_0, so
    |E[Q_l - Q]| ~ M_l^-alpha of Sec. 2.3 gives |Y-hat_l| ~ 8^-alpha l, and Eq. 12's
    V[Y_l] <= C_v M_l^-beta, C_l <= C_c M_l^gamma give the other two): minus the
    least-squares slope of log_8 |value| against l, from the normal equations of the
    line fit with exactly rounded sums. Needs at least two distinct levels."""
    if len(levels) < 2 or len(set(levels)) < 2:
        raise ValueError("a rate needs at least two distinct levels")
    x = [float(l) for l in levels]
    y = [math.log(abs(v)) / math.log(8.0) for v in values]
    n = float(len(x))
    sx, sy = math.fsum(x), math.fsum(y)
    sxx = math.fsum(a * a for a in x)
    sxy = math.fsum(a * b for a, b in zip(x, y))
    slope = (n * sxy - sx * sy) / (n * sxx - sx * sx)
    return -slope
