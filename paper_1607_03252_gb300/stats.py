"""Host-side MLMC bookkeeping of the product path (no GPU work).

  - Chan et al.'s pairwise merge of per-level (N, mean, M2) records, used to combine the
    level statistics of independent replicas (one per GPU) into the estimator's;
  - the sample sizes of Eq. 11 / Eq. 15 (Sec. 2.2-2.3) and the eps split of Eq. 6;
  - the MLMC estimate of Eq. 8 and its sampling variance (Eq. 10);
  - the decay rates alpha, beta, gamma of Eqs. 12 and 14 on a hierarchy with M_l ~ 8^l.
"""
from __future__ import annotations

import math
from typing import Iterable, Sequence

import numpy as np


def chan_merge(records: Iterable[Sequence[float]]):
    """Merge (N, mean, M2) records of disjoint sample sets, in the given order."""
    n, mean, m2 = 0.0, 0.0, 0.0
    for nb, mb, m2b in records:
        if nb == 0:
            continue
        tot = n + nb
        d = mb - mean
        mean = mean + d * nb / tot
        m2 = m2 + m2b + d * d * n * nb / tot
        n = tot
    return n, mean, m2


def merge_levels(per_rank):
    """per_rank: list (ranks) of lists (levels) of (N, mean, M2) -> merged list per level."""
    levels = len(per_rank[0])
    return [chan_merge([r[l] for r in per_rank]) for l in range(levels)]


def eps_split(eps: float, theta: float = 0.5):
    """(eps_s, eps_b) with eps_s^2 = theta eps^2, eps_b^2 = (1 - theta) eps^2 (Eq. 6)."""
    return math.sqrt(theta) * eps, math.sqrt(1.0 - theta) * eps


def sample_sizes(V: Sequence[float], C: Sequence[float], eps_s: float, minimum: int = 2):
    """N_l = ceil(eps_s^-2 (sum_k sqrt(V_k C_k)) sqrt(V_l / C_l)) (Eq. 11 / Eq. 15)."""
    total = sum(math.sqrt(v * c) for v, c in zip(V, C))
    return [max(minimum, int(math.ceil(total * math.sqrt(v / c) / (eps_s * eps_s)))) for v, c in zip(V, C)]


def mlmc_estimate(means: Sequence[float], variances: Sequence[float], N: Sequence[float]):
    """(Q-hat^ML = sum of level means (Eq. 8), its sampling variance sum V_l / N_l (Eq. 10))."""
    return math.fsum(means), math.fsum(v / n for v, n in zip(variances, N))


def fit_rate(levels: Sequence[int], values: Sequence[float]):
    """a in |value_l| ~ c 8^(-a l): minus the slope of the degree-1 least-squares fit of
    log_8 |value| against l; None with fewer than two distinct levels."""
    if len(set(levels)) < 2 or any(v == 0 for v in values):
        return None
    slope = np.polyfit(np.asarray(levels, dtype=np.float64), np.log(np.abs(np.asarray(values, dtype=np.float64)))
                       / math.log(8.0), 1)[0]
    return -float(slope)
