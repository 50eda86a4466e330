"""Level-record bookkeeping of the product path, through the library's host-only calls.

  - chan_merge / merge_levels: Chan et al.'s pairwise merge of (N, mean, M2) records of
    disjoint sample sets (mlmc_merge_records), used to combine the level statistics of
    replicas (one per GPU), level lanes and sample chunks;
  - sample_sizes: N_l of Eq. 11 / Eq. 15 for the eps split of Eq. 6 (mlmc_sample_sizes).

The arithmetic runs in libmlmc_gb300.so; this module only marshals arguments.
"""
from __future__ import annotations

import ctypes
from typing import Iterable, Sequence

from . import _capi


def chan_merge(records: Iterable[Sequence[float]]):
    """Merge (N, mean, M2) records of disjoint sample sets, in the given order."""
    recs = [float(x) for r in records for x in r]
    arr = (ctypes.c_double * max(len(recs), 1))(*recs)
    out = (ctypes.c_double * 3)()
    _capi._check(_capi.lib().mlmc_merge_records(arr, len(recs) // 3, out), "mlmc_merge_records")
    return out[0], out[1], out[2]


def merge_levels(per_rank):
    """per_rank: list (ranks) of lists (levels) of (N, mean, M2) -> merged list per level."""
    levels = len(per_rank[0])
    return [chan_merge([r[l] for r in per_rank]) for l in range(levels)]


def sample_sizes(V: Sequence[float], C: Sequence[float], eps: float, theta: float = 0.5):
    """N_l = ceil(eps_s^-2 (sum_k sqrt(V_k C_k)) sqrt(V_l / C_l)), at least 2, eps_s^2 =
    theta eps^2 (Eqs. 6, 11, 15)."""
    n = len(V)
    v = (ctypes.c_double * n)(*[float(x) for x in V])
    c = (ctypes.c_double * n)(*[float(x) for x in C])
    out = (ctypes.c_int64 * n)()
    _capi._check(_capi.lib().mlmc_sample_sizes(v, c, n, float(eps), float(theta), out), "mlmc_sample_sizes")
    return [int(x) for x in out]
