"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds no arithmetic of the method: only seeds, sample ids, grid sizes and
the configuration parameters of the six workloads, plus seeded random arrays used
as inputs to the batched solver. Both the CUDA path and the CPU oracle receive the
same values from here; neither side's computation lives here.

Grid sizes follow the uniform refinement h_l = 2^-l h_0 of Sec. 2 (n_l = 2^(l+4) + 1
nodes per axis, so level 0 is 17^3 and level 5 is 513^3). Sample ids give every MLMC
level its own stream of realisations (independent samples across levels, Sec. 2.2,
below Eq. 9); the fine and coarse solve of one Y_l share one id (Algorithm 1).
"""
from __future__ import annotations

import numpy as np

RUN_SEED = 1607032520


def level_n(level: int) -> int:
    """Nodes per axis of MLMC level `level` (17, 33, 65, 129, 257, 513 for 0..5)."""
    return 2 ** (level + 4) + 1


def sample_id(level: int, i: int) -> int:
    """Realisation id of sample i on MLMC level `level`: (level << 48) | i."""
    return (int(level) << 48) | int(i)


def sample_ids(level: int, first: int, count: int) -> np.ndarray:
    return np.array([sample_id(level, first + i) for i in range(count)], dtype=np.uint64)


# The five workloads (unit cube, homogeneous Dirichlet data, f = 1, V(2,2) red-black
# Gauss-Seidel, full weighting, trilinear prolongation, QoI = mean of u over [0.25,0.75]^3).
CONFIGS = {
    # single-level plain MC at 33^3, FP64
    "c1": dict(name="c1_mc_33", levels=[1], single_level=True, N=[64], sigma2=1.0, ell=0.3, M=256,
               precision="f64", rtol=1e-10, nu1=2, nu2=2),
    # plain 4-level MLMC, FP64, batched
    "c2": dict(name="c2_mlmc4_f64", levels=[0, 1, 2, 3], single_level=False, N=[4096, 1024, 256, 64],
               sigma2=1.0, ell=0.3, M=256, precision="f64", rtol=1e-10, nu1=2, nu2=2),
    # mixed-precision 5-level MLMC; N_l from Eq. 11 for eps = 1e-3 after a pilot
    "c3": dict(name="c3_mlmc5_mixed", levels=[0, 1, 2, 3, 4], single_level=False, N_init=[1024, 256, 64, 16, 16],
               eps=1e-3, theta=0.5, sigma2=2.0, ell=0.1, M=256, precision="mixed", accel="cg", rtol=1e-10,
               nu1=2, nu2=2),
    # serving: Poisson single-sample requests over levels 0..4 (C3's field)
    "c4": dict(name="c4_serving", levels=[0, 1, 2, 3, 4], sigma2=2.0, ell=0.1, M=256, precision="mixed",
               rtol=1e-10, nu1=2, nu2=2),
    # the paper's static 4-level run (Sec. 7.1: P1 elements, one FMG-2V(4,4) cycle per solve,
    # the point QoI, N = (4123, 688, 108, 16)) on 17^3..129^3, exponential covariance with
    # a correlation length of ~20 finest-grid spacings, as in the paper
    "c6": dict(name="c6_e9_fe_fmg", levels=[0, 1, 2, 3], single_level=False, N=[4123, 688, 108, 16],
               sigma2=1.0, ell=0.15, M=256, cov="exp", precision="f64", disc="fe", accel="fmg", qoi="point",
               nu1=4, nu2=4, cycles=2, rtol=0.0),
    # 6-level adaptive MLMC to RMS tolerance 2e-4
    "c5": dict(name="c5_mlmc6_adaptive", levels=[0, 1, 2, 3, 4, 5], single_level=False,
               N_init=[256, 64, 16, 8, 4, 2], eps=2e-4, theta=0.5, sigma2=1.0, ell=0.05, M=1024,
               precision="mixed", rtol=1e-10, nu1=2, nu2=2),
}


def random_coefficient(n: int, seed: int, sigma: float = 1.0) -> np.ndarray:
    """Nodal coefficient exp(sigma * g), g i.i.d. standard normal per node: a rough
    positive input for the batched solver (shape (n, n, n), [z, y, x])."""
    rng = np.random.default_rng(seed)
    return np.exp(sigma * rng.standard_normal((n, n, n)))


def random_rhs(n: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, size=(n, n, n))


def poisson_arrivals(rate_per_s: float, count: int, seed: int) -> np.ndarray:
    """Arrival times (s) of an open-loop Poisson stream."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=count))


def level_draws(probs, count: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    p = np.asarray(probs, dtype=np.float64)
    return rng.choice(len(p), size=count, p=p / p.sum())
