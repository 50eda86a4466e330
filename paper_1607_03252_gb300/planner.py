"""Host planner of MLMC work: the paper's performance model and scheduling strategies
(Secs. 4-5), and their one-GPU form, the lane plan of a step.

The paper distributes the samples of each level over processor blocks of a cluster:
a sample of level l runs on 2^(3l + theta) P0_min processors, theta in 0..S (the solver's
scalability window). This module restates, from the paper's definitions:

  - the Amdahl surrogate of the strong-scaling time and efficiency (Eq. amdahls):
    t_{l,theta} = t_{l,0} (B + 2^-theta (1 - B)), Eff(theta) = 1 / (2^theta B + 1 - B);
  - blocks, sequential steps and load imbalance of a level (Eq. seqsteps) and the level
    efficiency eta = (1 - Imb) Eff (Eq. effs); the optimal mean run-time (Eq. optruntime);
  - the homogeneous strategies: theta_l minimising k_seq(theta) t_{l,theta} per level
    (SaSyHom / LeSyHom, Sec. 5.1), the run-time robust choice from a run-time histogram
    (RuRoHom, Eq. maxrsM, Sec. 5.2), and the dynamic assignment of samples to blocks
    (DyLeSyHom, Sec. 5.3);
  - the heterogeneous bulk-synchronous schedule (Sec. 5.4): the proportional start of
    Eq. simpleestimation and the minimal run-time over N_{l,theta} >= 0 with sum_theta
    N_{l,theta} k_{l,theta} >= N_l and at most P_max processors. The paper searches that
    space with simulated annealing; here it is solved exactly: the run-time is one of the
    values t_{l,theta} k, and for a candidate T each level's cheapest cover of its N_l
    samples by blocks (each theta-block finishing floor(T / t_{l,theta}) samples on
    2^(3l+theta) P0_min processors) is a small unbounded-knapsack minimisation.

On one GPU the processor blocks are CUDA streams fed by host threads (lanes) and the block
size is a batch of samples; `lane_plan` assigns a step's levels (split into sample chunks
when one level exceeds a lane's share) longest first to the least-loaded lane, the
dynamic variant's greedy rule with measured per-level times (the step's bench path uses
it).
"""
from __future__ import annotations

import heapq
import math
import random
from typing import List, Sequence


# ---- performance model (Sec. 4.1) ------------------------------------------------------
def amdahl_time(t0: float, B: float, theta: int) -> float:
    """t_{l,theta} = t_{l,0} (B + 2^-theta (1 - B))."""
    return t0 * (B + (1.0 - B) / (1 << theta))


def amdahl_efficiency(B: float, theta: int) -> float:
    """Eff(theta) = t_{l,0} / (2^theta t_{l,theta}) = 1 / (2^theta B + 1 - B)."""
    return 1.0 / ((1 << theta) * B + 1.0 - B)


def blocks(l: int, theta: int, P_max: int, P0_min: int) -> int:
    """J_l(theta): samples of level l computed at once on 2^(3l+theta) P0_min processors each."""
    return P_max // ((1 << (3 * l + theta)) * P0_min)


def seq_steps(N_l: int, l: int, theta: int, P_max: int, P0_min: int):
    """(J_l, k_seq, Imb_l) of Eq. seqsteps; J_l = 0 (the level does not fit) gives k = inf."""
    J = blocks(l, theta, P_max, P0_min)
    if J == 0:
        return 0, math.inf, 1.0
    k = -(-N_l // J)
    imb = 1.0 - ((1 << (3 * l + theta)) * P0_min * N_l) / (k * P_max)
    return J, k, imb


def level_efficiency(N_l: int, l: int, theta: int, P_max: int, P0_min: int, B: float) -> float:
    """eta_l(theta) = (1 - Imb_l(theta)) Eff_l(theta) (Eq. effs)."""
    _, _, imb = seq_steps(N_l, l, theta, P_max, P0_min)
    return (1.0 - imb) * amdahl_efficiency(B, theta)


def optimal_runtime(N: Sequence[int], t0: Sequence[float], EC: Sequence[float], P_max: int, P0_min: int) -> float:
    """t_mlmc^opt = (P0_min / P_max) sum_l N_l 2^(3l) E[C_{l,0}] t_{l,0} (Eq. optruntime)."""
    return P0_min / P_max * math.fsum(n * (1 << (3 * l)) * c * t for l, (n, c, t) in enumerate(zip(N, EC, t0)))


# ---- homogeneous strategies (Secs. 5.1-5.3) ------------------------------------------------
def theta_homogeneous(N_l: int, l: int, S: int, P_max: int, P0_min: int, t_row=None, B=None) -> int:
    """The largest theta in 0..S minimising k_seq(theta) t_{l,theta} (SaSyHom / LeSyHom);
    t_{l,theta} from measured times t_row, else the Amdahl surrogate with serial fraction B."""
    best, arg = math.inf, 0
    for th in range(S + 1):
        _, k, _ = seq_steps(N_l, l, th, P_max, P0_min)
        t = t_row[th] if t_row is not None else (B + (1.0 - B) / (1 << th))
        v = k * t
        if v <= best * (1 + 1e-12):
            best, arg = min(best, v), th
    return arg


def expected_level_time(N_l: int, l: int, theta: int, P_max: int, P0_min: int, t_theta: float,
                        histogram: Sequence[float], mu: int, rng: random.Random) -> float:
    """E-hat_{l,theta}(mu) of Eq. maxrsM: the mean over mu draws of the slowest block's sum
    of k_seq cost factors, times t_{l,theta}; a cost factor is a run-time of the level-0
    histogram drawn uniformly, normalised by the histogram's mean."""
    J, k, _ = seq_steps(N_l, l, theta, P_max, P0_min)
    if J == 0:
        return math.inf
    K = len(histogram)
    mean = math.fsum(histogram) / K
    total = 0.0
    for _ in range(mu):
        slowest = 0.0
        for _ in range(J):
            s = 0.0
            for _ in range(k):
                s += histogram[rng.randrange(K)] / mean
            slowest = max(slowest, s)
        total += slowest
    return total / mu * t_theta


def theta_runtime_robust(N_l: int, l: int, S: int, P_max: int, P0_min: int, histogram: Sequence[float],
                         t_row=None, B=None, seed: int = 0, mu0: int = 8, mu_max: int = 512) -> int:
    """RuRoHom: theta minimising E-hat_{l,theta}(mu), mu doubled until mu and mu/2 agree."""

    def choose(mu):
        rng = random.Random(seed)
        vals = []
        for th in range(S + 1):
            t = t_row[th] if t_row is not None else (B + (1.0 - B) / (1 << th))
            vals.append(expected_level_time(N_l, l, th, P_max, P0_min, t, histogram, mu, rng))
        return min(range(S + 1), key=lambda th: vals[th])

    mu, prev = mu0, choose(mu0 // 2 if mu0 > 1 else 1)
    while True:
        cur = choose(mu)
        if cur == prev or mu >= mu_max:
            return cur
        prev, mu = cur, 2 * mu


def sync_makespan(times: Sequence[float], J: int) -> float:
    """SaSyHom: the samples run in steps of J at a time with a synchronisation after each
    step; the run-time is the sum over the steps of the slowest sample of the step."""
    return math.fsum(max(times[i:i + J]) for i in range(0, len(times), J))


def static_makespan(times: Sequence[float], J: int) -> float:
    """LeSyHom without synchronisation: block j runs samples j, j + J, j + 2J, ... back to back."""
    return max(math.fsum(times[j::J]) for j in range(min(J, len(times))))


def dynamic_makespan(times: Sequence[float], J: int) -> float:
    """DyLeSyHom: the next sample goes to the first block that becomes free."""
    free = [0.0] * min(J, len(times))
    heapq.heapify(free)
    end = 0.0
    for t in times:
        start = heapq.heappop(free)
        heapq.heappush(free, start + t)
        end = max(end, start + t)
    return end


# ---- heterogeneous bulk-synchronous schedule (Sec. 5.4) ----------------------------------------
def hetero_simple(N: Sequence[int], t0: Sequence[float], P_max: int, P0_min: int):
    """Eq. simpleestimation: N_{l,0} = floor(P_max N_l t_{l,0} / sum_i N_i 2^(3i) P0_min t_{i,0});
    returns (N_{l,0}, run-time max_l t_{l,0} ceil(N_l / N_{l,0}), processors)."""
    den = math.fsum(n * (1 << (3 * i)) * P0_min * t for i, (n, t) in enumerate(zip(N, t0)))
    Nl0 = [max(1, int(math.floor(P_max * n * t / den))) for n, t in zip(N, t0)]
    run = max(t * -(-n // m) for n, t, m in zip(N, t0, Nl0))
    procs = sum(m * (1 << (3 * l)) * P0_min for l, m in enumerate(Nl0))
    return Nl0, run, procs


def _level_cover(N_l: int, l: int, T: float, t_row: Sequence[float], P0_min: int):
    """Cheapest processor count covering N_l samples by theta-blocks within time T, and
    the block counts per theta (unbounded knapsack over the samples still to cover)."""
    opts = []
    for th, t in enumerate(t_row):
        k = int(math.floor(T / t * (1 + 1e-12)))
        if k > 0:
            opts.append((th, k, (1 << (3 * l + th)) * P0_min))
    if not opts:
        return math.inf, None
    INF = math.inf
    cost = [0] + [INF] * N_l
    pick = [None] * (N_l + 1)
    for s in range(1, N_l + 1):
        for th, k, c in opts:
            v = cost[max(0, s - k)] + c
            if v < cost[s]:
                cost[s], pick[s] = v, (th, k)
    counts = [0] * len(t_row)
    s = N_l
    while s > 0:
        th, k = pick[s]
        counts[th] += 1
        s = max(0, s - k)
    return cost[N_l], counts


def hetero_exact(N: Sequence[int], t: Sequence[Sequence[float]], P_max: int, P0_min: int):
    """The minimal bulk-synchronous run-time over N_{l,theta} (t[l][theta], theta in
    0..S = len(t[l]) - 1) with at most P_max processors, and at that run-time the
    allocation using the fewest processors: returns (T, N_{l,theta} lists, processors)."""
    cands = sorted({tt * k for l, row in enumerate(t) for tt in row
                    for k in range(1, int(N[l]) + 1)})
    lo, hi = 0, len(cands) - 1
    # the total cover cost falls as T grows: bisection for the first feasible candidate

    def total(T):
        tot, alloc = 0, []
        for l, row in enumerate(t):
            c, counts = _level_cover(int(N[l]), l, T, row, P0_min)
            tot += c
            alloc.append(counts)
        return tot, alloc

    if total(cands[hi])[0] > P_max:
        raise ValueError("no schedule fits P_max processors")
    while lo < hi:
        mid = (lo + hi) // 2
        if total(cands[mid])[0] <= P_max:
            hi = mid
        else:
            lo = mid + 1
    T = cands[lo]
    procs, alloc = total(T)
    return T, alloc, procs


# ---- the one-GPU form: lanes of a step -----------------------------------------------------
def lane_plan(levels: Sequence[int], N: Sequence[int], times, lanes: int) -> List[list]:
    """Work items (level, first, last) of one step on `lanes` concurrent streams: a level
    whose measured time exceeds the per-lane share is split into sample chunks (a sample's
    result does not depend on its batch); items go longest first onto the least-loaded
    lane. Returns a list of lanes, each a list of (level, first, last)."""
    lanes = max(1, lanes)
    total = sum(times[l] for l in levels)
    share = total / lanes
    items = []
    for l, n in zip(levels, N):
        k = 1
        if lanes > 1 and times[l] > share and n > 1:
            k = min(n, lanes, int(math.ceil(times[l] / share)))
        for c in range(k):
            a, b = n * c // k, n * (c + 1) // k
            items.append((l, a, b, times[l] * (b - a) / n))
    loads, out = [0.0] * lanes, [[] for _ in range(lanes)]
    for l, a, b, cost in sorted(items, key=lambda it: -it[3]):
        i = min(range(lanes), key=lambda k: loads[k])
        out[i].append((l, a, b))
        loads[i] += cost
    return [o for o in out if o]
