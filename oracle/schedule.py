"""The paper's MLMC performance model and scheduling rules (Secs. 4-5), written out plainly
(test infrastructure only).

Each function follows one definition of the paper: the Amdahl surrogate (Eq. amdahls),
blocks / sequential steps / imbalance (Eq. seqsteps), level efficiency (Eq. effs), the
optimal mean run-time (Eq. optruntime), the homogeneous choice of theta (Sec. 5.1), the
static and dynamic block assignments (Secs. 5.1, 5.3), the proportional heterogeneous
start (Eq. simpleestimation), and the heterogeneous optimum by exhaustive search over the
block counts N_{l,theta} (Sec. 5.4's problem; feasible for small P_max only).
"""
from __future__ import annotations

import itertools
import math


def amdahl_time(t0, B, theta):
    return t0 * (B + 2.0 ** (-theta) * (1.0 - B))


def amdahl_efficiency(B, theta):
    """t_{l,0} / (2^theta t_{l,theta}) with the Amdahl time."""
    return 1.0 / (2.0 ** theta * (B + 2.0 ** (-theta) * (1.0 - B)))


def seq_steps(N_l, l, theta, P_max, P0_min):
    procs = 2 ** (3 * l + theta) * P0_min
    J = P_max // procs
    if J == 0:
        return 0, math.inf, 1.0
    k = math.ceil(N_l / J)
    return J, k, 1.0 - procs * N_l / (k * P_max)


def level_efficiency(N_l, l, theta, P_max, P0_min, B):
    J, k, imb = seq_steps(N_l, l, theta, P_max, P0_min)
    return (1.0 - imb) * amdahl_efficiency(B, theta)


def optimal_runtime(N, t0, EC, P_max, P0_min):
    s = 0.0
    for l in range(len(N)):
        s += N[l] * 2 ** (3 * l) * EC[l] * t0[l]
    return P0_min / P_max * s


def theta_homogeneous(N_l, l, S, P_max, P0_min, t_row=None, B=None):
    """The largest theta with the least k_seq(theta) t_{l,theta}."""
    vals = []
    for th in range(S + 1):
        J, k, imb = seq_steps(N_l, l, th, P_max, P0_min)
        t = t_row[th] if t_row is not None else amdahl_time(1.0, B, th)
        vals.append(k * t)
    m = min(vals)
    return max(th for th in range(S + 1) if vals[th] <= m * (1 + 1e-12))


def sync_makespan(times, J):
    """Steps of J samples, each as slow as its slowest sample, one after the other."""
    total = 0.0
    for start in range(0, len(times), J):
        total += max(times[start:start + J])
    return total


def static_makespan(times, J):
    """Block j computes samples j, j + J, j + 2J, ...; the run-time is the slowest block's."""
    sums = [0.0] * J
    for i, t in enumerate(times):
        sums[i % J] += t
    return max(sums[: min(J, len(times))])


def dynamic_makespan(times, J):
    """Discrete-event simulation: when a block finishes, it takes the next sample."""
    finish = [0.0] * min(J, len(times))
    for t in times:
        b = min(range(len(finish)), key=lambda j: (finish[j], j))
        finish[b] += t
    return max(finish)


def hetero_simple(N, t0, P_max, P0_min):
    den = sum(N[i] * 2 ** (3 * i) * P0_min * t0[i] for i in range(len(N)))
    Nl0 = [max(1, math.floor(P_max * N[l] * t0[l] / den)) for l in range(len(N))]
    run = max(t0[l] * math.ceil(N[l] / Nl0[l]) for l in range(len(N)))
    procs = sum(Nl0[l] * 2 ** (3 * l) * P0_min for l in range(len(N)))
    return Nl0, run, procs


def hetero_bruteforce(N, t, P_max, P0_min):
    """Minimal run-time over every N_{l,theta} >= 0 with sum_{l,theta} N_{l,theta}
    2^(3l+theta) P0_min <= P_max and, per level, some theta-blocks: the samples of level l
    run on its blocks, a theta-block finishing floor(T / t_{l,theta}) of them by time T, so
    the run-time of an allocation is the least T whose blocks cover every N_l. Returns
    (T, fewest processors at T)."""
    L = len(N)
    per_level = []
    for l in range(L):
        S = len(t[l]) - 1
        caps = [P_max // (2 ** (3 * l + th) * P0_min) for th in range(S + 1)]
        opts = []
        for counts in itertools.product(*[range(c + 1) for c in caps]):
            procs = sum(counts[th] * 2 ** (3 * l + th) * P0_min for th in range(S + 1))
            if procs == 0 or procs > P_max:
                continue
            # least T at which these blocks finish N_l samples
            best = math.inf
            for th in range(S + 1):
                if counts[th] == 0:
                    continue
                for k in range(1, N[l] + 1):
                    T = t[l][th] * k
                    done = sum(counts[u] * math.floor(T / t[l][u] * (1 + 1e-12)) for u in range(S + 1))
                    if done >= N[l]:
                        best = min(best, T)
                        break
            opts.append((best, procs))
        per_level.append(opts)
    best_T, best_p = math.inf, None
    for combo in itertools.product(*per_level):
        procs = sum(c[1] for c in combo)
        if procs > P_max:
            continue
        T = max(c[0] for c in combo)
        if T < best_T - 1e-9 or (abs(T - best_T) <= 1e-9 and procs < best_p):
            best_T, best_p = T, procs
    return best_T, best_p
