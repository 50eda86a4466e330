"""Pins for the oracle's scheduling model (Secs. 4-5) against the paper's worked numbers
and closed forms, and the planner (product host logic) against the oracle."""
import json
import math
import os
import random

import pytest

from oracle import schedule as osch
from paper_1607_03252_gb300 import planner

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
# Sec. 5.4's example (tests/golden/schedule_sec54_example.json, with its citation)
EX = json.load(open(os.path.join(GOLDEN, "schedule_sec54_example.json")))
N_EX, T_EX = EX["N"], EX["t"]
EX52 = json.load(open(os.path.join(GOLDEN, "schedule_sec52_example.json")))


def test_seq_steps_paper_example():
    """2048 level-0 samples on 512 processors each of a 524288-processor machine: two
    sequential steps (Sec. 5.2)."""
    J, k, imb = osch.seq_steps(EX52["N0"], 0, 0, EX52["P_max"], EX52["P0_min"])
    assert (J, k, imb) == (1024, EX52["k_seq"], 0.0)
    # one sample more leaves most of the third step idle
    J, k, imb = osch.seq_steps(2049, 0, 0, 524288, 512)
    assert k == 3 and imb == pytest.approx(1 - 2049 / 3072)


def test_amdahl_closed_forms():
    for th in range(5):
        assert osch.amdahl_efficiency(0.0, th) == 1.0
        assert osch.amdahl_efficiency(1.0, th) == pytest.approx(2.0 ** -th)
        for B in (0.01, 0.03, 0.5):
            t = osch.amdahl_time(100.0, B, th)
            assert osch.amdahl_efficiency(B, th) == pytest.approx(100.0 / (2 ** th * t))


def test_simple_heterogeneous_start_paper_example():
    """Eq. simpleestimation on the example: run-time 716 s. The paper prints the split
    (1314, 221, 36, 5); the floor of the formula gives (1305, 223, 36, 5). Both take
    716 s within 8192 processors."""
    Nl0, run, procs = osch.hetero_simple(N_EX, [r[0] for r in T_EX], EX["P_max"], EX["P0_min"])
    assert run == EX["simple_runtime"]
    assert Nl0 == [1305, 223, 36, 5] and procs <= EX["P_max"]
    printed = EX["simple_split_printed"]
    assert max(T_EX[l][0] * math.ceil(N_EX[l] / printed[l]) for l in range(4)) == EX["simple_runtime"]
    assert sum(printed[l] * 8 ** l for l in range(4)) <= EX["P_max"]


def test_optimal_s0_schedule_paper_example():
    """The paper's optimum for S = 0: 684 s with (1031, 172, 36, 6) on 7783 processors.
    Hand check: every faster run-time needs more than 8192 processors."""
    alloc = EX["optimal_s0_split"]
    assert max(T_EX[l][0] * math.ceil(N_EX[l] / alloc[l]) for l in range(4)) == EX["optimal_s0_runtime"]
    assert sum(alloc[l] * 8 ** l for l in range(4)) == EX["optimal_s0_processors"]
    below = max(T_EX[l][0] * k for l in range(4) for k in range(1, 40) if T_EX[l][0] * k < 684)
    need = sum(math.ceil(N_EX[l] / math.floor(below / T_EX[l][0])) * 8 ** l for l in range(4))
    assert need > 8192
    T, N_lt, procs = planner.hetero_exact(N_EX, [[r[0]] for r in T_EX], 8192, 1)
    assert T == EX["optimal_s0_runtime"] and procs == EX["optimal_s0_processors"]
    assert [row[0] for row in N_lt] == alloc  # the paper's allocation itself


def test_exact_s4_schedule_beats_the_annealing_result():
    """With the full window (S = 4) the paper's simulated annealing reached 627.6 s at
    best; the exact minimum can only be lower or equal."""
    T, N_lt, procs = planner.hetero_exact(N_EX, T_EX, 8192, 1)
    assert T <= EX["annealing_s4_best"] and procs <= 8192
    # the allocation covers every level within T
    for l in range(4):
        done = sum(N_lt[l][th] * math.floor(T / T_EX[l][th] * (1 + 1e-12)) for th in range(5))
        assert done >= N_EX[l]


def test_exact_schedule_equals_brute_force_on_small_machines():
    rng = random.Random(3)
    for _ in range(25):
        L = rng.choice([1, 2])
        S = rng.choice([0, 1])
        P = rng.choice([8, 16, 24])
        N = [rng.randint(1, 30) for _ in range(L)]
        t = [[round(rng.uniform(5, 20) * (1 + 0.3 * l), 2)] for l in range(L)]
        for l in range(L):
            for th in range(1, S + 1):
                t[l].append(round(t[l][0] * (0.05 + 0.95 / 2 ** th) * rng.uniform(0.95, 1.1), 2))
        if sum(8 ** l for l in range(L)) > P:
            continue
        Tb, pb = osch.hetero_bruteforce(N, t, P, 1)
        Te, alloc, pe = planner.hetero_exact(N, t, P, 1)
        assert Te == pytest.approx(Tb) and pe == pb, (N, t, P)


def test_planner_matches_oracle_model():
    rng = random.Random(7)
    for _ in range(200):
        l, th = rng.randint(0, 3), rng.randint(0, 4)
        Nl, P, P0 = rng.randint(1, 5000), rng.choice([4096, 8192, 65536]), rng.choice([1, 2, 8])
        assert planner.seq_steps(Nl, l, th, P, P0) == pytest.approx(osch.seq_steps(Nl, l, th, P, P0))
        B = rng.uniform(0, 0.2)
        assert planner.level_efficiency(Nl, l, th, P, P0, B) == pytest.approx(
            osch.level_efficiency(Nl, l, th, P, P0, B))
        S = 4
        row = [100 * (B + (1 - B) / 2 ** k) for k in range(S + 1)]
        assert planner.theta_homogeneous(Nl, l, S, P, P0, t_row=row) == osch.theta_homogeneous(Nl, l, S, P, P0, row)
        assert planner.theta_homogeneous(Nl, l, S, P, P0, B=B) == osch.theta_homogeneous(Nl, l, S, P, P0, B=B)
    N, t0, EC = [100, 20, 3], [1.0, 1.2, 1.5], [1.0, 1.1, 1.3]
    assert planner.optimal_runtime(N, t0, EC, 4096, 2) == pytest.approx(
        2 / 4096 * (100 * 1.0 + 20 * 8 * 1.1 * 1.2 + 3 * 64 * 1.3 * 1.5))
    assert planner.hetero_simple(N_EX, [r[0] for r in T_EX], 8192, 1) == osch.hetero_simple(
        N_EX, [r[0] for r in T_EX], 8192, 1)


def test_dynamic_and_static_assignment():
    rng = random.Random(11)
    for _ in range(50):
        times = [rng.uniform(1, 5) for _ in range(rng.randint(1, 60))]
        J = rng.randint(1, 12)
        s, d = planner.static_makespan(times, J), planner.dynamic_makespan(times, J)
        assert s == pytest.approx(osch.static_makespan(times, J))
        assert d == pytest.approx(osch.dynamic_makespan(times, J))
        # greedy list scheduling: within the largest task of the average load
        assert d <= sum(times) / min(J, len(times)) + max(times) + 1e-9
    # constant run-times: both are ceil(N / J) steps
    assert planner.static_makespan([2.0] * 10, 4) == planner.dynamic_makespan([2.0] * 10, 4) == 6.0


def test_runtime_robust_equals_homogeneous_for_constant_times():
    """With a constant run-time histogram RuRoHom chooses LeSyHom's theta (Sec. 5.2)."""
    for Nl, l in ((2048, 0), (300, 1), (40, 2)):
        a = planner.theta_runtime_robust(Nl, l, 4, 65536, 16, [10.0] * 20, B=0.02, seed=1)
        b = planner.theta_homogeneous(Nl, l, 4, 65536, 16, B=0.02)
        assert a == b


def test_runtime_variation_example_of_sec_5_2():
    """Sec. 5.2: 2048 level-0 samples on 512-processor blocks of a 524288-processor machine
    (two sequential steps), 3 of them slow (50 s against 45 s). Sample-synchronous steps
    take 100 s unless all three slow samples share a step: probability
    1 - 2 C(1024,3) / C(2048,3) = 0.750 ("about 75%"); level-synchronous blocks take 100 s
    only if two slow samples share a block: 1 - 2044/2047 = 0.15% ("less than 1%"), and
    95 s otherwise ("<= 96 s")."""
    J, k, _ = osch.seq_steps(2048, 0, 0, 524288, 512)
    assert (J, k) == (1024, 2)
    p_sync = 1 - 2 * math.comb(1024, 3) / math.comb(2048, 3)
    p_level = 1 - 2044 / 2047
    assert p_sync == pytest.approx(EX52["p_sync_about"], abs=0.01) and p_level < EX52["p_level_below"]
    rng = random.Random(17)
    base = [45.0] * (EX52["N0"] - EX52["slow_samples"]) + [float(EX52["slow_time"])] * EX52["slow_samples"]
    hits_sync = hits_level = 0
    trials = 4000
    for _ in range(trials):
        times = base[:]
        rng.shuffle(times)
        s = planner.sync_makespan(times, J)
        assert s == osch.sync_makespan(times, J) and s in (95.0, 100.0)
        hits_sync += s == 100.0
        lv = planner.static_makespan(times, J)
        assert lv == osch.static_makespan(times, J) and (lv == 100.0 or lv <= EX52["level_otherwise_at_most"])
        hits_level += lv == 100.0
    assert abs(hits_sync / trials - p_sync) < 5 * math.sqrt(p_sync * (1 - p_sync) / trials)
    assert abs(hits_level / trials - p_level) < 5 * math.sqrt(p_level * (1 - p_level) / trials) + 1 / trials
