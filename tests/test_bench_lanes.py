"""Host logic of the bench's step schedule: levels (and chunks of a level's samples) on
concurrent streams cover every sample exactly once, in contiguous id ranges."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def covered(lanes):
    seen = {}
    for its in lanes:
        for (l, a, b) in its:
            assert a < b
            seen.setdefault(l, []).append((a, b))
    return {l: sorted(v) for l, v in seen.items()}


@pytest.mark.parametrize("lanes", [1, 2, 3, 4, 8])
def test_every_sample_once(bench, lanes):
    levels, N = [0, 1, 2, 3, 4], [170, 4, 2, 2, 2]
    times = {0: 4.2, 1: 4.8, 2: 5.9, 3: 12.8, 4: 65.8}
    out = bench.lane_items(levels, N, times, lanes)
    assert 1 <= len(out) <= lanes
    cov = covered(out)
    for l, n in zip(levels, N):
        spans = cov[l]
        assert spans[0][0] == 0 and spans[-1][1] == n
        for (a0, b0), (a1, b1) in zip(spans, spans[1:]):
            assert b0 == a1  # contiguous, disjoint


def test_long_level_is_split_and_balanced(bench):
    levels, N = [0, 1, 2, 3, 4], [170, 4, 2, 2, 2]
    times = {0: 4.2, 1: 4.8, 2: 5.9, 3: 12.8, 4: 65.8}
    out = bench.lane_items(levels, N, times, 4)
    cov = covered(out)
    assert len(cov[4]) == 2  # level 4 (2 samples, far above a quarter of the step) is split
    loads = [sum(times[l] * (b - a) / dict(zip(levels, N))[l] for (l, a, b) in its) for its in out]
    assert max(loads) <= 0.5 * sum(times.values()) + 1e-9


def test_one_lane_keeps_levels_whole(bench):
    out = bench.lane_items([0, 1, 2, 3], [4096, 1024, 256, 64], {0: 52, 1: 75, 2: 131, 3: 245}, 1)
    assert out == [[(3, 0, 64), (2, 0, 256), (1, 0, 1024), (0, 0, 4096)]]
