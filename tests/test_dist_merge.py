"""Multi-rank path on the CPU: two gloo ranks each hold the level statistics of their own
sample ids (the sharding of bench.py under torchrun) and merge them with Chan's formula
after an all-gather; the merged record equals the single-process statistics."""
import math
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1607_03252_gb300.stats import chan_merge, merge_levels, sample_sizes


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _level_values(level, first, count):
    rng = np.random.default_rng(1000 * level + 7)
    allv = rng.standard_normal(4096) * 10.0 ** (-level) + 0.05 / (level + 1)
    return allv[first:first + count]


def _record(v):
    m = float(np.mean(v))
    return (float(len(v)), m, float(np.sum((v - m) ** 2)))


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    N = [512, 128, 32]
    rec = torch.tensor([_record(_level_values(l, rank * n, n)) for l, n in enumerate(N)], dtype=torch.float64)
    parts = [torch.empty_like(rec) for _ in range(world)]
    dist.all_gather(parts, rec)
    merged = merge_levels([[tuple(r) for r in p.numpy()] for p in parts])
    if rank == 0:
        out.put(merged)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_merge_equals_single_process():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    merged = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for l, n in enumerate([512, 128, 32]):
        ref = _record(_level_values(l, 0, world * n))
        assert merged[l][0] == ref[0]
        assert merged[l][1] == pytest.approx(ref[1], rel=1e-13, abs=1e-16)
        assert merged[l][2] == pytest.approx(ref[2], rel=1e-12)


def test_chan_merge_matches_direct_statistics():
    v = np.random.default_rng(3).standard_normal(1000) + 5.0
    parts = [v[:100], v[100:101], v[101:700], v[700:]]
    n, m, m2 = chan_merge(_record(p) for p in parts)
    assert n == 1000 and m == pytest.approx(v.mean(), rel=1e-14)
    assert m2 == pytest.approx(((v - v.mean()) ** 2).sum(), rel=1e-12)


def test_sample_sizes_host_logic():
    # eps = 0.1 sqrt(2), theta = 1/2: eps_s = 0.1, the hand-worked case of Eq. 11
    assert sample_sizes([1.0, 0.25, 0.0625], [1.0, 8.0, 64.0], 0.1 * math.sqrt(2.0), 0.5) == [442, 79, 14]
    assert sample_sizes([1e-12], [1.0], 1.0, 0.5) == [2]  # at least two samples per level
