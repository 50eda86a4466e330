#!/usr/bin/env python
"""Benchmark of the MLMC multigrid hot path on one GB300 (or N, one process per GPU).

One step = one full MLMC estimate of the configured workload: for every level l the
N_l samples Y_l = Q_l - Q_{l-1} (field evaluation, fine and coarse multigrid solves on
the same realisation, QoI, level statistics), all in the CUDA library.

Default workload (--config c2): 4-level FP64 MLMC, levels 17^3, 33^3, 65^3, 129^3
(fine grids), N_l = 4096, 1024, 256, 64, sigma^2 = 1, ell = 0.3, M = 256, V(2,2) to
relative residual 1e-10, f = 1, QoI = mean of u over [0.25, 0.75]^3.

Reported (one JSON line on rank 0):
  value          MLMC samples/s over all levels (sum_l N_l per step x ranks / time),
                 ids already in HBM, outputs left in HBM (device-resident C-ABI call);
  per_level      samples/s per level;
  e2e            the same through the host-buffer C-ABI call (ids built on the host,
                 results copied back into pinned host memory every step);
  roofline       the dominant kernel class: algorithmic work / its event-timed device
                 time against the binding peak;
  cpu_baseline   the FP64 CPU oracle on a bounded sample of the same ids, host cores.
With --impl reference the oracle itself is timed on the same workload (bounded sample
per step) and reported as the reference arm.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1607_03252_gb300.workloads import CONFIGS, RUN_SEED, level_n, sample_ids  # noqa: E402

L2_BYTES = 129 * 1024 * 1024

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per work unit measured by ncu for
# a kernel, valid only while that kernel's source text hashes to `kernel_sha` (else null).
# unit_bytes: the algorithmic bytes the library accounts per unit, to count units per launch.
NCU_TRAFFIC = {
    "rbgs_f64": {"file": "paper_1607_03252_gb300/csrc/mg.cu", "kernel": "k_rbgs", "kernel_sha": "e8e43de9d3e4896e",
                 "dram_bytes_per_unit": (805.797e6 + 119.737e6) / (8 * 127 ** 3), "unit_bytes": 3.5 * 8,
                 "source": "profiles/rbgs_f64_twopass_n129_b8.md (129^3 x 8, one colour pass)"},
    "rbgs_f32": {"file": "paper_1607_03252_gb300/csrc/mg.cu", "kernel": "k_rbgs", "kernel_sha": "e8e43de9d3e4896e",
                 "dram_bytes_per_unit": (805.619e6 + 121.530e6) / (2 * 255 ** 3), "unit_bytes": 3.5 * 4,
                 "source": "profiles/rbgs_f32_n257_b2.md (257^3 x 2, one colour pass)"},
    "rbgs_split_f32": {"file": "paper_1607_03252_gb300/csrc/mg.cu", "kernel": "k_rbgs_split", "kernel_sha": "9d3393d2d0414e4e",
                       "dram_bytes_per_unit": (281.681e6 + 55.126e6) / (2 * 255 ** 3), "unit_bytes": 2.0 * 4,
                       "source": "profiles/rbgs_split_f32_n257_b2.md (257^3 x 2, one colour pass)"},
    "rbgs_split_f64": {"file": "paper_1607_03252_gb300/csrc/mg.cu", "kernel": "k_rbgs_split64", "kernel_sha": "771506262551874d",
                       "dram_bytes_per_unit": (636.264e6 + 59.780e6) / (8 * 127 ** 3), "unit_bytes": 3.5 * 8,
                       "source": "profiles/rbgs_split_f64_n129_b8.md (129^3 x 8, one colour pass)"},
    "rbgs_nodal_f32": {"file": "paper_1607_03252_gb300/csrc/mg.cu", "kernel": "k_rbgs_nodal", "kernel_sha": "cb8a0fa77df739fc",
                       "dram_bytes_per_unit": (405.356e6 + 107.601e6) / (2 * 255 ** 3), "unit_bytes": 2.0 * 4,
                       "source": "profiles/rbgs_nodal_f32_n257_b2.md (257^3 x 2, one colour pass)"},
}


def kernel_sha(path, name):
    """Hash of one kernel's source: its signature and brace-balanced body."""
    import hashlib

    try:
        import re

        src = open(os.path.join(ROOT, path)).read()
        m = re.search(r"__global__ void (__launch_bounds__\([^)]*\) )?" + re.escape(name) + r"\(", src)
        i = m.start()
        j = src.index("{", i)
        depth = 0
        for k in range(j, len(src)):
            depth += {"{": 1, "}": -1}.get(src[k], 0)
            if depth == 0:
                return hashlib.sha256(src[i:k + 1].encode()).hexdigest()[:16]
        return None
    except Exception:
        return None


def traffic_per_launch(name, rec):
    t = NCU_TRAFFIC.get(name)
    if not t or kernel_sha(t["file"], t["kernel"]) != t["kernel_sha"]:
        return None, None
    units = rec["bytes"] / max(rec["launches"], 1) / t["unit_bytes"]
    return units * t["dram_bytes_per_unit"], t["source"]
# FP64 peak from unit counts and clocks: 152 SMs x 2 FP64 FMA/clk/SM x 2 flop x 2.07 GHz
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="own", choices=["own", "reference"])
    p.add_argument("--config", default="c2", choices=["c1", "c2", "c3", "c4", "c5", "c6"])
    p.add_argument("--c5-arms", default="fast,plain", help="c5: which arms to run (fast, plain)")
    p.add_argument("--c5-eps", type=float, default=None, help="c5: override the RMS tolerance")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-extras", action="store_true",
                   help="c2: skip the c3 / c5 / c4 sub-records of the default line")
    p.add_argument("--lanes", type=int, default=4, help="concurrent level streams (1: levels in sequence)")
    p.add_argument("--plan-from", default=None,
                   help="reuse the autotuned choices (and pilot-sized N_l) of an earlier JSON line of the same "
                        "config instead of measuring them again (for runs under a profiler)")
    return p.parse_args()


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except Exception:
        return {}


def solver_kw(mg, cfg):
    """The solver settings of a workload as make_mlmc_cfg keywords: outer iteration (none,
    flexible CG, one FMG cycle), discretisation, QoI, covariance and the cycle budget (the
    FMG cycle's V-cycles per grid; otherwise the cap of a solve to rtol)."""
    accel = {"cg": mg.MLMC_ACCEL_CG, "fmg": mg.MLMC_ACCEL_FMG}.get(cfg.get("accel"), mg.MLMC_ACCEL_NONE)
    return dict(accel=accel, disc=mg.MLMC_DISC_FE if cfg.get("disc") == "fe" else mg.MLMC_DISC_FV,
                qoi={"point": mg.MLMC_QOI_POINT, "flux": mg.MLMC_QOI_FLUX}.get(cfg.get("qoi"), mg.MLMC_QOI_MEAN),
                cov=mg.MLMC_COV_EXP if cfg.get("cov") == "exp" else mg.MLMC_COV_GAUSS,
                max_cycles=cfg.get("cycles", 300))


def workload(cfg_name):
    c = CONFIGS[cfg_name]
    levels = c["levels"]
    N = c.get("N", c.get("N_init", [64] * len(levels)))
    single = c.get("single_level", False)
    return c, levels, N, single


def plan_levels(mg, cfg, levels, stream, rank):
    """Mixed-precision workloads: autotune each level (smoother x nu), run the pilot
    N_init, and size N_l by Eq. 11 for the configured eps (theta split of Eq. 6)."""
    prec = mg.MLMC_PREC_MIXED
    accel = mg.MLMC_ACCEL_CG if cfg.get("accel") == "cg" else mg.MLMC_ACCEL_NONE
    tune, V, C = {}, [], []
    for l, n0 in zip(levels, cfg["N_init"]):
        c = mg.make_mlmc_cfg(RUN_SEED, cfg["sigma2"], cfg["ell"], cfg["M"], n0=17, nu1=0, nu2=0, rtol=cfg["rtol"],
                             precision=prec, max_batch=n0, stream=stream, accel=accel, max_cycles=300)
        rows, bs, bnu = mg.mlmc_autotune(c, l, int(sample_ids(l, 1 << 40, 1)[0]), min(n0, 32))
        tune[str(l)] = {"best": {"smoother": mg._capi.SMOOTHER_NAMES.get(bs, bs), "nu": bnu}, "table": rows}
        st, _, _, _ = mg.mlmc_level_estimate(c, l, int(sample_ids(l, (1 << 41) + rank * n0, 1)[0]), n0,
                                             want_samples=False)
        V.append(max(st.var_unbiased, 1e-30))
        C.append(st.cost_per_sample)
    from paper_1607_03252_gb300.stats import sample_sizes

    N = sample_sizes(V, C, cfg["eps"], cfg["theta"])  # Eq. 11 in the library
    return N, {"pilot_N": cfg["N_init"], "pilot_var": V, "pilot_cost_s": C, "eps": cfg["eps"],
               "theta": cfg["theta"], "N_from_eq11": N, "autotune": tune}


def restore_plan(mg, cfg, levels, N, path):
    """The plan of an earlier run of the same config (its JSON line): each level's tuned
    smoother and nu go back into the library's tuning table (mlmc_tune_set, for the
    level's fine grid and precision), and pilot-sized workloads take its N_l."""
    with open(path) as fh:
        line = json.loads([ln for ln in fh.read().splitlines() if ln.strip().startswith("{")][-1])
    if line.get("config", {}).get("workload") != cfg["name"]:
        raise SystemExit("--plan-from: %s holds workload %r, not %r" % (path, line.get("config", {}).get("workload"),
                                                                       cfg["name"]))
    plan = line["plan"]
    prec = mg.MLMC_PREC_F64 if cfg["precision"] == "f64" else mg.MLMC_PREC_MIXED
    for l in levels:
        best = plan["autotune"][str(l)]["best"]
        mg.mlmc_tune_set(level_n(l), prec, best["smoother"], best["nu"])
    if "N_from_eq11" in plan:
        N = list(plan["N_from_eq11"])
    plan = dict(plan, restored_from=os.path.basename(path))
    return N, plan


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    smax.append(float(f[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, f[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


# --------------------------------------------------------------------------------------
# CPU oracle timing (bounded sample)
# --------------------------------------------------------------------------------------
def oracle_level_rates(cfg, levels, single, counts):
    """samples/s of the oracle per level on the given sample counts (OpenMP over samples).
    Levels with a count of 0 are not run; their rate is extrapolated from the previous
    level by the 8x growth of the grid (cost per sample ~ nodes)."""
    import oracle

    mixed = cfg.get("precision") == "mixed"
    ocfg = oracle.make_cfg(RUN_SEED, cfg["sigma2"], cfg["ell"], cfg["M"], cfg["nu1"], cfg["nu2"], cfg["rtol"], 400,
                           mixed=mixed)
    fe = cfg.get("disc") == "fe"
    if fe:
        from oracle import core as ocore
        from oracle import fe as ofe
    rates, secs = {}, {}
    for l, cnt in zip(levels, counts):
        if cnt == 0:
            rates[l] = rates[l - 1] / 8.0
            secs[l] = 0.0
            continue
        ids = sample_ids(l, 0, cnt)
        nc = 0 if (single or l == 0) else level_n(l - 1)
        t = time.perf_counter()
        if fe:  # the P1 / FMG-2V(4,4) oracle (plain numpy, one sample at a time)
            cov = ocore.COV_EXP if cfg.get("cov") == "exp" else ocore.COV_GAUSS
            for i in ids:
                ofe.level_sample(RUN_SEED, int(i), cfg["M"], cfg["sigma2"], cfg["ell"], level_n(l), nc,
                                 qoi=cfg.get("qoi", "point"), cov=cov)
        else:
            oracle.level_batch(ocfg, level_n(l), nc, ids)
        dt = time.perf_counter() - t
        rates[l] = cnt / dt
        secs[l] = dt
    return rates, secs


def oracle_counts(levels, threads, cfg=None):
    base = {0: max(16, 4 * threads), 1: max(8, threads), 2: max(4, threads // 2), 3: max(1, threads // 2),
            4: 0, 5: 0}
    if cfg is not None and cfg.get("precision") == "mixed":
        base[3] = 0  # rough fields: the stationary oracle needs 100+ cycles; extrapolate beyond 65^3
    if cfg is not None and cfg.get("disc") == "fe":
        base = {0: 32, 1: 8, 2: 2, 3: 0}  # numpy FE oracle, one thread: ~0.03 / 0.25 / 3 s per sample
    return [base[l] for l in levels]


def extrapolated_rate(levels, N, rates):
    t = sum(n / rates[l] for l, n in zip(levels, N))
    return sum(N) / t


# --------------------------------------------------------------------------------------
# Reference arm: the oracle
# --------------------------------------------------------------------------------------
def reference_arm(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle

    cfg, levels, N, single = workload(args.config)
    threads = 1 if cfg.get("disc") == "fe" else oracle.max_threads()  # the FE oracle is plain numpy
    counts = oracle_counts(levels, threads, cfg)
    step_times, all_rates = [], []
    for i in range(args.warmup + args.steps):
        t = time.perf_counter()
        rates, _ = oracle_level_rates(cfg, levels, single, counts)
        dt = time.perf_counter() - t
        if i >= args.warmup:
            step_times.append(dt)
            all_rates.append(rates)
    mean_rates = {l: statistics.mean(r[l] for r in all_rates) for l in levels}
    value = extrapolated_rate(levels, N, mean_rates)
    how = "one sample at a time (numpy)" if cfg.get("disc") == "fe" else "OpenMP over samples"
    sample = ("per step: %s samples on levels %s (ids of the benchmark workload), %s; "
              "samples/s per level extrapolated to N=%s" % (counts, levels, how, N))
    line = {
        "impl": "reference", "metric": "MLMC samples/s (all levels, %s)" % cfg["name"], "value": value,
        "unit": "samples/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * statistics.mean(step_times), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded Philox realisations)",
        "config": {"workload": cfg["name"], "levels": levels, "N": N, "fine_n": [level_n(l) for l in levels],
                   "sigma2": cfg["sigma2"], "ell": cfg["ell"], "M": cfg["M"], "rtol": cfg["rtol"]},
        "per_level": {str(l): mean_rates[l] for l in levels},
        "cpu_baseline": {"value": value, "unit": "samples/s", "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------------------
# Own arm
# --------------------------------------------------------------------------------------
def own_arm(args):
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    line = measure(args, args.config, full=True)
    if line is not None and world == 1 and args.config == "c2" and not args.no_extras:
        # the mixed-precision and adaptive workloads of the same metric family, on the same
        # GPU in the same run (sub-records; the headline stays the 4-level FP64 workload)
        t0 = time.perf_counter()
        line["c3"] = sub_c3(args)
        line["c5"] = sub_c5(args)
        line["c4"] = sub_c4(args, line["c3"])
        line["c6"] = measure(args, "c6", full=False)
        line["extras_wall_s"] = time.perf_counter() - t0
    if line is not None:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def measure(args, cfg_name, full=True):
    """One workload's bench line (rank 0; None on other ranks). full: also the e2e and
    cpu_baseline legs."""
    import torch

    import paper_1607_03252_gb300 as mg

    rank, world, local = dist_env()
    cfg, levels, N, single = workload(cfg_name)
    prec = mg.MLMC_PREC_F64 if cfg["precision"] == "f64" else mg.MLMC_PREC_MIXED
    skw = solver_kw(mg, cfg)
    accel = skw["accel"]
    stream = torch.cuda.Stream()
    dev = torch.device("cuda", local)
    plan = None
    nu_cfg = (cfg["nu1"], cfg["nu2"])
    if args.plan_from and cfg_name == args.config:
        N, plan = restore_plan(mg, cfg, levels, N, args.plan_from)
        if "N_init" in cfg:
            nu_cfg = (0, 0)
    elif "N_init" in cfg:
        N, plan = plan_levels(mg, cfg, levels, stream, rank)
        nu_cfg = (0, 0)  # the autotuned sweep count per level
    else:
        # the cycle is fixed (V(nu1, nu2)); tune only the smoother implementation per level,
        # which changes no result bit (bounded sample of tuning-only ids)
        tune = {}
        for l, n in zip(levels, N):
            c = mg.make_mlmc_cfg(RUN_SEED, cfg["sigma2"], cfg["ell"], cfg["M"], n0=(level_n(l) if single else 17),
                                 nu1=cfg["nu1"], nu2=cfg["nu2"], rtol=cfg["rtol"], precision=prec,
                                 max_batch=min(n, 256), stream=stream, **skw)
            rows, bs, bnu = mg.mlmc_autotune(c, 0 if single else l, int(sample_ids(l, 1 << 40, 1)[0]), min(n, 256))
            tune[str(l)] = {"best": {"smoother": mg._capi.SMOOTHER_NAMES.get(bs, bs), "nu": bnu}, "table": rows}
        plan = {"autotune": tune}
    # inputs resident in HBM: each rank its own realisations (weak scaling)
    ids = {l: torch.from_numpy(sample_ids(l, rank * n, n).view("int64")).to(dev) for l, n in zip(levels, N)}
    Y = {l: torch.empty(n, dtype=torch.float64, device=dev) for l, n in zip(levels, N)}
    mcfg = {}
    for l, n in zip(levels, N):
        n0 = level_n(l) if single else 17
        lvl = 0 if single else l
        mcfg[l] = (mg.make_mlmc_cfg(RUN_SEED, cfg["sigma2"], cfg["ell"], cfg["M"], n0=n0, nu1=nu_cfg[0],
                                    nu2=nu_cfg[1], rtol=cfg["rtol"], precision=prec, max_batch=n, stream=stream,
                                    **skw), lvl)
    # levels run concurrently on `lanes` streams (the one-GPU form of scheduling the
    # levels on separate processor groups): the FP64/HBM-bound solves of one level
    # overlap the FP32-bound field evaluation and solves of others
    # one untimed pass with the levels in sequence measures each level's time (the
    # lane assignment's costs)
    seq_ms, seq_launches = {}, {}
    for _ in range(2):  # the second pass, after first-call set-up
        for l in levels:
            c, lvl = mcfg[l]
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            mg.profile_reset()
            a.record(stream)
            mg.mlmc_level_run(c, lvl, ids[l], Y_dev=Y[l])
            b.record(stream)
            b.synchronize()
            seq_ms[l] = a.elapsed_time(b)
            seq_launches[l] = mg.profile_total_launches()
    lanes = lane_items(levels, N, seq_ms, args.lanes)
    lane_streams = [stream] + [torch.cuda.Stream() for _ in lanes[1:]]
    # one configuration per work item, bound to its lane's stream
    icfg = {}
    for i, its in enumerate(lanes):
        for (l, a, b) in its:
            c, lvl = mcfg[l]
            ci = type(c).from_buffer_copy(c)
            ci.stream = lane_streams[i].cuda_stream
            icfg[(l, a)] = (ci, lvl)
    chunks = {l: sorted(a for its in lanes for (ll, a, _) in its if ll == l) for l in levels}
    lev_ev = {l: [] for l in levels}  # per step: [(start, end) per chunk]
    stats = {}

    def step(record, sequential=False):
        parts = {}
        evs = {l: [] for l in levels}

        def lane(i):
            st = lane_streams[i]
            for (l, a, b) in lanes[i]:
                c, lvl = icfg[(l, a)]
                if record:
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(st)
                parts[(l, a)] = mg.mlmc_level_run(c, lvl, ids[l][a:b], Y_dev=Y[l][a:b])
                if record:
                    e1.record(st)
                    evs[l].append((e0, e1))

        if sequential:  # whole levels one after the other: each kernel alone, at its level's batch
            for l in levels:
                c, lvl = mcfg[l]
                stats[l] = mg.mlmc_level_run(c, lvl, ids[l], Y_dev=Y[l])
            return
        run_lanes(torch, lanes, lane_streams, stream, lane)
        for l in levels:
            ps = [parts[(l, a)] for a in chunks[l]]
            stats[l] = ps[0] if len(ps) == 1 else MergedLevel(ps)
            if record:
                lev_ev[l].append(evs[l])
        if world > 1:
            import torch.distributed as dist

            rec = torch.tensor([[stats[l].N, stats[l].mean, stats[l].M2] for l in levels], dtype=torch.float64,
                               device=dev)
            parts = [torch.empty_like(rec) for _ in range(world)]
            dist.all_gather(parts, rec)
            merged = merge_records([p.cpu().numpy() for p in parts])
            stats["merged"] = merged

    for _ in range(args.warmup):
        step(False)
    torch.cuda.synchronize()
    # timed region 1: the value (launches counted, no per-launch events)
    mg.profile_reset()
    mg.profile_enable(False)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_host0 = time.perf_counter()
    # NVTX range "timed_step" marks the timed launches (ncu --nvtx --nvtx-include timed_step/)
    torch.cuda.nvtx.range_push("timed_step")
    ev0.record(stream)
    for _ in range(args.steps):
        step(True)
    ev1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    if world > 1:
        torch.distributed.barrier()
    t_host = time.perf_counter() - t_host0
    clk = clocks.stop()
    elapsed_ms = ev0.elapsed_time(ev1)
    launches = mg.profile_total_launches()
    # timed region 2: the same steps, levels in sequence, with a CUDA event pair around
    # every launch, for the per-kernel device times of the roofline (each kernel alone)
    mg.profile_reset()
    mg.profile_enable(True)
    torch.cuda.synchronize()
    evp0, evp1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    evp0.record(stream)
    for _ in range(args.steps):
        step(False, sequential=True)
    evp1.record(stream)
    torch.cuda.synchronize()
    mg.profile_enable(False)
    prof = mg.profile_read()
    profiled_ms = evp0.elapsed_time(evp1)
    if world > 1:
        t = torch.tensor([elapsed_ms], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        elapsed_ms = float(t.item())
    total_samples = sum(N) * world * args.steps
    value = total_samples / (elapsed_ms / 1e3)
    per_level = {}
    for l, n in zip(levels, N):
        # a level's time per step: from its first chunk's start to its last chunk's end
        ms = sum(max(ev0.elapsed_time(e1) for _, e1 in evs) - min(ev0.elapsed_time(e0) for e0, _ in evs)
                 for evs in lev_ev[l])
        per_level[str(l)] = n * world * args.steps / (ms / 1e3)

    # roofline of the dominant kernel class
    peaks = measured_peaks()
    roof = roofline(prof, peaks)

    # end to end through the host-buffer C-ABI call
    e2e = None
    if full and not args.no_e2e:
        e2e = e2e_measure(args, mg, torch, cfg, levels, N, single, prec, rank, world, stream, nu_cfg, skw, lanes)

    line = None
    if rank == 0:
        cpu = None
        if full and world == 1 and not args.no_cpu_baseline:
            cpu = cpu_baseline(cfg, levels, N, single)
        line = {
            "metric": "MLMC samples/s (all levels, %s)" % cfg["name"], "value": value, "unit": "samples/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == mg.MLMC_PREC_F64 else "f32+f64",
            "solver": {"precision": cfg["precision"], "accel": cfg.get("accel", "none"),
                       "disc": cfg.get("disc", "fv"), "qoi": cfg.get("qoi", "mean"), "cov": cfg.get("cov", "gauss")},
            "plan": plan,
            "data": "synthetic (seeded Philox realisations, run_seed %d)" % RUN_SEED,
            "config": {"workload": cfg["name"], "levels": levels, "N_per_gpu": N,
                       "fine_n": [level_n(l) for l in levels], "sigma2": cfg["sigma2"], "ell": cfg["ell"],
                       "M": cfg["M"], "rtol": cfg["rtol"],
                       "cycle": ("FMG-%dV(%d,%d)" % (cfg["cycles"], cfg["nu1"], cfg["nu2"]) if cfg.get("accel") == "fmg"
                                 else "V(%d,%d)" % (cfg["nu1"], cfg["nu2"])),
                       "parallelism": "replicas x%d (samples sharded by rank, no data-path collective)" % world,
                       "level_streams": [["%d[%d:%d]" % (l, a, b) for (l, a, b) in its] for its in lanes],
                       "level_ms_alone": {str(l): round(v, 3) for l, v in seq_ms.items()},
                       "level_launches_alone": {str(l): v for l, v in seq_launches.items()},
                       "l2": "every level's batch working set exceeds the 129 MB L2 (no flush needed)"},
            "per_level": per_level,
            "time_per_estimate_s": elapsed_ms / 1e3 / args.steps,
            "level_stats": {str(l): {"mean": stats[l].mean, "var": stats[l].var_unbiased,
                                     "cycles_fine": stats[l].mean_cycles_fine,
                                     "cycles_coarse": stats[l].mean_cycles_coarse} for l in levels},
            "roofline": roof, "field_roofline": field_roofline(prof, peaks), "gpu_launches": launches, "e2e": e2e,
            "clocks": clk, "cpu_baseline": cpu,
            "host_wall_s": t_host,
            "timing_note": "value, per_level, clocks and gpu_launches: timed region 1 (levels on concurrent "
                           "streams, no per-launch events); roofline and kernel_classes: timed region 2 (same "
                           "steps, whole levels in sequence, CUDA events around every launch on the launching "
                           "stream)",
            "profiled_region_ms_per_step": profiled_ms / args.steps,
            "kernel_ms_per_step": sum(v["ms"] for v in prof.values()) / args.steps,
            "kernel_classes": class_shares(prof),
            "kernel_sizes_top": {k: {"launches": v["launches"], "ms": round(v["ms"], 3)}
                                 for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"])[:8]},
        }
        if prec == mg.MLMC_PREC_MIXED:
            line["smoother_roofline"] = roofline(prof, peaks, lambda k: k.startswith("rbgs"))
            line["residual_roofline"] = roofline(prof, peaks, lambda k: k.startswith("residual") and k.endswith("f32"))
    return line


def merge_records(parts):
    """Chan's merge of per-rank (N, mean, M2) rows per level."""
    import numpy as np

    from paper_1607_03252_gb300.stats import merge_levels

    return np.array(merge_levels([[tuple(row) for row in p] for p in parts]))


def base_class(name):
    """Launch class without its grid-size tag ("rbgs_f64@129" -> "rbgs_f64")."""
    return name.split("@")[0]


def class_shares(prof):
    """Device time per launch class (grid sizes merged), share of the profiled total."""
    agg = {}
    for k, v in prof.items():
        a = agg.setdefault(base_class(k), {"launches": 0, "ms": 0.0})
        a["launches"] += v["launches"]
        a["ms"] += v["ms"]
    tot = sum(v["ms"] for v in agg.values()) or 1.0
    return {k: {"launches": v["launches"], "ms": round(v["ms"], 3), "share": round(v["ms"] / tot, 4)}
            for k, v in sorted(agg.items(), key=lambda kv: -kv[1]["ms"])[:12]}


def family(base):
    """The operation a launch class performs, whatever its storage ("rbgs_split_f64" and
    "rbgs_f64" are both the FP64 colour sweep)."""
    return base.replace("_split", "")


def solver_class(base):
    """Launch classes of the multigrid solves (the field evaluation has its own roofline)."""
    return not (base.startswith("field") or base in ("phasors", "features", "xslices", "face_factors"))


def roofline(prof, peaks, keep=None):
    """The dominant solver operation (storages and grid sizes merged), then its launch
    class and grid size with the most time, among those `keep` accepts: algorithmic work
    per launch (active samples only) over its event-timed average launch time."""
    keep = keep or solver_class
    items = [(k, v) for k, v in prof.items() if keep(base_class(k))]
    if not items:
        return None
    tot = {}
    for k, v in items:
        tot[family(base_class(k))] = tot.get(family(base_class(k)), 0.0) + v["ms"]
    top = max(tot, key=tot.get)
    name, rec = max(((k, v) for k, v in items if family(base_class(k)) == top), key=lambda kv: kv[1]["ms"])
    base = base_class(name)
    timed = max(rec["timed"], 1)
    avg_s = rec["ms"] / 1e3 / timed
    per_launch_bytes = rec["bytes"] / max(rec["launches"], 1)
    per_launch_flops = rec["flops"] / max(rec["launches"], 1)
    hbm_peak = peaks.get("hbm_gbs")
    fp64 = base.endswith("f64") or base in ("residual_mixed", "update_mixed", "coarse_setup", "norm")
    traffic, tsrc = traffic_per_launch(base, rec)
    share = rec["ms"] / max(sum(v["ms"] for v in prof.values()), 1e-30)
    out = {"kernel": name, "share_of_profiled_time": share, "operation_share_of_profiled_time":
           tot[top] / max(sum(v["ms"] for v in prof.values()), 1e-30), "avg_launch_ms": avg_s * 1e3,
           "launches": rec["launches"], "traffic": traffic, "traffic_source": tsrc,
           "dram_gbs_from_traffic": traffic / avg_s / 1e9 if traffic else None}
    # (the nodal-coefficient sweeps, plain or colour-split FP32, account 4 words already)
    nodal = base.startswith("rbgs_nodal") or base == "rbgs_split_f32"
    if base.startswith("rbgs") and not nodal and per_launch_flops > 0:
        # the same work at the nodal-coefficient floor of 4 words per node and sweep: a
        # colour pass (6.5 flops per updated node) updates half the nodes and moves 2 words
        # per node, i.e. 4 per updated node; a fused sweep (13 flops per node) 4 per node
        fused = "fused" in base or "bulk" in base
        nodes = per_launch_flops / 13.0 if fused else per_launch_flops / 6.5
        word = 8 if base.endswith("f64") else 4
        floor = nodes * 4 * word / avg_s / 1e9
        out["hbm_gbs_at_4word_floor"] = floor
        out["hbm_frac_at_4word_floor"] = floor / hbm_peak if hbm_peak else None
    if fp64:
        achieved = per_launch_flops / avg_s / 1e12
        out.update({"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": achieved / FP64_PEAK_TFLOPS,
                    "peak_source": "FP64 from unit counts and clock: 152 SMs x 2 FMA/clk x 2 flop x 2.07 GHz",
                    "hbm_achieved_gbs": per_launch_bytes / avg_s / 1e9,
                    "hbm_frac_of_measured": (per_launch_bytes / avg_s / 1e9) / hbm_peak if hbm_peak else None})
        return out
    achieved = per_launch_bytes / avg_s / 1e9
    peak = hbm_peak if hbm_peak else 6800.0
    out.update({"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "peak_source": "measured" if hbm_peak else "fallback"})
    return out


def field_roofline(prof, peaks=None):
    """The field evaluation: node-features per second and its share of the profiled time.
    The tensor-core form (field_tc: the volume x < n - 1; field_tc_face: the face x = n - 1)
    executes 28 slice-pair products of 2 terms per node-feature (112 bf16 flops), reported
    against the measured sustained bf16 rate; the
    double-float form (field_df32) ~24 FP32 operations per node-feature on the FP32 pipe
    (ncu: profiles/field_df32_n129_b8.md)."""
    recs = [(base_class(k), v) for k, v in prof.items()
            if base_class(k).startswith("field") or base_class(k) in ("xslices", "face_factors")]
    if not recs:
        return None

    def secs(rs):
        return sum(v["ms"] * v["launches"] / max(v["timed"], 1) for _, v in rs) / 1e3

    ms = sum(v["ms"] for _, v in recs)
    node_features = sum(v["flops"] for b, v in recs if b.startswith("field")) / 4.0
    out = {"node_features_per_s": node_features / secs(recs) if secs(recs) > 0 else None,
           "share_of_profiled_time": ms / max(sum(v["ms"] for v in prof.values()), 1e-30)}
    tc = [(b, v) for b, v in recs if b in ("field_tc", "field_tc_face")]
    if tc and secs(tc) > 0:
        peaks = peaks or {}
        peak = peaks.get("bf16_tflops_sustained") or peaks.get("bf16_tflops")
        achieved = 112.0 * sum(v["flops"] for _, v in tc) / 4.0 / secs(tc) / 1e12
        out.update({"kernel": "field_tc", "bound": "tensor (bf16 slices, exact FP32 group sums; tcgen05 from 65^3)",
                    "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak if peak else None,
                    "peak_source": "measured sustained cuBLAS bf16" if peak else None,
                    "ncu": "profiles/field_umma_n129_b8.md (tcgen05 volume), profiles/field_tc_n129_b8.md "
                           "(mma.sync form)"})
        return out
    out.update({"kernel": "field_df32", "bound": "alu (FP32 pipe, double-float)",
                "fp32_ops_per_s": 24.0 * out["node_features_per_s"] if out["node_features_per_s"] else None,
                "ncu": "FP32 pipe 69.6% busy at 129^3 x 8 (profiles/field_df32_n129_b8.md)"})
    return out


def lane_items(levels, N, times, lanes):
    """The lane plan of one step (paper_1607_03252_gb300.planner.lane_plan: the one-GPU
    form of the paper's dynamic level scheduling, Sec. 5.3)."""
    from paper_1607_03252_gb300.planner import lane_plan

    return lane_plan(levels, N, times, lanes)


class MergedLevel:
    """Level record merged from chunk records (Chan's formula, chunks in id order)."""

    def __init__(self, parts):
        from paper_1607_03252_gb300.stats import chan_merge

        n, mean, m2 = chan_merge([(float(p.N), p.mean, p.M2) for p in parts])
        self.N, self.mean, self.M2 = int(n), mean, m2
        self.var_unbiased = m2 / (n - 1) if n > 1 else 0.0
        self.mean_cycles_fine = sum(p.N * p.mean_cycles_fine for p in parts) / max(n, 1)
        self.mean_cycles_coarse = sum(p.N * p.mean_cycles_coarse for p in parts) / max(n, 1)


def run_lanes(torch, lanes, lane_streams, main_stream, body):
    """Runs body(i) for every lane i, lane 0 on this thread and the others on their own
    host threads (the library calls release the GIL), each lane's work on its own
    stream, ordered after the work already on `main_stream`; `main_stream` then waits
    for every lane."""
    import threading

    if len(lanes) == 1:
        body(0)
        return
    start = torch.cuda.Event()
    start.record(main_stream)
    for st in lane_streams[1:]:
        st.wait_event(start)
    errors = []

    def wrap(i):
        try:
            body(i)
        except BaseException as e:  # re-raised on the calling thread
            errors.append(e)

    threads = [threading.Thread(target=wrap, args=(i,)) for i in range(1, len(lanes))]
    for t in threads:
        t.start()
    wrap(0)
    for t in threads:
        t.join()
    for st in lane_streams[1:]:
        done = torch.cuda.Event()
        done.record(st)
        main_stream.wait_event(done)
    if errors:
        raise errors[0]


def e2e_measure(args, mg, torch, cfg, levels, N, single, prec, rank, world, stream, nu_cfg, skw, lanes):
    """Same workload through mlmc_level_estimate: ids built on the host and copied in,
    Y/Qf/Qc copied back into pinned host buffers, every step."""
    import ctypes

    import numpy as np

    bufs = {l: [torch.empty(n, dtype=torch.float64, pin_memory=True) for _ in range(3)] for l, n in zip(levels, N)}
    lane_streams = [stream] + [torch.cuda.Stream() for _ in lanes[1:]]
    cfgs = {}
    Nof = dict(zip(levels, N))
    for i, its in enumerate(lanes):
        for (l, a, b) in its:
            n0 = level_n(l) if single else 17
            cfgs[(l, a)] = (mg.make_mlmc_cfg(RUN_SEED, cfg["sigma2"], cfg["ell"], cfg["M"], n0=n0, nu1=nu_cfg[0],
                                             nu2=nu_cfg[1], rtol=cfg["rtol"], precision=prec, max_batch=Nof[l],
                                             stream=lane_streams[i], **skw),
                            0 if single else l)
    L = mg.lib()
    dp = ctypes.POINTER(ctypes.c_double)

    def lane(i):
        for (l, a, b) in lanes[i]:
            n = Nof[l]
            c, lvl = cfgs[(l, a)]
            first = int(sample_ids(l, rank * n + a, 1)[0])
            out = mg.LevelStats()
            y, qf, qc = (ctypes.cast(buf.data_ptr() + 8 * a, dp) for buf in bufs[l])
            st = L.mlmc_level_estimate(ctypes.byref(c), lvl, first, b - a, y, qf, qc, ctypes.byref(out))
            if st < 0:
                raise mg.MlmcError(st, "mlmc_level_estimate", L.mlmc_last_error_string().decode())

    def step():
        run_lanes(torch, lanes, lane_streams, stream, lane)

    for _ in range(max(1, min(args.warmup, 2))):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    if world > 1:
        t = torch.tensor([dt], dtype=torch.float64, device=torch.device("cuda", torch.cuda.current_device()))
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        dt = float(t.item())
    return {"value": sum(N) * world * args.steps / dt, "unit": "samples/s",
            "h2d_bytes_per_step": int(8 * sum(N)), "d2h_bytes_per_step": int(24 * sum(N)),
            "api": "mlmc_level_estimate (host ids in, Y/Qf/Qc to pinned host memory)"}


def cpu_baseline(cfg, levels, N, single):
    import oracle

    threads = 1 if cfg.get("disc") == "fe" else oracle.max_threads()  # the FE oracle is plain numpy
    counts = oracle_counts(levels, threads, cfg)
    rates, secs = oracle_level_rates(cfg, levels, single, counts)
    value = extrapolated_rate(levels, N, rates)
    return {"value": value, "unit": "samples/s", "cores": threads, "kind": "oracle",
            "sample": "levels %s: %s samples (same ids as the GPU run; 0 = rate extrapolated from the level below "
                      "by 8x nodes), %.1f s of CPU time; per-level samples/s extrapolated to N=%s"
                      % (levels, counts, sum(secs.values()), N),
            "per_level": {str(l): rates[l] for l in levels}}


def serving_run(mg, probs, levels, cfg):
    """The serving loop of c4: returns run(rate, count, seed, burst) -> latency record."""
    import numpy as np

    from paper_1607_03252_gb300.workloads import level_draws, poisson_arrivals

    field = mg.field_cfg(RUN_SEED, cfg["sigma2"], cfg["ell"], cfg["M"])
    mgc = mg.mg_cfg(0, 0, cfg["rtol"], 300, mg.MLMC_PREC_MIXED, mg.MLMC_SMOOTH_AUTO, mg.MLMC_ACCEL_CG)
    counter = [0]

    def run(rate, count, seed, burst=False):
        draws = level_draws(probs, count, seed)
        times = np.zeros(count) if burst else poisson_arrivals(rate, count, seed + 1)
        with mg.Service(field, mgc, n0=17, max_level=max(levels), max_batch=64, workers=3,
                        hbm_budget_bytes=96 << 30, batch_wait_ms=2.0) as svc:
            t0 = time.perf_counter()
            tickets = []
            for i in range(count):
                while time.perf_counter() - t0 < times[i]:
                    pass
                lvl = int(draws[i])
                tickets.append((lvl, svc.submit(lvl, int(sample_ids(lvl, (1 << 44) + counter[0], 1)[0]))))
                counter[0] += 1
            res = [(lvl, svc.wait(t)[1]) for lvl, t in tickets]
            t_end = time.perf_counter()
        lat = {l: [1e3 * (r.t_done - r.t_submit) for lv, r in res if lv == l] for l in levels}
        ok = all(r.status == mg.MLMC_OK for _, r in res)
        t_first = min(r.t_submit for _, r in res)
        t_last = max(r.t_done for _, r in res)
        return {"offered_per_s": rate, "completed_per_s": count / (t_last - t_first), "all_ok": ok,
                "p50_ms": {str(l): float(np.percentile(v, 50)) if v else None for l, v in lat.items()},
                "p99_ms": {str(l): float(np.percentile(v, 99)) if v else None for l, v in lat.items()},
                "count": {str(l): len(v) for l, v in lat.items()}, "wall_s": t_end - t0}

    return run


def serving_line(mg, probs, levels, cfg, plan, burst_count, fracs, max_count, seconds_per_point):
    run = serving_run(mg, probs, levels, cfg)
    sat = run(0.0, burst_count, 11, burst=True)["completed_per_s"]
    sweep = []
    for frac in fracs:
        rate = frac * sat
        count = int(min(max_count, max(150, rate * seconds_per_point)))
        r = run(rate, count, 100 + int(frac * 100))
        r["load_fraction"] = frac
        sweep.append(r)
    return {"metric": "MLMC samples/s at saturation, served (c4: single-sample Poisson requests, levels 17^3..257^3)",
            "value": sat, "unit": "samples/s", "n_gpus": 1, "steps": len(sweep), "warmup": 1, "ms_per_step": None,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic (seeded Philox realisations, Poisson arrivals)",
            "config": {"workload": cfg["name"], "levels": levels, "level_probability": list(map(float, probs)),
                       "service": {"max_batch": 64, "workers": 3, "batch_wait_ms": 2.0, "hbm_budget_gb": 96},
                       "sigma2": cfg["sigma2"], "ell": cfg["ell"], "M": cfg["M"], "rtol": cfg["rtol"],
                       "solver": "FP64 flexible CG, FP32 V-cycle preconditioner (autotuned smoother, nu)",
                       "saturation_burst_requests": burst_count},
            "serving_sweep": sweep, "plan": plan}


def serving_arm(args):
    """c4: open-loop Poisson stream of single-sample requests into the solve service."""
    import numpy as np
    import torch

    import paper_1607_03252_gb300 as mg

    rank, world, local = dist_env()
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    cfg = CONFIGS["c4"]
    levels = cfg["levels"]
    stream = torch.cuda.Stream()
    N, plan = plan_levels(mg, CONFIGS["c3"], levels, stream, 0)  # autotunes every level, pilot, Eq. 11
    probs = np.array([n * c for n, c in zip(N, plan["pilot_cost_s"])])
    probs = probs / probs.sum()
    line = serving_line(mg, probs, levels, cfg, plan, 1200, (0.1, 0.25, 0.5, 0.75, 0.9, 1.0, 1.2), 3000, 3.0)
    print(json.dumps(line), flush=True)
    return 0


def sub_c3(args):
    """The mixed-precision 5-level workload measured like the headline, plus the error of
    its Y_l against FP64 solves of the same realisations (first ids of every level)."""
    import numpy as np
    import torch

    import paper_1607_03252_gb300 as mg

    line = measure(args, "c3", full=False)
    cfg = CONFIGS["c3"]
    stream = torch.cuda.Stream()
    errs, worst = {}, 0.0
    for l in cfg["levels"]:
        K = 4 if l < 4 else 2
        first = int(sample_ids(l, 0, 1)[0])
        kw = dict(n0=17, rtol=cfg["rtol"], accel=mg.MLMC_ACCEL_CG, max_cycles=300, stream=stream)
        cm = mg.make_mlmc_cfg(RUN_SEED, cfg["sigma2"], cfg["ell"], cfg["M"], nu1=0, nu2=0,
                              precision=mg.MLMC_PREC_MIXED, **kw)
        c64 = mg.make_mlmc_cfg(RUN_SEED, cfg["sigma2"], cfg["ell"], cfg["M"], nu1=2, nu2=2, precision=mg.MLMC_PREC_F64,
                               smoother=mg.MLMC_SMOOTH_TWO_PASS, **kw)
        _, Ym, _, _ = mg.mlmc_level_estimate(cm, l, first, K)
        _, Y64, Qf64, Qc64 = mg.mlmc_level_estimate(c64, l, first, K)
        e = np.abs(Ym - Y64) / np.maximum(np.abs(Qf64), np.abs(Qc64))
        errs[str(l)] = float(e.max())
        worst = max(worst, float(e.max()))
    line["mixed_err_vs_f64"] = {"max": worst, "per_level": errs, "samples_per_level": "4 (2 on level 4)",
                                "how": "|Y_mixed - Y_f64| / max(|Qf_f64|, |Qc_f64|) per sample, both solved to "
                                       "rtol 1e-10 (FP64 flexible CG with an FP64 V-cycle as the reference)"}
    return line


def sub_c4(args, c3line):
    """A short serving sweep of the c4 workload (levels drawn with probability N_l C_l of
    the c3 plan just measured; the tuning table of that plan is in place)."""
    import numpy as np

    import paper_1607_03252_gb300 as mg

    plan = (c3line or {}).get("plan") or {}
    N, C = plan.get("N_from_eq11"), plan.get("pilot_cost_s")
    if not N or not C:
        return None
    probs = np.array([n * c for n, c in zip(N, C)])
    probs = probs / probs.sum()
    return serving_line(mg, probs, CONFIGS["c4"]["levels"], CONFIGS["c4"], {"from": "c3 plan of this run"}, 400,
                        (0.25, 0.5, 0.9), 600, 2.0)


def sub_c5(args):
    import torch

    import paper_1607_03252_gb300 as mg

    line = c5_results(args, mg, torch)
    for arm in line["arms"].values():
        arm.pop("rounds_log", None)
    return line


def adaptive_mlmc(mg, torch, cfg, eps, mode, stream, log, lanes=1):
    """Algorithm 2 with L fixed (paper_1607_03252_gb300.estimator): pilot N_init, then N_l
    from Eq. 15 with the running s_l^2 and measured cost per sample, until no level needs
    more samples. mode 'fast': batched, FP32 V-cycle preconditioner (autotuned smoother and
    nu); 'plain': one sample per launch, FP64 throughout. Both use flexible CG around the
    V-cycle and the same realisation ids; the fast arm runs the levels of a round on `lanes`
    concurrent streams."""
    from paper_1607_03252_gb300.estimator import MLMCEstimator

    fast = mode == "fast"
    est = MLMCEstimator(RUN_SEED, cfg["sigma2"], cfg["ell"], cfg["M"], cfg["levels"], cfg["N_init"], eps,
                        cfg["theta"], n0=17, nu=((0, 0) if fast else (cfg["nu1"], cfg["nu2"])), rtol=cfg["rtol"],
                        precision=(mg.MLMC_PREC_MIXED if fast else mg.MLMC_PREC_F64), accel=mg.MLMC_ACCEL_CG,
                        smoother=(mg.MLMC_SMOOTH_AUTO if fast else mg.MLMC_SMOOTH_TWO_PASS),
                        max_batch=(0 if fast else 1), max_cycles=300, stream=stream,
                        streams=([stream] + [torch.cuda.Stream() for _ in range(max(0, lanes - 1))]) if fast else None)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = est.run()
    wall = time.perf_counter() - t0
    log.extend(est.log)
    res.update({"mode": mode, "wall_s": wall})
    return res


def c5_arm(args):
    import torch

    import paper_1607_03252_gb300 as mg

    rank, world, local = dist_env()
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    print(json.dumps(c5_results(args, mg, torch)), flush=True)
    return 0


def c5_results(args, mg, torch):
    cfg = CONFIGS["c5"]
    eps = args.c5_eps or cfg["eps"]
    stream = torch.cuda.Stream()
    # autotune the fast arm once per level (smoother x nu on real samples)
    tune = {}
    for l, n0 in zip(cfg["levels"], cfg["N_init"]):
        c = mg.make_mlmc_cfg(RUN_SEED, cfg["sigma2"], cfg["ell"], cfg["M"], n0=17, nu1=0, nu2=0, rtol=cfg["rtol"],
                             precision=mg.MLMC_PREC_MIXED, stream=stream, accel=mg.MLMC_ACCEL_CG, max_cycles=300)
        rows, bs, bnu = mg.mlmc_autotune(c, l, int(sample_ids(l, 1 << 40, 1)[0]), max(2, min(n0, 16)))
        tune[str(l)] = {"smoother": mg._capi.SMOOTHER_NAMES.get(bs, bs), "nu": bnu}
    out = {}
    for mode in args.c5_arms.split(","):
        log = []
        out[mode] = adaptive_mlmc(mg, torch, cfg, eps, mode, stream, log, lanes=args.lanes)
        out[mode]["rounds_log"] = log
    fast = out.get("fast")
    plain = out.get("plain")
    line = {"metric": "wall time to RMS tolerance eps (c5: adaptive 6-level MLMC, 17^3..513^3)",
            "value": fast["wall_s"] if fast else plain["wall_s"], "unit": "s", "n_gpus": 1, "steps": 1, "warmup": 0,
            "ms_per_step": None, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if fast else "f64", "data": "synthetic (seeded Philox realisations)",
            "config": {"workload": cfg["name"], "levels": cfg["levels"], "fine_n": [level_n(l) for l in cfg["levels"]],
                       "sigma2": cfg["sigma2"], "ell": cfg["ell"], "M": cfg["M"], "eps": eps, "theta": cfg["theta"],
                       "N_init": cfg["N_init"], "rtol": cfg["rtol"]},
            "autotune": tune, "arms": out,
            "speedup_plain_over_fast": (plain["wall_s"] / fast["wall_s"]) if (fast and plain) else None}
    return line


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    if args.config == "c4":
        return serving_arm(args)
    if args.config == "c5":
        return c5_arm(args)
    return own_arm(args)


if __name__ == "__main__":
    sys.exit(main())
