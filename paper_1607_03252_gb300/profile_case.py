"""One small batched field evaluation + multigrid solve, for kernel profiling.

  python -m paper_1607_03252_gb300.profile_case --n 129 --batch 8 --prec f64 --cycles 2 \
      [--smoother two-pass|32x8|32x16|64x8|bulk32x8|bulk32x16|bulk64x8|nodal|split] [--accel cg] [--timing]
      [--field gauss|exp|spde] [--level L --n0 17] [--disc fv|fe] [--accel fmg] [--qoi mean|point|flux]
  python -m paper_1607_03252_gb300.profile_case --fma-peak
  python -m paper_1607_03252_gb300.profile_case --level 0 --batch 64 --engine cta|batched --timing

Evaluates the lognormal field (sigma^2 = 1, ell = 0.3, M = 256 unless given) for `batch`
realisations on an n^3 grid and runs exactly `cycles` V(2,2) cycles (rtol = 0; or V(nu, nu)
to --rtol) through the C ABI, so
that every kernel class launches with the sizes of that grid. With --timing the solve runs
twice and the second run records CUDA events around every launch: per kernel class it
prints launches, device time per launch and algorithmic GB/s, and the same for the field
evaluation (Fourier features, or the SPDE sampler of Sec. 3.2), with its wall time
(MLMC_FIELD_ARITH=0..3 selects the field's arithmetic; 3, the tensor-core form, is the
default). With --level
it instead runs mlmc_level_estimate for `batch` samples of that MLMC level (grids from n0;
the precision, smoother and field as given, rtol 1e-10) and, with --timing, prints the
per-class profile of a second run. With --fma-peak it prints the measured FP64 and FP32
FMA throughput (mlmc_profile_fma_peak) instead. Exits 0 on success.
"""
from __future__ import annotations

import argparse
import sys


def main(argv=None):
    import torch

    import paper_1607_03252_gb300 as mg
    from paper_1607_03252_gb300.workloads import RUN_SEED, sample_ids

    p = argparse.ArgumentParser()
    p.add_argument("--n", type=int, default=129)
    p.add_argument("--batch", type=int, default=8)
    p.add_argument("--prec", choices=["f64", "mixed"], default="f64")
    p.add_argument("--cycles", type=int, default=2)
    p.add_argument("--M", type=int, default=256)
    p.add_argument("--smoother", choices=["auto", "two-pass", "32x8", "32x16", "64x8", "bulk32x8", "bulk32x16",
                                          "bulk64x8", "nodal", "split"], default="auto")
    p.add_argument("--accel", choices=["none", "cg", "fmg"], default="none")
    p.add_argument("--disc", choices=["fv", "fe"], default="fv")
    p.add_argument("--qoi", choices=["mean", "point", "flux"], default="mean")
    p.add_argument("--timing", action="store_true")
    p.add_argument("--nu", type=int, default=2, help="V(nu, nu)")
    p.add_argument("--rtol", type=float, default=0.0, help="stop at this relative residual (0: exactly --cycles)")
    p.add_argument("--sigma2", type=float, default=1.0)
    p.add_argument("--ell", type=float, default=0.3)
    p.add_argument("--field", choices=["gauss", "exp", "spde"], default="gauss")
    p.add_argument("--level", type=int, default=-1, help="run one MLMC level estimate instead")
    p.add_argument("--n0", type=int, default=17)
    p.add_argument("--fma-peak", action="store_true", help="print the measured FP64 and FP32 FMA throughput and exit")
    p.add_argument("--engine", choices=["auto", "batched", "cta"], default="auto",
                   help="execution engine of the solves (mg_cfg.engine)")
    a = p.parse_args(argv)
    if a.fma_peak:
        f64 = mg.profile_fma_peak(mg.MLMC_PREC_F64)
        f32 = mg.profile_fma_peak(mg.MLMC_PREC_MIXED)
        print("fma peak: FP64 %.3f TFLOP/s, FP32 %.2f TFLOP/s, ratio %.1f (%s)"
              % (f64, f32, f32 / f64, torch.cuda.get_device_name()))
        return 0
    prec = mg.MLMC_PREC_F64 if a.prec == "f64" else mg.MLMC_PREC_MIXED
    sm = {"auto": mg.MLMC_SMOOTH_AUTO, "two-pass": mg.MLMC_SMOOTH_TWO_PASS, "32x8": mg.MLMC_SMOOTH_FUSED_32x8,
          "32x16": mg.MLMC_SMOOTH_FUSED_32x16, "64x8": mg.MLMC_SMOOTH_FUSED_64x8,
          "bulk32x8": mg.MLMC_SMOOTH_BULK_32x8, "bulk32x16": mg.MLMC_SMOOTH_BULK_32x16,
          "bulk64x8": mg.MLMC_SMOOTH_BULK_64x8, "nodal": mg.MLMC_SMOOTH_NODAL,
          "split": mg.MLMC_SMOOTH_SPLIT}[a.smoother]
    accel = {"none": mg.MLMC_ACCEL_NONE, "cg": mg.MLMC_ACCEL_CG, "fmg": mg.MLMC_ACCEL_FMG}[a.accel]
    disc = mg.MLMC_DISC_FE if a.disc == "fe" else mg.MLMC_DISC_FV
    qoi = {"mean": mg.MLMC_QOI_MEAN, "point": mg.MLMC_QOI_POINT, "flux": mg.MLMC_QOI_FLUX}[a.qoi]
    cov = {"gauss": mg.MLMC_COV_GAUSS, "exp": mg.MLMC_COV_EXP, "spde": mg.MLMC_COV_SPDE}[a.field]
    fcfg = mg.field_cfg(RUN_SEED, a.sigma2, a.ell, a.M, cov=cov)
    engine = {"auto": mg.MLMC_ENGINE_AUTO, "batched": mg.MLMC_ENGINE_BATCHED, "cta": mg.MLMC_ENGINE_CTA}[a.engine]
    if a.level >= 0:
        fmg = accel == mg.MLMC_ACCEL_FMG
        lcfg = mg.make_mlmc_cfg(RUN_SEED, a.sigma2, a.ell, a.M, n0=a.n0, nu1=a.nu, nu2=a.nu,
                                rtol=0.0 if fmg else 1e-10, max_cycles=a.cycles if fmg else 300, precision=prec,
                                smoother=sm, accel=accel, cov=cov, disc=disc, qoi=qoi, engine=engine)
        first = sample_ids(a.level, 0, 1)[0]
        st, *_ = mg.mlmc_level_estimate(lcfg, a.level, int(first), a.batch, want_samples=False)
        print("level=%d n0=%d samples=%d field=%s mean=%.6e var=%.3e" % (a.level, a.n0, a.batch, a.field, st.mean,
                                                                       st.var_unbiased))
        if a.timing:
            import time

            torch.cuda.synchronize()
            mg.profile_reset()
            t0 = time.perf_counter()
            mg.mlmc_level_estimate(lcfg, a.level, int(first), a.batch, want_samples=False)
            dt = time.perf_counter() - t0
            print("  level estimate wall time: %.3f ms (%.1f samples/s), %d launches (engine %s)"
                  % (dt * 1e3, a.batch / dt, mg.profile_total_launches(), a.engine))
            mg.profile_reset()
            mg.profile_enable(True)
            mg.mlmc_level_estimate(lcfg, a.level, int(first), a.batch, want_samples=False)
            torch.cuda.synchronize()
            mg.profile_enable(False)
            _print_profile(mg.profile_read())
        return 0
    k = torch.empty((a.batch, a.n, a.n, a.n), dtype=torch.float64, device="cuda")
    mg.mlmc_field_eval(fcfg, sample_ids(3, 0, a.batch), k)
    u = torch.zeros_like(k)
    cfg = mg.mg_cfg(a.nu, a.nu, a.rtol, a.cycles, prec, sm, accel, disc, engine)
    cyc, rel, st = mg.mg_solve_batch(cfg, k, u)
    torch.cuda.synchronize()
    print("n=%d batch=%d prec=%s cycles=%s rel_res=%.3e" % (a.n, a.batch, a.prec, cyc.tolist(), rel.max()))
    if a.timing:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        mg.mlmc_field_eval(fcfg, sample_ids(3, 0, a.batch), k)
        e1.record()
        torch.cuda.synchronize()
        print("  %s field wall time: %.3f ms (%.1f samples/s)" % (a.field, e0.elapsed_time(e1),
                                                                a.batch / (e0.elapsed_time(e1) * 1e-3)))
        mg.profile_reset()
        mg.profile_enable(True)
        mg.mlmc_field_eval(fcfg, sample_ids(3, 0, a.batch), k)
        torch.cuda.synchronize()
        mg.profile_enable(False)
        _print_profile(mg.profile_read())
    if a.timing:
        # wall time of a solve on a created stream (graph replay on), then the per-kernel
        # device times with events around every launch (graphs off)
        side = torch.cuda.Stream()
        u.zero_()
        side.wait_stream(torch.cuda.current_stream())
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(side)
        mg.mg_solve_batch(cfg, k, u, stream=side)
        e1.record(side)
        torch.cuda.synchronize()
        print("  solve wall time (graph replay): %.3f ms" % e0.elapsed_time(e1))
        u.zero_()
        mg.profile_reset()
        mg.profile_enable(True)
        mg.mg_solve_batch(cfg, k, u)
        torch.cuda.synchronize()
        mg.profile_enable(False)
        _print_profile(mg.profile_read())
    return 0


def _print_profile(prof):
    for name, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"]):
        if v["timed"] == 0:
            continue
        per = v["ms"] / v["timed"]
        gbs = v["bytes"] / v["launches"] / (per * 1e-3) / 1e9 if per > 0 else 0.0
        print("  %-22s launches %5d  %9.3f us/launch  %8.1f GB/s algorithmic" % (name, v["launches"], per * 1e3, gbs))


if __name__ == "__main__":
    sys.exit(main())
