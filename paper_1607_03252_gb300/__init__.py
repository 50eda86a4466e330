"""GB300-native (sm_103a) multilevel Monte Carlo multigrid library.

The hot path -- Philox-seeded lognormal field, batched geometric multigrid solves of
-div(k grad u) = 1 on the unit cube, and coupled fine/coarse solves on one realisation
giving Y_l = Q_l - Q_{l-1} (Gmeiner et al., Sec. 2.2, Eq. 8, Algorithm 1) -- runs in
hand-written CUDA behind the C ABI of include/mlmc.h (libmlmc_gb300.so). This package
is a thin ctypes binding with the same names; PyTorch provides device memory and
streams only.

The library is loaded lazily on first use, so that `workloads` (seeded inputs) can be
imported on machines without a GPU.
"""
from ._capi import (  # noqa: F401
    MLMC_ERR_BUSY, MLMC_ERR_CANCELLED, MLMC_ERR_CUDA, MLMC_ERR_INVALID, MLMC_ERR_NOT_CONVERGED, MLMC_ERR_NOT_FOUND, MLMC_ERR_OOM,
    MLMC_ACCEL_FMG, MLMC_ENGINE_AUTO, MLMC_ENGINE_BATCHED, MLMC_ENGINE_CTA, MLMC_COV_EXP, MLMC_COV_GAUSS, MLMC_COV_SPDE, MLMC_DISC_FE, MLMC_DISC_FV, MLMC_QOI_FLUX,
    MLMC_QOI_MEAN, MLMC_QOI_POINT, MLMC_ERR_TIMEOUT, MLMC_F32, MLMC_F64, MLMC_OK, MLMC_PENDING, MLMC_PREC_F64, MLMC_PREC_MIXED, MLMC_ACCEL_NONE, MLMC_ACCEL_CG, MLMC_SMOOTH_AUTO,
    MLMC_SMOOTH_BULK_32x8, MLMC_SMOOTH_BULK_32x16, MLMC_SMOOTH_BULK_64x8, MLMC_SMOOTH_NODAL, MLMC_SMOOTH_SPLIT, MLMC_SMOOTH_FUSED_32x8,
    MLMC_SMOOTH_FUSED_32x16, MLMC_SMOOTH_FUSED_64x8, MLMC_SMOOTH_TWO_PASS, SIGNATURES,
    FieldCfg, LevelStats, MgCfg, MgStats, MlmcCfg, MlmcError, field_cfg, lib, library_path, make_mlmc_cfg, mg_cfg,
    mg_solve_batch, mlmc_field_eval, mlmc_level_estimate, mlmc_level_run, mlmc_autotune, mlmc_tune_set, profile_enable, profile_fma_peak, profile_read,
    profile_reset, profile_total_launches, Service, set_wait_budget, inject_alloc_failure, inject_wait_failure,
)
