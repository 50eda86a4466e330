"""ctypes binding of include/mlmc.h (argument marshalling only).

Every computation runs in libmlmc_gb300.so. Grid arrays are torch CUDA tensors of
shape (B, n, n, n) (x fastest), passed by data_ptr; streams are torch.cuda.Stream
objects or None (the current torch stream). There is no CPU fallback: a missing
library or CUDA device raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

MLMC_OK = 0
MLMC_PENDING = 1
MLMC_ERR_INVALID = -1
MLMC_ERR_OOM = -2
MLMC_ERR_NOT_CONVERGED = -3
MLMC_ERR_TIMEOUT = -4
MLMC_ERR_CUDA = -5
MLMC_ERR_BUSY = -6
MLMC_ERR_NOT_FOUND = -7
MLMC_ERR_CANCELLED = -8

MLMC_F64 = 0
MLMC_F32 = 1
MLMC_PREC_F64 = 0
MLMC_PREC_MIXED = 1
MLMC_COV_GAUSS = 0
MLMC_COV_EXP = 1
MLMC_COV_SPDE = 2
MLMC_DISC_FV = 0
MLMC_DISC_FE = 1
MLMC_QOI_MEAN = 0
MLMC_QOI_POINT = 1
MLMC_QOI_FLUX = 2

_STATUS_NAMES = {
    MLMC_ERR_INVALID: "MLMC_ERR_INVALID",
    MLMC_ERR_OOM: "MLMC_ERR_OOM",
    MLMC_ERR_NOT_CONVERGED: "MLMC_ERR_NOT_CONVERGED",
    MLMC_ERR_TIMEOUT: "MLMC_ERR_TIMEOUT",
    MLMC_ERR_CUDA: "MLMC_ERR_CUDA",
    MLMC_ERR_BUSY: "MLMC_ERR_BUSY",
    MLMC_ERR_NOT_FOUND: "MLMC_ERR_NOT_FOUND",
    MLMC_ERR_CANCELLED: "MLMC_ERR_CANCELLED",
}


class MlmcError(RuntimeError):
    def __init__(self, status, func, msg):
        super().__init__("%s returned %s: %s" % (func, _STATUS_NAMES.get(status, status), msg))
        self.status = status


class FieldCfg(ctypes.Structure):
    _fields_ = [("run_seed", ctypes.c_uint64), ("sigma2", ctypes.c_double), ("ell", ctypes.c_double),
                ("M", ctypes.c_int), ("cov", ctypes.c_int)]


MLMC_SMOOTH_AUTO = 0
MLMC_SMOOTH_TWO_PASS = 1
MLMC_SMOOTH_FUSED_32x8 = 2
MLMC_SMOOTH_FUSED_32x16 = 3
MLMC_SMOOTH_FUSED_64x8 = 4
MLMC_SMOOTH_BULK_32x8 = 5
MLMC_SMOOTH_BULK_32x16 = 6
MLMC_SMOOTH_BULK_64x8 = 7
MLMC_SMOOTH_NODAL = 8
MLMC_SMOOTH_SPLIT = 9


MLMC_ACCEL_NONE = 0
MLMC_ACCEL_CG = 1
MLMC_ACCEL_FMG = 2


MLMC_ENGINE_AUTO = 0
MLMC_ENGINE_BATCHED = 1
MLMC_ENGINE_CTA = 2


class MgCfg(ctypes.Structure):
    _fields_ = [("nu1", ctypes.c_int), ("nu2", ctypes.c_int), ("rtol", ctypes.c_double),
                ("max_cycles", ctypes.c_int), ("precision", ctypes.c_int), ("smoother", ctypes.c_int),
                ("accel", ctypes.c_int), ("disc", ctypes.c_int), ("engine", ctypes.c_int)]


class MgStats(ctypes.Structure):
    _fields_ = [("cycles", ctypes.c_int), ("rel_res", ctypes.c_double)]


class MlmcCfg(ctypes.Structure):
    _fields_ = [("field", FieldCfg), ("mg", MgCfg), ("n0", ctypes.c_int), ("max_batch", ctypes.c_int),
                ("stream", ctypes.c_void_p), ("qoi", ctypes.c_int)]


class LevelStats(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64), ("mean", ctypes.c_double), ("var_biased", ctypes.c_double),
                ("var_unbiased", ctypes.c_double), ("sum", ctypes.c_double), ("sum_comp", ctypes.c_double),
                ("M2", ctypes.c_double), ("mean_cycles_fine", ctypes.c_double),
                ("mean_cycles_coarse", ctypes.c_double), ("max_cycles_seen", ctypes.c_int),
                ("seconds", ctypes.c_double), ("cost_per_sample", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ServiceCfg(ctypes.Structure):
    _fields_ = [("field", FieldCfg), ("mg", MgCfg), ("n0", ctypes.c_int), ("max_level", ctypes.c_int),
                ("max_batch", ctypes.c_int), ("workers", ctypes.c_int), ("queue_capacity", ctypes.c_int),
                ("hbm_budget_bytes", ctypes.c_size_t), ("batch_wait_ms", ctypes.c_double)]


class Request(ctypes.Structure):
    _fields_ = [("level", ctypes.c_int), ("sample_id", ctypes.c_uint64)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("level", ctypes.c_int), ("sample_id", ctypes.c_uint64),
                ("Y", ctypes.c_double), ("Qf", ctypes.c_double), ("Qc", ctypes.c_double),
                ("cycles_fine", ctypes.c_int), ("cycles_coarse", ctypes.c_int), ("t_submit", ctypes.c_double),
                ("t_start", ctypes.c_double), ("t_done", ctypes.c_double)]


class ServiceReport(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("rejected", ctypes.c_int64),
                ("pending", ctypes.c_int64), ("cancelled", ctypes.c_int64), ("inflight_batches", ctypes.c_int),
                ("bytes_in_use", ctypes.c_size_t),
                ("samples_per_s", ctypes.c_double), ("count", ctypes.c_int64 * 9), ("p50_ms", ctypes.c_double * 9),
                ("p99_ms", ctypes.c_double * 9)]


MLMC_MAX_LEVELS = 9
MLMC_COST_MEASURED = 0
MLMC_COST_NODES = 1
_L9 = MLMC_MAX_LEVELS


class AdaptiveCfg(ctypes.Structure):
    _fields_ = [("level", MlmcCfg), ("L0", ctypes.c_int), ("max_level", ctypes.c_int),
                ("N_init", ctypes.c_int64 * _L9), ("eps", ctypes.c_double), ("theta", ctypes.c_double),
                ("cost_model", ctypes.c_int), ("alpha", ctypes.c_double), ("alpha0", ctypes.c_double),
                ("alpha_floor", ctypes.c_double), ("lanes", ctypes.c_int), ("lane_streams", ctypes.c_void_p * 8)]


class AdaptiveRound(ctypes.Structure):
    _fields_ = [("round", ctypes.c_int), ("L", ctypes.c_int), ("grow", ctypes.c_int),
                ("have", ctypes.c_int64 * _L9), ("N_next", ctypes.c_int64 * _L9), ("alpha", ctypes.c_double),
                ("bias", ctypes.c_double)]


class AdaptiveSummary(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int), ("rounds", ctypes.c_int), ("bias_ok", ctypes.c_int), ("Q_hat", ctypes.c_double),
                ("sampling_var", ctypes.c_double), ("eps_s2", ctypes.c_double), ("alpha", ctypes.c_double),
                ("beta", ctypes.c_double), ("gamma", ctypes.c_double), ("bias", ctypes.c_double),
                ("N", ctypes.c_int64 * _L9), ("mean", ctypes.c_double * _L9), ("var", ctypes.c_double * _L9),
                ("M2", ctypes.c_double * _L9), ("cost", ctypes.c_double * _L9), ("seconds", ctypes.c_double * _L9)]


class AdaptiveState(ctypes.Structure):
    _fields_ = [("magic", ctypes.c_uint32), ("version", ctypes.c_uint32), ("L", ctypes.c_int),
                ("rounds", ctypes.c_int), ("have", ctypes.c_int64 * _L9), ("target", ctypes.c_int64 * _L9),
                ("N", ctypes.c_double * _L9), ("mean", ctypes.c_double * _L9), ("M2", ctypes.c_double * _L9),
                ("seconds", ctypes.c_double * _L9)]


LEVEL_SAMPLER = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_int64,
                                 ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                 ctypes.POINTER(ctypes.c_double))


class TuneEntry(ctypes.Structure):
    _fields_ = [("smoother", ctypes.c_int), ("nu", ctypes.c_int), ("seconds_per_sample", ctypes.c_double),
                ("mean_cycles", ctypes.c_double)]


_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_u64p = ctypes.POINTER(ctypes.c_uint64)

# name -> (restype, argtypes); the exported symbols of include/mlmc.h
SIGNATURES = {
    "mlmc_field_eval": (ctypes.c_int, [ctypes.POINTER(FieldCfg), _u64p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       _vp, _vp]),
    "mlmc_field_eval_pair": (ctypes.c_int, [ctypes.POINTER(FieldCfg), _u64p, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_int, ctypes.c_int, _vp, _vp]),
    "mg_solve_batch": (ctypes.c_int, [ctypes.POINTER(MgCfg), ctypes.c_int, ctypes.c_int, _vp, _vp, _vp,
                                      ctypes.POINTER(MgStats), _vp]),
    "mg_solve_batch_noalloc": (ctypes.c_int, [ctypes.POINTER(MgCfg), ctypes.c_int, ctypes.c_int, _vp, _vp, _vp,
                                              ctypes.POINTER(MgStats), _vp]),
    "mlmc_level_estimate": (ctypes.c_int, [ctypes.POINTER(MlmcCfg), ctypes.c_int, ctypes.c_uint64, ctypes.c_int,
                                           _dp, _dp, _dp, ctypes.POINTER(LevelStats)]),
    "mlmc_level_run": (ctypes.c_int, [ctypes.POINTER(MlmcCfg), ctypes.c_int, _vp, ctypes.c_int, _vp, _vp, _vp,
                                      ctypes.POINTER(LevelStats)]),
    "mlmc_service_create": (ctypes.c_void_p, [ctypes.POINTER(ServiceCfg)]),
    "mlmc_service_destroy": (None, [ctypes.c_void_p]),
    "mlmc_submit": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]),
    "mlmc_poll": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(Result)]),
    "mlmc_wait": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_double, ctypes.POINTER(Result)]),
    "mlmc_cancel": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64]),
    "mlmc_service_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ServiceReport)]),
    "mlmc_set_wait_budget": (ctypes.c_int, [ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]),
    "mlmc_inject_alloc_failure": (ctypes.c_int, [ctypes.c_int64]),
    "mlmc_inject_wait_failure": (ctypes.c_int, [ctypes.c_int]),
    "mlmc_tune_set": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "mlmc_autotune": (ctypes.c_int, [ctypes.POINTER(MlmcCfg), ctypes.c_int, ctypes.c_uint64, ctypes.c_int,
                                     ctypes.POINTER(TuneEntry), ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "mlmc_sample_sizes": (ctypes.c_int, [_dp, _dp, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                         ctypes.POINTER(ctypes.c_int64)]),
    "mlmc_merge_records": (ctypes.c_int, [_dp, ctypes.c_int, _dp]),
    "mlmc_adaptive_create": (ctypes.c_void_p, [ctypes.POINTER(AdaptiveCfg)]),
    "mlmc_adaptive_destroy": (None, [ctypes.c_void_p]),
    "mlmc_adaptive_set_sampler": (ctypes.c_int, [ctypes.c_void_p, LEVEL_SAMPLER, ctypes.c_void_p]),
    "mlmc_adaptive_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]),
    "mlmc_adaptive_run": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "mlmc_adaptive_result": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(AdaptiveSummary)]),
    "mlmc_adaptive_log_count": (ctypes.c_int, [ctypes.c_void_p]),
    "mlmc_adaptive_log_get": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(AdaptiveRound)]),
    "mlmc_adaptive_get_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(AdaptiveState)]),
    "mlmc_adaptive_set_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(AdaptiveState)]),
    "mlmc_profile_enable": (ctypes.c_int, [ctypes.c_int]),
    "mlmc_profile_reset": (ctypes.c_int, []),
    "mlmc_profile_count": (ctypes.c_int, []),
    "mlmc_profile_total_launches": (ctypes.c_int64, []),
    "mlmc_profile_get": (ctypes.c_int, [ctypes.c_int, ctypes.c_char_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                                        ctypes.POINTER(ctypes.c_int64), _dp, _dp, _dp]),
    "mlmc_profile_fma_peak": (ctypes.c_int, [ctypes.c_int, _dp]),
    "mlmc_last_error_string": (ctypes.c_char_p, []),
    "mlmc_version": (ctypes.c_char_p, []),
}

_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = True):
    """Load libmlmc_gb300.so (building it with nvcc if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if build_if_missing else _build.LIB
            if not os.path.exists(path):
                raise RuntimeError("libmlmc_gb300.so not built (%s); run paper_1607_03252_gb300/build.py" % path)
            L = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(status, func):
    if status < 0:
        raise MlmcError(status, func, lib().mlmc_last_error_string().decode())
    return status


def _stream_ptr(stream):
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _grid_tensor(t, dtype, name):
    import torch

    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype or not t.is_contiguous() or t.dim() != 4 or not (t.shape[1] == t.shape[2] == t.shape[3]):
        raise ValueError("%s must be a contiguous %s tensor of shape (B, n, n, n)" % (name, dtype))
    return t


def field_cfg(run_seed, sigma2, ell, M, cov=MLMC_COV_GAUSS):
    return FieldCfg(int(run_seed), float(sigma2), float(ell), int(M), int(cov))


def mg_cfg(nu1=2, nu2=2, rtol=1e-10, max_cycles=100, precision=MLMC_PREC_F64, smoother=MLMC_SMOOTH_AUTO,
           accel=MLMC_ACCEL_NONE, disc=MLMC_DISC_FV, engine=MLMC_ENGINE_AUTO):
    return MgCfg(int(nu1), int(nu2), float(rtol), int(max_cycles), int(precision), int(smoother), int(accel),
                 int(disc), int(engine))


def mlmc_field_eval(cfg: FieldCfg, sample_ids, k_out, stream=None, n_fine=None):
    """k_out (B, n, n, n) float64 or float32 CUDA tensor <- k of the given sample ids; with
    n_fine (n or 2n - 1) the grid's field as a grid of the pair whose fine grid is n_fine
    (mlmc_field_eval_pair)."""
    import torch

    ids = np.ascontiguousarray(np.asarray(sample_ids, dtype=np.uint64))
    if k_out.dtype == torch.float64:
        dt = MLMC_F64
    elif k_out.dtype == torch.float32:
        dt = MLMC_F32
    else:
        raise ValueError("k_out must be float64 or float32")
    _grid_tensor(k_out, k_out.dtype, "k_out")
    if k_out.shape[0] != len(ids):
        raise ValueError("k_out batch %d != %d ids" % (k_out.shape[0], len(ids)))
    if n_fine is None:
        st = lib().mlmc_field_eval(ctypes.byref(cfg), ids.ctypes.data_as(_u64p), len(ids), k_out.shape[1], dt,
                                   ctypes.c_void_p(k_out.data_ptr()), _stream_ptr(stream))
        _check(st, "mlmc_field_eval")
    else:
        st = lib().mlmc_field_eval_pair(ctypes.byref(cfg), ids.ctypes.data_as(_u64p), len(ids), k_out.shape[1],
                                        int(n_fine), dt, ctypes.c_void_p(k_out.data_ptr()), _stream_ptr(stream))
        _check(st, "mlmc_field_eval_pair")


def mg_solve_batch(cfg: MgCfg, k, u, f=None, stream=None, allow_not_converged=False):
    """Solve in place into u; returns (cycles int array, rel_res float array, status)."""
    import torch

    _grid_tensor(k, torch.float64, "k")
    _grid_tensor(u, torch.float64, "u")
    if f is not None:
        _grid_tensor(f, torch.float64, "f")
    if k.shape != u.shape or (f is not None and f.shape != k.shape):
        raise ValueError("k, u (and f) must have the same shape")
    B, n = k.shape[0], k.shape[1]
    stats = (MgStats * B)()
    st = lib().mg_solve_batch(ctypes.byref(cfg), B, n, ctypes.c_void_p(k.data_ptr()),
                              ctypes.c_void_p(f.data_ptr() if f is not None else 0), ctypes.c_void_p(u.data_ptr()),
                              stats, _stream_ptr(stream))
    if not (allow_not_converged and st == MLMC_ERR_NOT_CONVERGED):
        _check(st, "mg_solve_batch")
    cyc = np.array([s.cycles for s in stats], dtype=np.int32)
    rel = np.array([s.rel_res for s in stats], dtype=np.float64)
    return cyc, rel, st


def mlmc_level_estimate(cfg: MlmcCfg, level: int, first_id: int, N: int, want_samples=True,
                        allow_not_converged=False):
    """Returns (LevelStats, Y, Qf, Qc) with numpy arrays (or None when want_samples is False)."""
    Y = np.zeros(N) if want_samples else None
    Qf = np.zeros(N) if want_samples else None
    Qc = np.zeros(N) if want_samples else None
    out = LevelStats()

    def p(a):
        return a.ctypes.data_as(_dp) if a is not None else None

    st = lib().mlmc_level_estimate(ctypes.byref(cfg), int(level), int(first_id), int(N), p(Y), p(Qf), p(Qc),
                                   ctypes.byref(out))
    if not (allow_not_converged and st == MLMC_ERR_NOT_CONVERGED):
        _check(st, "mlmc_level_estimate")
    return out, Y, Qf, Qc


def mlmc_level_run(cfg: MlmcCfg, level: int, ids_dev, Y_dev=None, Qf_dev=None, Qc_dev=None,
                   allow_not_converged=False):
    """Device-resident level run: ids_dev is a uint64-compatible CUDA tensor (int64 dtype);
    outputs are optional float64 CUDA tensors of N entries. Returns LevelStats."""
    N = int(ids_dev.numel())
    out = LevelStats()

    def p(t):
        return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)

    st = lib().mlmc_level_run(ctypes.byref(cfg), int(level), p(ids_dev), N, p(Y_dev), p(Qf_dev), p(Qc_dev),
                              ctypes.byref(out))
    if not (allow_not_converged and st == MLMC_ERR_NOT_CONVERGED):
        _check(st, "mlmc_level_run")
    return out


SMOOTHER_NAMES = {MLMC_SMOOTH_TWO_PASS: "two-pass", MLMC_SMOOTH_FUSED_32x8: "fused 32x8",
                  MLMC_SMOOTH_FUSED_32x16: "fused 32x16", MLMC_SMOOTH_FUSED_64x8: "fused 64x8",
                  MLMC_SMOOTH_BULK_32x8: "bulk 32x8", MLMC_SMOOTH_BULK_32x16: "bulk 32x16",
                  MLMC_SMOOTH_BULK_64x8: "bulk 64x8", MLMC_SMOOTH_NODAL: "nodal", MLMC_SMOOTH_SPLIT: "split"}


def mlmc_autotune(cfg: MlmcCfg, level: int, first_id: int, samples: int):
    """Returns (table as list of dicts, best smoother, best nu); the choice is stored
    for the level's fine grid in the library's tuning table."""
    cap = 64  # 9 smoothers x 4 sweep counts at most
    tab = (TuneEntry * cap)()
    cnt, bs, bnu = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().mlmc_autotune(ctypes.byref(cfg), int(level), int(first_id), int(samples), tab, cap,
                               ctypes.byref(cnt), ctypes.byref(bs), ctypes.byref(bnu)), "mlmc_autotune")
    rows = [dict(smoother=SMOOTHER_NAMES.get(t.smoother, t.smoother), nu=t.nu,
                 ms_per_sample=1e3 * t.seconds_per_sample, cycles=t.mean_cycles)
            for t in tab[:min(cnt.value, cap)]]
    return rows, bs.value, bnu.value


SMOOTHER_IDS = {v: k for k, v in {MLMC_SMOOTH_TWO_PASS: "two-pass", MLMC_SMOOTH_FUSED_32x8: "fused 32x8",
                                   MLMC_SMOOTH_FUSED_32x16: "fused 32x16", MLMC_SMOOTH_FUSED_64x8: "fused 64x8",
                                   MLMC_SMOOTH_BULK_32x8: "bulk 32x8", MLMC_SMOOTH_BULK_32x16: "bulk 32x16",
                                   MLMC_SMOOTH_BULK_64x8: "bulk 64x8", MLMC_SMOOTH_NODAL: "nodal",
                                   MLMC_SMOOTH_SPLIT: "split"}.items()}


def mlmc_tune_set(n: int, precision: int, smoother, nu: int):
    """Stores a tuning choice (smoother id or name, V(nu, nu)) for n^3 grids at `precision`."""
    sm = SMOOTHER_IDS[smoother] if isinstance(smoother, str) else int(smoother)
    _check(lib().mlmc_tune_set(int(n), int(precision), sm, int(nu)), "mlmc_tune_set")


def profile_enable(on=True):
    lib().mlmc_profile_enable(1 if on else 0)


def profile_reset():
    lib().mlmc_profile_reset()


def profile_total_launches():
    return int(lib().mlmc_profile_total_launches())


def profile_fma_peak(precision=MLMC_PREC_F64) -> float:
    """Measured FMA throughput in TFLOP/s (FP64 for MLMC_PREC_F64, FP32 for MLMC_PREC_MIXED)."""
    t = ctypes.c_double()
    _check(lib().mlmc_profile_fma_peak(int(precision), ctypes.byref(t)), "mlmc_profile_fma_peak")
    return t.value


def profile_read():
    """{class: dict(launches, timed, ms, bytes, flops)} (synchronises on recorded events)."""
    L = lib()
    res = {}
    for i in range(L.mlmc_profile_count()):
        name = ctypes.create_string_buffer(128)
        la, ti = ctypes.c_int64(), ctypes.c_int64()
        ms, by, fl = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check(L.mlmc_profile_get(i, name, 128, ctypes.byref(la), ctypes.byref(ti), ctypes.byref(ms), ctypes.byref(by),
                                  ctypes.byref(fl)), "mlmc_profile_get")
        res[name.value.decode()] = dict(launches=la.value, timed=ti.value, ms=ms.value, bytes=by.value,
                                        flops=fl.value)
    return res


def set_wait_budget(clocks: int) -> int:
    """Budget (SM clocks) of the kernels' bounded waits; returns the previous one."""
    prev = ctypes.c_int64()
    _check(lib().mlmc_set_wait_budget(int(clocks), ctypes.byref(prev)), "mlmc_set_wait_budget")
    return prev.value


def inject_alloc_failure(after: int):
    """After `after` more successful device allocations every later one fails with
    MLMC_ERR_OOM (-1: off)."""
    _check(lib().mlmc_inject_alloc_failure(int(after)), "mlmc_inject_alloc_failure")


def inject_wait_failure(launches: int):
    """The next `launches` launches of the tcgen05 field kernel wait on an mbarrier that
    nothing arrives on, so the wait runs out after the wait budget (0: off)."""
    _check(lib().mlmc_inject_wait_failure(int(launches)), "mlmc_inject_wait_failure")


def make_mlmc_cfg(run_seed, sigma2, ell, M, n0=17, nu1=2, nu2=2, rtol=1e-10, max_cycles=100,
                  precision=MLMC_PREC_F64, max_batch=0, stream=None, smoother=MLMC_SMOOTH_AUTO,
                  accel=MLMC_ACCEL_NONE, cov=MLMC_COV_GAUSS, disc=MLMC_DISC_FV, qoi=MLMC_QOI_MEAN,
                  engine=MLMC_ENGINE_AUTO):
    sp = ctypes.c_void_p(0)
    if stream is not None:
        sp = ctypes.c_void_p(stream.cuda_stream)
    return MlmcCfg(field_cfg(run_seed, sigma2, ell, M, cov),
                   mg_cfg(nu1, nu2, rtol, max_cycles, precision, smoother, accel, disc, engine), int(n0),
                   int(max_batch), sp, int(qoi))


class Service:
    """Thin wrapper of the mlmc_service_* calls (continuous-batching solve service)."""

    def __init__(self, field, mg, n0=17, max_level=4, max_batch=64, workers=2, queue_capacity=100000,
                 hbm_budget_bytes=64 << 30, batch_wait_ms=2.0):
        self.cfg = ServiceCfg(field, mg, int(n0), int(max_level), int(max_batch), int(workers), int(queue_capacity),
                              int(hbm_budget_bytes), float(batch_wait_ms))
        self.h = lib().mlmc_service_create(ctypes.byref(self.cfg))
        if not self.h:
            raise MlmcError(MLMC_ERR_INVALID, "mlmc_service_create", lib().mlmc_last_error_string().decode())

    def submit(self, level, sample_id):
        """Returns a ticket, or None when the queue is full (MLMC_ERR_BUSY)."""
        t = ctypes.c_uint64()
        st = lib().mlmc_submit(self.h, ctypes.byref(Request(int(level), int(sample_id))), ctypes.byref(t))
        if st == MLMC_ERR_BUSY:
            return None
        _check(st, "mlmc_submit")
        return t.value

    def poll(self, ticket):
        """(status, Result): status MLMC_PENDING or MLMC_OK."""
        r = Result()
        st = lib().mlmc_poll(self.h, int(ticket), ctypes.byref(r))
        if st < 0:
            _check(st, "mlmc_poll")
        return st, r

    def wait(self, ticket, timeout_ms=60000.0):
        r = Result()
        st = lib().mlmc_wait(self.h, int(ticket), float(timeout_ms), ctypes.byref(r))
        if st == MLMC_ERR_TIMEOUT:
            return st, r
        _check(st, "mlmc_wait")
        return st, r

    def cancel(self, ticket):
        """MLMC_OK if the queued request was withdrawn, MLMC_ERR_BUSY if it already ran
        or is running."""
        st = lib().mlmc_cancel(self.h, int(ticket))
        if st in (MLMC_OK, MLMC_ERR_BUSY):
            return st
        _check(st, "mlmc_cancel")
        return st

    def report(self):
        r = ServiceReport()
        _check(lib().mlmc_service_stats(self.h, ctypes.byref(r)), "mlmc_service_stats")
        return r

    def close(self):
        if self.h:
            lib().mlmc_service_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
