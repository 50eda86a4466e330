"""CPU checks of the C-ABI library: it builds, loads, and exports every function that
include/*.h declares; argument validation runs on the host without touching a GPU."""
import ctypes
import glob
import os
import re

import pytest

import paper_1607_03252_gb300 as mg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", text, flags=re.M):
            if not m.group(0).lstrip().startswith(("#", "typedef", "return")):
                names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary_calls():
    names = declared_functions()
    for required in ("mlmc_field_eval", "mg_solve_batch", "mlmc_level_estimate", "mlmc_last_error_string"):
        assert required in names


def test_library_exports_every_declared_symbol():
    L = ctypes.CDLL(mg.library_path())
    for name in declared_functions():
        assert hasattr(L, name), name


def test_binding_covers_every_declared_symbol():
    assert set(declared_functions()) <= set(mg.SIGNATURES)


def test_version_string():
    assert b"sm_103a" in mg.lib().mlmc_version()


def _no_gpu():
    try:
        import torch

        return not torch.cuda.is_available()
    except Exception:
        return True


# Tests that pass placeholder device pointers (address 8) rely on the argument checks to
# reject the call before any launch; they run only where no CUDA device is visible, so
# that a regression in those checks can never make a kernel touch that address.
host_only = pytest.mark.skipif(not _no_gpu(), reason="placeholder device pointers: run only without a GPU")


@host_only
def test_invalid_grid_rejected_on_host():
    L = mg.lib()
    cfg = mg.mg_cfg()
    st = L.mg_solve_batch(ctypes.byref(cfg), 1, 6, ctypes.c_void_p(8), None, ctypes.c_void_p(8), None, None)
    assert st == mg.MLMC_ERR_INVALID
    assert b"2^p+1" in L.mlmc_last_error_string()
    st = L.mg_solve_batch(ctypes.byref(cfg), 0, 9, ctypes.c_void_p(8), None, ctypes.c_void_p(8), None, None)
    assert st == mg.MLMC_ERR_INVALID
    bad = mg.mg_cfg(max_cycles=0)
    st = L.mg_solve_batch(ctypes.byref(bad), 1, 9, ctypes.c_void_p(8), None, ctypes.c_void_p(8), None, None)
    assert st == mg.MLMC_ERR_INVALID


@host_only
def test_invalid_field_cfg_rejected_on_host():
    L = mg.lib()
    ids = (ctypes.c_uint64 * 1)(1)
    for cfg in (mg.field_cfg(1, 1.0, 0.0, 8), mg.field_cfg(1, -1.0, 0.3, 8), mg.field_cfg(1, 1.0, 0.3, 0),
                mg.field_cfg(1, 1.0, 0.3, 8, cov=3), mg.field_cfg(1, 1.0, 0.3, 8, cov=-1)):
        st = L.mlmc_field_eval(ctypes.byref(cfg), ids, 1, 9, mg.MLMC_F64, ctypes.c_void_p(8), None)
        assert st == mg.MLMC_ERR_INVALID


@pytest.mark.skipif(not _no_gpu(), reason="checks the no-device path")
def test_no_cpu_fallback_without_device():
    L = mg.lib()
    cfg = mg.make_mlmc_cfg(1, 1.0, 0.3, 8)
    out = mg.LevelStats()
    st = L.mlmc_level_estimate(ctypes.byref(cfg), 0, 0, 1, None, None, None, ctypes.byref(out))
    assert st == mg.MLMC_ERR_CUDA


def test_tune_set_validates_on_host():
    """mlmc_tune_set is host-only: valid entries are stored, invalid ones rejected, no GPU.
    (The stored entries equal the untuned defaults, so later solves in this process are
    unaffected.)"""
    L = mg.lib()
    assert L.mlmc_tune_set(33, mg.MLMC_PREC_MIXED, mg.MLMC_SMOOTH_TWO_PASS, 2) == mg.MLMC_OK
    assert L.mlmc_tune_set(34, mg.MLMC_PREC_MIXED, mg.MLMC_SMOOTH_TWO_PASS, 3) == mg.MLMC_ERR_INVALID
    assert L.mlmc_tune_set(33, 7, mg.MLMC_SMOOTH_TWO_PASS, 3) == mg.MLMC_ERR_INVALID
    assert L.mlmc_tune_set(33, mg.MLMC_PREC_F64, mg.MLMC_SMOOTH_AUTO, 3) == mg.MLMC_ERR_INVALID
    assert L.mlmc_tune_set(33, mg.MLMC_PREC_F64, mg.MLMC_SMOOTH_SPLIT + 1, 3) == mg.MLMC_ERR_INVALID
    assert L.mlmc_tune_set(33, mg.MLMC_PREC_F64, mg.MLMC_SMOOTH_TWO_PASS, 0) == mg.MLMC_ERR_INVALID
    mg.mlmc_tune_set(65, mg.MLMC_PREC_F64, "two-pass", 2)


def test_field_cfg_layout_and_cov_default():
    """cov occupies the former tail padding of mlmc_field_cfg: the size stays 32 bytes and
    a zero-filled struct selects the Gaussian covariance."""
    import ctypes

    assert ctypes.sizeof(mg.FieldCfg) == 32
    assert mg.FieldCfg.cov.offset == 28
    assert mg.field_cfg(1, 1.0, 0.3, 8).cov == mg.MLMC_COV_GAUSS
    assert mg.field_cfg(1, 1.0, 0.3, 8, cov=mg.MLMC_COV_EXP).cov == 1


def test_solver_and_level_cfg_layouts():
    import ctypes

    assert ctypes.sizeof(mg.MgCfg) == 40 and mg.MgCfg.disc.offset == 32
    assert ctypes.sizeof(mg.MlmcCfg) == 96 and mg.MlmcCfg.qoi.offset == 88
    c = mg.make_mlmc_cfg(1, 1.0, 0.3, 8)
    assert c.mg.disc == mg.MLMC_DISC_FV and c.qoi == mg.MLMC_QOI_MEAN


@host_only
def test_fe_and_fmg_cfg_rejected_on_host():
    L = mg.lib()
    for cfg in (mg.mg_cfg(disc=2), mg.mg_cfg(accel=3), mg.mg_cfg(precision=mg.MLMC_PREC_MIXED, disc=mg.MLMC_DISC_FE),
                mg.mg_cfg(precision=mg.MLMC_PREC_MIXED, accel=mg.MLMC_ACCEL_FMG)):
        st = L.mg_solve_batch(ctypes.byref(cfg), 1, 9, ctypes.c_void_p(8), None, ctypes.c_void_p(8), None, None)
        assert st == mg.MLMC_ERR_INVALID
    fmg = mg.mg_cfg(4, 4, 0.0, 2, accel=mg.MLMC_ACCEL_FMG, disc=mg.MLMC_DISC_FE)
    st = L.mg_solve_batch(ctypes.byref(fmg), 1, 9, ctypes.c_void_p(8), ctypes.c_void_p(8), ctypes.c_void_p(8), None,
                          None)
    assert st == mg.MLMC_ERR_INVALID  # FMG solves f = 1 only


@host_only
def test_noalloc_rejects_unsupported_cfgs_on_host():
    L = mg.lib()
    for cfg in (mg.mg_cfg(accel=mg.MLMC_ACCEL_FMG, disc=mg.MLMC_DISC_FE), mg.mg_cfg(disc=5),
                mg.mg_cfg(precision=mg.MLMC_PREC_MIXED, disc=mg.MLMC_DISC_FE)):
        st = L.mg_solve_batch_noalloc(ctypes.byref(cfg), 1, 9, ctypes.c_void_p(8), None, ctypes.c_void_p(8), None,
                                      None)
        assert st == mg.MLMC_ERR_INVALID
