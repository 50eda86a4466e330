"""ctypes wrapper over the plain-C FP64 oracle (test infrastructure only).

Arrays are numpy float64 of shape (n, n, n) indexed [z, y, x] (x fastest in memory),
boundary nodes included, as in mlmc_oracle.c.
"""
from __future__ import annotations

import ctypes
import threading

import numpy as np

from .build import build as _build_oracle

ORC_OK = 0
ORC_ERR_INVALID = -1
ORC_ERR_OOM = -2
ORC_ERR_NOT_CONVERGED = -3

# covariance families of the field (Gaussian; exponential, Sec. 3.2)
COV_GAUSS = 0
COV_EXP = 1
COV_SPDE = 2

_lib = None
_lock = threading.Lock()

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_u64p = ctypes.POINTER(ctypes.c_uint64)


class OrcCfg(ctypes.Structure):
    _fields_ = [
        ("run_seed", ctypes.c_uint64),
        ("sigma2", ctypes.c_double),
        ("ell", ctypes.c_double),
        ("M", ctypes.c_int),
        ("nu1", ctypes.c_int),
        ("nu2", ctypes.c_int),
        ("rtol", ctypes.c_double),
        ("max_cycles", ctypes.c_int),
        ("mixed", ctypes.c_int),
        ("cov", ctypes.c_int),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(_build_oracle())
            L.orc_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
            L.orc_philox4x64_10.argtypes = [_u64p, _u64p, _u64p]
            L.orc_uniforms.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, _dp]
            L.orc_features.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                       _dp, _dp]
            L.orc_logk_point.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_double, ctypes.c_double]
            L.orc_logk_point.restype = ctypes.c_double
            L.orc_field.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_int, ctypes.c_int, _dp]
            L.orc_apply.argtypes = [ctypes.c_int, _dp, _dp, _dp, ctypes.c_int, ctypes.c_double]
            L.orc_residual.argtypes = [ctypes.c_int, _dp, _dp, _dp, _dp, ctypes.c_int, ctypes.c_double]
            L.orc_rbgs_sweep.argtypes = [ctypes.c_int, _dp, _dp, _dp, ctypes.c_int, ctypes.c_double]
            L.orc_restrict_fw.argtypes = [ctypes.c_int, _dp, _dp]
            L.orc_prolong_add.argtypes = [ctypes.c_int, _dp, _dp]
            L.orc_coarse_solve.argtypes = [ctypes.c_int, _dp, _dp, _dp, ctypes.c_int, ctypes.c_double]
            L.orc_mg_solve.argtypes = [ctypes.c_int, _dp, _dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                       ctypes.c_int, ctypes.c_int, ctypes.c_double, _ip, _dp, _dp]
            L.orc_qoi.argtypes = [ctypes.c_int, _dp]
            L.orc_qoi.restype = ctypes.c_double
            L.orc_sample.argtypes = [ctypes.POINTER(OrcCfg), ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                     _dp, _dp, _ip, _ip]
            L.orc_level_batch.argtypes = [ctypes.POINTER(OrcCfg), ctypes.c_int, ctypes.c_int, _u64p, ctypes.c_int,
                                          _dp, _dp, _dp, _ip, _ip, ctypes.c_int]
            L.orc_max_threads.restype = ctypes.c_int
            L.orc_log_series.argtypes = [ctypes.c_float]
            L.orc_log_series.restype = ctypes.c_float
            L.orc_octant_normal.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
            L.orc_octant_normal.restype = ctypes.c_float
            L.orc_spde_noise.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, ctypes.c_int, _dp]
            L.orc_spde_apply.argtypes = [ctypes.c_int, ctypes.c_double, _dp, _dp]
            L.orc_spde_solve.argtypes = [ctypes.c_int, ctypes.c_double, _dp, _dp]
            L.orc_spde_field.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_int, ctypes.c_int, _dp]
            L.orc_assemble_csr.argtypes = [ctypes.c_int, _dp, ctypes.c_int, ctypes.c_double, _ip, _ip, _dp]
            L.orc_assemble_csr.restype = ctypes.c_int
            _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(_dp)


def _grid(a, n):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.shape != (n, n, n):
        raise ValueError("expected shape (%d,%d,%d), got %s" % (n, n, n, a.shape))
    return a


def philox4x32(ctr, key):
    c = (ctypes.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (ctypes.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(x) for x in o]


def philox4x64(ctr, key):
    m = (1 << 64) - 1
    c = (ctypes.c_uint64 * 4)(*[int(x) & m for x in ctr])
    k = (ctypes.c_uint64 * 2)(*[int(x) & m for x in key])
    o = (ctypes.c_uint64 * 4)()
    lib().orc_philox4x64_10(c, k, o)
    return [int(x) for x in o]


def uniforms(run_seed, sample_id, m):
    U = np.zeros(6)
    lib().orc_uniforms(run_seed, sample_id, m, _d(U))
    return U


def features(run_seed, sample_id, M, ell, cov=COV_GAUSS):
    w = np.zeros((M, 3))
    b = np.zeros(M)
    lib().orc_features(run_seed, sample_id, M, ell, int(cov), _d(w), _d(b))
    return w, b


def logk_point(w, b, sigma, x, y, z):
    w = np.ascontiguousarray(w, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    return lib().orc_logk_point(_d(w), _d(b), len(b), sigma, x, y, z)


def field(run_seed, sample_id, M, sigma2, ell, n, cov=COV_GAUSS):
    k = np.zeros((n, n, n))
    st = lib().orc_field(run_seed, sample_id, M, float(np.sqrt(sigma2)), ell, int(cov), n, _d(k))
    if st != ORC_OK:
        raise ValueError("orc_field failed: %d" % st)
    return k


def apply(k, u, mixed=False, c=0.0):
    n = k.shape[0]
    k = _grid(k, n)
    u = _grid(u, n)
    out = np.zeros_like(k)
    lib().orc_apply(n, _d(k), _d(u), _d(out), int(mixed), float(c))
    return out


def residual(k, f, u, mixed=False, c=0.0):
    n = k.shape[0]
    k = _grid(k, n)
    u = _grid(u, n)
    fp = None if f is None else _grid(f, n)
    r = np.zeros_like(k)
    lib().orc_residual(n, _d(k), None if fp is None else _d(fp), _d(u), _d(r), int(mixed), float(c))
    return r


def rbgs_sweep(k, f, u, mixed=False, c=0.0):
    """One red-then-black sweep; returns a new array."""
    n = k.shape[0]
    k = _grid(k, n)
    u = _grid(u, n).copy()
    fp = None if f is None else _grid(f, n)
    lib().orc_rbgs_sweep(n, _d(k), None if fp is None else _d(fp), _d(u), int(mixed), float(c))
    return u


def restrict_fw(r):
    nf = r.shape[0]
    r = _grid(r, nf)
    nc = (nf + 1) // 2
    rc = np.zeros((nc, nc, nc))
    lib().orc_restrict_fw(nf, _d(r), _d(rc))
    return rc


def prolong_add(ec, u):
    nc = ec.shape[0]
    nf = 2 * nc - 1
    ec = _grid(ec, nc)
    u = _grid(u, nf).copy()
    lib().orc_prolong_add(nf, _d(ec), _d(u))
    return u


def coarse_solve(k, f=None, mixed=False, c=0.0):
    n = k.shape[0]
    k = _grid(k, n)
    fp = None if f is None else _grid(f, n)
    u = np.zeros_like(k)
    st = lib().orc_coarse_solve(n, _d(k), None if fp is None else _d(fp), _d(u), int(mixed), float(c))
    if st != ORC_OK:
        raise ValueError("orc_coarse_solve failed: %d" % st)
    return u


def mg_solve(k, f=None, u0=None, nu1=2, nu2=2, rtol=1e-10, max_cycles=100, mixed=False, c=0.0):
    """Returns (u, status, cycles, relres, per-cycle relative residuals)."""
    n = k.shape[0]
    k = _grid(k, n)
    fp = None if f is None else _grid(f, n)
    u = np.zeros_like(k) if u0 is None else _grid(u0, n).copy()
    cyc = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    hist = np.zeros(max(max_cycles, 1))
    st = lib().orc_mg_solve(n, _d(k), None if fp is None else _d(fp), _d(u), nu1, nu2, rtol, max_cycles,
                            int(mixed), float(c), ctypes.byref(cyc), ctypes.byref(rr), _d(hist))
    if st == ORC_ERR_INVALID or st == ORC_ERR_OOM:
        raise ValueError("orc_mg_solve failed: %d" % st)
    return u, st, cyc.value, rr.value, hist[: cyc.value].copy()


def qoi(u):
    n = u.shape[0]
    u = _grid(u, n)
    return lib().orc_qoi(n, _d(u))


def make_cfg(run_seed, sigma2, ell, M, nu1=2, nu2=2, rtol=1e-10, max_cycles=100, mixed=False, cov=COV_GAUSS):
    return OrcCfg(run_seed, sigma2, ell, M, nu1, nu2, rtol, max_cycles, int(mixed), int(cov))


def sample(cfg, n_fine, n_coarse, sample_id):
    qf = ctypes.c_double()
    qc = ctypes.c_double()
    cf = ctypes.c_int()
    cc = ctypes.c_int()
    st = lib().orc_sample(ctypes.byref(cfg), n_fine, n_coarse, sample_id, ctypes.byref(qf), ctypes.byref(qc),
                          ctypes.byref(cf), ctypes.byref(cc))
    return st, qf.value, qc.value, cf.value, cc.value


def level_batch(cfg, n_fine, n_coarse, ids, nthreads=0):
    """Y, Qf, Qc, cycles_f, cycles_c, status for the given sample ids (OpenMP over samples)."""
    ids = np.ascontiguousarray(ids, dtype=np.uint64)
    N = len(ids)
    Y = np.zeros(N)
    Qf = np.zeros(N)
    Qc = np.zeros(N)
    cf = np.zeros(N, dtype=np.int32)
    cc = np.zeros(N, dtype=np.int32)
    st = lib().orc_level_batch(ctypes.byref(cfg), n_fine, n_coarse, ids.ctypes.data_as(_u64p), N, _d(Y), _d(Qf),
                               _d(Qc), cf.ctypes.data_as(_ip), cc.ctypes.data_as(_ip), nthreads)
    return Y, Qf, Qc, cf, cc, st


def max_threads():
    return lib().orc_max_threads()


def assemble_csr(k, mixed=False, c=0.0):
    """scipy.sparse CSR matrix of the operator on the interior nodes (x fastest)."""
    import scipy.sparse as sp

    n = k.shape[0]
    k = _grid(k, n)
    m = n - 2
    N = m ** 3
    indptr = np.zeros(N + 1, dtype=np.int32)
    indices = np.zeros(7 * N, dtype=np.int32)
    data = np.zeros(7 * N)
    nnz = lib().orc_assemble_csr(n, _d(k), int(mixed), float(c), indptr.ctypes.data_as(_ip),
                                 indices.ctypes.data_as(_ip), _d(data))
    return sp.csr_matrix((data[:nnz], indices[:nnz], indptr), shape=(N, N))


# ---- SPDE field sampler (Sec. 3.2) ---------------------------------------------------
def log_series(s):
    """The FP32 natural logarithm the octant normals use (float in, float out)."""
    return lib().orc_log_series(float(s))


def octant_normal(run_seed, sample_id, octant):
    return lib().orc_octant_normal(int(run_seed), int(sample_id), int(octant))


def spde_noise(run_seed, sample_id, n, n_noise=None):
    """Scaled right-hand side g = W(cell) / h on the C^3 cells (C = 2(n-1)) of level grid
    n, shape (C, C, C) indexed [z, y, x]; the noise lives on the octants of grid n_noise."""
    n_noise = n if n_noise is None else n_noise
    C = 2 * (n - 1)
    g = np.zeros((C, C, C))
    st = lib().orc_spde_noise(int(run_seed), int(sample_id), n, n_noise, _d(g))
    if st != ORC_OK:
        raise ValueError("orc_spde_noise failed: %d" % st)
    return g


def spde_apply(Z, ch2):
    Z = np.ascontiguousarray(Z, dtype=np.float64)
    out = np.zeros_like(Z)
    lib().orc_spde_apply(Z.shape[0], float(ch2), _d(Z), _d(out))
    return out


def spde_solve(g, ch2):
    g = np.ascontiguousarray(g, dtype=np.float64)
    Z = np.zeros_like(g)
    st = lib().orc_spde_solve(g.shape[0], float(ch2), _d(g), _d(Z))
    if st != ORC_OK:
        raise ValueError("orc_spde_solve failed: %d" % st)
    return Z


def spde_field(run_seed, sample_id, sigma2, ell, n, n_noise=None):
    """k on the n^3 grid of D from the SPDE sampler (Sec. 3.2)."""
    n_noise = n if n_noise is None else n_noise
    k = np.zeros((n, n, n))
    st = lib().orc_spde_field(int(run_seed), int(sample_id), float(sigma2), float(ell), n, n_noise, _d(k))
    if st != ORC_OK:
        raise ValueError("orc_spde_field failed: %d" % st)
    return k
