"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances (derived in the design notes):
  - field k (FP64): 1e-12 relative (the GPU sums separable phasor products, the oracle
    calls cos per node; both are FP64 and differ by a few ulp per term);
  - u after a FIXED number of cycles: 1e-10 relative in the max norm (the same
    algorithm step by step; only rounding order differs);
  - converged u (rtol 1e-12): 1e-9 relative in the max norm;
  - Y_l: |dY| <= 1e-9 * max(|Q_l|, |Q_{l-1}|) per sample (scale-normalised: Y_l << Q_l),
    in FP64 and in mixed precision alike: the mixed form (FP32 V-cycle corrections of
    residuals taken on the FP64 operator) converges to the FP64 solution, so it is
    compared with the FP64 oracle, and its error against FP64 is printed per result
    ("mixed vs FP64"), far inside the 1e-7 that mixed precision is allowed;
  - cycle counts equal the oracle's within one cycle (a sample near the threshold may
    stop one cycle apart).
"""
import numpy as np
import pytest

import paper_1607_03252_gb300 as mg
from paper_1607_03252_gb300.workloads import RUN_SEED, level_n, random_coefficient, random_rhs, sample_ids

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def gpu_solve(ks, fs=None, precision=mg.MLMC_PREC_F64, rtol=1e-12, max_cycles=100, nu=(2, 2), allow_nc=False):
    k = to_dev(np.stack(ks))
    u = torch.zeros_like(k)
    f = to_dev(np.stack(fs)) if fs is not None else None
    cyc, rel, st = mg.mg_solve_batch(mg.mg_cfg(nu[0], nu[1], rtol, max_cycles, precision), k, u, f,
                                     allow_not_converged=allow_nc)
    torch.cuda.synchronize()
    return u.cpu().numpy(), cyc, rel, st


def relmax(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("n,sigma2,ell,M", [(9, 1.0, 0.3, 256), (17, 2.0, 0.1, 256), (33, 1.0, 0.05, 64)])
def test_field_eval_f64_matches_oracle(orc, n, sigma2, ell, M):
    ids = sample_ids(2, 5, 3)
    k = torch.zeros((3, n, n, n), dtype=torch.float64, device=DEV)
    mg.mlmc_field_eval(mg.field_cfg(RUN_SEED, sigma2, ell, M), ids, k)
    k = k.cpu().numpy()
    for s, sid in enumerate(ids):
        ko = orc.field(RUN_SEED, int(sid), M, sigma2, ell, n)
        assert relmax(k[s], ko) < 1e-12


def test_field_eval_f32_is_rounded_f64(orc):
    n, ids = 17, sample_ids(1, 0, 2)
    cfg = mg.field_cfg(RUN_SEED, 1.0, 0.3, 256)
    k32 = torch.zeros((2, n, n, n), dtype=torch.float32, device=DEV)
    mg.mlmc_field_eval(cfg, ids, k32)
    for s, sid in enumerate(ids):
        ko = orc.field(RUN_SEED, int(sid), 256, 1.0, 0.3, n).astype(np.float32)
        diff_ulps = np.abs(k32[s].cpu().numpy().view(np.int32) - ko.view(np.int32))
        assert diff_ulps.max() <= 1


def test_field_sigma_zero_is_one():
    k = torch.zeros((1, 9, 9, 9), dtype=torch.float64, device=DEV)
    mg.mlmc_field_eval(mg.field_cfg(RUN_SEED, 0.0, 0.3, 16), [7], k)
    assert torch.all(k == 1.0)


@pytest.mark.parametrize("n", [5, 9, 17, 33])
def test_fixed_cycles_match_oracle_step_by_step(orc, n):
    """rtol = 0 runs exactly c cycles: any difference in smoother order, transfer or
    coarse solve shows up at O(1e-3), far above rounding."""
    ks = [random_coefficient(n, 100 + s, 1.0) for s in range(3)]
    fs = [random_rhs(n, 200 + s) for s in range(3)]
    for cycles in (1, 3):
        u, cyc, rel, st = gpu_solve(ks, fs, rtol=0.0, max_cycles=cycles)
        assert st == 0 and np.all(cyc == cycles)
        for s in range(3):
            uo, _, co, rro, _ = orc.mg_solve(ks[s], fs[s], rtol=0.0, max_cycles=cycles)
            assert co == cycles
            assert relmax(u[s], uo) < 1e-10, (n, cycles, s)
            assert rel[s] == pytest.approx(rro, rel=1e-8)


@pytest.mark.parametrize("nu", [(1, 1), (2, 2), (3, 1)])
def test_fixed_cycles_other_smoothing_counts(orc, nu):
    n = 17
    ks = [random_coefficient(n, 7, 1.0)]
    u, cyc, rel, st = gpu_solve(ks, None, rtol=0.0, max_cycles=2, nu=nu)
    uo, *_ = orc.mg_solve(ks[0], None, nu1=nu[0], nu2=nu[1], rtol=0.0, max_cycles=2)
    assert relmax(u[0], uo) < 1e-10


@pytest.mark.parametrize("n", [9, 17, 33, 65])
def test_converged_solution_matches_oracle(orc, n):
    B = 3 if n < 65 else 2
    ks = [orc.field(RUN_SEED, int(i), 256, 1.0, 0.3, n) for i in sample_ids(3, 0, B)]
    u, cyc, rel, st = gpu_solve(ks, rtol=1e-12)
    assert st == 0 and np.all(rel <= 1e-12)
    for s in range(B):
        uo, sto, co, rro, _ = orc.mg_solve(ks[s], None, rtol=1e-12)
        assert relmax(u[s], uo) < 1e-9
        assert abs(int(cyc[s]) - co) <= 1
    # production tolerance: same cycle counts within one
    u2, cyc2, rel2, st2 = gpu_solve(ks, rtol=1e-10)
    for s in range(B):
        _, _, co, _, _ = orc.mg_solve(ks[s], None, rtol=1e-10)
        assert abs(int(cyc2[s]) - co) <= 1


def test_mixed_precision_converges_to_the_fp64_solution(orc):
    n = 33
    ks = [orc.field(RUN_SEED, int(i), 256, 2.0, 0.1, n) for i in sample_ids(2, 0, 2)]
    u, cyc, rel, st = gpu_solve(ks, precision=mg.MLMC_PREC_MIXED, rtol=1e-12)
    assert st == 0 and np.all(rel <= 1e-12)
    for s in range(2):
        u64, *_ = orc.mg_solve(ks[s], None, rtol=1e-12)
        um, *_ = orc.mg_solve(ks[s], None, rtol=1e-12, mixed=True)
        err = relmax(u[s], u64)
        print("mixed vs FP64 (u, max norm, sample %d): %.2e" % (s, err))
        assert err < 1e-9
        # the FP32-faced operator's solution is a different one (about 1e-7 away), so the
        # test would see a solver that stopped at the FP32 operator
        assert relmax(um, u64) > 10 * err


def test_batch_composition_does_not_change_results():
    n = 17
    ks = [random_coefficient(n, 300 + s, 1.0) for s in range(5)]
    for prec in (mg.MLMC_PREC_F64, mg.MLMC_PREC_MIXED):
        ub, cb, rb, _ = gpu_solve(ks, precision=prec, rtol=1e-10)
        for s in (0, 3):
            ua, ca, ra, _ = gpu_solve([ks[s]], precision=prec, rtol=1e-10)
            assert np.array_equal(ua[0], ub[s]) and ca[0] == cb[s]


def test_not_converged_status_and_output_written():
    n = 17
    ks = [random_coefficient(n, 9, 1.0)]
    u, cyc, rel, st = gpu_solve(ks, rtol=1e-10, max_cycles=1, allow_nc=True)
    assert st == mg.MLMC_ERR_NOT_CONVERGED and cyc[0] == 1 and rel[0] > 1e-10
    assert np.abs(u).max() > 0


def test_invalid_arguments_rejected():
    k = torch.ones((1, 6, 6, 6), dtype=torch.float64, device=DEV)
    with pytest.raises(mg.MlmcError) as e:
        mg.mg_solve_batch(mg.mg_cfg(), k, torch.zeros_like(k))
    assert e.value.status == mg.MLMC_ERR_INVALID
    k = torch.ones((1, 9, 9, 9), dtype=torch.float64, device=DEV)
    with pytest.raises(mg.MlmcError):
        mg.mg_solve_batch(mg.mg_cfg(nu1=9, nu2=2), k, torch.zeros_like(k))
    with pytest.raises(mg.MlmcError):
        mg.mg_solve_batch(mg.mg_cfg(smoother=99), k, torch.zeros_like(k))
    with pytest.raises(mg.MlmcError):
        mg.mlmc_field_eval(mg.field_cfg(RUN_SEED, 1.0, -1.0, 8), [1], k)


def _exp_field_tol(orc, sid, M, sigma2, ell):
    """Relative k tolerance for the exponential covariance. Its Cauchy frequencies reach
    |w| ~ 1e4 / ell, and the GPU rounds w_x x, w_y y, w_z z + b separately where the oracle
    rounds their sum: per feature the phases differ by at most ~4 eps (|w|_1 + 2 pi), so
    log k differs by sigma sqrt(2/M) times the sum of those bounds, plus the 1e-12 of the
    Gaussian case (the separable products in double-float)."""
    w, _ = orc.features(RUN_SEED, int(sid), M, ell, cov=orc.COV_EXP)
    eps = np.finfo(np.float64).eps
    phase = np.sum(4.0 * eps * (np.abs(w).sum(axis=1) + 2.0 * np.pi))
    return 1e-12 + np.sqrt(sigma2) * np.sqrt(2.0 / M) * phase


@pytest.mark.parametrize("n,sigma2,ell,M", [(9, 1.0, 0.3, 256), (17, 2.0, 0.1, 256), (33, 1.0, 0.05, 64)])
def test_field_eval_exp_covariance_matches_oracle(orc, n, sigma2, ell, M):
    ids = sample_ids(2, 5, 3)
    k = torch.zeros((3, n, n, n), dtype=torch.float64, device=DEV)
    mg.mlmc_field_eval(mg.field_cfg(RUN_SEED, sigma2, ell, M, cov=mg.MLMC_COV_EXP), ids, k)
    k = k.cpu().numpy()
    for s, sid in enumerate(ids):
        ko = orc.field(RUN_SEED, int(sid), M, sigma2, ell, n, cov=orc.COV_EXP)
        assert np.max(np.abs(k[s] - ko) / ko) < _exp_field_tol(orc, sid, M, sigma2, ell)
        # and it is not the Gaussian field of the same draws
        assert relmax(k[s], orc.field(RUN_SEED, int(sid), M, sigma2, ell, n)) > 1e-3


def _y_tol(Qf, Qc, tol):
    return tol * np.maximum(np.abs(Qf), np.abs(Qc))


@pytest.mark.parametrize("level", [0, 1, 2])
def test_level_estimate_matches_oracle(orc, level):
    ids = sample_ids(level, 0, 6)
    cfg = mg.make_mlmc_cfg(RUN_SEED, 1.0, 0.3, 256, n0=17, rtol=1e-12)
    stats, Y, Qf, Qc = mg.mlmc_level_estimate(cfg, level, int(ids[0]), len(ids))
    ocfg = orc.make_cfg(RUN_SEED, 1.0, 0.3, 256, rtol=1e-12)
    nf = level_n(level)
    nc = level_n(level - 1) if level > 0 else 0
    Yo, Qfo, Qco, cfo, cco, sto = orc.level_batch(ocfg, nf, nc, ids)
    assert sto == 0
    assert np.all(np.abs(Y - Yo) <= _y_tol(Qfo, Qco, 1e-9))
    assert np.all(np.abs(Qf - Qfo) <= 1e-9 * np.abs(Qfo))
    assert stats.N == len(ids)
    assert stats.mean == pytest.approx(orc.stats.level_mean(list(Yo)), abs=1e-9 * np.abs(Qfo).mean())
    if level == 0:
        assert np.all(Qc == 0)


def _mixed_err(Y, Y64, Qf64, Qc64, what):
    err = np.abs(Y - Y64) / np.maximum(np.abs(Qf64), np.abs(Qc64))
    print("mixed vs FP64 (%s, |dY| / max|Q| per sample): %s" % (what, " ".join("%.1e" % e for e in err)))
    return err


def test_level_estimate_mixed_matches_oracle(orc):
    # sigma^2 = 2, ell = 0.2: the stationary V(2,2) cycle converges on every sample
    # (at ell = 0.1 some samples need far more than 100 cycles, on both sides)
    level, ids = 1, sample_ids(1, 10, 4)
    cfg = mg.make_mlmc_cfg(RUN_SEED, 2.0, 0.2, 256, n0=17, rtol=1e-11, precision=mg.MLMC_PREC_MIXED)
    _, Y, Qf, Qc = mg.mlmc_level_estimate(cfg, level, int(ids[0]), len(ids))
    Y64, Qf64, Qc64, *_ = orc.level_batch(orc.make_cfg(RUN_SEED, 2.0, 0.2, 256, rtol=1e-11), 33, 17, ids)
    assert np.all(_mixed_err(Y, Y64, Qf64, Qc64, "level 1, iterative refinement") <= 1e-9)


@pytest.mark.parametrize("level", [0, 1, 2])
def test_level_estimate_exp_covariance_matches_oracle(orc, level):
    """The paper's exponential covariance (rougher fields, 15-25 cycles at rtol 1e-12)."""
    ids = sample_ids(level, 40, 5)
    cfg = mg.make_mlmc_cfg(RUN_SEED, 1.0, 0.1, 256, n0=17, rtol=1e-12, max_cycles=300, cov=mg.MLMC_COV_EXP)
    stats, Y, Qf, Qc = mg.mlmc_level_estimate(cfg, level, int(ids[0]), len(ids))
    ocfg = orc.make_cfg(RUN_SEED, 1.0, 0.1, 256, rtol=1e-12, max_cycles=300, cov=orc.COV_EXP)
    nf = level_n(level)
    nc = level_n(level - 1) if level > 0 else 0
    Yo, Qfo, Qco, cfo, cco, sto = orc.level_batch(ocfg, nf, nc, ids)
    assert sto == 0
    assert np.all(np.abs(Y - Yo) <= _y_tol(Qfo, Qco, 1e-9))
    assert np.all(np.abs(Qf - Qfo) <= 1e-9 * np.abs(Qfo))
    assert stats.N == len(ids)


def test_level_estimate_exp_covariance_mixed(orc):
    level, ids = 1, sample_ids(1, 50, 4)
    kw = dict(rtol=1e-11, max_cycles=300)
    cfg = mg.make_mlmc_cfg(RUN_SEED, 1.0, 0.1, 256, n0=17, precision=mg.MLMC_PREC_MIXED, accel=mg.MLMC_ACCEL_CG,
                           cov=mg.MLMC_COV_EXP, **kw)
    _, Y, Qf, Qc = mg.mlmc_level_estimate(cfg, level, int(ids[0]), len(ids))
    Y64, Qf64, Qc64, *_ = orc.level_batch(orc.make_cfg(RUN_SEED, 1.0, 0.1, 256, cov=orc.COV_EXP, **kw), 33, 17, ids)
    assert np.all(_mixed_err(Y, Y64, Qf64, Qc64, "level 1, exponential covariance, CG") <= 1e-9)


def test_level_estimate_batch_size_invariant():
    cfg1 = mg.make_mlmc_cfg(RUN_SEED, 1.0, 0.3, 64, n0=17, rtol=1e-10, max_batch=3)
    cfg2 = mg.make_mlmc_cfg(RUN_SEED, 1.0, 0.3, 64, n0=17, rtol=1e-10, max_batch=0)
    s1, Y1, _, _ = mg.mlmc_level_estimate(cfg1, 1, int(sample_ids(1, 0, 1)[0]), 7)
    s2, Y2, _, _ = mg.mlmc_level_estimate(cfg2, 1, int(sample_ids(1, 0, 1)[0]), 7)
    assert np.array_equal(Y1, Y2)
    assert s1.mean == s2.mean and s1.M2 == s2.M2


def test_c2_level3_full_size_sampled(orc):
    """Level 3 of the 4-level FP64 workload (129^3 fine, 65^3 coarse) in the batch size
    the benchmark uses (64); three samples of the batch recomputed by the oracle."""
    ids = sample_ids(3, 0, 64)
    cfg = mg.make_mlmc_cfg(RUN_SEED, 1.0, 0.3, 256, n0=17, rtol=1e-10, max_batch=64)
    stats, Y, Qf, Qc = mg.mlmc_level_estimate(cfg, 3, int(ids[0]), 64)
    pick = [0, 31, 63]
    ocfg = orc.make_cfg(RUN_SEED, 1.0, 0.3, 256, rtol=1e-10)
    Yo, Qfo, Qco, cfo, cco, sto = orc.level_batch(ocfg, 129, 65, ids[pick])
    assert sto == 0
    # rtol 1e-10 on both sides: the stopping points may differ by one cycle (error ~1e-10)
    assert np.all(np.abs(Y[pick] - Yo) <= _y_tol(Qfo, Qco, 1e-8))
    assert np.all(np.isfinite(Y)) and stats.max_cycles_seen < 30


SMOOTHERS = [mg.MLMC_SMOOTH_TWO_PASS, mg.MLMC_SMOOTH_FUSED_32x8, mg.MLMC_SMOOTH_FUSED_32x16, mg.MLMC_SMOOTH_FUSED_64x8,
             mg.MLMC_SMOOTH_BULK_32x8, mg.MLMC_SMOOTH_BULK_32x16, mg.MLMC_SMOOTH_BULK_64x8]


@pytest.mark.parametrize("prec", [mg.MLMC_PREC_F64, mg.MLMC_PREC_MIXED])
@pytest.mark.parametrize("n", [9, 17, 33, 65])
def test_smoother_variants_identical_fixed_cycles(prec, n):
    """The fused one-pass sweep (every tile shape) performs the same operations on the
    same operands as the two-pass colour sweep: identical iterates, bit for bit (batched
    engine: the kernels themselves)."""
    B = 3
    k = to_dev(np.stack([random_coefficient(n, 500 + s, 1.0) for s in range(B)]))
    f = to_dev(np.stack([random_rhs(n, 600 + s) for s in range(B)]))
    outs = []
    for sm in SMOOTHERS:
        u = torch.zeros_like(k)
        cyc, rel, st = mg.mg_solve_batch(mg.mg_cfg(2, 2, 0.0, 3, prec, sm, engine=mg.MLMC_ENGINE_BATCHED), k, u, f)
        outs.append((u.cpu().numpy(), rel))
    for u, rel in outs[1:]:
        assert np.array_equal(u, outs[0][0])
        assert np.array_equal(rel, outs[0][1])


@pytest.mark.parametrize("prec", [mg.MLMC_PREC_F64, mg.MLMC_PREC_MIXED])
def test_smoother_variants_identical_with_masking(prec, orc):
    """Samples that converge at different cycle counts: finished samples must keep
    their iterate under the double-buffered fused sweep."""
    n, B = 33, 4
    ks = [orc.field(RUN_SEED, int(i), 256, 1.0 + 0.5 * s, 0.15, n) for s, i in enumerate(sample_ids(4, 0, B))]
    k = to_dev(np.stack(ks))
    outs = []
    for sm in SMOOTHERS:
        u = torch.zeros_like(k)
        cyc, rel, st = mg.mg_solve_batch(mg.mg_cfg(2, 2, 1e-10, 200, prec, sm, engine=mg.MLMC_ENGINE_BATCHED), k, u)
        outs.append((u.cpu().numpy(), cyc))
    assert len(set(outs[0][1].tolist())) > 1  # the samples did stop at different cycles
    for u, cyc in outs[1:]:
        assert np.array_equal(cyc, outs[0][1])
        assert np.array_equal(u, outs[0][0])


GRAPH_CASES = [(mg.MLMC_PREC_F64, mg.MLMC_ACCEL_NONE, mg.MLMC_SMOOTH_TWO_PASS),
               (mg.MLMC_PREC_F64, mg.MLMC_ACCEL_NONE, mg.MLMC_SMOOTH_FUSED_32x16),
               (mg.MLMC_PREC_MIXED, mg.MLMC_ACCEL_NONE, mg.MLMC_SMOOTH_FUSED_32x8),
               (mg.MLMC_PREC_MIXED, mg.MLMC_ACCEL_CG, mg.MLMC_SMOOTH_FUSED_64x8),
               (mg.MLMC_PREC_MIXED, mg.MLMC_ACCEL_CG, mg.MLMC_SMOOTH_NODAL),
               (mg.MLMC_PREC_MIXED, mg.MLMC_ACCEL_CG, mg.MLMC_SMOOTH_SPLIT),
               (mg.MLMC_PREC_MIXED, mg.MLMC_ACCEL_NONE, mg.MLMC_SMOOTH_SPLIT),
               (mg.MLMC_PREC_F64, mg.MLMC_ACCEL_NONE, mg.MLMC_SMOOTH_SPLIT),
               (mg.MLMC_PREC_F64, mg.MLMC_ACCEL_CG, mg.MLMC_SMOOTH_TWO_PASS)]


@pytest.mark.parametrize("prec,accel,sm", GRAPH_CASES)
def test_graph_replay_matches_direct_launches(orc, prec, accel, sm):
    """On a created stream the V-cycle is captured once and replayed as a CUDA graph; on
    the legacy default stream every kernel is launched directly. Same iterates, cycle
    counts and residuals, bit for bit, with samples finishing at different cycles."""
    n, B = 33, 4
    ks = [orc.field(RUN_SEED, int(i), 256, 1.0 + 0.5 * s, 0.15, n) for s, i in enumerate(sample_ids(4, 0, B))]
    k = to_dev(np.stack(ks))
    cfg = mg.mg_cfg(2, 2, 1e-10, 200, prec, sm, accel, engine=mg.MLMC_ENGINE_BATCHED)
    u0 = torch.zeros_like(k)
    cyc0, rel0, st0 = mg.mg_solve_batch(cfg, k, u0)
    side = torch.cuda.Stream()
    u1 = torch.zeros_like(k)
    side.wait_stream(torch.cuda.current_stream())
    cyc1, rel1, st1 = mg.mg_solve_batch(cfg, k, u1, stream=side)
    torch.cuda.synchronize()
    assert st0 == st1 == 0
    assert np.array_equal(cyc0, cyc1) and np.array_equal(rel0, rel1)
    assert np.array_equal(u0.cpu().numpy(), u1.cpu().numpy())
    if accel == mg.MLMC_ACCEL_NONE:
        assert len(set(cyc0.tolist())) > 1  # masking was exercised


@pytest.mark.parametrize("accel", [mg.MLMC_ACCEL_NONE, mg.MLMC_ACCEL_CG])
def test_nodal_smoother_reaches_the_same_solution(orc, accel):
    """The nodal-coefficient sweep smooths an operator within a few ulps of the stored
    FP32 one; the FP64 outer residual (FP64 faces) fixes the solution, so it converges
    to the FP64 solution like the stored-face smoothers (not bit for bit)."""
    n, B = 33, 3
    ks = [orc.field(RUN_SEED, int(i), 256, 1.0, 0.2, n) for i in sample_ids(2, 60, B)]
    k = to_dev(np.stack(ks))
    out = {}
    for sm in (mg.MLMC_SMOOTH_TWO_PASS, mg.MLMC_SMOOTH_NODAL):
        u = torch.zeros_like(k)
        cyc, rel, st = mg.mg_solve_batch(mg.mg_cfg(2, 2, 1e-12, 200, mg.MLMC_PREC_MIXED, sm, accel, engine=mg.MLMC_ENGINE_BATCHED), k, u)
        assert st == 0 and np.all(rel <= 1e-12)
        out[sm] = (u.cpu().numpy(), cyc)
    for s in range(B):
        u64, *_ = orc.mg_solve(ks[s], None, rtol=1e-12)
        assert relmax(out[mg.MLMC_SMOOTH_NODAL][0][s], u64) < 1e-9
        assert relmax(out[mg.MLMC_SMOOTH_NODAL][0][s], out[mg.MLMC_SMOOTH_TWO_PASS][0][s]) < 1e-9
    # the smoother's operator differs by ulps: the cycle counts stay within one of each other
    assert np.all(np.abs(out[mg.MLMC_SMOOTH_NODAL][1] - out[mg.MLMC_SMOOTH_TWO_PASS][1]) <= 1)


@pytest.mark.parametrize("accel", [mg.MLMC_ACCEL_NONE, mg.MLMC_ACCEL_CG])
@pytest.mark.parametrize("n", [9, 17, 33, 65, 129])
def test_split_storage_equals_nodal_sweep_bitwise(orc, accel, n):
    """MLMC_SMOOTH_SPLIT runs the nodal-coefficient sweep, residual, transfers and coarse
    solve on colour-split storage with the same operations in the same order: iterates,
    cycle counts and residuals equal MLMC_SMOOTH_NODAL's bit for bit, samples stopping at
    different cycles."""
    B = 4 if n < 65 else 2  # 129^3: the sweeps stage their rows through shared memory
    ks = [orc.field(RUN_SEED, int(i), 256, 1.0 + 0.5 * s, 0.15, n) for s, i in enumerate(sample_ids(4, 0, B))]
    k = to_dev(np.stack(ks))
    out = {}
    for sm in (mg.MLMC_SMOOTH_NODAL, mg.MLMC_SMOOTH_SPLIT):
        u = torch.zeros_like(k)
        cyc, rel, st = mg.mg_solve_batch(mg.mg_cfg(2, 2, 1e-10, 200, mg.MLMC_PREC_MIXED, sm, accel, engine=mg.MLMC_ENGINE_BATCHED), k, u)
        assert st == 0
        out[sm] = (u.cpu().numpy(), cyc, rel)
    a, b = out[mg.MLMC_SMOOTH_NODAL], out[mg.MLMC_SMOOTH_SPLIT]
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
    assert np.array_equal(a[0], b[0])


@pytest.mark.parametrize("n", [9, 17, 33, 65, 129])
def test_split_storage_fp64_equals_two_pass_bitwise(orc, n):
    """FP64 stationary cycles with MLMC_SMOOTH_SPLIT: stored faces, D, 1/D, u, g and r in
    colour-split storage, the two-pass sweep's, residual's and transfers' operations in
    their order, the convergence residual on the same partition. Iterates, cycle counts
    and residuals equal MLMC_SMOOTH_TWO_PASS's bit for bit, samples stopping at different
    cycles, with and without a right-hand side."""
    B = 4 if n < 65 else 2
    ks = [orc.field(RUN_SEED, int(i), 256, 1.0 + 0.5 * s, 0.15, n) for s, i in enumerate(sample_ids(4, 0, B))]
    k = to_dev(np.stack(ks))
    f = to_dev(np.stack([random_rhs(n, 700 + s) for s in range(B)]))
    for rhs in (None, f):
        out = {}
        for sm in (mg.MLMC_SMOOTH_TWO_PASS, mg.MLMC_SMOOTH_SPLIT):
            u = torch.zeros_like(k)
            cfg = mg.mg_cfg(2, 2, 1e-10, 200, mg.MLMC_PREC_F64, sm, engine=mg.MLMC_ENGINE_BATCHED)
            cyc, rel, st = mg.mg_solve_batch(cfg, k, u, rhs)
            assert st == 0
            out[sm] = (u.cpu().numpy(), cyc, rel)
        a, b = out[mg.MLMC_SMOOTH_TWO_PASS], out[mg.MLMC_SMOOTH_SPLIT]
        assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
        assert np.array_equal(a[0], b[0])
        if rhs is None and n >= 17:
            assert len(set(a[1].tolist())) > 1  # masking was exercised


def test_split_storage_fp64_fixed_cycles_from_a_nonzero_guess(orc):
    """The initial guess enters the split storage and the result leaves it: three fixed
    cycles from a random interior guess equal the two-pass iterate bit for bit."""
    n, B = 65, 3
    k = to_dev(np.stack([random_coefficient(n, 800 + s, 1.0) for s in range(B)]))
    rng = np.random.default_rng(5)
    u0 = np.zeros((B, n, n, n))
    u0[:, 1:-1, 1:-1, 1:-1] = rng.standard_normal((B, n - 2, n - 2, n - 2))
    res = []
    for sm in (mg.MLMC_SMOOTH_TWO_PASS, mg.MLMC_SMOOTH_SPLIT):
        u = to_dev(u0)
        cyc, rel, st = mg.mg_solve_batch(mg.mg_cfg(2, 2, 0.0, 3, mg.MLMC_PREC_F64, sm,
                                                   engine=mg.MLMC_ENGINE_BATCHED), k, u)
        res.append((u.cpu().numpy(), rel))
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])
    assert not np.array_equal(res[0][0], u0)


@pytest.mark.parametrize("disc,accel", [(mg.MLMC_DISC_FE, mg.MLMC_ACCEL_FMG), (mg.MLMC_DISC_FE, mg.MLMC_ACCEL_NONE),
                                         (mg.MLMC_DISC_FV, mg.MLMC_ACCEL_FMG)])
@pytest.mark.parametrize("n", [17, 65])
def test_split_storage_fe_and_fmg_equal_two_pass_bitwise(orc, disc, accel, n):
    """P1 elements (faces assembled plain and copied into the split storage, P1 transfers
    on split storage) and the FMG cycle (every grid's right-hand side, interpolation and
    cycles on split storage): the iterate and residual of MLMC_SMOOTH_TWO_PASS bit for bit."""
    B = 3
    k = to_dev(np.stack([orc.field(RUN_SEED, int(i), 64, 1.0, 0.3, n) for i in sample_ids(2, 90, B)]))
    fmg = accel == mg.MLMC_ACCEL_FMG
    out = {}
    for sm in (mg.MLMC_SMOOTH_TWO_PASS, mg.MLMC_SMOOTH_SPLIT):
        u = torch.zeros_like(k)
        cfg = mg.mg_cfg(4 if fmg else 2, 4 if fmg else 2, 0.0 if fmg else 1e-10, 2 if fmg else 200,
                        mg.MLMC_PREC_F64, sm, accel, disc, engine=mg.MLMC_ENGINE_BATCHED)
        cyc, rel, st = mg.mg_solve_batch(cfg, k, u)
        assert st == 0
        out[sm] = (u.cpu().numpy(), cyc, rel)
    a, b = out[mg.MLMC_SMOOTH_TWO_PASS], out[mg.MLMC_SMOOTH_SPLIT]
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
    assert np.array_equal(a[0], b[0])


def test_split_storage_fp64_level_estimate_matches_oracle(orc):
    level, ids = 2, sample_ids(2, 30, 3)
    cfg = mg.make_mlmc_cfg(RUN_SEED, 1.0, 0.2, 256, n0=17, rtol=1e-11, smoother=mg.MLMC_SMOOTH_SPLIT,
                           engine=mg.MLMC_ENGINE_BATCHED)
    _, Y, Qf, Qc = mg.mlmc_level_estimate(cfg, level, int(ids[0]), len(ids))
    Y64, Qf64, Qc64, *_ = orc.level_batch(orc.make_cfg(RUN_SEED, 1.0, 0.2, 256, rtol=1e-11), 65, 33, ids)
    scale = np.max(np.abs(Qf64))
    assert np.max(np.abs(Y - Y64)) <= 1e-9 * scale
    assert np.max(np.abs(Qf - Qf64)) <= 1e-9 * scale


def test_split_storage_level_estimate_matches_oracle(orc):
    level, ids = 2, sample_ids(2, 30, 3)
    cfg = mg.make_mlmc_cfg(RUN_SEED, 2.0, 0.2, 256, n0=17, rtol=1e-11, precision=mg.MLMC_PREC_MIXED,
                           smoother=mg.MLMC_SMOOTH_SPLIT, accel=mg.MLMC_ACCEL_CG, engine=mg.MLMC_ENGINE_BATCHED)
    _, Y, Qf, Qc = mg.mlmc_level_estimate(cfg, level, int(ids[0]), len(ids))
    Y64, Qf64, Qc64, *_ = orc.level_batch(orc.make_cfg(RUN_SEED, 2.0, 0.2, 256, rtol=1e-11), 65, 33, ids)
    assert np.all(_mixed_err(Y, Y64, Qf64, Qc64, "level 2, colour-split storage, CG") <= 1e-9)


def test_nodal_smoother_level_estimate_matches_oracle(orc):
    level, ids = 1, sample_ids(1, 30, 4)
    cfg = mg.make_mlmc_cfg(RUN_SEED, 2.0, 0.2, 256, n0=17, rtol=1e-11, precision=mg.MLMC_PREC_MIXED,
                           smoother=mg.MLMC_SMOOTH_NODAL, accel=mg.MLMC_ACCEL_CG)
    _, Y, Qf, Qc = mg.mlmc_level_estimate(cfg, level, int(ids[0]), len(ids))
    Y64, Qf64, Qc64, *_ = orc.level_batch(orc.make_cfg(RUN_SEED, 2.0, 0.2, 256, rtol=1e-11), 33, 17, ids)
    assert np.all(_mixed_err(Y, Y64, Qf64, Qc64, "level 1, nodal smoother, CG") <= 1e-9)


def _direct(orc, k, mixed=False, f=None):
    import scipy.sparse.linalg as spl

    A = orc.assemble_csr(k, mixed)
    n = k.shape[0]
    rhs = np.ones(A.shape[0]) if f is None else f[1:-1, 1:-1, 1:-1].ravel()
    u = np.zeros_like(k)
    u[1:-1, 1:-1, 1:-1] = spl.spsolve(A.tocsc(), rhs).reshape(n - 2, n - 2, n - 2)
    return u


@pytest.mark.parametrize("prec", [mg.MLMC_PREC_F64, mg.MLMC_PREC_MIXED])
@pytest.mark.parametrize("n", [17, 33])
def test_cg_matches_sparse_direct_on_rough_field(orc, prec, n):
    """sigma^2 = 2, ell = 0.1: the stationary V(2,2) cycle needs 100+ cycles on some
    realisations; flexible CG with the same cycle as preconditioner reaches the same
    discrete solution (the oracle's sparse matrix solved directly)."""
    ids = sample_ids(1, 10, 4)
    ks = [orc.field(RUN_SEED, int(i), 256, 2.0, 0.1, n) for i in ids]
    rtol = 1e-12 if prec == mg.MLMC_PREC_F64 else 1e-11
    k = to_dev(np.stack(ks))
    u = torch.zeros_like(k)
    cyc, rel, st = mg.mg_solve_batch(mg.mg_cfg(2, 2, rtol, 200, prec, accel=mg.MLMC_ACCEL_CG), k, u)
    assert st == 0 and np.all(rel <= rtol)
    assert cyc.max() < 45
    u = u.cpu().numpy()
    for s in range(len(ids)):
        ud = _direct(orc, ks[s])  # both precisions solve the FP64 operator
        assert relmax(u[s], ud) < 1e-9


def test_cg_with_rhs_and_smoothers(orc):
    n = 17
    ks = [random_coefficient(n, 700 + s, 1.0) for s in range(3)]
    fs = [random_rhs(n, 800 + s) for s in range(3)]
    ref = None
    for sm in SMOOTHERS:
        u, cyc, rel, st = gpu_solve(ks, fs, rtol=1e-12, max_cycles=100)
        k = to_dev(np.stack(ks))
        ug = torch.zeros_like(k)
        cyc, rel, st = mg.mg_solve_batch(mg.mg_cfg(2, 2, 1e-12, 100, mg.MLMC_PREC_F64, sm, mg.MLMC_ACCEL_CG, engine=mg.MLMC_ENGINE_BATCHED), k, ug,
                                         to_dev(np.stack(fs)))
        ug = ug.cpu().numpy()
        for s in range(3):
            assert relmax(ug[s], _direct(orc, ks[s], f=fs[s])) < 1e-9
        if ref is None:
            ref = ug
        assert np.array_equal(ug, ref)


def test_cg_batch_composition_does_not_change_results(orc):
    n = 17
    ks = [orc.field(RUN_SEED, int(i), 256, 2.0, 0.1, n) for i in sample_ids(2, 40, 5)]
    for prec in (mg.MLMC_PREC_F64, mg.MLMC_PREC_MIXED):
        cfg = mg.mg_cfg(2, 2, 1e-10, 200, prec, accel=mg.MLMC_ACCEL_CG)
        k = to_dev(np.stack(ks))
        ub = torch.zeros_like(k)
        cb, _, _ = mg.mg_solve_batch(cfg, k, ub)
        for s in (1, 4):
            ka = to_dev(ks[s][None])
            ua = torch.zeros_like(ka)
            ca, _, _ = mg.mg_solve_batch(cfg, ka, ua)
            assert ca[0] == cb[s] and torch.equal(ua[0], ub[s])


def test_autotune_records_choice():
    cfg = mg.make_mlmc_cfg(RUN_SEED, 1.0, 0.3, 64, n0=17, nu1=0, nu2=0, rtol=1e-10, precision=mg.MLMC_PREC_MIXED)
    rows, best_sm, best_nu = mg.mlmc_autotune(cfg, 1, int(sample_ids(1, 900, 1)[0]), 16)
    assert len(rows) == 36 and best_nu in (1, 2, 3, 4)  # 9 smoothers x nu in {1, 2, 3, 4}
    assert all(r["ms_per_sample"] > 0 for r in rows)
    # a level run with AUTO smoother and nu = 0 uses the choice and matches an explicit run
    s_auto, Ya, _, _ = mg.mlmc_level_estimate(cfg, 1, int(sample_ids(1, 0, 1)[0]), 8)
    cfg2 = mg.make_mlmc_cfg(RUN_SEED, 1.0, 0.3, 64, n0=17, nu1=best_nu, nu2=best_nu, rtol=1e-10,
                            precision=mg.MLMC_PREC_MIXED, smoother=best_sm)
    s_exp, Ye, _, _ = mg.mlmc_level_estimate(cfg2, 1, int(sample_ids(1, 0, 1)[0]), 8)
    assert s_auto.mean_cycles_fine == s_exp.mean_cycles_fine


def test_autotune_fp64_candidates():
    """FP64 stationary cycles on finite volumes: 8 candidates (the colour-split stored-face
    sweep, no nodal-coefficient sweep); with CG: 7."""
    for accel, count in ((mg.MLMC_ACCEL_NONE, 8), (mg.MLMC_ACCEL_CG, 7)):
        cfg = mg.make_mlmc_cfg(RUN_SEED, 1.0, 0.3, 64, n0=9, nu1=2, nu2=2, rtol=1e-10, accel=accel)
        rows, best_sm, best_nu = mg.mlmc_autotune(cfg, 1, int(sample_ids(1, 950, 1)[0]), 8)
        assert len(rows) == count and best_nu == 2
        sms = [r["smoother"] for r in rows]
        assert "nodal" not in sms
        assert ("split" in sms) == (accel == mg.MLMC_ACCEL_NONE)
