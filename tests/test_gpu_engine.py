"""The small-grid engine (MLMC_ENGINE_CTA: one persistent launch per solve, one CTA per
sample at a time) against the batched engine: every mode it runs -- FP64 stationary
cycles, mixed-precision refinement, flexible CG in FP64 and mixed precision -- with
every smoother family (two-pass, fused and bulk sweeps share the two-pass arithmetic;
nodal and colour-split share the nodal one) gives the same iterates, cycle counts and
residuals bit for bit, with samples stopping at different cycles; and the same level
statistics. The engine must also launch far fewer kernels."""
import numpy as np
import pytest

import paper_1607_03252_gb300 as mg
from paper_1607_03252_gb300.workloads import RUN_SEED, sample_ids

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [(mg.MLMC_PREC_F64, mg.MLMC_ACCEL_NONE, mg.MLMC_SMOOTH_TWO_PASS),
         (mg.MLMC_PREC_F64, mg.MLMC_ACCEL_NONE, mg.MLMC_SMOOTH_BULK_32x8),
         (mg.MLMC_PREC_F64, mg.MLMC_ACCEL_CG, mg.MLMC_SMOOTH_TWO_PASS),
         (mg.MLMC_PREC_MIXED, mg.MLMC_ACCEL_NONE, mg.MLMC_SMOOTH_TWO_PASS),
         (mg.MLMC_PREC_MIXED, mg.MLMC_ACCEL_NONE, mg.MLMC_SMOOTH_NODAL),
         (mg.MLMC_PREC_MIXED, mg.MLMC_ACCEL_CG, mg.MLMC_SMOOTH_NODAL),
         (mg.MLMC_PREC_MIXED, mg.MLMC_ACCEL_CG, mg.MLMC_SMOOTH_SPLIT),
         (mg.MLMC_PREC_MIXED, mg.MLMC_ACCEL_CG, mg.MLMC_SMOOTH_FUSED_32x8)]


def _solve(k, prec, accel, sm, engine, rtol=1e-10, maxc=200, stream=None):
    u = torch.zeros_like(k)
    cyc, rel, st = mg.mg_solve_batch(mg.mg_cfg(2, 2, rtol, maxc, prec, sm, accel, engine=engine), k, u,
                                     stream=stream, allow_not_converged=True)
    torch.cuda.synchronize()
    return u.cpu().numpy(), cyc, rel, st


@pytest.mark.parametrize("prec,accel,sm", CASES)
@pytest.mark.parametrize("n", [9, 17, 33])
def test_cta_engine_equals_batched_bitwise(orc, prec, accel, sm, n):
    B = 5
    ks = [orc.field(RUN_SEED, int(i), 256, 1.0 + 0.5 * (s % 3), 0.15, n) for s, i in enumerate(sample_ids(4, 7, B))]
    k = torch.from_numpy(np.stack(ks)).cuda()
    ub, cb, rb, sb = _solve(k, prec, accel, sm, mg.MLMC_ENGINE_BATCHED)
    uc, cc, rc, sc = _solve(k, prec, accel, sm, mg.MLMC_ENGINE_CTA)
    assert sb == sc == 0
    assert np.array_equal(cb, cc) and np.array_equal(rb, rc)
    assert np.array_equal(ub, uc)
    if accel == mg.MLMC_ACCEL_NONE:
        assert len(set(cb.tolist())) > 1  # the samples stopped at different cycles


def test_cta_engine_not_converged_and_created_stream(orc):
    n, B = 17, 3
    ks = [orc.field(RUN_SEED, int(i), 64, 1.0, 0.2, n) for i in sample_ids(2, 3, B)]
    k = torch.from_numpy(np.stack(ks)).cuda()
    ub, cb, rb, sb = _solve(k, mg.MLMC_PREC_F64, mg.MLMC_ACCEL_NONE, mg.MLMC_SMOOTH_TWO_PASS,
                            mg.MLMC_ENGINE_BATCHED, rtol=1e-10, maxc=3)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    uc, cc, rc, sc = _solve(k, mg.MLMC_PREC_F64, mg.MLMC_ACCEL_NONE, mg.MLMC_SMOOTH_TWO_PASS, mg.MLMC_ENGINE_CTA,
                            rtol=1e-10, maxc=3, stream=side)
    assert sb == sc == mg.MLMC_ERR_NOT_CONVERGED
    assert np.all(cc == 3) and np.array_equal(ub, uc) and np.array_equal(rb, rc)


@pytest.mark.parametrize("prec,accel", [(mg.MLMC_PREC_F64, mg.MLMC_ACCEL_NONE), (mg.MLMC_PREC_MIXED, mg.MLMC_ACCEL_CG)])
@pytest.mark.parametrize("level", [0, 1])
def test_cta_engine_level_estimate_equal_and_fewer_launches(prec, accel, level):
    ids = sample_ids(level, 0, 24)
    out = {}
    for eng in (mg.MLMC_ENGINE_BATCHED, mg.MLMC_ENGINE_CTA):
        # the stationary FP64 cycle on the four-level workload's field; CG on the rough one
        sig2, ell = (1.0, 0.3) if accel == mg.MLMC_ACCEL_NONE else (2.0, 0.1)
        cfg = mg.make_mlmc_cfg(RUN_SEED, sig2, ell, 256, n0=17, nu1=2, nu2=2, rtol=1e-10, max_cycles=300,
                               precision=prec, accel=accel, engine=eng)
        mg.profile_reset()
        st, Y, Qf, Qc = mg.mlmc_level_estimate(cfg, level, int(ids[0]), len(ids))
        out[eng] = (Y, st.mean, st.M2, st.mean_cycles_fine, mg.profile_total_launches())
    a, b = out[mg.MLMC_ENGINE_BATCHED], out[mg.MLMC_ENGINE_CTA]
    assert np.array_equal(a[0], b[0]) and a[1:4] == b[1:4]
    print("launches per level call, batched %d, CTA engine %d" % (a[4], b[4]))
    assert b[4] * 3 <= a[4]


def test_engine_argument_checked():
    k = torch.ones((1, 9, 9, 9), dtype=torch.float64, device="cuda")
    with pytest.raises(mg.MlmcError) as e:
        mg.mg_solve_batch(mg.mg_cfg(engine=7), k, torch.zeros_like(k))
    assert e.value.status == mg.MLMC_ERR_INVALID
