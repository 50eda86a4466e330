"""GPU parity of the P1 finite-element discretisation, the FMG-2V(4,4) cycle and the
point and flux QoIs (Secs. 3.1, 7) against the oracle (tests/test_oracle_fe.py pins it).

Tolerances: the converged FE solve against the oracle's direct solve, 1e-9 relative in
the max norm (rtol 1e-12 on the GPU); FMG-2V(4,4) against the oracle's FMG (the same
steps in the same order: red-black Gauss-Seidel, P1 transfers, exact 5^3 solve), 1e-11
relative (rounding order only); Y_l, 1e-10 of max(|Q_l|, |Q_{l-1}|).
"""
import numpy as np
import pytest

import paper_1607_03252_gb300 as mg
from paper_1607_03252_gb300.workloads import RUN_SEED, random_coefficient, sample_ids

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _fields(orc, n, ids, sigma2=1.0, ell=0.3, M=64):
    return np.stack([orc.field(RUN_SEED, int(s), M, sigma2, ell, n) for s in ids])


def _solve(k, cfg):
    kt = torch.from_numpy(k).to(DEV)
    u = torch.zeros_like(kt)
    cyc, rel, st = mg.mg_solve_batch(cfg, kt, u, allow_not_converged=True)
    torch.cuda.synchronize()
    return u.cpu().numpy(), cyc, rel


@pytest.mark.parametrize("n", [9, 17, 33])
def test_fe_operator_converged_matches_direct_solve(n):
    from oracle import fe

    import oracle as orc
    ids = sample_ids(1, 3, 2)
    k = _fields(orc, n, ids)
    u, cyc, rel = _solve(k, mg.mg_cfg(2, 2, 1e-12, 200, smoother=mg.MLMC_SMOOTH_TWO_PASS, disc=mg.MLMC_DISC_FE))
    for s in range(len(ids)):
        ud = fe.solve_direct(n, k[s])
        assert np.abs(u[s] - ud).max() <= 1e-9 * np.abs(ud).max()


@pytest.mark.parametrize("n", [9, 17, 33])
@pytest.mark.parametrize("sm", [mg.MLMC_SMOOTH_TWO_PASS, mg.MLMC_SMOOTH_FUSED_32x8])
def test_fmg_matches_oracle_fmg(n, sm):
    from oracle import fe

    import oracle as orc
    ids = sample_ids(2, 7, 2)
    k = _fields(orc, n, ids)
    cfg = mg.mg_cfg(4, 4, 0.0, 2, smoother=sm, accel=mg.MLMC_ACCEL_FMG, disc=mg.MLMC_DISC_FE)
    u, cyc, rel = _solve(k, cfg)
    assert np.all(cyc == 2)
    for s in range(len(ids)):
        uo = fe.fmg(n, k[s])
        assert np.abs(u[s] - uo).max() <= 1e-11 * np.abs(uo).max()


@pytest.mark.parametrize("level", [0, 1, 2])
@pytest.mark.parametrize("qoi", ["point", "flux"])
def test_fe_fmg_level_estimate_matches_oracle(orc, level, qoi):
    from oracle import fe

    ids = sample_ids(level, 20, 3)
    q = mg.MLMC_QOI_POINT if qoi == "point" else mg.MLMC_QOI_FLUX
    cfg = mg.make_mlmc_cfg(RUN_SEED, 1.0, 0.3, 64, n0=9, nu1=4, nu2=4, rtol=0.0, max_cycles=2,
                           accel=mg.MLMC_ACCEL_FMG, disc=mg.MLMC_DISC_FE, qoi=q)
    st, Y, Qf, Qc = mg.mlmc_level_estimate(cfg, level, int(ids[0]), len(ids))
    nf = 8 * 2 ** level + 1
    nc = 8 * 2 ** (level - 1) + 1 if level > 0 else 0
    for s, sid in enumerate(ids):
        qf, qc = fe.level_sample(RUN_SEED, int(sid), 64, 1.0, 0.3, nf, nc, qoi)
        scale = max(abs(qf), abs(qc))
        assert abs(Qf[s] - qf) <= 1e-10 * scale
        assert abs(Y[s] - (qf - qc)) <= 1e-10 * scale


@pytest.mark.parametrize("level", [0, 1, 2])
def test_fe_fmg_exponential_covariance_level_matches_oracle(orc, level):
    """The settings of the paper's static run (Sec. 7.1) as the c6 workload uses them: P1
    elements, one FMG-2V(4,4) cycle, the point QoI, exponential covariance with a short
    correlation length (ell = 0.15, M = 256), grids 17^3..65^3."""
    from oracle import core, fe

    ids = sample_ids(level, 40, 3)
    cfg = mg.make_mlmc_cfg(RUN_SEED, 1.0, 0.15, 256, n0=17, nu1=4, nu2=4, rtol=0.0, max_cycles=2,
                           accel=mg.MLMC_ACCEL_FMG, disc=mg.MLMC_DISC_FE, qoi=mg.MLMC_QOI_POINT,
                           cov=mg.MLMC_COV_EXP)
    st, Y, Qf, Qc = mg.mlmc_level_estimate(cfg, level, int(ids[0]), len(ids))
    nf = 16 * 2 ** level + 1
    nc = 16 * 2 ** (level - 1) + 1 if level > 0 else 0
    for s, sid in enumerate(ids):
        qf, qc = fe.level_sample(RUN_SEED, int(sid), 256, 1.0, 0.15, nf, nc, "point", cov=core.COV_EXP)
        scale = max(abs(qf), abs(qc))
        # 1e-9: the exponential covariance's heavy-tailed frequencies round the phases of
        # the field to a few ulps of |w| (as in the FV exponential-covariance level test)
        assert abs(Qf[s] - qf) <= 1e-9 * scale
        assert abs(Y[s] - (qf - qc)) <= 1e-9 * scale


FMG_GRAPH_CHILD = r"""
import sys
import numpy as np, torch
import paper_1607_03252_gb300 as mg
from paper_1607_03252_gb300.workloads import random_coefficient
n, B = 65, 3
k = torch.from_numpy(np.stack([random_coefficient(n, 300 + s, 1.0) for s in range(B)])).cuda()
out = {}
for sm in (mg.MLMC_SMOOTH_TWO_PASS, mg.MLMC_SMOOTH_SPLIT):
    cfg = mg.mg_cfg(4, 4, 0.0, 2, mg.MLMC_PREC_F64, sm, mg.MLMC_ACCEL_FMG, mg.MLMC_DISC_FE,
                    engine=mg.MLMC_ENGINE_BATCHED)
    u0 = torch.zeros_like(k)
    _, rel0, st0 = mg.mg_solve_batch(cfg, k, u0)  # legacy default stream: direct launches
    side = torch.cuda.Stream()
    u1 = torch.zeros_like(k)
    side.wait_stream(torch.cuda.current_stream())
    _, rel1, st1 = mg.mg_solve_batch(cfg, k, u1, stream=side)  # created stream: graph replay
    torch.cuda.synchronize()
    assert st0 == st1 == 0
    assert np.array_equal(rel0, rel1)
    assert np.array_equal(u0.cpu().numpy(), u1.cpu().numpy())
print("ok")
"""


def test_fmg_graph_replay_matches_direct_launches():
    """With MLMC_FMG_GRAPHS=1 (read once per process, so in a child process) the FMG cycle
    on a created stream replays each grid's V-cycles from one captured graph; on the
    legacy default stream every kernel is launched directly: the same iterate and
    residual bit for bit, on the plain and the colour-split storage."""
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, MLMC_FMG_GRAPHS="1")
    res = subprocess.run([sys.executable, "-c", FMG_GRAPH_CHILD], cwd=root, env=env, capture_output=True, text=True,
                         timeout=600)
    assert res.returncode == 0 and "ok" in res.stdout, res.stdout[-2000:] + res.stderr[-4000:]


def test_qoi_choice_on_the_fv_path(orc):
    """The point QoI reads u(1/4, 1/4, 1/4) of the finite-volume solution as well."""
    ids = sample_ids(0, 1, 2)
    base = dict(n0=17, rtol=1e-12)
    _, _, Qm, _ = mg.mlmc_level_estimate(mg.make_mlmc_cfg(RUN_SEED, 1.0, 0.3, 256, **base), 0, int(ids[0]), 2)
    _, _, Qp, _ = mg.mlmc_level_estimate(mg.make_mlmc_cfg(RUN_SEED, 1.0, 0.3, 256, qoi=mg.MLMC_QOI_POINT, **base), 0,
                                         int(ids[0]), 2)
    for s, sid in enumerate(ids):
        u, *_ = orc.mg_solve(orc.field(RUN_SEED, int(sid), 256, 1.0, 0.3, 17), rtol=1e-12)
        assert Qp[s] == pytest.approx(u[4, 4, 4], rel=1e-9)
        assert Qm[s] == pytest.approx(orc.qoi(u), rel=1e-9)
