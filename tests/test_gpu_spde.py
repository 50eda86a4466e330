"""GPU parity of the SPDE field sampler (Sec. 3.2) against the oracle.

The oracle solves each SPDE system exactly (eigenvectors of the zero-flux second
difference); the GPU runs cell-centred multigrid to a relative residual of 1e-12, with
the same white noise bit for bit (polar normals from correctly rounded FP32 steps). The
field tolerance is 1e-9 relative in k: the residual bound times the operator's condition
number (c h^2 + 12) / (c h^2) stays below 1e-9 / |log k| at the sizes tested. Y_l: the
scale-normalised 1e-9 of the other covariances.
"""
import numpy as np
import pytest

import paper_1607_03252_gb300 as mg
from paper_1607_03252_gb300.workloads import RUN_SEED, level_n, sample_ids

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _field(cfg, ids, n, n_fine=None, dtype=torch.float64):
    k = torch.zeros((len(ids), n, n, n), dtype=dtype, device=DEV)
    mg.mlmc_field_eval(cfg, ids, k, n_fine=n_fine)
    torch.cuda.synchronize()
    return k.cpu().numpy()


@pytest.mark.parametrize("n,sigma2,ell", [(5, 1.0, 0.3), (9, 1.0, 0.3), (17, 2.0, 0.1), (33, 1.0, 0.05)])
def test_spde_field_matches_oracle(orc, n, sigma2, ell):
    ids = sample_ids(2, 11, 3)
    cfg = mg.field_cfg(RUN_SEED, sigma2, ell, 1, cov=mg.MLMC_COV_SPDE)
    k = _field(cfg, ids, n)
    for s, sid in enumerate(ids):
        ko = orc.spde_field(RUN_SEED, int(sid), sigma2, ell, n)
        assert np.max(np.abs(k[s] - ko) / ko) < 1e-9


@pytest.mark.parametrize("nf", [9, 17, 33])
def test_spde_coarse_of_pair_matches_oracle(orc, nf):
    nc = (nf + 1) // 2
    ids = sample_ids(3, 2, 2)
    cfg = mg.field_cfg(RUN_SEED, 1.0, 0.2, 1, cov=mg.MLMC_COV_SPDE)
    k = _field(cfg, ids, nc, n_fine=nf)
    for s, sid in enumerate(ids):
        ko = orc.spde_field(RUN_SEED, int(sid), 1.0, 0.2, nc, nf)
        assert np.max(np.abs(k[s] - ko) / ko) < 1e-9
    # it is a different field from the coarse grid's own (its noise is the fine grid's)
    own = _field(cfg, ids, nc)
    assert np.max(np.abs(own - k)) > 1e-3


def test_spde_field_f32_is_rounded_f64():
    ids = sample_ids(1, 0, 2)
    cfg = mg.field_cfg(RUN_SEED, 1.0, 0.3, 1, cov=mg.MLMC_COV_SPDE)
    k64 = _field(cfg, ids, 17)
    k32 = _field(cfg, ids, 17, dtype=torch.float32)
    assert np.array_equal(k64.astype(np.float32), k32)


def test_spde_batch_composition_does_not_change_results():
    cfg = mg.field_cfg(RUN_SEED, 1.0, 0.3, 1, cov=mg.MLMC_COV_SPDE)
    ids = sample_ids(0, 5, 4)
    together = _field(cfg, ids, 17)
    alone = _field(cfg, ids[2:3], 17)
    assert np.array_equal(together[2], alone[0])


@pytest.mark.parametrize("level", [0, 1, 2])
def test_spde_level_estimate_matches_oracle(orc, level):
    ids = sample_ids(level, 70, 4)
    cfg = mg.make_mlmc_cfg(RUN_SEED, 1.0, 0.2, 1, n0=9, rtol=1e-12, max_cycles=200, cov=mg.MLMC_COV_SPDE)
    stats, Y, Qf, Qc = mg.mlmc_level_estimate(cfg, level, int(ids[0]), len(ids))
    nf = 8 * 2 ** level + 1
    nc = 8 * 2 ** (level - 1) + 1 if level > 0 else 0
    Yo, Qfo, Qco, cfo, cco, sto = orc.level_batch(
        orc.make_cfg(RUN_SEED, 1.0, 0.2, 1, rtol=1e-12, max_cycles=200, cov=orc.COV_SPDE), nf, nc, ids)
    assert sto == 0
    assert np.all(np.abs(Y - Yo) <= 1e-9 * np.maximum(np.abs(Qfo), np.abs(Qco)))
    assert np.all(np.abs(Qf - Qfo) <= 1e-9 * np.abs(Qfo))
    assert stats.N == len(ids)


def test_spde_level_estimate_mixed_precision(orc):
    level, ids = 1, sample_ids(1, 90, 3)
    kw = dict(rtol=1e-11, max_cycles=300)
    cfg = mg.make_mlmc_cfg(RUN_SEED, 1.0, 0.2, 1, n0=9, precision=mg.MLMC_PREC_MIXED, accel=mg.MLMC_ACCEL_CG,
                           cov=mg.MLMC_COV_SPDE, **kw)
    _, Y, Qf, Qc = mg.mlmc_level_estimate(cfg, level, int(ids[0]), len(ids))
    Y64, Qf64, Qc64, *_ = orc.level_batch(orc.make_cfg(RUN_SEED, 1.0, 0.2, 1, cov=orc.COV_SPDE, **kw), 17, 9, ids)
    err = np.abs(Y - Y64) / np.maximum(np.abs(Qf64), np.abs(Qc64))
    print("mixed vs FP64 (SPDE level 1, |dY| / max|Q|): %s" % " ".join("%.1e" % e for e in err))
    assert np.all(err <= 1e-9)


def test_spde_pair_argument_checked():
    cfg = mg.field_cfg(RUN_SEED, 1.0, 0.3, 1, cov=mg.MLMC_COV_SPDE)
    k = torch.zeros((1, 9, 9, 9), dtype=torch.float64, device=DEV)
    with pytest.raises(mg.MlmcError):
        mg.mlmc_field_eval(cfg, [1], k, n_fine=11)
