"""Pins for the oracle's SPDE field sampler (Sec. 3.2).

Z solves (kappa^2 - Laplace) Z = W on a zero-flux box around D by cell-centred finite
volumes; log k = sqrt(8 pi kappa sigma^2) Z with kappa = 1 / ell. Pinned by:
  - the FP32 logarithm of the polar normals against math.log (its error bound), and the
    normals against N(0, 1);
  - the white-noise cell sums against an independent aggregation (numpy reshape-sums of
    the octant normals) for the fine grid and for the coupled coarse grid;
  - the operator by hand (2^3 cells, constants) and the exact solve against it;
  - the sampled covariance of log k against the exact covariance of the discrete model,
    h A^-2 scaled (eigenvectors of the zero-flux second difference), and that model
    against Whittle's closed form sigma^2 exp(-r / ell) as h -> 0.
"""
import math

import numpy as np
import pytest

from paper_1607_03252_gb300.workloads import RUN_SEED, sample_id


def test_log_series_error_bound(orc):
    xs = np.exp(np.linspace(math.log(2.0 ** -48), math.log(0.999999), 4001)).astype(np.float32)
    for x in xs:
        got = orc.log_series(float(x))
        ref = math.log(float(x))
        # 2^-22 relative (two FP32 ulps), or an absolute 2^-24 near s = 1 where ln s -> 0
        assert abs(got - ref) <= max(2.0 ** -22 * abs(ref), 2.0 ** -24), (x, got, ref)
    assert orc.log_series(0.5) == pytest.approx(-math.log(2.0), rel=2.0 ** -22)


def test_octant_normals_are_standard_normal(orc):
    sst = pytest.importorskip("scipy.stats")
    z = np.array([orc.octant_normal(RUN_SEED, sample_id(3, 1), o) for o in range(60000)])
    assert sst.kstest(z, "norm").pvalue > 1e-4
    assert abs(z.mean()) < 5 / math.sqrt(len(z))
    assert abs(z.var() - 1.0) < 5 * math.sqrt(2.0 / len(z))
    # independent across octants and samples
    z2 = np.array([orc.octant_normal(RUN_SEED, sample_id(3, 2), o) for o in range(60000)])
    assert abs(np.corrcoef(z, z2)[0, 1]) < 5 / math.sqrt(len(z))
    assert abs(np.corrcoef(z[1:], z[:-1])[0, 1]) < 5 / math.sqrt(len(z))


def _octants(orc, sid, n_f):
    Mo = 4 * (n_f - 1) + 1
    a = np.array([orc.octant_normal(RUN_SEED, sid, o) for o in range(Mo ** 3)], dtype=np.float64)
    return a.reshape(Mo, Mo, Mo)  # [z, y, x]


@pytest.mark.parametrize("n_f", [9, 17])
def test_noise_cells_are_octant_sums(orc, n_f):
    """Fine cells: octants 1 .. 2C of the union box (2 per axis); coarse cells of the pair
    (spacing 2 h_f): octants 0 .. 4 C_c - 1 (4 per axis). Each octant carries
    (h_f/2)^(3/2) xi and g = W / h."""
    sid = sample_id(2, 4)
    O = _octants(orc, sid, n_f)
    hf = 1.0 / (n_f - 1)
    w = (hf / 2) ** 1.5
    C = 2 * (n_f - 1)
    fine = O[1:1 + 2 * C, 1:1 + 2 * C, 1:1 + 2 * C].reshape(C, 2, C, 2, C, 2).sum(axis=(1, 3, 5)) * w / hf
    np.testing.assert_allclose(orc.spde_noise(RUN_SEED, sid, n_f), fine, rtol=1e-13, atol=1e-13)
    n_c = (n_f + 1) // 2
    Cc = 2 * (n_c - 1)
    coarse = O[:4 * Cc, :4 * Cc, :4 * Cc].reshape(Cc, 4, Cc, 4, Cc, 4).sum(axis=(1, 3, 5)) * w / (2 * hf)
    np.testing.assert_allclose(orc.spde_noise(RUN_SEED, sid, n_c, n_f), coarse, rtol=1e-13, atol=1e-13)


def test_noise_variance_is_cell_volume(orc):
    """W(cell) ~ N(0, h^3), so g = W / h has variance h."""
    n = 9
    g = np.concatenate([orc.spde_noise(RUN_SEED, sample_id(4, i), n).ravel() for i in range(6)])
    h = 1.0 / (n - 1)
    assert abs(g.var() / h - 1.0) < 5 * math.sqrt(2.0 / g.size)


def test_operator_by_hand_and_constants(orc):
    ch2 = 0.7
    Z = np.arange(8, dtype=np.float64).reshape(2, 2, 2) + 1.0
    AZ = orc.spde_apply(Z, ch2)
    # every cell of the 2^3 box has three face neighbours
    for z in range(2):
        for y in range(2):
            for x in range(2):
                nb = Z[1 - z, y, x] + Z[z, 1 - y, x] + Z[z, y, 1 - x]
                assert AZ[z, y, x] == pytest.approx((ch2 + 3) * Z[z, y, x] - nb, rel=1e-15)
    # zero flux: a constant field only feels the reaction term
    C = 6
    one = np.ones((C, C, C))
    np.testing.assert_allclose(orc.spde_apply(one, ch2), ch2 * one, rtol=1e-15)
    np.testing.assert_allclose(orc.spde_solve(ch2 * one, ch2), one, rtol=1e-12)


@pytest.mark.parametrize("n", [5, 9, 17])
def test_exact_solve_against_operator(orc, n):
    h = 1.0 / (n - 1)
    ch2 = (h / 0.2) ** 2
    g = orc.spde_noise(RUN_SEED, sample_id(1, n), n)
    Z = orc.spde_solve(g, ch2)
    r = g - orc.spde_apply(Z, ch2)
    assert np.linalg.norm(r) <= 1e-13 * np.linalg.norm(g) * (2 * (n - 1))
    # symmetric operator: <A x, y> = <x, A y>
    x = np.random.default_rng(1).standard_normal(Z.shape)
    y = np.random.default_rng(2).standard_normal(Z.shape)
    assert np.vdot(orc.spde_apply(x, ch2), y) == pytest.approx(np.vdot(x, orc.spde_apply(y, ch2)), rel=1e-12)


def _model_cov(n, ell, cells):
    """Covariance of log k between cells (x, y, z) of the discrete model for sigma^2 = 1:
    8 pi kappa h [A^-2], from the eigenvectors of the zero-flux second difference."""
    C = 2 * (n - 1)
    h = 1.0 / (n - 1)
    kappa = 1.0 / ell
    a = np.arange(C)
    w = np.where(a == 0, math.sqrt(1.0 / C), math.sqrt(2.0 / C))
    Phi = w[:, None] * np.cos(np.pi * a[:, None] * (a[None, :] + 0.5) / C)
    l1 = 4 * np.sin(np.pi * a / (2 * C)) ** 2
    mu = (kappa * h) ** 2 + l1[:, None, None] + l1[None, :, None] + l1[None, None, :]

    def phi3(p):
        return Phi[:, p[2]][:, None, None] * Phi[:, p[1]][None, :, None] * Phi[:, p[0]][None, None, :]

    f0 = phi3(cells[0])
    return [8 * math.pi * kappa * h * float(np.sum(f0 * phi3(q) / mu ** 2)) for q in cells]


def test_model_covariance_tends_to_whittle():
    """sigma^2 exp(-r / ell) at D's centre: the model's variance approaches 1 from above
    as h -> 0 and its correlations stay within a few per cent of exp(-r / ell)."""
    ell = 0.3
    errs = []
    for n in (9, 17, 33):
        h = 1.0 / (n - 1)
        c = n - 1  # cell of D's centre node
        d1, d2 = round(0.125 / h), round(0.25 / h)
        v, c1, c2 = _model_cov(n, ell, [(c, c, c), (c, c, c + d1), (c, c, c + d2)])
        errs.append(v - 1.0)
        assert abs(c1 / v - math.exp(-0.125 / ell)) < 0.03
        assert abs(c2 / v - math.exp(-0.25 / ell)) < 0.03
    assert 0 < errs[2] < errs[1] < errs[0] < 0.08


def test_sampled_covariance_matches_model(orc):
    n, ell, sigma2, N = 9, 0.3, 1.5, 1500
    c = (n - 1) // 2
    vals = np.zeros((N, 3))
    for i in range(N):
        logk = np.log(orc.spde_field(RUN_SEED, sample_id(6, i), sigma2, ell, n))
        vals[i] = logk[c, c, c], logk[c, c, c + 1], logk[c, c, c + 2]
    C = n - 1
    model = [sigma2 * v for v in _model_cov(n, ell, [(C, C, C), (C, C, C + 1), (C, C, C + 2)])]
    assert np.all(np.abs(vals.mean(axis=0)) < 5 * math.sqrt(model[0] / N))
    emp = [np.mean(vals[:, 0] * vals[:, j]) for j in range(3)]
    for e, m in zip(emp, model):
        # product of two N(0, v) variables: standard deviation <= v sqrt(2) / sqrt(N)
        assert abs(e - m) < 5 * model[0] * math.sqrt(2.0 / N), (e, m)


def test_fine_and_coarse_fields_share_the_noise(orc):
    """The pair's coarse field is built from the fine grid's octants: at a common node it
    is strongly correlated with the fine field of the same sample (0.78 measured at 9^3 /
    5^3, where the two discretisations still differ much), and not with other samples."""
    n_f, n_c, ell, N = 9, 5, 0.3, 400
    a, b, other = [], [], []
    for i in range(N):
        sid = sample_id(7, i)
        kf = np.log(orc.spde_field(RUN_SEED, sid, 1.0, ell, n_f))
        kc = np.log(orc.spde_field(RUN_SEED, sid, 1.0, ell, n_c, n_f))
        ko = np.log(orc.spde_field(RUN_SEED, sample_id(7, i + 5000), 1.0, ell, n_c, n_f))
        a.append(kf[4, 4, 4])
        b.append(kc[2, 2, 2])
        other.append(ko[2, 2, 2])
    assert np.corrcoef(a, b)[0, 1] > 0.7
    assert abs(np.corrcoef(a, other)[0, 1]) < 5 / math.sqrt(N)


def test_spde_level_differences_decay(orc):
    """MLMC levels on the SPDE field (each Y_l on one shared noise realisation): the
    variance of Y_l falls with l, as the coupling must make it (Sec. 2.2)."""
    cfg = orc.make_cfg(RUN_SEED, 1.0, 0.3, 1, rtol=1e-10, cov=orc.COV_SPDE)
    V = []
    for l, (nf, nc) in enumerate([(9, 0), (17, 9), (33, 17)]):
        ids = np.array([sample_id(l, i) for i in range(24)], dtype=np.uint64)
        Y, Qf, Qc, cf, cc, st = orc.level_batch(cfg, nf, nc, ids)
        assert st == 0
        V.append(Y.var(ddof=1))
    assert V[0] > V[1] > V[2]
