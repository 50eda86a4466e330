"""Pins for the oracle's lognormal random field.

log k(x) = sigma sqrt(2/M) sum_m cos(w_m . x + b_m) with w_m ~ N(0, I/ell^2) and
b_m ~ U[0, 2 pi) has, for any M, mean 0 and covariance
sigma^2 exp(-|x - y|^2 / (2 ell^2)) (random Fourier features of the Gaussian kernel).
A wrong normaliser, a w scaled by ell instead of 1/ell, or a biased phase all break
one of these closed forms. The exponential covariance (the paper's, Sec. 3.2) is pinned
below by the closed forms of its spectral law.
"""
import math

import numpy as np
import pytest

from paper_1607_03252_gb300.workloads import RUN_SEED, sample_id


@pytest.fixture(scope="module")
def logk_samples(orc):
    sigma2, ell, M, N = 2.0, 0.1, 256, 4000
    x0 = np.array([0.3, 0.4, 0.5])
    offsets = [0.0, 0.05, 0.1, 0.2]
    direction = np.array([1.0, 2.0, -2.0]) / 3.0
    vals = np.zeros((N, len(offsets)))
    for i in range(N):
        w, b = orc.features(RUN_SEED, sample_id(7, i), M, ell)
        for j, r in enumerate(offsets):
            x = x0 + r * direction
            vals[i, j] = orc.logk_point(w, b, math.sqrt(sigma2), *x)
    return sigma2, ell, offsets, vals


def test_field_mean_zero(logk_samples):
    sigma2, _, _, vals = logk_samples
    N = vals.shape[0]
    assert np.all(np.abs(vals.mean(axis=0)) < 5 * math.sqrt(sigma2 / N))


def test_field_variance_sigma2(logk_samples):
    sigma2, _, _, vals = logk_samples
    N = vals.shape[0]
    v = vals[:, 0].var()
    # the sample variance of a near-Gaussian variable has std sigma^2 sqrt(2/N)
    assert abs(v - sigma2) < 5 * sigma2 * math.sqrt(2.0 / N)


def test_field_gaussian_covariance(logk_samples):
    sigma2, ell, offsets, vals = logk_samples
    N = vals.shape[0]
    for j, r in enumerate(offsets[1:], start=1):
        c = np.mean(vals[:, 0] * vals[:, j])
        expected = sigma2 * math.exp(-r * r / (2 * ell * ell))
        assert abs(c - expected) < 5 * sigma2 * math.sqrt(2.0 / N), (r, c, expected)


def test_field_nested_grids_injection_equal(orc):
    """Each grid evaluates the field at its own nodes; the nodes of the 17^3 grid are
    the even nodes of the 33^3 grid (dyadic coordinates), so the values agree exactly."""
    kf = orc.field(RUN_SEED, sample_id(1, 3), 64, 1.0, 0.3, 33)
    kc = orc.field(RUN_SEED, sample_id(1, 3), 64, 1.0, 0.3, 17)
    assert np.array_equal(kf[::2, ::2, ::2], kc)


def test_field_is_exp_of_logk(orc):
    n, M, sigma2, ell = 9, 32, 1.0, 0.3
    k = orc.field(RUN_SEED, 99, M, sigma2, ell, n)
    w, b = orc.features(RUN_SEED, 99, M, ell)
    h = 1.0 / (n - 1)
    for (z, y, x) in [(0, 0, 0), (3, 5, 7), (8, 8, 8), (1, 0, 6)]:
        direct = sum(math.cos(w[m, 0] * x * h + w[m, 1] * y * h + w[m, 2] * z * h + b[m]) for m in range(M))
        assert k[z, y, x] == pytest.approx(math.exp(math.sqrt(sigma2) * math.sqrt(2.0 / M) * direct), rel=1e-13)
    assert np.all(k > 0)


def test_sigma_zero_gives_unit_coefficient(orc):
    k = orc.field(RUN_SEED, 5, 16, 0.0, 0.3, 9)
    assert np.all(k == 1.0)


# ---- exponential covariance sigma^2 exp(-r / ell) (Sec. 3.2) --------------------------
# Its spectral density in 3-D is proportional to (1 + ell^2 |w|^2)^-2, the multivariate
# Cauchy law: s = ell |w| has density (4/pi) s^2 / (1 + s^2)^2, so
# P(s <= t) = (2/pi) (atan t - t / (1 + t^2)), directions are uniform on the sphere, and
# E[cos(w . r)] = exp(-|r| / ell) (the covariance is the characteristic function).


def _exp_features(orc, ell, count=80, M=256):
    W = [orc.features(RUN_SEED, sample_id(9, i), M, ell, cov=orc.COV_EXP)[0] for i in range(count)]
    return np.concatenate(W)


def test_exp_features_radial_law(orc):
    sst = pytest.importorskip("scipy.stats")
    ell = 0.1
    s = np.linalg.norm(_exp_features(orc, ell), axis=1) * ell

    def cdf(t):
        return (2.0 / math.pi) * (np.arctan(t) - t / (1.0 + t * t))

    assert sst.kstest(s, cdf).pvalue > 1e-4
    # the Gaussian law of the other covariance fails the same test by far
    g = np.linalg.norm(orc.features(RUN_SEED, 5, 20000, ell)[0], axis=1) * ell
    assert sst.kstest(g, cdf).pvalue < 1e-10


def test_exp_features_isotropic(orc):
    W = _exp_features(orc, 0.3)
    d = W / np.linalg.norm(W, axis=1, keepdims=True)
    N = len(d)
    assert np.all(np.abs(d.mean(axis=0)) < 5 * math.sqrt(1.0 / 3.0 / N))
    # E[d_i^2] = 1/3 with variance 4/45 on the unit sphere
    assert np.all(np.abs((d * d).mean(axis=0) - 1.0 / 3.0) < 5 * math.sqrt(4.0 / 45.0 / N))
    assert np.all(np.isfinite(W))


def test_exp_features_characteristic_function(orc):
    ell = 0.1
    W = _exp_features(orc, ell)
    N = len(W)
    direction = np.array([2.0, -1.0, 2.0]) / 3.0
    for r in (0.02, 0.05, 0.1, 0.2, 0.4):
        c = np.cos(W @ (r * direction))
        expected = math.exp(-r / ell)
        # |cos| <= 1 bounds the standard deviation of the mean by 1/sqrt(N)
        assert abs(c.mean() - expected) < 5.0 / math.sqrt(N), (r, c.mean(), expected)
        # and it tells the exponential law from the Gaussian one where the two differ
        gauss = math.exp(-r * r / (2 * ell * ell))
        if abs(expected - gauss) > 0.1:
            assert abs(c.mean() - gauss) > 0.05


def test_exp_field_covariance(orc):
    sigma2, ell, M, N = 2.0, 0.1, 256, 4000
    x0 = np.array([0.3, 0.4, 0.5])
    direction = np.array([1.0, 2.0, -2.0]) / 3.0
    offsets = [0.0, 0.05, 0.1, 0.2]
    vals = np.zeros((N, len(offsets)))
    for i in range(N):
        w, b = orc.features(RUN_SEED, sample_id(8, i), M, ell, cov=orc.COV_EXP)
        for j, r in enumerate(offsets):
            vals[i, j] = orc.logk_point(w, b, math.sqrt(sigma2), *(x0 + r * direction))
    assert abs(vals[:, 0].var() - sigma2) < 5 * sigma2 * math.sqrt(2.0 / N)
    for j, r in enumerate(offsets[1:], start=1):
        c = np.mean(vals[:, 0] * vals[:, j])
        assert abs(c - sigma2 * math.exp(-r / ell)) < 5 * sigma2 * math.sqrt(2.0 / N), (r, c)


def test_exp_field_is_exp_of_logk(orc):
    n, M, sigma2, ell = 9, 32, 1.0, 0.3
    k = orc.field(RUN_SEED, 77, M, sigma2, ell, n, cov=orc.COV_EXP)
    w, b = orc.features(RUN_SEED, 77, M, ell, cov=orc.COV_EXP)
    wg, bg = orc.features(RUN_SEED, 77, M, ell)
    # same phases, same directions; only the radius of w differs between the two laws
    assert np.array_equal(b, bg)
    assert np.allclose(w / np.linalg.norm(w, axis=1, keepdims=True), wg / np.linalg.norm(wg, axis=1, keepdims=True),
                       rtol=0, atol=1e-14)
    h = 1.0 / (n - 1)
    for (z, y, x) in [(0, 0, 0), (3, 5, 7), (8, 8, 8)]:
        direct = sum(math.cos(w[m, 0] * x * h + w[m, 1] * y * h + w[m, 2] * z * h + b[m]) for m in range(M))
        assert k[z, y, x] == pytest.approx(math.exp(math.sqrt(sigma2) * math.sqrt(2.0 / M) * direct), rel=1e-13)
