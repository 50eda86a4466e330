"""Pins for the oracle's discrete operator, smoother, grid transfers, coarse solve,
V-cycle and quantity of interest.

Closed forms and invariants used:
  - k = 1 and f = sin(pi x) sin(pi y) sin(pi z) at the nodes: the discrete solution
    is f / lambda_h with lambda_h = (12 / h^2) sin^2(pi h / 2);
  - manufactured smooth solutions converge at O(h^2) (error ratio ~4 per refinement),
    for k = 1 and for a smooth variable k;
  - the multigrid fixed point equals a dense direct solve (scipy) on 9^3;
  - the operator matrix is symmetric with zero row sums away from the boundary;
  - full weighting and trilinear prolongation are exact on trilinear functions and
    adjoint up to the factor 8;
  - after a red-black sweep every black node satisfies its own equation;
  - the V(2,2) convergence factor does not grow with 1/h;
  - the trapezoid QoI is exact on multilinear functions, with error h^2/6 for x^2.
"""
import math

import numpy as np
import pytest
import scipy.linalg

from paper_1607_03252_gb300.workloads import RUN_SEED, random_coefficient, random_rhs, sample_id


def coords(n):
    h = 1.0 / (n - 1)
    x = np.arange(n) * h
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    return X, Y, Z, h


def interior(n):
    m = np.zeros((n, n, n), dtype=bool)
    m[1:-1, 1:-1, 1:-1] = True
    return m


def dense_matrix(orc, k, mixed=False):
    n = k.shape[0]
    idx = np.argwhere(interior(n))
    N = len(idx)
    A = np.zeros((N, N))
    e = np.zeros((n, n, n))
    for c, (z, y, x) in enumerate(idx):
        e[z, y, x] = 1.0
        Ae = orc.apply(k, e, mixed)
        A[:, c] = Ae[interior(n)]
        e[z, y, x] = 0.0
    return A


def test_operator_matrix_symmetric_m_matrix(orc):
    n = 9
    k = orc.field(RUN_SEED, sample_id(0, 1), 32, 1.0, 0.3, n)
    A = dense_matrix(orc, k)
    assert np.array_equal(A, A.T)
    assert np.all(np.diag(A) > 0)
    off = A - np.diag(np.diag(A))
    assert np.all(off <= 0)
    assert np.all((off != 0).sum(axis=1) <= 6)
    # zero row sums for nodes with no boundary neighbour, positive otherwise
    idx = np.argwhere(interior(n))
    far = np.all((idx >= 2) & (idx <= n - 3), axis=1)
    rs = A.sum(axis=1)
    assert np.all(np.abs(rs[far]) < 1e-12 * np.abs(np.diag(A)[far]))
    assert np.all(rs[~far] > 0)


def test_operator_against_independent_assembly(orc):
    """Assemble the harmonic-mean 7-point matrix directly from its definition and
    compare with the oracle's operator applied to unit vectors."""
    n = 5
    k = random_coefficient(n, 11, 1.0)
    h = 1.0 / (n - 1)
    idx = [tuple(p) for p in np.argwhere(interior(n))]
    pos = {p: i for i, p in enumerate(idx)}
    A = np.zeros((len(idx), len(idx)))
    for p in idx:
        for d in [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]:
            q = (p[0] + d[0], p[1] + d[1], p[2] + d[2])
            kpq = 2 * k[p] * k[q] / (k[p] + k[q])
            A[pos[p], pos[p]] += kpq / h ** 2
            if q in pos:
                A[pos[p], pos[q]] -= kpq / h ** 2
    np.testing.assert_allclose(dense_matrix(orc, k), A, rtol=1e-14, atol=0)


def test_mixed_faces_are_fp32_harmonic_means(orc):
    n = 5
    k = random_coefficient(n, 12, 1.5)
    h2 = (1.0 / (n - 1)) ** 2
    A = dense_matrix(orc, k, mixed=True)
    idx = [tuple(p) for p in np.argwhere(interior(n))]
    pos = {p: i for i, p in enumerate(idx)}
    for p in idx:
        q = (p[0], p[1], p[2] + 1)
        if q in pos:
            a, b = np.float32(k[p]), np.float32(k[q])
            kf = np.float32(np.float32(np.float32(2.0) * a) * b) / np.float32(a + b)
            assert -A[pos[p], pos[q]] * h2 == pytest.approx(float(kf), rel=1e-15)


@pytest.mark.parametrize("n", [17, 33])
def test_discrete_eigenfunction_exact(orc, n):
    X, Y, Z, h = coords(n)
    f = np.sin(math.pi * X) * np.sin(math.pi * Y) * np.sin(math.pi * Z)
    lam = 12.0 / h ** 2 * math.sin(math.pi * h / 2) ** 2
    u, st, cyc, rr, _ = orc.mg_solve(np.ones((n, n, n)), f, rtol=1e-13)
    assert st == 0
    np.testing.assert_allclose(u[interior(n)], (f / lam)[interior(n)], rtol=1e-11, atol=1e-14)


@pytest.mark.parametrize("c", [0.5, 40.0])
def test_discrete_eigenfunction_with_reaction(orc, c):
    """-Laplace u + c u: the same eigenfunction with eigenvalue lambda_h + c, through the
    apply, the smoother, the coarse solve and the cycle."""
    n = 17
    X, Y, Z, h = coords(n)
    f = np.sin(math.pi * X) * np.sin(math.pi * Y) * np.sin(math.pi * Z)
    lam = 12.0 / h ** 2 * math.sin(math.pi * h / 2) ** 2
    k = np.ones((n, n, n))
    np.testing.assert_allclose(orc.apply(k, f, c=c)[interior(n)], ((lam + c) * f)[interior(n)], rtol=1e-12,
                               atol=1e-12)
    u, st, cyc, rr, _ = orc.mg_solve(k, f, rtol=1e-13, c=c)
    assert st == 0
    np.testing.assert_allclose(u[interior(n)], (f / (lam + c))[interior(n)], rtol=1e-11, atol=1e-14)
    A = orc.assemble_csr(k, c=c)
    np.testing.assert_allclose(A @ f[interior(n)].ravel(order="C"), ((lam + c) * f)[interior(n)].ravel(), rtol=1e-12,
                               atol=1e-12)


def _manufactured_errors(orc, ns, variable_k):
    errs = []
    for n in ns:
        X, Y, Z, h = coords(n)
        pi = math.pi
        u_star = np.sin(pi * X) * np.sin(pi * Y) * np.sin(pi * Z)
        if variable_k:
            logk = 0.5 * np.sin(2 * pi * X) * np.cos(pi * Y) + 0.3 * Z
            k = np.exp(logk)
            glx = 0.5 * 2 * pi * np.cos(2 * pi * X) * np.cos(pi * Y)
            gly = -0.5 * pi * np.sin(2 * pi * X) * np.sin(pi * Y)
            glz = 0.3 * np.ones_like(X)
            ux = pi * np.cos(pi * X) * np.sin(pi * Y) * np.sin(pi * Z)
            uy = pi * np.sin(pi * X) * np.cos(pi * Y) * np.sin(pi * Z)
            uz = pi * np.sin(pi * X) * np.sin(pi * Y) * np.cos(pi * Z)
            # -div(k grad u) = -k (lap u + grad(log k) . grad u)
            f = -k * (-3 * pi * pi * u_star + glx * ux + gly * uy + glz * uz)
        else:
            k = np.ones_like(X)
            f = 3 * pi * pi * u_star
        u, st, _, _, _ = orc.mg_solve(k, f, rtol=1e-12)
        assert st == 0
        errs.append(np.abs(u - u_star)[interior(n)].max())
    return errs


def test_manufactured_solution_second_order_constant_k(orc):
    e = _manufactured_errors(orc, [9, 17, 33, 65], False)
    ratios = [e[i] / e[i + 1] for i in range(len(e) - 1)]
    assert all(3.6 < r < 4.4 for r in ratios), ratios


def test_manufactured_solution_second_order_variable_k(orc):
    e = _manufactured_errors(orc, [17, 33, 65], True)
    ratios = [e[i] / e[i + 1] for i in range(len(e) - 1)]
    assert all(3.4 < r < 4.6 for r in ratios), ratios


def test_multigrid_equals_dense_direct_solve(orc):
    n = 9
    k = orc.field(RUN_SEED, sample_id(0, 2), 256, 1.0, 0.3, n)
    A = dense_matrix(orc, k)
    f = np.ones(A.shape[0])
    u_direct = scipy.linalg.solve(A, f, assume_a="pos")
    u, st, _, _, _ = orc.mg_solve(k, None, rtol=1e-14, max_cycles=60)
    assert st == 0
    np.testing.assert_allclose(u[interior(n)], u_direct, rtol=1e-12)
    # random rhs as well
    fr = random_rhs(n, 3)
    u2, st, _, _, _ = orc.mg_solve(k, fr, rtol=1e-14, max_cycles=60)
    np.testing.assert_allclose(u2[interior(n)], scipy.linalg.solve(A, fr[interior(n)], assume_a="pos"),
                               rtol=1e-10, atol=1e-13 * np.abs(u2).max())


def test_coarse_solve_matches_dense(orc):
    n = 5
    k = random_coefficient(n, 4, 1.0)
    f = random_rhs(n, 5)
    A = dense_matrix(orc, k)
    u = orc.coarse_solve(k, f)
    np.testing.assert_allclose(u[interior(n)], np.linalg.solve(A, f[interior(n)]), rtol=1e-12)
    assert np.all(u[~interior(n)] == 0)


def trilinear(X, Y, Z):
    return (1 + X) * (2 - Y) * (0.5 + Z) + 0.25 * X * Y * Z


def test_full_weighting_exact_on_trilinear(orc):
    nf = 17
    X, Y, Z, _ = coords(nf)
    rc = orc.restrict_fw(trilinear(X, Y, Z))
    Xc, Yc, Zc, _ = coords(9)
    ic = interior(9)
    np.testing.assert_allclose(rc[ic], trilinear(Xc, Yc, Zc)[ic], rtol=1e-14)
    assert np.all(rc[~ic] == 0)
    # weights sum to one
    np.testing.assert_allclose(orc.restrict_fw(np.ones((nf, nf, nf)))[ic], 1.0, rtol=1e-15)


def test_prolongation_exact_on_trilinear(orc):
    nc, nf = 9, 17
    Xc, Yc, Zc, _ = coords(nc)
    X, Y, Z, _ = coords(nf)
    u = orc.prolong_add(trilinear(Xc, Yc, Zc), np.zeros((nf, nf, nf)))
    i = interior(nf)
    np.testing.assert_allclose(u[i], trilinear(X, Y, Z)[i], rtol=1e-14)
    assert np.all(u[~i] == 0)


def test_restriction_is_one_eighth_prolongation_adjoint(orc):
    nf, nc = 17, 9
    rng = np.random.default_rng(0)
    r = rng.standard_normal((nf, nf, nf)) * interior(nf)
    e = rng.standard_normal((nc, nc, nc)) * interior(nc)
    lhs = 8.0 * np.sum(orc.restrict_fw(r) * e)
    rhs = np.sum(r * orc.prolong_add(e, np.zeros((nf, nf, nf))))
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_rbgs_black_nodes_satisfied_after_sweep(orc):
    n = 9
    k = random_coefficient(n, 6, 1.0)
    f = random_rhs(n, 7)
    u0 = random_rhs(n, 8) * interior(n)
    u1 = orc.rbgs_sweep(k, f, u0)
    r = orc.residual(k, f, u1)
    X = np.indices((n, n, n)).sum(axis=0)
    black = interior(n) & (X % 2 == 1)
    red = interior(n) & (X % 2 == 0)
    scale = np.abs(f).max()
    assert np.abs(r[black]).max() < 1e-12 * scale
    assert np.abs(r[red]).max() > 1e-3 * scale
    # the discrete solution is a fixed point of the sweep
    u_ex, st, _, _, _ = orc.mg_solve(k, f, rtol=1e-14, max_cycles=60)
    np.testing.assert_allclose(orc.rbgs_sweep(k, f, u_ex), u_ex, rtol=0, atol=1e-12 * np.abs(u_ex).max())


def test_vcycle_convergence_factor_h_independent(orc):
    rhos = []
    for n in (17, 33, 65):
        _, st, cyc, _, hist = orc.mg_solve(np.ones((n, n, n)), random_rhs(n, 9), rtol=0, max_cycles=8)
        rho = (hist[7] / hist[2]) ** (1.0 / 5.0)
        rhos.append(rho)
    assert max(rhos) < 0.15, rhos
    assert max(rhos) / min(rhos) < 1.25, rhos


def test_vcycle_converges_on_rough_lognormal_field(orc):
    n = 33
    for sigma2 in (1.0, 2.0):
        k = orc.field(RUN_SEED, sample_id(1, 0), 256, sigma2, 0.1, n)
        _, st, cyc, rr, hist = orc.mg_solve(k, None, rtol=1e-10, max_cycles=60)
        assert st == 0 and rr <= 1e-10
        rho = (hist[-1] / hist[0]) ** (1.0 / max(len(hist) - 1, 1))
        assert rho < 0.5


def test_not_converged_is_reported(orc):
    k = np.ones((17, 17, 17))
    u, st, cyc, rr, _ = orc.mg_solve(k, None, rtol=1e-10, max_cycles=1)
    assert st == -3 and cyc == 1 and rr > 1e-10


def test_invalid_grid_rejected(orc):
    with pytest.raises(ValueError):
        orc.mg_solve(np.ones((6, 6, 6)))
    with pytest.raises(ValueError):
        orc.mg_solve(np.ones((3, 3, 3)))


def test_coarsest_grid_solved_in_one_cycle(orc):
    k = random_coefficient(5, 13, 1.0)
    u, st, cyc, rr, _ = orc.mg_solve(k, None, rtol=1e-12)
    assert st == 0 and cyc == 1 and rr < 1e-13


def test_qoi_trapezoid_exact_cases(orc):
    for n in (5, 9, 17, 33):
        X, Y, Z, h = coords(n)
        assert orc.qoi(np.ones((n, n, n))) == pytest.approx(1.0, rel=1e-15)
        # multilinear: the trapezoid rule is exact; mean of (1+x)(2-y)(0.5+z) is 1.5*1.5*1.0
        assert orc.qoi((1 + X) * (2 - Y) * (0.5 + Z)) == pytest.approx(2.25, rel=1e-14)
        # x^2: trapezoid mean exceeds the exact mean 13/48 by h^2/6
        assert orc.qoi(X * X) == pytest.approx(13.0 / 48.0 + h * h / 6.0, rel=1e-14)
        # values outside [0.25, 0.75]^3 do not contribute
        outside = (X < 0.25) | (X > 0.75) | (Y < 0.25) | (Y > 0.75) | (Z < 0.25) | (Z > 0.75)
        assert orc.qoi(np.where(outside, 1e6, 0.0)) == 0.0


def test_mixed_operator_solution_close_to_fp64(orc):
    n = 17
    k = orc.field(RUN_SEED, sample_id(0, 4), 256, 2.0, 0.1, n)
    u64, st, _, _, _ = orc.mg_solve(k, None, rtol=1e-12)
    u32, st2, _, _, _ = orc.mg_solve(k, None, rtol=1e-12, mixed=True)
    rel = np.abs(u32 - u64).max() / np.abs(u64).max()
    assert st == 0 and st2 == 0
    assert 1e-10 < rel < 1e-6
