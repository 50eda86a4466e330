"""Pins for the oracle's P1 finite elements on the tetrahedral mesh, its transfers, its
FMG-2V(4,4) cycle and the two quantities of interest of Sec. 7."""
import math

import numpy as np
import pytest

from oracle import fe
from paper_1607_03252_gb300.workloads import RUN_SEED, sample_id


def _nodes(n):
    h = 1.0 / (n - 1)
    x = np.arange(n) * h
    return np.meshgrid(x, x, x, indexing="ij")  # Z, Y, X


@pytest.fixture(scope="module")
def kfield(orc):
    return {n: orc.field(RUN_SEED, sample_id(1, 2), 64, 1.0, 0.3, n) for n in (5, 9, 17, 33)}


def test_assembly_symmetric_conservative_and_load(kfield):
    n = 9
    A, F = fe.assemble(n, kfield[n])
    assert abs(A - A.T).max() < 1e-14 * abs(A).max()
    # the pure stiffness annihilates constants (every row, boundary rows included)
    assert np.abs(A @ np.ones(n ** 3)).max() < 1e-13 * abs(A).max()
    h = 1.0 / (n - 1)
    I = fe.interior_mask(n)
    assert np.allclose(F[I], h ** 3, rtol=1e-14)  # int phi_i = h^3 for an interior node


def test_stiffness_couples_only_axis_neighbours(kfield):
    """On this mesh every element's stiffness couples only the three axis edges of its
    vertex path (grad lambda_i . grad lambda_j = 0 across the diagonal edges), so the
    operator is a seven-point stencil even for an element-wise varying coefficient."""
    n = 9
    A, _ = fe.assemble(n, kfield[n])
    C = A.tocoo()
    big = abs(C.data) > 1e-13 * abs(C.data).max()
    r, c = C.row[big], C.col[big]
    dr = np.stack(np.unravel_index(r, (n, n, n)), -1) - np.stack(np.unravel_index(c, (n, n, n)), -1)
    steps = np.abs(dr).sum(axis=1)
    assert set(steps.tolist()) <= {0, 1}


def test_constant_coefficient_is_the_seven_point_laplacian():
    n = 9
    h = 1.0 / (n - 1)
    A, _ = fe.assemble(n, np.full((n, n, n), 2.5))
    p = fe.node_index(n, 4, 4, 4)
    row = A[p].toarray().ravel()
    assert row[p] == pytest.approx(2.5 * 6 * h)
    for q in (p - 1, p + 1, p - n, p + n, p - n * n, p + n * n):
        assert row[q] == pytest.approx(-2.5 * h)
    assert np.count_nonzero(np.abs(row) > 1e-15) == 7


def test_face_coefficient_closed_form(kfield):
    """The x-face between P and P + e_x is shared by six elements: -A/h = (k_P + k_{P+x})/4
    + (k_{P+x+y} + k_{P+x+z} + k_{P+x+y+z} + k_{P-y} + k_{P-z} + k_{P-y-z})/12."""
    n = 9
    k = kfield[n]
    A, _ = fe.assemble(n, k)
    h = 1.0 / (n - 1)
    for (x, y, z) in [(2, 3, 4), (1, 1, 1), (6, 2, 5)]:
        p = fe.node_index(n, x, y, z)
        K = lambda dx, dy, dz: k[z + dz, y + dy, x + dx]
        want = (K(0, 0, 0) + K(1, 0, 0)) / 4 + (K(1, 1, 0) + K(1, 0, 1) + K(1, 1, 1) + K(0, -1, 0) + K(0, 0, -1)
                                               + K(0, -1, -1)) / 12
        assert -A[p, p + 1] / h == pytest.approx(want, rel=1e-13)


def test_patch_test_linear_functions():
    n = 9
    Z, Y, X = _nodes(n)
    A, _ = fe.assemble(n, np.full((n, n, n), 1.7))
    u = (0.3 + 1.1 * X - 0.7 * Y + 2.0 * Z).ravel()
    I = fe.interior_mask(n)
    assert np.abs((A @ u)[I]).max() < 1e-13


def test_manufactured_solution_second_order():
    errs = []
    for n in (9, 17, 33):
        Z, Y, X = _nodes(n)
        pi = math.pi
        u_star = np.sin(pi * X) * np.sin(pi * Y) * np.sin(pi * Z)
        k = np.exp(0.4 * np.sin(2 * pi * X) * np.cos(pi * Y) + 0.3 * Z)
        glx = 0.4 * 2 * pi * np.cos(2 * pi * X) * np.cos(pi * Y)
        gly = -0.4 * pi * np.sin(2 * pi * X) * np.sin(pi * Y)
        glz = 0.3
        ux = pi * np.cos(pi * X) * np.sin(pi * Y) * np.sin(pi * Z)
        uy = pi * np.sin(pi * X) * np.cos(pi * Y) * np.sin(pi * Z)
        uz = pi * np.sin(pi * X) * np.sin(pi * Y) * np.cos(pi * Z)
        f = -k * (-3 * pi * pi * u_star + glx * ux + gly * uy + glz * uz)
        u = fe.solve_direct(n, k, f)
        errs.append(np.abs(u - u_star).max())
    assert 3.0 < errs[0] / errs[1] < 5.0 and 3.0 < errs[1] / errs[2] < 5.0


def test_prolongation_reproduces_linear_functions():
    nc = 5
    P = fe.prolongation(nc)
    assert np.allclose(np.asarray(P.sum(axis=1)).ravel(), 1.0)
    Zc, Yc, Xc = _nodes(nc)
    Zf, Yf, Xf = _nodes(2 * nc - 1)
    lin = lambda X, Y, Z: 0.2 - X + 3 * Y + 0.5 * Z
    assert np.abs(P @ lin(Xc, Yc, Zc).ravel() - lin(Xf, Yf, Zf).ravel()).max() < 1e-14


def test_prolongation_equals_node_by_node_kuhn_interpolation():
    """The vectorised interpolation matrix against a plain loop over the fine nodes of
    5^3 -> 9^3: per fine node, its coarse cube, the Kuhn tetrahedron holding it (the one
    whose vertex path steps along the axes in decreasing order of the local coordinates)
    and its barycentric weights; a coarse P1 function (random nodal values) is evaluated
    there and compared with P applied to the same values."""
    nc = 5
    nf = 2 * nc - 1
    P = fe.prolongation(nc).toarray()
    vals = np.random.default_rng(3).standard_normal(nc ** 3)

    def cidx(x, y, z):
        return (z * nc + y) * nc + x

    for z in range(nf):
        for y in range(nf):
            for x in range(nf):
                p = [x / 2.0, y / 2.0, z / 2.0]
                o = [min(int(c), nc - 2) for c in p]
                loc = [p[a] - o[a] for a in range(3)]
                axes = sorted(range(3), key=lambda a: -loc[a])
                w = [1.0 - loc[axes[0]], loc[axes[0]] - loc[axes[1]], loc[axes[1]] - loc[axes[2]], loc[axes[2]]]
                v = list(o)
                ref = w[0] * vals[cidx(*v)]
                for step in range(3):
                    v[axes[step]] += 1
                    ref += w[step + 1] * vals[cidx(*v)]
                got = P[(z * nf + y) * nf + x] @ vals
                assert abs(got - ref) <= 1e-14 * (1 + abs(ref))


def test_fmg_reaches_discretisation_accuracy(kfield):
    """One FMG-2V(4,4) cycle leaves an algebraic error far below the discretisation error
    (the property the paper relies on, Sec. 7): at 17^3, 4.6e-4 against 2.2e-2 (the
    change to the 33^3 solution of the same field)."""
    k17, k33 = kfield[17], kfield[33]
    u17 = fe.solve_direct(17, k17)
    alg = np.abs(fe.fmg(17, k17) - u17).max() / np.abs(u17).max()
    disc = np.abs(u17 - fe.solve_direct(33, k33)[::2, ::2, ::2]).max() / np.abs(u17).max()
    assert alg < 1e-3 and alg < 0.05 * disc, (alg, disc)


def test_vcycle_convergence_factor(kfield):
    n = 17
    k = kfield[n]
    levels, P = fe.hierarchy(n, k)
    L = levels[0]
    u = np.zeros(len(L.I))
    res = [np.linalg.norm(L.F)]
    for _ in range(4):
        u = fe.vcycle(levels, P, 0, u, L.F, 4, 4)
        res.append(np.linalg.norm(L.F - L.A @ u))
    rho = (res[-1] / res[1]) ** (1 / 3)
    assert rho < 0.1


def test_qoi_point_and_flux_closed_forms():
    n = 17
    Z, Y, X = _nodes(n)
    u = 0.5 * X + 2.0 * Y
    assert fe.qoi_point(u) == pytest.approx(0.5 * 0.25 + 2.0 * 0.25)
    # u = 2 y with k = 3: k du/dx_2 = 6 everywhere, so the flux across x_2 = 1/4 is 6
    assert fe.qoi_flux(2.0 * Y, np.full((n, n, n), 3.0)) == pytest.approx(6.0, rel=1e-13)
    # a field varying in x and z: the layer mean of k du/dx_2 with du/dx_2 = 1
    k = 1.0 + X + Z
    assert fe.qoi_flux(Y, k) == pytest.approx(2.0, rel=1e-12)
