"""P1 finite elements on the structured tetrahedral mesh and FMG (test infrastructure only).

The paper's discretisation (Sec. 3.1) and cycle (Sec. 7): standard P1 elements on a
simplicial mesh of D = (0,1)^3, the stiffness assembled element by element with the
four-vertex quadrature of the coefficient,
    A_ij = sum_tau grad phi_i . grad phi_j |_tau (|tau| / 4) sum_{vertices x of tau} k(x),
    F_i = int f phi_i,
solved by one FMG-2V(4,4) cycle (nested iteration with two V(4,4) cycles per new level),
and the two quantities of interest of Sec. 7: the point value u(1/4, 1/4, 1/4) and the
flux of k du/dn across the plane x_2 = 1/4.

Readings (the mesh is not specified beyond "uniformly refined"):
  - the mesh: every grid cube of side h is cut into the six tetrahedra
    {O, O + h e_a, O + h(e_a + e_b), O + h(1,1,1)} over the permutations (a, b, c)
    (Kuhn / Freudenthal), which uniform refinement reproduces;
  - the transfers: P1 interpolation from the coarse mesh (the coarse function evaluated
    at the fine nodes) and its transpose;
  - the smoother: red-black Gauss-Seidel (the stiffness couples only the axis
    neighbours on this mesh, see the pins), red = (i + j + k) even first;
  - coarse operators: the same assembly on each grid with k injected; coarsest grid 5^3
    solved exactly;
  - the flux: the mean of k du/dx_2 over the layer of elements between x_2 = 1/4 - h and
    1/4 (du/dx_2 is constant on each element), times the plane's area 1.

Everything here is plain numpy / scipy: barycentric gradients from the 4x4 vertex matrix,
assembly by scattering element matrices, Gauss-Seidel as colour-wise exact updates.
"""
from __future__ import annotations

import functools
import itertools

import numpy as np
import scipy.sparse as sp

PERMS = list(itertools.permutations(range(3)))


def _tet_offsets():
    """The six tetrahedra of the unit cube as 4 x 3 integer vertex offsets (x, y, z)."""
    out = []
    for a, b, c in PERMS:
        v = [np.zeros(3, dtype=int)]
        for ax in (a, b, c):
            w = v[-1].copy()
            w[ax] += 1
            v.append(w)
        out.append(np.array(v))
    return out


TETS = _tet_offsets()


def _bary_gradients(verts):
    """Gradients of the four barycentric functions of a tetrahedron (rows), from the
    inverse of [[1, x_v]] (lambda_i(x) = [1, x] . column i of the inverse)."""
    M = np.hstack([np.ones((4, 1)), verts])
    return np.linalg.inv(M)[1:, :].T


def node_index(n, i, j, k):
    return (k * n + j) * n + i


def assemble(n, k, f=1.0):
    """Full stiffness matrix (all n^3 nodes, boundary rows included) and load vector of
    grid n for the nodal coefficient k[z, y, x]; f a constant, or nodal values (n, n, n)
    integrated by the vertex rule (each element gives |tau|/4 f(x_i) to node i)."""
    h = 1.0 / (n - 1)
    kf = np.asarray(k, dtype=np.float64).ravel()
    rows, cols, vals = [], [], []
    F = np.zeros(n ** 3)
    fn = np.broadcast_to(np.asarray(f, dtype=np.float64), (n, n, n)).ravel()
    O = np.stack(np.meshgrid(np.arange(n - 1), np.arange(n - 1), np.arange(n - 1), indexing="ij"), -1).reshape(-1, 3)
    for T in TETS:
        G = _bary_gradients(T * h)  # same shape for every cube
        vol = abs(np.linalg.det(np.vstack([T[1] - T[0], T[2] - T[0], T[3] - T[0]]) * h)) / 6.0
        vidx = [node_index(n, O[:, 0] + T[v, 0], O[:, 1] + T[v, 1], O[:, 2] + T[v, 2]) for v in range(4)]
        kbar = sum(kf[vi] for vi in vidx) / 4.0
        for a in range(4):
            np.add.at(F, vidx[a], fn[vidx[a]] * vol / 4.0)
            for b in range(4):
                g = float(G[a] @ G[b])
                if g == 0.0:
                    continue
                rows.append(vidx[a])
                cols.append(vidx[b])
                vals.append(kbar * vol * g)
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n ** 3, n ** 3))
    return A.tocsr(), F


def interior_mask(n):
    m = np.zeros((n, n, n), dtype=bool)
    m[1:-1, 1:-1, 1:-1] = True
    return m.ravel()


def solve_direct(n, k, f=1.0):
    """The discrete solution (u = 0 on the boundary), shape (n, n, n)."""
    import scipy.sparse.linalg as spl

    A, F = assemble(n, k, f)
    I = np.flatnonzero(interior_mask(n))
    u = np.zeros(n ** 3)
    u[I] = spl.spsolve(A[I][:, I].tocsc(), F[I])
    return u.reshape(n, n, n)


@functools.lru_cache(maxsize=None)
def prolongation(nc):
    """P1 interpolation from grid nc to grid 2 nc - 1: each fine node's value is the coarse
    P1 function at that point (the Kuhn tetrahedron containing it, barycentric weights),
    evaluated for all fine nodes at once."""
    nf = 2 * nc - 1
    Zf, Yf, Xf = np.meshgrid(np.arange(nf), np.arange(nf), np.arange(nf), indexing="ij")
    x = np.stack([Xf.ravel(), Yf.ravel(), Zf.ravel()], -1) / 2.0  # coarse index units (x, y, z)
    o = np.minimum(np.floor(x).astype(int), nc - 2)
    loc = x - o
    order = np.argsort(-loc, axis=1, kind="stable")  # x_a >= x_b >= x_c per node
    srt = np.take_along_axis(loc, order, axis=1)
    lam = np.stack([1.0 - srt[:, 0], srt[:, 0] - srt[:, 1], srt[:, 1] - srt[:, 2], srt[:, 2]], -1)
    verts = [o.copy()]
    v = o.copy()
    for step in range(3):
        v = v.copy()
        v[np.arange(len(v)), order[:, step]] += 1
        verts.append(v)
    fine = node_index(nf, Xf.ravel(), Yf.ravel(), Zf.ravel())
    rows, cols, vals = [], [], []
    for w, vv in zip(lam.T, verts):
        keep = w != 0.0
        rows.append(fine[keep])
        cols.append(node_index(nc, vv[keep, 0], vv[keep, 1], vv[keep, 2]))
        vals.append(w[keep])
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(nf ** 3, nc ** 3))


class Level:
    def __init__(self, n, k, f):
        self.n = n
        A, F = assemble(n, k, f)
        I = np.flatnonzero(interior_mask(n))
        self.I = I
        self.A = A[I][:, I].tocsr()
        self.F = F[I]
        ijk = np.stack(np.unravel_index(I, (n, n, n)), -1)  # (z, y, x)
        red = (ijk.sum(axis=1) % 2) == 0
        self.colours = [np.flatnonzero(red), np.flatnonzero(~red)]
        self.D = self.A.diagonal()
        self.blocks = []
        for c in self.colours:
            Ac = self.A[c]
            self.blocks.append(Ac)


def _gs_colour(L, u, b, ci):
    c = L.colours[ci]
    Ac = L.blocks[ci]
    # Gauss-Seidel on an independent set: every node of the colour from the others' values
    r = b[c] - Ac @ u + L.D[c] * u[c]
    u[c] = r / L.D[c]


def _smooth(L, u, b, nu):
    for _ in range(nu):
        _gs_colour(L, u, b, 0)
        _gs_colour(L, u, b, 1)


def _embed(L, v):
    full = np.zeros(L.n ** 3)
    full[L.I] = v
    return full


def vcycle(levels, P, l, u, b, nu1, nu2):
    """One V(nu1, nu2) cycle on level l (0 = finest) for A_l u = b (interior vectors)."""
    L = levels[l]
    if l == len(levels) - 1:
        return np.linalg.solve(L.A.toarray(), b)
    _smooth(L, u, b, nu1)
    r = b - L.A @ u
    Lc = levels[l + 1]
    rc = (P[l].T @ _embed(L, r))[Lc.I]
    ec = vcycle(levels, P, l + 1, np.zeros(len(Lc.I)), rc, nu1, nu2)
    u = u + (P[l] @ _embed(Lc, ec))[L.I]
    _smooth(L, u, b, nu2)
    return u


def hierarchy(n, k, f=1.0):
    """Grids n, (n+1)/2, ..., 5 with k injected, and the prolongations between them."""
    levels, P = [], []
    kk = np.asarray(k, dtype=np.float64)
    nn = n
    while True:
        levels.append(Level(nn, kk, f))
        if nn == 5:
            break
        P.append(prolongation((nn + 1) // 2))
        kk = kk[::2, ::2, ::2]
        nn = (nn + 1) // 2
    return levels, P


def fmg(n, k, f=1.0, nu=4, vcycles=2):
    """One FMG-2V(nu, nu) cycle: exact solve on 5^3, then on each finer grid the P1
    interpolation of the coarser solution followed by `vcycles` V(nu, nu) cycles."""
    levels, P = hierarchy(n, k, f)
    Lc = levels[-1]
    u = np.linalg.solve(Lc.A.toarray(), Lc.F)
    for l in range(len(levels) - 2, -1, -1):
        L = levels[l]
        u = (P[l] @ _embed(levels[l + 1], u))[L.I]
        for _ in range(vcycles):
            u = vcycle(levels, P, l, u, L.F, nu, nu)
    out = np.zeros(n ** 3)
    out[levels[0].I] = u
    return out.reshape(n, n, n)


def qoi_point(u):
    n = u.shape[0]
    q = (n - 1) // 4
    return float(u[q, q, q])


def qoi_flux(u, k):
    """Mean of k du/dx_2 over the elements between x_2 = 1/4 - h and 1/4 (times area 1):
    (1/h) sum_tau |tau| kbar_tau d_2 u|_tau over that layer."""
    n = u.shape[0]
    h = 1.0 / (n - 1)
    j0 = (n - 1) // 4 - 1
    uf = np.asarray(u).ravel()
    kf = np.asarray(k, dtype=np.float64).ravel()
    total = 0.0
    O = np.stack(np.meshgrid(np.arange(n - 1), np.arange(n - 1), indexing="ij"), -1).reshape(-1, 2)
    for T in TETS:
        G = _bary_gradients(T * h)
        vol = h ** 3 / 6.0
        vidx = [node_index(n, O[:, 0] + T[v, 0], j0 + T[v, 1], O[:, 1] + T[v, 2]) for v in range(4)]
        kbar = sum(kf[vi] for vi in vidx) / 4.0
        d2 = sum(G[v, 1] * uf[vidx[v]] for v in range(4))
        total += float(np.sum(vol * kbar * d2))
    return total / h


def level_sample(run_seed, sample_id, M, sigma2, ell, nf, nc, qoi="point", cov=None):
    """(Q_f, Q_c) of one MLMC sample on the FE discretisation: the Fourier-feature field
    of the sample on each grid (orc_field; cov: the covariance, Gaussian by default), one
    FMG-2V(4,4) cycle each, the QoI ("point": u(1/4, 1/4, 1/4); "flux": across x_2 = 1/4);
    Q_c = 0 when nc = 0."""
    from . import core

    cv = core.COV_GAUSS if cov is None else cov

    def q(n):
        k = core.field(run_seed, sample_id, M, sigma2, ell, n, cov=cv)
        u = fmg(n, k)
        return qoi_point(u) if qoi == "point" else qoi_flux(u, k)

    return q(nf), (q(nc) if nc else 0.0)
