"""Pins of the oracle's Hodge stars and Laplacian (Sec. 3.1.1, Eq. hodge0-laplacian).

The Hodge stars are checked against an independent construction of the
circumcentric dual from actual circumcentres (dual edge lengths and dual cell
areas), the Laplacian against the textbook 5-point matrix on the structured
unit-square triangulation, and the discretisation against O(h^2) convergence.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import workloads as W
from oracle import dec, mesh as M, multigrid as mg


def _circumcentre(P0, P1, P2):
    a = P1 - P0
    b = P2 - P0
    axb = np.cross(a, b)
    num = np.cross(np.sum(a * a, axis=1)[:, None] * b - np.sum(b * b, axis=1)[:, None] * a, axb)
    return P0 + num / (2.0 * np.sum(axb * axb, axis=1))[:, None]


def _as3d(v):
    return v if v.shape[1] == 3 else np.concatenate([v, np.zeros((len(v), 1))], axis=1)


def _geometric_stars(m):
    """Dual edge length / primal length and dual cell area, from circumcentres."""
    V = _as3d(m.verts)
    P = V[m.tris]
    C = _circumcentre(P[:, 0], P[:, 1], P[:, 2])
    nrm = np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0])
    nrm = nrm / np.linalg.norm(nrm, axis=1)[:, None]
    s1 = np.zeros(m.ne)
    s0 = np.zeros(m.nv)
    for k in range(3):
        A, B, O = P[:, k], P[:, (k + 1) % 3], P[:, (k + 2) % 3]
        mid = 0.5 * (A + B)
        d = (B - A) / np.linalg.norm(B - A, axis=1)[:, None]
        toward = (O - mid) - np.sum((O - mid) * d, axis=1)[:, None] * d
        toward /= np.linalg.norm(toward, axis=1)[:, None]
        signed = np.sum((C - mid) * toward, axis=1)
        np.add.at(s1, m.tri_edges[:, k], signed / np.linalg.norm(B - A, axis=1))
        # dual-cell piece at vertex k: quad (P_k, mid(k,k+1), C, mid(k,k+2))
        mp = 0.5 * (A + B)
        mq = 0.5 * (A + P[:, (k + 2) % 3])
        area = 0.5 * (np.sum(np.cross(mp - A, C - A) * nrm, axis=1) + np.sum(np.cross(C - A, mq - A) * nrm, axis=1))
        np.add.at(s0, m.tris[:, k], area)
    return s0, s1


def _jittered_grid(seed=0):
    v, t = W.grid_mesh(6, 5)
    rng = np.random.default_rng(seed)
    inner = (v[:, 0] > 0) & (v[:, 0] < 1) & (v[:, 1] > 0) & (v[:, 1] < 1)
    v = v + inner[:, None] * rng.uniform(-0.06, 0.06, size=v.shape)
    return M.build_mesh(v, t)


@pytest.mark.parametrize("case", ["jitter", "ico", "square"])
def test_stars_match_circumcentric_geometry(case):
    if case == "jitter":
        m = _jittered_grid()
    elif case == "ico":
        v, t = W.icosahedron(); m = M.refine(v, t, 2, sphere=True)[0][-1]
    else:
        v, t = W.unit_square(); m = M.refine(v, t, 2)[0][-1]
    g0, g1 = _geometric_stars(m)
    assert np.allclose(dec.hodge_star1(m), g1, rtol=1e-12, atol=1e-13)
    assert np.allclose(dec.hodge_star0(m), g0, rtol=1e-12, atol=1e-14)
    if case == "jitter":
        # the jitter makes some angles obtuse: negative contributions must be kept
        assert (dec.opposite_cotangents(m) < 0).any()


def test_star0_sums_to_area():
    m = _jittered_grid(1)
    assert abs(dec.hodge_star0(m).sum() - 1.0) < 1e-14
    v, t = W.icosahedron()
    meshes, _ = M.refine(v, t, 4, sphere=True)
    errs = []
    for m in meshes[1:]:
        s = dec.hodge_star0(m).sum()
        assert abs(s - dec.triangle_areas(m).sum()) < 1e-12
        errs.append(abs(s - 4.0 * math.pi))
    # flat-facet area converges to 4 pi at second order
    for e0, e1 in zip(errs[:-1], errs[1:]):
        assert 3.5 < e0 / e1 < 4.5


def _grid_index(m, h):
    ij = np.rint(m.verts / h).astype(int)
    return ij


def test_square_is_textbook_five_point():
    # *1 = 1 on interior axis edges, 1/2 on boundary edges, exactly 0 on the diagonals;
    # *0 = h^2 inside, so L is the 5-point Laplacian / h^2 on the interior
    v, t = W.unit_square()
    nsub = 3
    m = M.refine(v, t, nsub)[0][-1]
    N = 2 ** nsub
    h = 1.0 / N
    s0 = dec.hodge_star0(m)
    s1 = dec.hodge_star1(m)
    ij = _grid_index(m, h)
    d = np.abs(ij[m.edges[:, 1]] - ij[m.edges[:, 0]])
    diag_e = (d[:, 0] == 1) & (d[:, 1] == 1)
    bnd_e = M.boundary_edges(m)
    assert np.all(s1[diag_e] == 0.0)
    assert np.all(s1[bnd_e] == 0.5)
    assert np.all(s1[~diag_e & ~bnd_e] == 1.0)
    interior = (ij[:, 0] > 0) & (ij[:, 0] < N) & (ij[:, 1] > 0) & (ij[:, 1] < N)
    assert np.all(s0[interior] == h * h)
    L = dec.laplacian(m, s0, s1)
    idx = np.flatnonzero(interior)
    order = idx[np.lexsort((ij[idx, 0], ij[idx, 1]))]
    Lii = L[order][:, order].toarray()
    T1 = sp.diags([-np.ones(N - 2), 2 * np.ones(N - 1), -np.ones(N - 2)], [-1, 0, 1])
    I1 = sp.identity(N - 1)
    five = ((sp.kron(I1, T1) + sp.kron(T1, I1)) / (h * h)).toarray()
    assert np.array_equal(Lii, five)


@pytest.mark.parametrize("case", ["jitter", "ico"])
def test_laplacian_kernel_and_symmetry(case):
    if case == "jitter":
        m = _jittered_grid(2)
    else:
        v, t = W.icosahedron(); m = M.refine(v, t, 3, sphere=True)[0][-1]
    s0 = dec.hodge_star0(m)
    s1 = dec.hodge_star1(m)
    A = dec.stiffness(m, s1)
    L = dec.laplacian(m, s0, s1)
    scale = abs(L).max()
    assert np.max(np.abs(L @ np.ones(m.nv))) < 1e-13 * scale
    assert abs(A - A.T).max() == 0.0
    # L is self-adjoint in the *0 inner product
    rng = np.random.default_rng(3)
    x, y = rng.standard_normal((2, m.nv))
    assert abs(np.dot(s0 * x, L @ y) - np.dot(s0 * y, L @ x)) < 1e-12 * abs(np.dot(s0 * x, L @ y))
    # and positive semidefinite with a one-dimensional kernel on a connected mesh
    ev = np.linalg.eigvalsh(A.toarray())
    assert ev[0] > -1e-12 and ev[1] > 1e-8


def test_unit_square_closed_form_discrete_solution():
    # -Delta u = 2 pi^2 sin(pi x) sin(pi y): the grid restriction of sin(pi x) sin(pi y) is an
    # eigenvector of the 5-point matrix, so u_h = 2 pi^2 / lambda_11 * sin sin exactly
    v, t = W.unit_square()
    h = mg.build_hierarchy(v, t, 5, 1, "dirichlet")
    lev = h.finest
    b = W.rhs_sin_square(lev.mesh.verts)
    x = mg.direct_solve(h, b)
    hh = 1.0 / 32
    lam11 = 8.0 / hh ** 2 * math.sin(math.pi * hh / 2) ** 2
    u_h = 2 * math.pi ** 2 / lam11 * W.u_sin_square(lev.mesh.verts)
    assert np.max(np.abs(x - u_h)) / np.max(np.abs(u_h)) < 1e-13


def test_square_second_order_convergence():
    v, t = W.unit_square()
    meshes, par = M.refine(v, t, 6)
    errs = []
    for nsub in (3, 4, 5, 6):
        h = mg.build_hierarchy(v, t, nsub, 1, "dirichlet", meshes=meshes[: nsub + 1], parents=par[:nsub])
        lev = h.finest
        x = mg.direct_solve(h, W.rhs_sin_square(lev.mesh.verts))
        errs.append(np.max(np.abs(x - W.u_sin_square(lev.mesh.verts))))
    for e0, e1 in zip(errs[:-1], errs[1:]):
        assert 3.8 < e0 / e1 < 4.2


def test_sphere_second_order_convergence():
    # L Y = l(l+1) Y for a degree-2 harmonic on the unit sphere; the discrete solution converges at O(h^2)
    v, t = W.icosahedron()
    meshes, par = M.refine(v, t, 5, sphere=True)
    errs = []
    for nsub in (2, 3, 4, 5):
        h = mg.build_hierarchy(v, t, nsub, 1, "gauge", sphere=True, meshes=meshes[: nsub + 1], parents=par[:nsub])
        lev = h.finest
        p = lev.mesh.verts
        Y = 3.0 * p[:, 2] ** 2 - 1.0 + p[:, 0] * p[:, 1]
        x = mg.direct_solve(h, 6.0 * Y)
        Yc = mg.project_mean_zero(lev, Y)
        errs.append(mg.star0_norm(lev, x - Yc) / mg.star0_norm(lev, Yc))
    for e0, e1 in zip(errs[:-1], errs[1:]):
        assert 3.5 < e0 / e1 < 4.5
