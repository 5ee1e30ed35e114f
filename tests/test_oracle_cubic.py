"""Pins of the oracle's cubic (1->9) subdivision and its geometric-map transfers (Sec. 2.2.1)."""
import math
import os

import numpy as np
import pytest

import workloads as W
from oracle import dec, mesh as M, multigrid as mg

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("base", ["square", "ico", "grid"])
def test_cubic_counting(base):
    # V' = V + 2E + T (two points per edge, one per triangle), T' = 9T, E' = 3E + 9T
    if base == "square":
        v, t = W.unit_square(); meshes, maps = M.refine(v, t, 3, scheme="cubic")
    elif base == "ico":
        v, t = W.icosahedron(); meshes, maps = M.refine(v, t, 2, sphere=True, scheme="cubic")
    else:
        v, t = W.grid_mesh(3, 4); meshes, maps = M.refine(v, t, 2, scheme="cubic")
    for c, f, Mf in zip(meshes[:-1], meshes[1:], maps):
        assert (f.nv, f.ne, f.nt) == (c.nv + 2 * c.ne + c.nt, 3 * c.ne + 9 * c.nt, 9 * c.nt)
        assert Mf.shape == (c.nv, f.nv)
        # every fine vertex's global barycentric coordinates sum to one: interpolation keeps constants
        assert np.allclose(np.asarray(Mf.sum(axis=0)).ravel(), 1.0, rtol=0, atol=1e-15)
        assert np.array_equal(f.verts[: c.nv], c.verts)
        if base != "ico":
            # planar: the map reproduces positions (affine functions) exactly up to rounding
            assert np.allclose(Mf.T @ c.verts, f.verts, rtol=0, atol=1e-15)
    if base == "ico":
        for m in meshes:
            assert m.nv - m.ne + m.nt == 2
            assert np.allclose(np.linalg.norm(m.verts, axis=1), 1.0, atol=1e-15)


def test_cubic_triangles_keep_orientation_and_split_area_in_nine():
    v, t = W.unit_square()
    c = M.build_mesh(v, t)
    f, _ = M.subdivide_cubic(c)
    def areas(m):
        p = m.verts[m.tris]
        return 0.5 * ((p[:, 1, 0] - p[:, 0, 0]) * (p[:, 2, 1] - p[:, 0, 1]) - (p[:, 2, 0] - p[:, 0, 0]) * (p[:, 1, 1] - p[:, 0, 1]))
    ac, af = areas(c), areas(f)
    assert np.all(ac > 0) and np.all(af > 0)
    assert np.allclose(af.reshape(-1, 9), ac[:, None] / 9.0, rtol=1e-12)


def test_cubic_restriction_of_one_triangle_is_the_golden_matrix():
    rows = [[float(x) for x in ln.split()] for ln in open(os.path.join(GOLDEN, "restriction_cubic_one_triangle.txt"))
            if ln.strip() and not ln.startswith("#")]
    v, t = W.one_triangle()
    meshes, maps = M.refine(v, t, 1, scheme="cubic")
    R = mg.restriction(3, maps[0]).toarray()
    assert np.allclose(R, np.array(rows) / 10.0, rtol=0, atol=1e-15)
    # and the restriction keeps constants (row sums one)
    assert np.allclose(R.sum(axis=1), 1.0, atol=1e-15)


def test_cubic_square_hierarchy_reaches_the_discrete_closed_form():
    # unit square subdivided cubically k times is the (3^k + 1)^2 grid with its diagonals: the hypotenuse
    # *1 vanishes (up to rounding), L is the 5-point Laplacian, and -Delta of sin(pi x) sin(pi y) has the discrete solution
    # (2 pi^2 / lambda_11) sin(pi x) sin(pi y), lambda_11 = (8 / h^2) sin^2(pi h / 2), h = 3^-k
    v, t = W.unit_square()
    h = mg.build_hierarchy(v, t, 3, 3, "dirichlet", scheme="cubic")
    lev = h.finest
    assert lev.mesh.nv == 28 * 28
    s1 = dec.hodge_star1(lev.mesh)
    assert np.all((np.abs(s1) <= 1e-12) | (s1 > 0.25))  # k/27 coordinates: hypotenuses vanish up to rounding
    r = mg.mg_solve(h, W.rhs_sin_square(lev.mesh.verts), 1e-12, 200)
    hh = 1.0 / 27
    lam = 8.0 / hh ** 2 * math.sin(math.pi * hh / 2) ** 2
    u_h = 2 * math.pi ** 2 / lam * W.u_sin_square(lev.mesh.verts)
    assert r.rel_res <= 1e-12
    assert mg.star0_norm(lev, r.x - u_h) / mg.star0_norm(lev, u_h) < 1e-10
    rp = mg.pcg_solve(h, W.rhs_sin_square(lev.mesh.verts), 1e-12, 200)
    assert mg.star0_norm(lev, rp.x - u_h) / mg.star0_norm(lev, u_h) < 1e-10
