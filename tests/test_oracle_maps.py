"""Oracle pins for transfers by a general geometric map (Sec. 2.2, M(f); Sec. 2.2.1).

The hierarchy is four non-nested meshes of the unit square (jittered grids,
workloads.jittered_square_levels); the map sends each fine vertex to its own
position, given by the containing coarse triangle and barycentric
coordinates.  What the definitions fix:
  * each column of M(f) holds barycentric coordinates: non-negative, summing
    to 1, and M(f)^T applied to the coarse coordinates gives back the fine
    coordinates (the map is the identity embedding), so interpolation
    reproduces every affine function exactly;
  * the row-normalized restriction maps constants to constants (R 1 = 1);
  * the *0-adjoint restriction satisfies <R r, e>_*0c = <r, P e>_*0f;
  * multigrid on these levels converges to the direct solution.
"""
import numpy as np

import workloads as W
from oracle import mesh as omesh, multigrid as omg


def _hier(restriction="rownorm", smoother="jacobi", bc="dirichlet"):
    ms, mi, mw = W.jittered_square_levels(4, 5)
    meshes = [omesh.build_mesh(v, t) for v, t in ms]
    maps = [omg.map_matrix_from_table(meshes[l].nv, mi[l], mw[l]) for l in range(3)]
    opts = omg.MGOptions(smoother=smoother, restriction=restriction)
    return omg.build_hierarchy(None, None, 3, 4, bc, opts=opts, meshes=meshes, parents=maps), meshes, maps


def test_map_columns_are_barycentric_and_reproduce_affine_functions():
    h, meshes, maps = _hier()
    rng = np.random.default_rng(3)
    for l, M in enumerate(maps):
        M = M.toarray()
        assert M.min() >= 0.0
        assert np.allclose(M.sum(axis=0), 1.0, atol=1e-15, rtol=0)
        # the fine vertices are not on the coarse mesh: some columns mix three coarse vertices
        assert np.mean(np.count_nonzero(M, axis=0) == 3) > 0.5
        xc, xf = meshes[l].verts, meshes[l + 1].verts
        assert np.abs(M.T @ xc - xf).max() < 1e-14
        a, b, c = rng.standard_normal(3)
        P = h.P[l]
        assert np.abs(P @ (a + b * xc[:, 0] + c * xc[:, 1]) - (a + b * xf[:, 0] + c * xf[:, 1])).max() < 1e-13


def test_rownorm_restriction_preserves_constants_and_star0_restriction_is_adjoint():
    h, meshes, _ = _hier()
    for R in h.R:
        assert np.allclose(R @ np.ones(R.shape[1]), 1.0, atol=1e-14, rtol=0)
    h0, _, _ = _hier(restriction="star0")
    rng = np.random.default_rng(4)
    for l in range(3):
        lc, lf = h0.levels[l], h0.levels[l + 1]
        r, e = rng.standard_normal(lf.mesh.nv), rng.standard_normal(lc.mesh.nv)
        lhs = np.sum(lc.star0 * (h0.R[l] @ r) * e)
        rhs = np.sum(lf.star0 * r * (h0.P[l] @ e))
        assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + abs(rhs))


def test_multigrid_on_mapped_levels_reaches_the_direct_solution():
    for smoother in ("jacobi", "chebyshev"):
        h, _, _ = _hier(smoother=smoother)
        lev = h.finest
        b = W.uniform_field(lev.mesh.nv, 8)
        xs = omg.direct_solve(h, b)
        for res in (omg.mg_solve(h, b, 1e-11, 200), omg.pcg_solve(h, b, 1e-11, 100)):
            assert res.rel_res <= 1e-11
            assert omg.star0_norm(lev, res.x - xs) / omg.star0_norm(lev, xs) < 1e-8
        # a working hierarchy: clearly faster than plain CG
        cg = omg.pcg_solve(h, b, 1e-11, 2000, precondition=False)
        assert omg.pcg_solve(h, b, 1e-11, 100).iters * 3 < cg.iters
