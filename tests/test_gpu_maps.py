"""Hierarchies on caller-given meshes and geometric maps (dec_mg_build_maps) against the oracle.

Four non-nested meshes of the unit square (jittered grids) related by the
geometric map that sends each fine vertex to its own position (Sec. 2.2,
M(f)); interpolation is M(f)^T and restriction the transpose of the
row-normalized M(f) or the *0-adjoint of interpolation (Sec. 2.2.1).  The
map tables must come back bit for bit; one cycle must match the oracle's
to 1e-12 (FP64) and 2e-5 (FP32) in the *0 norm, as the subdivision
hierarchies' cycles do; solves must reach the direct solution; and malformed
maps must be refused.
"""
import numpy as np
import pytest

import workloads as W
from oracle import mesh as omesh, multigrid as omg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _pair(smoother="jacobi", restriction="rownorm", bc="dirichlet", nlev=4):
    import paper_2508_12501_gb300 as P
    ms, mi, mw = W.jittered_square_levels(nlev, 5)
    h = P.Hierarchy.from_maps([P.Mesh(v, t) for v, t in ms], mi, mw, bc=bc, smoother=smoother,
                              restriction=restriction)
    meshes = [omesh.build_mesh(v, t) for v, t in ms]
    maps = [omg.map_matrix_from_table(meshes[l].nv, mi[l], mw[l]) for l in range(nlev - 1)]
    oh = omg.build_hierarchy(None, None, nlev - 1, nlev, bc, opts=omg.MGOptions(smoother=smoother,
                                                                                  restriction=restriction),
                             meshes=meshes, parents=maps)
    return h, oh, mi, mw


def _rel(lev, a, b):
    return omg.star0_norm(lev, a - b) / omg.star0_norm(lev, b)


def test_map_tables_round_trip_bit_exact():
    h, oh, mi, mw = _pair()
    assert h.nv == [lev.mesh.nv for lev in oh.levels]
    for l in range(3):
        assert np.array_equal(h.table(l, "map_idx"), mi[l])
        assert np.array_equal(h.table(l, "map_w"), mw[l])
        assert np.array_equal(h.table(l, "star0"), oh.levels[l].star0) or \
            np.abs(h.table(l, "star0") - oh.levels[l].star0).max() <= 1e-13 * oh.levels[l].star0.max()


@pytest.mark.parametrize("smoother", ["jacobi", "chebyshev"])
@pytest.mark.parametrize("restriction", ["rownorm", "star0"])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_one_cycle_matches_oracle(smoother, restriction, prec):
    h, oh, _, _ = _pair(smoother, restriction)
    lev = oh.finest
    b = omg.prepare_rhs(oh, W.uniform_field(lev.mesh.nv, 21))
    ref = omg.vcycle(oh, b, np.zeros_like(b))
    dt = torch.float64 if prec == "f64" else torch.float32
    x = torch.zeros(lev.mesh.nv, dtype=dt, device="cuda")
    h.vcycle(torch.as_tensor(b, dtype=dt, device="cuda"), x)
    got = x.double().cpu().numpy()
    assert _rel(lev, got, ref) < (1e-12 if prec == "f64" else 2e-5)
    assert np.all(got[~lev.free] == 0.0)


@pytest.mark.parametrize("solver", ["mg", "mgpcg"])
@pytest.mark.parametrize("mode", ["f64", "mixed", "mixed_ff"])
def test_solve_matches_direct_solution(solver, mode):
    h, oh, _, _ = _pair("chebyshev")
    lev = oh.finest
    b = W.uniform_field(lev.mesh.nv, 31)
    x, st = h.solve(torch.as_tensor(b, device="cuda"), solver=solver, mode=mode, tol=1e-10, maxit=200)
    assert st.status == 0 and st.rel_res <= 1e-10
    xs = omg.direct_solve(oh, b)
    assert _rel(lev, x.cpu().numpy(), xs) < 1e-7
    if mode == "f64":
        ref = omg.mg_solve(oh, b, 1e-10, 200) if solver == "mg" else omg.pcg_solve(oh, b, 1e-10, 200)
        assert abs(st.iters - ref.iters) <= 1


def test_malformed_maps_are_refused():
    import paper_2508_12501_gb300 as P
    ms, mi, mw = W.jittered_square_levels(3, 5)
    meshes = [P.Mesh(v, t) for v, t in ms]
    bad_idx = [a.copy() for a in mi]
    bad_idx[1][7, 0] = meshes[1].nv  # out of range
    bad_w = [a.copy() for a in mw]
    bad_w[0][3] *= 1.5               # weights that do not sum to 1
    unused = [a.copy() for a in mi]
    unused_w = [a.copy() for a in mw]
    c = int(unused[0][0, 0])
    hit = np.flatnonzero((unused[0] == c) & (unused_w[0] != 0))
    rows = np.unique(hit // 3)
    for r in rows:  # move every weight off coarse vertex c: c carries no weight
        unused[0][r] = [int(unused[0][r][k]) if unused[0][r][k] != c else int(unused[0][r][(k + 1) % 3])
                        for k in range(3)]
    for idx, w in ((bad_idx, mw), (mi, bad_w), (unused, unused_w)):
        with pytest.raises(P.DecError) as ei:
            P.Hierarchy.from_maps(meshes, idx, w)
        assert ei.value.code == 1
