"""Fused cycle kernels (fuse=True: every DEC_FUSE_* bit) against one kernel per step (fuse=0).

The fused kernels recompute, per neighbour, the value the first kernel of
the pair would have stored, with the same operations in the same order:
  * the first two pre-smoothing steps from zero (k_smooth0 + k_smooth),
  * residual and restriction (k_residual + k_restrict; stencils of <= 7 slots),
  * interpolation with the first post-smoothing step (k_prolong + k_smooth),
and, without extra gathers,
  * restriction with the coarse level's first smoothing step (k_restrict + k_smooth0),
  * in MG-PCG with FP32 cycles, the outer update with the finest level's first
    smoothing step and the last post-smoothing step with the dot products.
So cycles and whole solves must agree bit for bit, for every smoother,
precision, restriction, sweep count and cycle shape; the parity of the
unfused cycle with the oracle is covered by tests/test_gpu_parity.py.
The fused path also runs the oracle's one-cycle parity cases here through
test_fused_matches_oracle, so the option stands on its own.
"""
import math

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _fan9():
    # valence 9 at the centre: 9 stencil slots, beyond the 8-lane residual/restriction groups
    ang = 2.0 * math.pi * np.arange(9) / 9.0
    verts = np.concatenate([[[0.0, 0.0]], np.stack([np.cos(ang), np.sin(ang)], axis=1)])
    tris = np.array([[0, 1 + k, 1 + (k + 1) % 9] for k in range(9)], dtype=np.int32)
    return verts, tris


CASES = {
    "square5": (W.unit_square, 5, 4, "dirichlet", False),
    "ico5": (W.icosahedron, 5, 4, "gauge", True),
    "fan7": (W.heptagon_fan, 3, 3, "dirichlet", False),
    "fan9": (_fan9, 3, 3, "dirichlet", False),
}


def _pair(name, **kw):
    import paper_2508_12501_gb300 as P
    base, nsub, nl, bc, sph = CASES[name]
    v, t = base()
    hs = [P.Hierarchy(P.Mesh(v, t), nsub, nl, bc=bc, sphere=sph, fuse=f, **kw) for f in (False, True)]
    return hs


def _cycles_equal(hs, dtype, seed):
    n = hs[0].n
    b = torch.as_tensor(W.uniform_field(n, seed), dtype=dtype, device="cuda")
    xs = []
    for h in hs:
        x = torch.zeros(n, dtype=dtype, device="cuda")
        h.vcycle(b, x)  # from zero: every fused kernel runs
        x1 = x.clone()
        h.vcycle(b, x)  # from a nonzero iterate
        xs.append((x1, x))
    assert torch.equal(xs[0][0], xs[1][0])
    assert torch.equal(xs[0][1], xs[1][1])
    assert torch.isfinite(xs[1][1]).all() and xs[1][1].abs().max() > 0


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("smoother", ["jacobi", "chebyshev"])
@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("restriction", ["rownorm", "star0"])
def test_fused_cycle_is_bitwise_equal(name, smoother, dtype, restriction):
    _cycles_equal(_pair(name, smoother=smoother, restriction=restriction), dtype, 5)


@pytest.mark.parametrize("nu", [(0, 1), (1, 0), (1, 1), (2, 2), (3, 1), (4, 3)])
@pytest.mark.parametrize("smoother", ["jacobi", "chebyshev"])
def test_fused_cycle_sweep_counts(nu, smoother):
    _cycles_equal(_pair("square5", smoother=smoother, nu1=nu[0], nu2=nu[1]), torch.float32, 7)


@pytest.mark.parametrize("gamma", [2, 3])
def test_fused_w_cycle(gamma):
    _cycles_equal(_pair("ico5", smoother="chebyshev", gamma=gamma), torch.float32, 9)


@pytest.mark.parametrize("mode", ["f64", "mixed", "mixed_ff"])
@pytest.mark.parametrize("solver", ["mg", "mgpcg"])
def test_fused_solve_is_bitwise_equal(mode, solver):
    hs = _pair("ico5", smoother="chebyshev")
    b = torch.as_tensor(W.uniform_field(hs[0].n, 11), device="cuda")
    out = [h.solve(b, solver=solver, mode=mode, tol=1e-10) for h in hs]
    assert out[0][1].iters == out[1][1].iters
    assert torch.equal(out[0][0], out[1][0])
    # fewer kernels per iteration
    assert out[1][1].launches < out[0][1].launches


@pytest.mark.parametrize("fuse", [1, 2, 4, 7, 8, 9, 10, 14])
def test_fused_masks_match_unfused(fuse):
    import paper_2508_12501_gb300 as P
    base, nsub, nl, bc, sph = CASES["square5"]
    v, t = base()
    hs = [P.Hierarchy(P.Mesh(v, t), nsub, nl, bc=bc, sphere=sph, smoother="chebyshev", fuse=f) for f in (0, fuse)]
    _cycles_equal(hs, torch.float32, 13)


def test_fused_matches_oracle():
    # one FP64 cycle from zero with every fusion, against the oracle's cycle (*0-norm, 1e-12)
    import paper_2508_12501_gb300 as P
    from oracle import multigrid as omg
    v, t = W.icosahedron()
    h = P.Hierarchy(P.Mesh(v, t), 4, 3, bc="gauge", sphere=True, smoother="chebyshev", fuse=True)
    oh = omg.build_hierarchy(v, t, 4, 3, "gauge", sphere=True, opts=omg.MGOptions(smoother="chebyshev"))
    b = omg.prepare_rhs(oh, W.uniform_field(h.n, 17))
    x = torch.zeros(h.n, dtype=torch.float64, device="cuda")
    h.vcycle(torch.as_tensor(b, device="cuda"), x)
    ref = omg.vcycle(oh, b, np.zeros_like(b))
    s0 = oh.finest.star0
    d = x.cpu().numpy() - ref
    assert np.sqrt(np.sum(s0 * d * d) / np.sum(s0 * ref * ref)) < 1e-12


@pytest.mark.parametrize("fuse", [8, 16, 24, 31])
@pytest.mark.parametrize("mode", ["mixed", "mixed_ff"])
@pytest.mark.parametrize("smoother", ["jacobi", "chebyshev"])
def test_outer_fusion_solves_match(fuse, mode, smoother):
    import paper_2508_12501_gb300 as P
    for name in ("square5", "ico5"):
        base, nsub, nl, bc, sph = CASES[name]
        v, t = base()
        hs = [P.Hierarchy(P.Mesh(v, t), nsub, nl, bc=bc, sphere=sph, smoother=smoother, fuse=f) for f in (0, fuse)]
        b = torch.as_tensor(W.uniform_field(hs[0].n, 19), device="cuda")
        out = [h.solve(b, solver="mgpcg", mode=mode, tol=1e-10) for h in hs]
        assert out[0][1].iters == out[1][1].iters
        assert torch.equal(out[0][0], out[1][0])
        out = [h.solve(b, solver="mgpcg", mode=mode, tol=1e-10, host_loop=True) for h in hs]
        assert torch.equal(out[0][0], out[1][0])


@pytest.mark.parametrize("name", ["square5", "ico5", "fan7"])
@pytest.mark.parametrize("smoother", ["jacobi", "chebyshev"])
@pytest.mark.parametrize("restriction", ["rownorm", "star0"])
def test_shared_memory_coarse_cycle_is_bitwise_equal(name, smoother, restriction):
    # DEC_FUSE_COARSE: the coarsest levels in one 1024-thread block out of shared memory
    import paper_2508_12501_gb300 as P
    base, nsub, nl, bc, sph = CASES[name]
    v, t = base()
    hs = [P.Hierarchy(P.Mesh(v, t), nsub, nl, bc=bc, sphere=sph, smoother=smoother, restriction=restriction,
                      fuse=f) for f in (0, 32, 56)]
    _cycles_equal(hs[:2], torch.float32, 23)
    _cycles_equal([hs[0], hs[2]], torch.float32, 23)
    b = torch.as_tensor(W.uniform_field(hs[0].n, 29), device="cuda")
    out = [h.solve(b, solver="mgpcg", mode="mixed_ff", tol=1e-10) for h in hs]
    assert out[0][1].iters == out[1][1].iters == out[2][1].iters
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][0], out[2][0])
    assert out[1][1].launches < out[0][1].launches


@pytest.mark.parametrize("nu", [(0, 1), (1, 0), (1, 1), (3, 2), (4, 4)])
def test_shared_memory_coarse_cycle_sweep_counts(nu):
    import paper_2508_12501_gb300 as P
    v, t = W.icosahedron()
    hs = [P.Hierarchy(P.Mesh(v, t), 5, 5, bc="gauge", sphere=True, smoother="chebyshev", nu1=nu[0], nu2=nu[1],
                      fuse=f) for f in (0, 32)]
    _cycles_equal(hs, torch.float32, 31)


def test_whole_small_hierarchy_in_one_block():
    # unit square x5 with 5 levels (1,089 vertices at most): every level fits, the whole cycle is one launch
    import paper_2508_12501_gb300 as P
    v, t = W.unit_square()
    hs = [P.Hierarchy(P.Mesh(v, t), 5, 5, bc="dirichlet", fuse=f) for f in (0, 32)]
    _cycles_equal(hs, torch.float32, 37)
    b = torch.as_tensor(W.rhs_sin_square(hs[0].table(-1, "verts")), device="cuda")
    out = [h.solve(b, solver="mg", mode="mixed_ff", tol=1e-10) for h in hs]
    assert torch.equal(out[0][0], out[1][0]) and out[0][1].iters == out[1][1].iters


def test_coarse_cycle_after_smaller_hierarchies():
    # the shared-memory limit of the block kernel belongs to the kernel, not to a hierarchy:
    # a large layout built first still launches after smaller hierarchies were built
    import paper_2508_12501_gb300 as P
    v, t = W.icosahedron()
    hs = [P.Hierarchy(P.Mesh(v, t), 7, 6, bc="gauge", sphere=True, smoother="chebyshev", fuse=f) for f in (0, 32)]
    vs, ts = W.unit_square()
    small = [P.Hierarchy(P.Mesh(vs, ts), n, n - 1, bc="dirichlet", fuse=32) for n in (5, 4)]
    b = torch.as_tensor(W.uniform_field(hs[0].n, 41), device="cuda")
    out = [h.solve(b, mode="mixed_ff", tol=1e-8) for h in hs]
    assert out[1][1].rel_res <= 1e-8 and torch.equal(out[0][0], out[1][0])
    bs = torch.as_tensor(W.uniform_field(small[0].n, 43), device="cuda")
    assert small[0].solve(bs, mode="mixed_ff", tol=1e-8)[1].rel_res <= 1e-8


@pytest.mark.parametrize("max_rows", [100, 300, 1000])
@pytest.mark.parametrize("smoother", ["jacobi", "chebyshev"])
@pytest.mark.parametrize("restriction", ["rownorm", "star0"])
def test_gathering_fusions_on_small_levels(max_rows, smoother, restriction):
    # fuse_max_rows: the gathering fusions only on levels of at most max_rows rows
    # (unit square x5: 9, 25, 81, 289, 1089 rows), the separate kernels above; still bitwise
    import paper_2508_12501_gb300 as P
    v, t = W.unit_square()
    hs = [P.Hierarchy(P.Mesh(v, t), 5, 5, bc="dirichlet", smoother=smoother, restriction=restriction, fuse=f,
                      fuse_max_rows=m) for f, m in ((0, 0), (31, max_rows), (63, max_rows))]
    _cycles_equal(hs[:2], torch.float32, 47)
    _cycles_equal([hs[0], hs[2]], torch.float32, 47)
    _cycles_equal(hs[:2], torch.float64, 47)
    b = torch.as_tensor(W.uniform_field(hs[0].n, 53), device="cuda")
    out = [h.solve(b, solver="mgpcg", mode="mixed_ff", tol=1e-10) for h in hs]
    assert out[0][1].iters == out[1][1].iters == out[2][1].iters
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][0], out[2][0])
    # fewer launches than the row-local fusions alone only when some level takes the gathering ones
    hr = P.Hierarchy(P.Mesh(v, t), 5, 5, bc="dirichlet", smoother=smoother, restriction=restriction, fuse=24)
    nr = hr.solve(b, solver="mgpcg", mode="mixed_ff", tol=1e-10)[1].launches
    assert out[1][1].launches < nr


def test_fuse_max_rows_is_validated():
    import paper_2508_12501_gb300 as P
    v, t = W.unit_square()
    with pytest.raises(P.DecError):
        P.Hierarchy(P.Mesh(v, t), 3, 3, bc="dirichlet", fuse_max_rows=-1)
