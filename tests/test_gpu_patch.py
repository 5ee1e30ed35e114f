"""Halo-tiled cycle levels (DEC_FUSE_PATCH) against the per-step kernels.

On a tiled level one block per tile runs the pre-smoothing steps, the
residual and the restriction in one launch, and the interpolation, the
correction and the post-smoothing steps in another, recomputing the values of
the vertices within nu edges of its own.  Every row takes the operations of
the per-step kernels in their order, so cycles and solves must agree bit for
bit with the hierarchy built without the bit -- for every smoother, sweep
count (1 to 3), restriction, precision, stencil width and tile size.  The
oracle check at the end holds the tiled cycle to the paper's cycle directly.
"""
import math

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BASE = 8 | 16 | 32  # the library's default fusions
PATCH = 64


def _fan9():
    # valence 9 at the centre: 9 stencil slots (the generic-width kernels)
    ang = 2.0 * math.pi * np.arange(9) / 9.0
    verts = np.concatenate([[[0.0, 0.0]], np.stack([np.cos(ang), np.sin(ang)], axis=1)])
    tris = np.array([[0, 1 + k, 1 + (k + 1) % 9] for k in range(9)], dtype=np.int32)
    return verts, tris


# base mesh, subdivisions, levels, boundary condition, sphere projection
CASES = {
    "square6": (W.unit_square, 6, 5, "dirichlet", False),
    "ico6": (W.icosahedron, 6, 5, "gauge", True),
    "fan9": (_fan9, 5, 4, "dirichlet", False),
}


def _pair(name, coarse_max_rows=60, **kw):
    import paper_2508_12501_gb300 as P
    base, nsub, nl, bc, sph = CASES[name]
    v, t = base()
    # a small shared-memory coarse block, so that FP32 cycles reach tiled levels too
    return [P.Hierarchy(P.Mesh(v, t), nsub, nl, bc=bc, sphere=sph, fuse=f, coarse_max_rows=coarse_max_rows, **kw)
            for f in (BASE, BASE | PATCH)]


def _tiled_launches(h, b, mode="mixed"):
    # kernels of the tiled levels in one solve (the profiled iteration graph records every launch)
    h.profile(2)
    h.solve(b, mode=mode, tol=1e-6, host_loop=True)
    torch.cuda.synchronize()
    ent = h.profile_read()
    h.profile(0)
    return sum(e["launches"] for e in ent if e["kind"] in ("patchdown", "patchup"))


def _cycles_equal(hs, dtype, seed, expect_tiles=True):
    n = hs[0].n
    b = torch.as_tensor(W.uniform_field(n, seed), dtype=dtype, device="cuda")
    assert sum(hs[0].tiles) == 0
    if expect_tiles:
        assert sum(hs[1].tiles) > 0
        bd = b.double()
        assert _tiled_launches(hs[1], bd, "f64" if dtype == torch.float64 else "mixed") > 0
    xs = []
    for h in hs:
        x = torch.zeros(n, dtype=dtype, device="cuda")
        h.vcycle(b, x)  # from zero
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
def test_tiled_cycle_is_bitwise_equal(name, smoother, dtype, restriction):
    _cycles_equal(_pair(name, smoother=smoother, restriction=restriction), dtype, 3)


@pytest.mark.parametrize("nu", [(1, 1), (2, 2), (3, 3), (1, 3), (3, 1), (2, 1)])
@pytest.mark.parametrize("smoother", ["jacobi", "chebyshev"])
@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_tiled_sweep_counts(nu, smoother, dtype):
    _cycles_equal(_pair("square6", smoother=smoother, nu1=nu[0], nu2=nu[1]), dtype, 7)


@pytest.mark.parametrize("chunk", [1, 5, 64, 100000])
def test_tile_size_does_not_change_results(chunk):
    # one coarse vertex per tile up to a single tile per level: the same bits
    hs = _pair("ico6", smoother="chebyshev", patch_chunk=chunk)
    _cycles_equal(hs, torch.float32, 11)


def test_unsupported_options_keep_per_step_kernels():
    # 4 smoothing steps (more rings than the tiles carry), W-cycles, multicolour GS: no tiles, same results
    for kw in (dict(nu1=4, nu2=2), dict(gamma=2), dict(smoother="mcgs")):
        _cycles_equal(_pair("square6", **kw), torch.float64, 5, expect_tiles=False)
        h = _pair("square6", **kw)[1]
        assert sum(h.tiles) == 0


def test_patch_max_rows_limits_tiled_levels():
    import paper_2508_12501_gb300 as P
    v, t = W.icosahedron()
    nvs = [10 * 4 ** k + 2 for k in range(7)]  # icosphere vertex counts
    h = P.Hierarchy(P.Mesh(v, t), 6, 5, bc="gauge", sphere=True, smoother="chebyshev", fuse=BASE | PATCH,
                    coarse_max_rows=60, patch_max_rows=nvs[4])
    b = torch.as_tensor(W.uniform_field(h.n, 4), device="cuda")
    h.profile(2)
    h.solve(b, mode="f64", tol=1e-6, host_loop=True)
    torch.cuda.synchronize()
    lv = sorted({e["level"] for e in h.profile_read() if e["kind"] == "patchdown"})
    h.profile(0)
    # levels 0..4 hold nvs[2..6] rows: the coarsest and the finest are never tiled, and level 3
    # (nvs[5] rows) is above the limit
    assert lv == [1, 2]
    assert [t > 0 for t in h.tiles] == [False, True, True, False, False]


@pytest.mark.parametrize("mode", ["f64", "mixed", "mixed_ff", "mixed_f32dot"])
@pytest.mark.parametrize("solver", ["mg", "mgpcg"])
def test_tiled_solve_is_bitwise_equal(mode, solver):
    hs = _pair("ico6", smoother="chebyshev")
    b = torch.as_tensor(W.uniform_field(hs[0].n, 23), device="cuda")
    out = [h.solve(b, solver=solver, mode=mode, tol=1e-10) for h in hs]
    assert out[0][1].iters == out[1][1].iters
    assert torch.equal(out[0][0], out[1][0])
    # fewer kernels per iteration
    assert out[1][1].launches < out[0][1].launches
    out = [h.solve(b, solver=solver, mode=mode, tol=1e-10, host_loop=True) for h in hs]
    assert torch.equal(out[0][0], out[1][0])


def test_tiled_adjoint_is_bitwise_equal():
    hs = _pair("square6", smoother="chebyshev")
    b = torch.as_tensor(W.uniform_field(hs[0].n, 29), device="cuda")
    g = torch.as_tensor(W.uniform_field(hs[0].n, 31), device="cuda")
    res = []
    for h in hs:
        u, _ = h.solve(b, mode="mixed", tol=1e-10)
        res.append(h.solve_backward(u, g, mode="mixed", tol=1e-10))
    assert torch.equal(res[0][0], res[1][0])
    assert torch.equal(res[0][1], res[1][1])


@pytest.mark.parametrize("smoother", ["jacobi", "chebyshev"])
@pytest.mark.parametrize("restriction", ["rownorm", "star0"])
def test_tiled_cycle_matches_oracle(smoother, restriction):
    # one FP64 cycle from zero with tiled levels against the oracle's cycle (*0 norm, 1e-12)
    import paper_2508_12501_gb300 as P
    from oracle import multigrid as omg
    v, t = W.icosahedron()
    h = P.Hierarchy(P.Mesh(v, t), 4, 4, bc="gauge", sphere=True, smoother=smoother, restriction=restriction,
                    fuse=BASE | PATCH)
    oh = omg.build_hierarchy(v, t, 4, 4, "gauge", sphere=True,
                             opts=omg.MGOptions(smoother=smoother, restriction=restriction))
    b = omg.prepare_rhs(oh, W.uniform_field(h.n, 17))
    assert sum(h.tiles) > 0
    x = torch.zeros(h.n, dtype=torch.float64, device="cuda")
    h.vcycle(torch.as_tensor(b, device="cuda"), x)
    ref = omg.vcycle(oh, b, np.zeros_like(b))
    s0 = oh.finest.star0
    d = x.cpu().numpy() - ref
    assert np.sqrt(np.sum(s0 * d * d) / np.sum(s0 * ref * ref)) < 1e-12


@pytest.mark.parametrize("threads", [32, 96, 256])
def test_block_size_does_not_change_results(threads):
    hs = _pair("square6", smoother="chebyshev", patch_threads=threads)
    _cycles_equal(hs, torch.float64, 13)
