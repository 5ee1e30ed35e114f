"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle.

Tolerances come from the arithmetic.  One operator row sums at most K terms
w_k (x_i - x_k); reordering that sum changes it by at most ~K eps times
s_i = sum_k |w_k| (|x_i| + |x_k|), so rows are compared against
TOL_ROW * eps * s_i (eps = 2^-53 for FP64, 2^-24 for FP32, where the FP32
weights add one more rounding per term).  Cycles and solves are compared in
the *0-norm: 1e-12 relative for an FP64 cycle, 2e-5 for an FP32 cycle, and
for solves the error bound implied by the requested relative residual.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import multigrid as omg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS64 = 2.0 ** -53
EPS32 = 2.0 ** -24
TOL_ROW = 16.0


def _lib():
    import paper_2508_12501_gb300 as P
    return P


def _dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


CASES = {
    # name: (base, nsub, nlevels, bc, sphere)
    "square5": (W.unit_square, 5, 5, "dirichlet", False),
    "ico5": (W.icosahedron, 5, 4, "gauge", True),
    "fan3": (W.heptagon_fan, 3, 3, "dirichlet", False),
    "grid_ragged": (lambda: W.grid_mesh(7, 5, 0.0, 1.3, 0.0, 0.9), 3, 3, "dirichlet", False),
}

_cache = {}


def _pair(name, smoother="jacobi", nu=2, restriction="rownorm"):
    key = (name, smoother, nu, restriction)
    if key not in _cache:
        P = _lib()
        base, nsub, nl, bc, sph = CASES[name]
        v, t = base()
        h = P.Hierarchy(P.Mesh(v, t), nsub, nl, bc=bc, sphere=sph, smoother=smoother, nu1=nu, nu2=nu,
                        restriction=restriction)
        oh = omg.build_hierarchy(v, t, nsub, nl, bc, sphere=sph,
                                 opts=omg.MGOptions(smoother=smoother, nu1=nu, nu2=nu, restriction=restriction))
        _cache[key] = (h, oh)
    return _cache[key]


def _row_scale(lev, x):
    # s_i = sum_k |w_k| (|x_i| + |x_k|) = (|L| |x|)_i
    return abs(lev.L) @ np.abs(x)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_laplace0_apply_matches_oracle(name, prec):
    h, oh = _pair(name)
    assert h.ell_width[-1] == (7 if name == "fan3" else 6)
    for l in range(h.nlevels):
        lev = oh.levels[l]
        x = W.uniform_field(lev.mesh.nv, 100 + l)
        if prec == "f32":
            x = x.astype(np.float32).astype(np.float64)  # exactly representable input
        y = h.laplace0_apply(_dev(x, torch.float64 if prec == "f64" else torch.float32), level=l).double().cpu().numpy()
        ref = np.where(lev.free, lev.L @ x, 0.0)
        eps = EPS64 if prec == "f64" else EPS32
        bound = TOL_ROW * eps * _row_scale(lev, x) + 1e-300
        assert np.all(np.abs(y - ref) <= bound), (l, np.max(np.abs(y - ref) / bound))


@pytest.mark.parametrize("name", ["square5", "ico5", "fan3"])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_residual_matches_oracle(name, prec):
    h, oh = _pair(name)
    lev = oh.finest
    x = W.uniform_field(lev.mesh.nv, 7)
    b = W.uniform_field(lev.mesh.nv, 8)
    if prec == "f32":
        x = x.astype(np.float32).astype(np.float64)
        b = b.astype(np.float32).astype(np.float64)
    dt = torch.float64 if prec == "f64" else torch.float32
    r = h.residual(_dev(b, dt), _dev(x, dt)).double().cpu().numpy()
    ref = np.where(lev.free, b - lev.L @ x, 0.0)
    eps = EPS64 if prec == "f64" else EPS32
    bound = TOL_ROW * eps * (_row_scale(lev, x) + np.abs(b)) + 1e-300
    assert np.all(np.abs(r - ref) <= bound)


def _s0_rel(lev, a, b):
    return omg.star0_norm(lev, a - b) / omg.star0_norm(lev, b)


@pytest.mark.parametrize("name", ["square5", "ico5", "fan3", "grid_ragged"])
@pytest.mark.parametrize("smoother", ["jacobi", "chebyshev", "mcgs"])
@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("restriction", ["rownorm", "star0"])
def test_one_cycle_matches_oracle(name, smoother, prec, restriction):
    h, oh = _pair(name, smoother, restriction=restriction)
    lev = oh.finest
    b = omg.prepare_rhs(oh, W.uniform_field(lev.mesh.nv, 21))
    ref = omg.vcycle(oh, b, np.zeros_like(b))
    dt = torch.float64 if prec == "f64" else torch.float32
    x = torch.zeros(lev.mesh.nv, dtype=dt, device="cuda")
    h.vcycle(_dev(b, dt), x)
    got = x.double().cpu().numpy()
    tol = 1e-12 if prec == "f64" else 2e-5
    assert _s0_rel(lev, got, ref) < tol
    assert np.all(got[~lev.free] == 0.0)


@pytest.mark.parametrize("name", ["square5", "ico5", "fan3"])
@pytest.mark.parametrize("solver", ["mg", "mgpcg", "cg"])
@pytest.mark.parametrize("mode", ["f64", "mixed", "mixed_ff"])
def test_solve_matches_oracle(name, solver, mode):
    h, oh = _pair(name)
    lev = oh.finest
    b = W.uniform_field(lev.mesh.nv, 31)
    tol = 1e-10
    xs = omg.direct_solve(oh, b)
    x, st = h.solve(_dev(b), solver=solver, mode=mode, tol=tol, maxit=1000 if solver == "cg" else 100)
    x = x.cpu().numpy()
    assert st.status == 0 and st.rel_res <= tol
    bp = omg.prepare_rhs(oh, b)
    # the true FP64 residual of the returned iterate, recomputed by the oracle
    assert omg.rel_residual(lev, bp, x) <= 4 * tol
    assert _s0_rel(lev, x, xs) < 1e-7
    if mode == "f64" and solver != "cg":
        # the same algorithm in the same precision takes the same number of steps
        ref = omg.mg_solve(oh, b, tol, 100) if solver == "mg" else omg.pcg_solve(oh, b, tol, 100)
        assert abs(st.iters - ref.iters) <= 1
    if mode == "f64" and solver == "cg":
        ref = omg.pcg_solve(oh, b, tol, 1000, precondition=False)
        assert abs(st.iters - ref.iters) <= max(2, 0.05 * ref.iters)


def test_config1_closed_form():
    # unit square x5, 5-level V(2,2) Jacobi, Dirichlet, -Delta of sin(pi x) sin(pi y), standalone MG to 1e-10
    h, oh = _pair("square5")
    lev = oh.finest
    assert h.nv == [9, 25, 81, 289, 1089]
    b = W.rhs_sin_square(lev.mesh.verts)
    x, st = h.solve(_dev(b), solver="mg", mode="f64", tol=1e-10, maxit=100)
    ref = omg.mg_solve(oh, b, 1e-10, 100)
    assert st.iters == ref.iters
    hh = 1.0 / 32
    lam11 = 8.0 / hh ** 2 * math.sin(math.pi * hh / 2) ** 2
    u_h = 2 * math.pi ** 2 / lam11 * W.u_sin_square(lev.mesh.verts)
    assert _s0_rel(lev, x.cpu().numpy(), u_h) < 1e-9


def test_host_buffers_and_warm_start():
    h, oh = _pair("ico5")
    lev = oh.finest
    b = torch.as_tensor(W.uniform_field(lev.mesh.nv, 41)).pin_memory()
    x, st = h.solve(b, tol=1e-9)
    assert x.device.type == "cpu" and st.rel_res <= 1e-9
    x2, st2 = h.solve(b.cuda(), x=x.cuda(), warm_start=True, tol=1e-9)
    assert st2.iters <= 1 and st2.rel_res0 <= 1e-8


@pytest.mark.parametrize("name", ["ico5", "square5"])
@pytest.mark.parametrize("mode", ["f64", "mixed", "mixed_ff"])
@pytest.mark.parametrize("pinned", [True, False])
def test_solve_host_matches_device(name, mode, pinned):
    # dec_solve_host runs the same kernels on copies of b and x: bitwise the device solve
    h, oh = _pair(name)
    b = W.uniform_field(oh.finest.mesh.nv, 43)
    bh = torch.as_tensor(b)
    if pinned:
        bh = bh.pin_memory()
    xd, sd = h.solve(_dev(b), mode=mode, tol=1e-10)
    xh, sh = h.solve(bh, mode=mode, tol=1e-10)
    assert xh.device.type == "cpu" and sh.iters == sd.iters and torch.equal(xh, xd.cpu())
    x0 = xh.clone().pin_memory() if pinned else xh.clone()
    x2, s2 = h.solve(bh, x0, warm_start=True, mode=mode, tol=1e-10)
    assert x2 is x0 and s2.iters <= 1 and s2.rel_res <= 1e-10


def test_error_paths():
    P = _lib()
    h, oh = _pair("ico5")
    n = oh.finest.mesh.nv
    b = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    with pytest.raises(P.DecError) as ei:
        h.solve(b)
    assert ei.value.code == 6  # DEC_ERR_NONFINITE
    b = _dev(W.uniform_field(n, 5))
    x, st = h.solve(b, maxit=1, raise_on_fail=False)
    assert st.status == 5 and st.iters == 1 and 0 < st.rel_res < st.rel_res0
    assert torch.isfinite(x).all()
    z, st = h.solve(torch.zeros(n, dtype=torch.float64, device="cuda"))
    assert st.iters == 0 and torch.count_nonzero(z) == 0
    with pytest.raises(TypeError):
        h.solve(b.float())


def test_single_level_hierarchy_is_direct_solve():
    P = _lib()
    v, t = W.icosahedron()
    h = P.Hierarchy(P.Mesh(v, t), 2, 1, bc="gauge", sphere=True)
    oh = omg.build_hierarchy(v, t, 2, 1, "gauge", sphere=True)
    b = omg.prepare_rhs(oh, W.uniform_field(h.n, 3))
    x = torch.zeros(h.n, dtype=torch.float64, device="cuda")
    h.vcycle(_dev(b), x)
    assert _s0_rel(oh.finest, x.cpu().numpy(), omg.direct_solve(oh, b)) < 1e-12


@pytest.mark.parametrize("solver", ["mg", "mgpcg"])
def test_host_and_device_loops_agree(solver):
    h, oh = _pair("ico5")
    b = _dev(W.uniform_field(oh.finest.mesh.nv, 51))
    x1, s1 = h.solve(b, solver=solver, tol=1e-10)
    x2, s2 = h.solve(b, solver=solver, tol=1e-10, host_loop=True, check_every=3)
    assert s1.iters == s2.iters
    assert torch.equal(x1, x2)  # same kernels in the same order: bitwise equal


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("name", ["square5", "ico5"])
def test_w_cycle_matches_oracle(name, prec):
    P = _lib()
    base, nsub, nl, bc, sph = CASES[name]
    v, t = base()
    h = P.Hierarchy(P.Mesh(v, t), nsub, nl, bc=bc, sphere=sph, gamma=2)
    oh = omg.build_hierarchy(v, t, nsub, nl, bc, sphere=sph, opts=omg.MGOptions(gamma=2))
    lev = oh.finest
    b = omg.prepare_rhs(oh, W.uniform_field(lev.mesh.nv, 61))
    ref = omg.vcycle(oh, b, np.zeros_like(b))
    dt = torch.float64 if prec == "f64" else torch.float32
    x = torch.zeros(lev.mesh.nv, dtype=dt, device="cuda")
    h.vcycle(_dev(b, dt), x)
    assert _s0_rel(lev, x.double().cpu().numpy(), ref) < (1e-12 if prec == "f64" else 2e-5)
    xs, st = h.solve(_dev(W.uniform_field(lev.mesh.nv, 62)), solver="mg", mode="f64", tol=1e-10)
    ref2 = omg.mg_solve(oh, W.uniform_field(lev.mesh.nv, 62), 1e-10, 100)
    assert abs(st.iters - ref2.iters) <= 1


@pytest.mark.parametrize("name", ["square5", "ico5"])
@pytest.mark.parametrize("smoother", ["jacobi", "chebyshev", "mcgs"])
@pytest.mark.parametrize("gamma", [1, 2])
def test_convergence_factor_matches_oracle(name, smoother, gamma):
    # standalone MG in FP64: geometric-mean residual reduction per cycle, GPU vs oracle
    P = _lib()
    base, nsub, nl, bc, sph = CASES[name]
    v, t = base()
    h = P.Hierarchy(P.Mesh(v, t), nsub, nl, bc=bc, sphere=sph, smoother=smoother, gamma=gamma)
    oh = omg.build_hierarchy(v, t, nsub, nl, bc, sphere=sph, opts=omg.MGOptions(smoother=smoother, gamma=gamma))
    b = W.uniform_field(oh.finest.mesh.nv, 71)
    _, st = h.solve(_dev(b), solver="mg", mode="f64", tol=1e-10, maxit=100)
    ref = omg.mg_solve(oh, b, 1e-10, 100)
    cf_gpu = (st.rel_res / st.rel_res0) ** (1.0 / st.iters)
    cf_ref = omg.convergence_factor(ref.history)
    assert abs(cf_gpu - cf_ref) <= 0.02, (cf_gpu, cf_ref)


@pytest.mark.parametrize("name", ["square5", "ico5"])
def test_morton_order_cycle_and_solve_match_oracle(name):
    # the opt-in space-filling-curve numbering: same tables as the oracle's, same cycle, same solution
    P = _lib()
    base, nsub, nl, bc, sph = CASES[name]
    v, t = base()
    h = P.Hierarchy(P.Mesh(v, t), nsub, nl, bc=bc, sphere=sph, smoother="chebyshev", order="morton")
    oh = omg.build_hierarchy(v, t, nsub, nl, bc, sphere=sph, opts=omg.MGOptions(smoother="chebyshev"),
                             order="morton")
    lev = oh.finest
    assert np.array_equal(h.table(-1, "verts"), lev.mesh.verts)
    b = omg.prepare_rhs(oh, W.uniform_field(lev.mesh.nv, 61))
    x = torch.zeros(h.n, dtype=torch.float64, device="cuda")
    h.vcycle(_dev(b), x)
    ref = omg.vcycle(oh, b, np.zeros_like(b))
    assert _s0_rel(lev, x.cpu().numpy(), ref) < 1e-12
    xs, st = h.solve(_dev(b), mode="mixed_ff", tol=1e-10)
    assert st.rel_res <= 1e-10
    assert _s0_rel(lev, xs.cpu().numpy(), omg.direct_solve(oh, b)) < 1e-7


@pytest.mark.parametrize("name", ["square5", "ico5", "fan3"])
@pytest.mark.parametrize("mode", ["f64", "mixed_ff"])
def test_mcgs_solves_match_oracle(name, mode):
    # the paper's Gauss-Seidel, multicoloured: standalone MG and MG-PCG reach the direct solution
    h, oh = _pair(name, smoother="mcgs")
    lev = oh.finest
    b = W.uniform_field(lev.mesh.nv, 67)
    xs = omg.direct_solve(oh, b)
    for solver in ("mg", "mgpcg"):
        x, st = h.solve(_dev(b), solver=solver, mode=mode, tol=1e-10, maxit=100)
        assert st.rel_res <= 1e-10
        assert _s0_rel(lev, x.cpu().numpy(), xs) < 1e-7
    if mode == "f64":
        ref = omg.mg_solve(oh, b, 1e-10, 100)
        _, st = h.solve(_dev(b), solver="mg", mode="f64", tol=1e-10, maxit=100)
        assert abs(st.iters - ref.iters) <= 1


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("name", ["square5", "ico5"])
@pytest.mark.parametrize("smoother", ["jacobi", "chebyshev"])
def test_f_cycle_matches_oracle(name, prec, smoother):
    # F-cycles: the coarse correction is an F-cycle then a V-cycle (4 levels: differs from V and W)
    P = _lib()
    base, nsub, nl, bc, sph = CASES[name]
    v, t = base()
    h = P.Hierarchy(P.Mesh(v, t), nsub, nl, bc=bc, sphere=sph, smoother=smoother, fcycle=True)
    oh = omg.build_hierarchy(v, t, nsub, nl, bc, sphere=sph, opts=omg.MGOptions(smoother=smoother, fcycle=True))
    lev = oh.finest
    b = omg.prepare_rhs(oh, W.uniform_field(lev.mesh.nv, 63))
    ref = omg.vcycle(oh, b, np.zeros_like(b))
    dt = torch.float64 if prec == "f64" else torch.float32
    x = torch.zeros(lev.mesh.nv, dtype=dt, device="cuda")
    h.vcycle(_dev(b, dt), x)
    assert _s0_rel(lev, x.double().cpu().numpy(), ref) < (1e-12 if prec == "f64" else 2e-5)
    b2 = W.uniform_field(lev.mesh.nv, 64)
    _, st = h.solve(_dev(b2), solver="mg", mode="f64", tol=1e-10)
    ref2 = omg.mg_solve(oh, b2, 1e-10, 100)
    assert abs(st.iters - ref2.iters) <= 1
    cf = (st.rel_res / st.rel_res0) ** (1.0 / st.iters)
    assert abs(cf - omg.convergence_factor(ref2.history)) <= 0.02
    xs, st = h.solve(_dev(b2), solver="mgpcg", mode="mixed_ff", tol=1e-10)
    assert st.rel_res <= 1e-10 and _s0_rel(lev, xs.cpu().numpy(), omg.direct_solve(oh, b2)) < 1e-7


CUBIC = {
    # name: (base, nsub, nlevels, bc, sphere)
    "square_cubic": (W.unit_square, 3, 3, "dirichlet", False),
    "ico_cubic": (W.icosahedron, 3, 3, "gauge", True),
}


@pytest.mark.parametrize("name", list(CUBIC))
@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("restriction", ["rownorm", "star0"])
@pytest.mark.parametrize("smoother", ["jacobi", "chebyshev"])
def test_cubic_cycle_matches_oracle(name, prec, restriction, smoother):
    # cubic (1->9) subdivision: interpolation by the geometric map, restriction by the transpose of its
    # row normalization (or the *0-adjoint), both as general gather kernels
    P = _lib()
    base, nsub, nl, bc, sph = CUBIC[name]
    v, t = base()
    h = P.Hierarchy(P.Mesh(v, t), nsub, nl, bc=bc, sphere=sph, smoother=smoother, restriction=restriction,
                    scheme="cubic")
    oh = omg.build_hierarchy(v, t, nsub, nl, bc, sphere=sph, scheme="cubic",
                             opts=omg.MGOptions(smoother=smoother, restriction=restriction))
    lev = oh.finest
    assert h.nv == [l.mesh.nv for l in oh.levels]
    b = omg.prepare_rhs(oh, W.uniform_field(lev.mesh.nv, 71))
    ref = omg.vcycle(oh, b, np.zeros_like(b))
    dt = torch.float64 if prec == "f64" else torch.float32
    x = torch.zeros(lev.mesh.nv, dtype=dt, device="cuda")
    h.vcycle(_dev(b, dt), x)
    assert _s0_rel(lev, x.double().cpu().numpy(), ref) < (1e-12 if prec == "f64" else 2e-5)


@pytest.mark.parametrize("name", list(CUBIC))
def test_cubic_solves_match_oracle(name):
    P = _lib()
    base, nsub, nl, bc, sph = CUBIC[name]
    v, t = base()
    h = P.Hierarchy(P.Mesh(v, t), nsub, nl, bc=bc, sphere=sph, smoother="chebyshev", scheme="cubic")
    oh = omg.build_hierarchy(v, t, nsub, nl, bc, sphere=sph, scheme="cubic", opts=omg.MGOptions(smoother="chebyshev"))
    lev = oh.finest
    b = W.uniform_field(lev.mesh.nv, 72)
    xs = omg.direct_solve(oh, b)
    for solver, mode in (("mg", "f64"), ("mgpcg", "mixed_ff"), ("mgpcg", "mixed")):
        x, st = h.solve(_dev(b), solver=solver, mode=mode, tol=1e-10, maxit=200)
        assert st.rel_res <= 1e-10
        assert _s0_rel(lev, x.cpu().numpy(), xs) < 1e-7
    _, st = h.solve(_dev(b), solver="mg", mode="f64", tol=1e-10, maxit=200)
    ref = omg.mg_solve(oh, b, 1e-10, 200)
    assert abs(st.iters - ref.iters) <= 1
    cf = (st.rel_res / st.rel_res0) ** (1.0 / st.iters)
    assert abs(cf - omg.convergence_factor(ref.history)) <= 0.02


def test_cubic_square_closed_form():
    # unit square cubed three times (28 x 28 grid): MG reaches the discrete solution of -Delta sin sin
    P = _lib()
    v, t = W.unit_square()
    h = P.Hierarchy(P.Mesh(v, t), 3, 3, bc="dirichlet", scheme="cubic")
    xy = h.table(-1, "verts")
    x, st = h.solve(_dev(W.rhs_sin_square(xy)), solver="mg", mode="f64", tol=1e-12, maxit=200)
    hh = 1.0 / 27
    u_h = 2 * math.pi ** 2 / (8.0 / hh ** 2 * math.sin(math.pi * hh / 2) ** 2) * W.u_sin_square(xy)
    s0 = h.table(-1, "star0")
    d = x.cpu().numpy() - u_h
    assert np.sqrt(np.sum(s0 * d * d) / np.sum(s0 * u_h * u_h)) < 1e-10


def test_interleaved_right_hand_sides_match_single_calls():
    # k = 3 interleaved columns ([v * k + j]): the operator and residual per column equal the single-column
    # calls bitwise (same per-row arithmetic); cycles and solves per column equal single-column ones
    import ctypes as C
    from paper_2508_12501_gb300 import _lib as L
    h, oh = _pair("ico5")
    lev = oh.finest
    n, k = lev.mesh.nv, 3
    X = np.stack([W.uniform_field(n, 300 + j) for j in range(k)], axis=1)
    Bm = np.stack([omg.prepare_rhs(oh, W.uniform_field(n, 310 + j)) for j in range(k)], axis=1)
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for dt, prec in ((torch.float64, L.DEC_F64), (torch.float32, L.DEC_F32)):
        x = torch.as_tensor(X, dtype=dt, device="cuda").contiguous()
        b = torch.as_tensor(Bm, dtype=dt, device="cuda").contiguous()
        y = torch.empty_like(x)
        r = torch.empty_like(x)
        assert L.lib.dec_laplace0_apply(h._h, h.nlevels - 1, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()), k,
                                        prec, st) == 0
        assert L.lib.dec_residual(h._h, h.nlevels - 1, C.c_void_p(b.data_ptr()), C.c_void_p(x.data_ptr()),
                                  C.c_void_p(r.data_ptr()), k, prec, st) == 0
        xv = x.clone()
        assert L.lib.dec_mg_vcycle(h._h, C.c_void_p(b.data_ptr()), C.c_void_p(xv.data_ptr()), k, prec, st) == 0
        for j in range(k):
            xj = x[:, j].contiguous()
            assert torch.equal(y[:, j], h.laplace0_apply(xj))
            rj = torch.empty_like(xj)
            assert L.lib.dec_residual(h._h, h.nlevels - 1, C.c_void_p(b[:, j].contiguous().data_ptr()),
                                      C.c_void_p(xj.data_ptr()), C.c_void_p(rj.data_ptr()), 1, prec, st) == 0
            assert torch.equal(r[:, j], rj)
            h.vcycle(b[:, j].contiguous(), xj)
            assert torch.equal(xv[:, j], xj)
    b = torch.as_tensor(np.stack([W.uniform_field(n, 320 + j) for j in range(k)], axis=1), device="cuda")
    x = torch.empty_like(b)
    o = L.dec_solve_opts()
    L.lib.dec_solve_default_opts(C.byref(o))
    o.tol = 1e-10
    sts = L.dec_stats()
    assert L.lib.dec_solve(h._h, C.c_void_p(b.data_ptr()), C.c_void_p(x.data_ptr()), k, C.byref(o), C.byref(sts),
                           st) == 0
    assert sts.rel_res <= 1e-10
    for j in range(k):
        xs = omg.direct_solve(oh, b[:, j].cpu().numpy())
        assert _s0_rel(lev, x[:, j].cpu().numpy(), xs) < 1e-7
