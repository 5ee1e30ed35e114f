"""Float-float outer iteration (mode "mixed_ff") and the benchmark workload at full size.

The ff outer iteration keeps x, r and q = L p as unevaluated sums of two
floats (about 48 bits) and the search direction in FP32.  What the oracle can
check at any size is the property the mode promises: the FP64 relative
residual ||b - L x|| / ||b|| of the returned x, recomputed on the CPU by the
oracle's own operator, meets the requested tolerance.  The outer vectors are
scaled by a power of two, so scaling b by 2^k scales x by exactly 2^k: the
results are compared bitwise, including a b far below the FP32 range.

The full-size case is the benchmark workload: icosphere x8 (655,362
vertices), levels 8..2, Chebyshev V(2,2), gauge, a sum of real spherical
harmonics l = 1..16 (seed 1), MG-PCG to 1e-8, in every precision mode.  Each
mode's solution is compared with the oracle's u*: the oracle's own flexible
MG-PCG (FP64, the same hierarchy and smoother) run to a relative residual of
1e-13, in the *0 norm, to the stated 1e-6.
"""
import numpy as np
import pytest

import workloads as W
from oracle import mesh as omesh, multigrid as omg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _lib():
    import paper_2508_12501_gb300 as P
    return P


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _s0_rel(s0, a, b):
    d = a - b
    return float(np.sqrt(np.sum(s0 * d * d) / np.sum(s0 * b * b)))


_full = {}


def _full_size():
    if not _full:
        P = _lib()
        v, t = W.icosahedron()
        h = P.Hierarchy(P.Mesh(v, t), 8, 7, bc="gauge", sphere=True, smoother="chebyshev")
        oh = omg.build_hierarchy(v, t, 8, 7, "gauge", sphere=True, opts=omg.MGOptions(smoother="chebyshev"))
        lev = oh.finest
        b = W.sh_sum(lev.mesh.verts, W.sh_coefficients(1))
        _full.update(h=h, oh=oh, lev=lev, b=b, bp=omg.project_mean_zero(lev, b))
    return _full


def _u_star():
    F = _full_size()
    if "ustar" not in F:
        ref = omg.pcg_solve(F["oh"], F["b"], 1e-13, 200)
        assert ref.rel_res <= 1e-13
        F["ustar"] = ref.x
    return F["ustar"]


MODES = ["f64", "mixed", "mixed_ff", "mixed_f32dot"]


@pytest.mark.parametrize("mode", MODES)
def test_benchmark_workload_true_residual(mode):
    F = _full_size()
    h, lev = F["h"], F["lev"]
    assert h.n == 655362
    x, st = h.solve(_dev(F["b"]), solver="mgpcg", mode=mode, tol=1e-8)
    x = x.cpu().numpy()
    assert st.status == 0 and st.rel_res <= 1e-8 and st.iters <= 10
    true = omg.rel_residual(lev, F["bp"], x)
    assert true <= 1e-8, true
    # the reported (updated) residual tracks the true one
    assert abs(true - st.rel_res) <= 1e-3 * 1e-8 + 0.05 * st.rel_res
    assert abs(omg.star0_mean(lev, x)) <= 1e-12 * np.sqrt(np.mean(x * x))
    F.setdefault("x", {})[mode] = x


def test_benchmark_workload_modes_agree():
    F = _full_size()
    xs = F.get("x", {})
    if len(xs) < len(MODES):
        pytest.skip("needs the solves above")
    s0 = F["lev"].star0
    # all at relative residual 1e-8: solutions agree far below the discretization error
    for m in MODES[1:]:
        assert _s0_rel(s0, xs[m], xs["f64"]) < 1e-7, m


@pytest.mark.parametrize("mode", MODES)
def test_benchmark_workload_solution_error_vs_oracle(mode):
    # ||u - u*||_*0 / ||u*||_*0 <= 1e-6 against the oracle's u* (its FP64 MG-PCG to 1e-13)
    F = _full_size()
    ustar = _u_star()
    x, st = F["h"].solve(_dev(F["b"]), solver="mgpcg", mode=mode, tol=1e-8)
    assert st.status == 0
    err = _s0_rel(F["lev"].star0, x.cpu().numpy(), ustar)
    print(f"icosphere x8 {mode}: iters {st.iters}, rel_res {st.rel_res:.3e}, *0 error vs oracle u* {err:.3e}")
    assert err <= 1e-6, err


@pytest.mark.parametrize("solver", ["mg", "mgpcg"])
@pytest.mark.parametrize("bc", ["gauge", "dirichlet"])
def test_power_of_two_scaling_is_exact(solver, bc):
    P = _lib()
    if bc == "gauge":
        v, t = W.icosahedron()
        h = P.Hierarchy(P.Mesh(v, t), 5, 4, bc="gauge", sphere=True)
    else:
        v, t = W.unit_square()
        h = P.Hierarchy(P.Mesh(v, t), 6, 5, bc="dirichlet")
    b = _dev(W.uniform_field(h.n, 91))
    x1, s1 = h.solve(b, solver=solver, mode="mixed_ff", tol=1e-10)
    for k in (-140, -60, 70):
        # 2^-140 b is below the smallest normal FP32 number: only the scaling keeps it solvable
        xk, sk = h.solve(b * 2.0 ** k, solver=solver, mode="mixed_ff", tol=1e-10)
        assert sk.iters == s1.iters
        assert torch.equal(xk, x1 * 2.0 ** k)


@pytest.mark.parametrize("solver", ["mg", "mgpcg"])
def test_ff_host_and_device_loops_agree(solver):
    P = _lib()
    v, t = W.icosahedron()
    h = P.Hierarchy(P.Mesh(v, t), 5, 4, bc="gauge", sphere=True, smoother="chebyshev")
    b = _dev(W.uniform_field(h.n, 93))
    x1, s1 = h.solve(b, solver=solver, mode="mixed_ff", tol=1e-10)
    x2, s2 = h.solve(b, solver=solver, mode="mixed_ff", tol=1e-10, host_loop=True, check_every=2)
    assert s1.iters == s2.iters
    assert torch.equal(x1, x2)


def test_ff_warm_start_and_star1_update():
    # new *1 weights reach the ff operator (w32 + wlo); a warm start from the solution converges at once
    from oracle import dec
    P = _lib()
    v, t = W.unit_square()
    h = P.Hierarchy(P.Mesh(v, t), 6, 5, bc="dirichlet")
    m = omesh.refine(v, t, 6)[0][-1]
    scale = W.lognormal_factors(m.ne, 7)
    lev = omg.make_level(m, "dirichlet", star1_scale=scale)
    h.set_star1(_dev(dec.hodge_star1(m, scale)))
    b = W.uniform_field(h.n, 95)
    x, st = h.solve(_dev(b), mode="mixed_ff", tol=1e-10, maxit=200)
    assert omg.rel_residual(lev, lev.free * b, x.cpu().numpy()) <= 4e-10
    x2, st2 = h.solve(_dev(b), x=x, warm_start=True, mode="mixed_ff", tol=1e-9)
    assert st2.iters <= 1


@pytest.mark.parametrize("mode", ["f64", "mixed", "mixed_ff"])
def test_tol_zero_stops_cleanly(mode):
    # tol = 0 is never met: the iteration runs until it cannot move in its precision (in the
    # mixed modes the FP32 dot products underflow near relative residual 1e-20) and then stops
    # with DEC_ERR_NOT_CONVERGED, a finite x and no NaN
    P = _lib()
    v, t = W.unit_square()
    h = P.Hierarchy(P.Mesh(v, t), 5, 5, bc="dirichlet", smoother="chebyshev")
    oh = omg.build_hierarchy(v, t, 5, 5, "dirichlet", opts=omg.MGOptions(smoother="chebyshev"))
    b = W.uniform_field(h.n, 97)
    x, st = h.solve(_dev(b), mode=mode, tol=0.0, maxit=400, raise_on_fail=False)
    assert st.status == 5 and torch.isfinite(x).all()
    assert st.rel_res < 1e-12
    xs = omg.direct_solve(oh, b)
    assert _s0_rel(oh.finest.star0, x.cpu().numpy(), xs) < 1e-10


@pytest.mark.parametrize("smoother", ["jacobi", "chebyshev"])
def test_kernel_timer(smoother):
    # back-to-back timing of the finest-level kernels of the float-float loop: positive times, the byte model,
    # argument checks, and a solve afterwards still converges (the timer only overwrote work vectors)
    import paper_2508_12501_gb300 as P
    v, t = W.icosahedron()
    h = P.Hierarchy(P.Mesh(v, t), 5, 4, bc="gauge", sphere=True, smoother=smoother)
    n, K = h.n, 6
    cheb = smoother == "chebyshev"
    want = {"smoothdots": n * (8 * K + 12 + (4 if cheb else 0) + 9), "spmv64": n * (12 * K + 16),
            "update": n * (44 + 8 + (4 if cheb else 0))}
    for kind, by in want.items():
        ms, b = h.time_kernel(kind, reps=5)
        assert ms > 0 and b == by
    ms, b = h.time_kernel("smooth", level=1, reps=5)
    assert ms > 0 and b > 0
    for bad in (dict(kind="spmv64", level=1), dict(kind="residual"), dict(kind="update", reps=0)):
        with pytest.raises(P.DecError):
            h.time_kernel(**bad)
    b = torch.as_tensor(W.uniform_field(n, 3), device="cuda")
    assert h.solve(b, mode="mixed_ff", tol=1e-10)[1].rel_res <= 1e-10


@pytest.mark.parametrize("bc", ["gauge", "dirichlet"])
@pytest.mark.parametrize("solver", ["mg", "mgpcg"])
def test_ff_cold_start_edges(bc, solver):
    # the two-kernel cold start (x = 0): b = 0, maxit = 0, a NaN on a free row, and agreement with a
    # warm start from x = 0, which forms r = b - L x and splits it the general way
    P = _lib()
    if bc == "gauge":
        v, t = W.icosahedron()
        h = P.Hierarchy(P.Mesh(v, t), 5, 4, bc="gauge", sphere=True, smoother="chebyshev")
    else:
        v, t = W.unit_square()
        h = P.Hierarchy(P.Mesh(v, t), 6, 5, bc="dirichlet", smoother="chebyshev")
    n = h.n
    z, st = h.solve(torch.zeros(n, dtype=torch.float64, device="cuda"), solver=solver, mode="mixed_ff")
    assert st.status == 0 and st.iters == 0 and torch.count_nonzero(z) == 0
    b = _dev(W.uniform_field(n, 99))
    x0, st0 = h.solve(b, solver=solver, mode="mixed_ff", maxit=0, raise_on_fail=False)
    assert st0.status == 5 and st0.iters == 0 and torch.count_nonzero(x0) == 0 and st0.rel_res == st0.rel_res0 == 1.0
    free = np.flatnonzero(h.table(-1, "free"))
    bn = b.clone()
    bn[int(free[len(free) // 2])] = float("nan")
    with pytest.raises(P.DecError) as ei:
        h.solve(bn, solver=solver, mode="mixed_ff")
    assert ei.value.code == 6
    xc, sc = h.solve(b, solver=solver, mode="mixed_ff", tol=1e-10)
    xw, sw = h.solve(b, torch.zeros(n, dtype=torch.float64, device="cuda"), solver=solver, mode="mixed_ff", tol=1e-10,
                     warm_start=True)
    assert sc.status == sw.status == 0 and sc.iters == sw.iters
    s0 = h.table(-1, "star0")
    assert _s0_rel(s0, xc.cpu().numpy(), xw.cpu().numpy()) < 1e-8
