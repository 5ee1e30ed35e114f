"""Pins of the oracle's multigrid and Krylov layer.

Smoothers are pinned against closed forms on diagonal operators (Jacobi and
Chebyshev polynomials) and against library triangular solves (Gauss-Seidel);
the coarse solve against a pseudo-inverse; unpreconditioned flexible CG
against scipy's CG on the equivalent symmetric system; MG and MG-PCG against
direct solves.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import workloads as W
from oracle import multigrid as mg


def _square(nsub, nlevels, **kw):
    v, t = W.unit_square()
    return mg.build_hierarchy(v, t, nsub, nlevels, "dirichlet", opts=mg.MGOptions(**kw))


def _square_gauge(nsub, nlevels, **kw):
    v, t = W.unit_square()
    return mg.build_hierarchy(v, t, nsub, nlevels, "gauge", opts=mg.MGOptions(**kw))


def _ico(nsub, nlevels, **kw):
    v, t = W.icosahedron()
    return mg.build_hierarchy(v, t, nsub, nlevels, "gauge", sphere=True, opts=mg.MGOptions(**kw))


def _diag_level(lams):
    n = len(lams)
    lev = mg.Level(mesh=None, star0=np.ones(n), star1=None, A=None, L=sp.diags(lams).tocsr(),
                   free=np.ones(n, dtype=bool), diag=np.ones(n))
    lev.lmax = float(max(lams))
    return lev


def test_jacobi_closed_form_on_diagonal_operator():
    lams = np.array([0.1, 0.5, 1.0, 1.7])
    lev = _diag_level(lams)
    for nu in (1, 2, 3):
        x = mg.jacobi(lev, np.zeros(4), np.ones(4), 0.7, nu)
        assert np.allclose(x, (1 - 0.7 * lams) ** nu, rtol=1e-14)


def _cheb_T(s, x):
    return np.cosh(s * np.arccosh(x)) if np.all(x >= 1) else np.cos(s * np.arccos(np.clip(x, -1, 1)))


def test_chebyshev_is_scaled_chebyshev_polynomial():
    # with b = 0 the error after s steps is T_s((theta - lam)/delta) / T_s(theta/delta)
    lams = np.linspace(0.35, 1.9, 9)
    lev = _diag_level(lams)
    lo, hi = 0.3, 1.1
    a, bb = lo * lev.lmax, hi * lev.lmax
    theta, delta = (a + bb) / 2, (bb - a) / 2
    for s in (1, 2, 3, 4):
        x = mg.chebyshev(lev, np.zeros(len(lams)), np.ones(len(lams)), s, lo, hi)
        expect = np.array([_cheb_T(s, np.array([(theta - l) / delta]))[0] for l in lams]) / _cheb_T(s, np.array([theta / delta]))[0]
        assert np.allclose(x, expect, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("kl", [(1, 1), (3, 2), (7, 11), (15, 15)])
def test_jacobi_damps_each_sine_mode_by_its_symbol(kl):
    # On the unit square L is the 5-point stencil (/h^2), whose Dirichlet eigenvectors are the sine modes
    # sin(k pi x) sin(l pi y) with D^-1 L eigenvalue sin^2(k pi h/2) + sin^2(l pi h/2): one damped-Jacobi
    # sweep with b = 0 multiplies the mode by exactly 1 - omega (that sum), on the DEC operator itself.
    k, l = kl
    v, t = W.unit_square()
    h = mg.build_hierarchy(v, t, 4, 1, "dirichlet")
    lev = h.finest
    xy = lev.mesh.verts
    e = np.sin(k * np.pi * xy[:, 0]) * np.sin(l * np.pi * xy[:, 1]) * lev.free
    hh = 1.0 / 16
    sym = np.sin(k * np.pi * hh / 2) ** 2 + np.sin(l * np.pi * hh / 2) ** 2
    for omega in (2.0 / 3.0, 0.8, 1.0):
        x = mg.jacobi(lev, np.zeros(lev.mesh.nv), e.copy(), omega, 1)
        assert np.max(np.abs(x - (1.0 - omega * sym) * e)) < 1e-13


def test_gauss_seidel_matches_sequential_sweep():
    h = _square(2, 2, smoother="gs")
    lev = h.finest
    rng = np.random.default_rng(0)
    b = lev.free * rng.standard_normal(lev.mesh.nv)
    x0 = lev.free * rng.standard_normal(lev.mesh.nv)
    got = mg.gauss_seidel(lev, b, x0, 2)
    L = lev.L.toarray()
    x = x0.copy()
    for _ in range(2):
        for i in range(len(x)):
            if lev.free[i]:
                s = sum(L[i, j] * x[j] for j in range(len(x)) if j != i and lev.free[j])
                x[i] = (b[i] - s) / L[i, i]
    assert np.allclose(got, x, rtol=1e-13, atol=1e-13)


def test_greedy_colouring_worked_example():
    # Heptagon fan: centre 0, rim 1..7 in cyclic order.  First fit in vertex order, worked by hand: the
    # centre takes 0; rim vertex 1 sees {0} -> 1; 2 sees {0, 1} -> 2; 3 sees {0, 2} -> 1; 4 -> 2; 5 -> 1;
    # 6 -> 2; 7 touches 0, 6 and 1, sees {0, 2, 1} -> 3 (an odd rim needs a third rim colour).  Any other
    # order (largest first, by degree, by colour class size) colours this fan differently.
    from oracle import mesh as om
    v, t = W.heptagon_fan()
    m = om.build_mesh(v, t)
    assert mg.greedy_colors(m).tolist() == [0, 1, 2, 1, 2, 1, 2, 3]
    # the same fan renumbered (rim starting one step later) moves the third rim colour with the numbering
    perm = np.array([0, 2, 3, 4, 5, 6, 7, 1])  # new vertex k is old vertex perm[k]
    inv = np.argsort(perm)
    m2 = om.build_mesh(v[perm], inv[t])
    assert mg.greedy_colors(m2).tolist() == [0, 1, 2, 1, 2, 1, 2, 3]


@pytest.mark.parametrize("mk", [lambda: _square(3, 2, smoother="mcgs"), lambda: _ico(2, 2, smoother="mcgs")])
def test_multicolour_gs_is_gs_in_colour_order(mk):
    h = mk()
    lev = h.finest
    col = lev.colors
    for a, b in lev.mesh.edges:
        assert col[a] != col[b]
    rng = np.random.default_rng(1)
    b = lev.free * rng.standard_normal(lev.mesh.nv)
    x0 = lev.free * rng.standard_normal(lev.mesh.nv)
    got = mg.mc_gauss_seidel(lev, b, x0, 1)
    perm = np.lexsort((np.arange(len(col)), col))
    F = sp.diags(lev.free.astype(float))
    Lf = (F @ lev.L @ F).tocsr() + sp.diags((~lev.free).astype(float))
    Lp = Lf[perm][:, perm]
    lo = sp.tril(Lp, 0).tocsr()
    up = sp.triu(Lp, 1).tocsr()
    xp = spla.spsolve_triangular(lo, (lev.free * b)[perm] - up @ x0[perm], lower=True)
    expect = np.empty_like(xp)
    expect[perm] = xp
    assert np.allclose(got, lev.free * expect, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("mk", [lambda: _square(4, 1), lambda: _ico(3, 1)])
def test_power_iteration_bounds_lambda_max(mk):
    h = mk()
    lev = h.finest
    idx = np.flatnonzero(lev.free)
    DL = (sp.diags(1.0 / lev.diag[idx]) @ lev.L[idx][:, idx]).toarray()
    true = np.max(np.linalg.eigvals(DL).real)
    assert lev.lmax <= true * (1 + 1e-12)
    assert lev.lmax > 0.9 * true


def test_gauge_coarse_solve_is_pseudo_inverse():
    h = _ico(1, 1)
    lev = h.finest
    b = mg.prepare_rhs(h, W.uniform_field(lev.mesh.nv, 7))
    x = mg.coarse_solve(h, lev, b)
    A = lev.A.toarray()
    xp = np.linalg.pinv(A) @ (lev.star0 * b)
    assert np.allclose(x, mg.project_mean_zero(lev, xp), atol=1e-12)
    assert abs(mg.star0_mean(lev, x)) < 1e-14


def test_dirichlet_coarse_solve_single_unknown():
    # 3x3 vertices, one interior unknown: *0 = 1/4, L_ii = 4 / h^2 with h = 1/2
    h = _square(1, 1)
    lev = h.finest
    b = np.ones(lev.mesh.nv)
    x = mg.coarse_solve(h, lev, b)
    assert np.count_nonzero(x) == 1
    assert np.isclose(x[lev.free][0], 1.0 / 16.0, rtol=1e-15)


def test_unpreconditioned_flexible_cg_is_cg():
    # CG on L in the *0 inner product == CG on A x = *0 b in the Euclidean one
    h = _square(3, 1)
    lev = h.finest
    b = mg.prepare_rhs(h, W.uniform_field(lev.mesh.nv, 3))
    idx = np.flatnonzero(lev.free)
    A = lev.A[idx][:, idx]
    iters = []
    spla.cg(A, lev.star0[idx] * b[idx], rtol=1e-30, maxiter=6, callback=lambda xk: iters.append(xk.copy()))
    for k in range(1, 6):
        res = mg.pcg_solve(h, b, 0.0, k, precondition=False)
        assert np.allclose(res.x[idx], iters[k - 1], rtol=1e-9, atol=1e-12)


def test_single_level_cycle_is_direct_solve():
    h = _ico(2, 1)
    lev = h.finest
    b = mg.prepare_rhs(h, W.uniform_field(lev.mesh.nv, 4))
    x = mg.vcycle(h, b, np.zeros_like(b))
    assert np.allclose(x, mg.direct_solve(h, b), atol=1e-12)


@pytest.mark.parametrize("smoother", ["jacobi", "chebyshev", "gs", "mcgs"])
@pytest.mark.parametrize("which", ["square", "ico"])
def test_mg_and_pcg_reach_direct_solution(smoother, which):
    h = _square(5, 4, smoother=smoother) if which == "square" else _ico(3, 3, smoother=smoother)
    lev = h.finest
    b = W.uniform_field(lev.mesh.nv, 11)
    xs = mg.direct_solve(h, b)
    r1 = mg.mg_solve(h, b, 1e-10, 60)
    r2 = mg.pcg_solve(h, b, 1e-10, 60)
    for r in (r1, r2):
        assert r.rel_res <= 1e-10
        assert mg.star0_norm(lev, r.x - xs) / mg.star0_norm(lev, xs) < 1e-8
    # Jacobi: the spectral radius of the V(2,2) error propagator of this operator and these transfers is
    # 0.31 (test_jacobi_v22_factor_is_the_dense_error_propagators_spectral_radius); the others converge faster
    band = {"jacobi": 0.32, "chebyshev": 0.3, "gs": 0.2, "mcgs": 0.2}[smoother]
    assert mg.convergence_factor(r1.history) < band
    assert r2.iters <= r1.iters


def test_config1_standalone_mg_matches_closed_form():
    # unit square x5, 5-level V(2,2), Dirichlet 0, RHS -Delta of sin(pi x) sin(pi y), to 1e-10
    h = _square(5, 5)
    lev = h.finest
    assert [l.mesh.nv for l in h.levels] == [9, 25, 81, 289, 1089]
    r = mg.mg_solve(h, W.rhs_sin_square(lev.mesh.verts), 1e-10, 100)
    hh = 1.0 / 32
    lam11 = 8.0 / hh ** 2 * math.sin(math.pi * hh / 2) ** 2
    u_h = 2 * math.pi ** 2 / lam11 * W.u_sin_square(lev.mesh.verts)
    assert r.rel_res <= 1e-10
    assert mg.star0_norm(lev, r.x - u_h) / mg.star0_norm(lev, u_h) < 1e-9


def test_w_cycle_converges_faster_than_v():
    hv = _square(5, 5)
    hw = _square(5, 5, gamma=2)
    b = W.uniform_field(hv.finest.mesh.nv, 12)
    rv = mg.mg_solve(hv, b, 1e-10, 60)
    rw = mg.mg_solve(hw, b, 1e-10, 60)
    assert rw.iters <= rv.iters
    assert np.allclose(rw.x, rv.x, atol=1e-9 * np.abs(rv.x).max())


@pytest.mark.parametrize("which", ["square", "ico"])
def test_star0_restriction_is_adjoint_of_interpolation(which):
    # <R r, e>_{*0 coarse} = <r, P e>_{*0 fine}, and on a uniform interior vertex it equals the paper's R
    if which == "square":
        h = _square(4, 2, restriction="star0"); hp = _square(4, 2)
    else:
        h = _ico(3, 2, restriction="star0"); hp = _ico(3, 2)
    c, f = h.levels[0], h.levels[1]
    rng = np.random.default_rng(5)
    r = rng.standard_normal(f.mesh.nv)
    e = rng.standard_normal(c.mesh.nv)
    lhs = np.sum(c.star0 * (h.R[0] @ r) * e)
    rhs = np.sum(f.star0 * r * (h.P[0] @ e))
    assert abs(lhs - rhs) <= 1e-13 * (abs(lhs) + np.sum(np.abs(c.star0 * e)) * np.abs(r).max())
    if which == "square":
        xy = c.mesh.verts
        inner = (xy[:, 0] > 0) & (xy[:, 0] < 1) & (xy[:, 1] > 0) & (xy[:, 1] < 1)
        assert np.allclose((h.R[0] @ r)[inner], (hp.R[0] @ r)[inner], rtol=1e-13, atol=1e-14)


def test_star0_restriction_keeps_pcg_stable_on_boundary_data():
    # data concentrated next to the boundary: the paper's R gives a non-symmetric preconditioner there
    h = _square_gauge(6, 5, restriction="star0")
    lev = h.finest
    y = lev.mesh.verts[:, 1]
    b = np.where(np.abs(y - (1 - 1.0 / 64)) < 1e-12, W.uniform_field(lev.mesh.nv, 9) * 1e5, 0.0)
    r = mg.pcg_solve(h, b, 1e-10, 60)
    assert r.rel_res <= 1e-10 and r.iters < 20


def test_f_cycle_on_three_levels_is_the_w_cycle():
    # F(2) = pre, [F(1) then V(1)], post and F(1) = V(1) (its coarse correction is exact): the W-cycle,
    # up to the rounding of the W-cycle's repeated exact coarse solve
    v, t = W.unit_square()
    hf = mg.build_hierarchy(v, t, 4, 3, "dirichlet", opts=mg.MGOptions(fcycle=True))
    hw = mg.build_hierarchy(v, t, 4, 3, "dirichlet", opts=mg.MGOptions(gamma=2))
    hv = mg.build_hierarchy(v, t, 4, 3, "dirichlet")
    b = W.uniform_field(hf.finest.mesh.nv, 13)
    x0 = np.zeros_like(b)
    xf, xw, xv = mg.vcycle(hf, b, x0), mg.vcycle(hw, b, x0), mg.vcycle(hv, b, x0)
    assert np.max(np.abs(xf - xw)) <= 1e-12 * np.max(np.abs(xw))
    assert np.max(np.abs(xf - xv)) > 1e-6 * np.max(np.abs(xv))


def test_f_cycle_between_v_and_w():
    # 5 levels: F differs from V and W; its convergence lies between theirs (and it reaches the solution)
    v, t = W.unit_square()
    b = W.uniform_field(mg.build_hierarchy(v, t, 6, 1, "dirichlet").finest.mesh.nv, 14)
    res = {}
    for name, o in (("V", mg.MGOptions()), ("F", mg.MGOptions(fcycle=True)), ("W", mg.MGOptions(gamma=2))):
        h = mg.build_hierarchy(v, t, 6, 5, "dirichlet", opts=o)
        r = mg.mg_solve(h, b, 1e-10, 60)
        assert r.rel_res <= 1e-10
        res[name] = mg.convergence_factor(r.history)
    assert res["W"] <= res["F"] * 1.05 and res["F"] <= res["V"] * 1.05, res
    assert res["F"] < res["V"], res


def _dense_vcycle_propagator(n, nlev, omega, nu1, nu2):
    """V-cycle error propagator on the interior of the (n+1)^2 grid of the unit square, built from the
    textbook definitions alone (not from the oracle): the 5-point operator (4 u_i - sum of the 4 neighbours)
    / h^2 -- the DEC operator on this triangulation, whose hypotenuses carry *1 = 0 -- damped Jacobi,
    interpolation linear on the triangles (a midpoint takes the mean of its edge's ends, the diagonal edges
    running (i,j)-(i+1,j+1)), restriction the row-normalized transpose of that map, the operator
    rediscretized on every level and an exact solve on the coarsest:
    E_l = S^nu2 (I - P (I - E_{l-1}) A_{l-1}^-1 R A_l) S^nu1."""
    m = n - 1
    A = np.zeros((m * m, m * m))
    for j in range(1, n):
        for i in range(1, n):
            k = (j - 1) * m + (i - 1)
            A[k, k] = 4.0 * n * n
            for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                if 1 <= i + di <= n - 1 and 1 <= j + dj <= n - 1:
                    A[k, (j + dj - 1) * m + (i + di - 1)] = -1.0 * n * n
    if nlev == 1:
        return np.zeros_like(A)
    nc = n // 2 + 1
    M = np.zeros((nc * nc, (n + 1) * (n + 1)))
    for j in range(n + 1):
        for i in range(n + 1):
            if i % 2 == 0 and j % 2 == 0:
                par = [(i // 2, j // 2, 1.0)]
            elif j % 2 == 0:
                par = [((i - 1) // 2, j // 2, 0.5), ((i + 1) // 2, j // 2, 0.5)]
            elif i % 2 == 0:
                par = [(i // 2, (j - 1) // 2, 0.5), (i // 2, (j + 1) // 2, 0.5)]
            else:
                par = [((i - 1) // 2, (j - 1) // 2, 0.5), ((i + 1) // 2, (j + 1) // 2, 0.5)]
            for I, J, w in par:
                M[J * nc + I, j * (n + 1) + i] = w
    R = M / M.sum(axis=1, keepdims=True)
    ic = [J * nc + I for J in range(1, nc - 1) for I in range(1, nc - 1)]
    jf = [j * (n + 1) + i for j in range(1, n) for i in range(1, n)]
    P, R = M[np.ix_(ic, jf)].T, R[np.ix_(ic, jf)]
    Ec = _dense_vcycle_propagator(n // 2, nlev - 1, omega, nu1, nu2)
    mc = n // 2 - 1
    Ac = np.zeros((mc * mc, mc * mc))
    nn = n // 2
    for j in range(1, nn):
        for i in range(1, nn):
            k = (j - 1) * mc + (i - 1)
            Ac[k, k] = 4.0 * nn * nn
            for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                if 1 <= i + di <= nn - 1 and 1 <= j + dj <= nn - 1:
                    Ac[k, (j + dj - 1) * mc + (i + di - 1)] = -1.0 * nn * nn
    S = np.eye(m * m) - omega * A / (4.0 * n * n)
    C = np.eye(m * m) - P @ (np.eye(mc * mc) - Ec) @ np.linalg.solve(Ac, R @ A)
    return np.linalg.matrix_power(S, nu2) @ C @ np.linalg.matrix_power(S, nu1)


def test_jacobi_v22_factor_is_the_dense_error_propagators_spectral_radius():
    # The paper's transfers with damped Jacobi (omega = 2/3) V(2,2) on config 1's 5 levels: the asymptotic
    # residual reduction per cycle is the spectral radius of the cycle's error propagator, 0.307 here (the
    # smoothing factor alone, (2/3)^4 = 0.198, ignores the coarse-grid correction's own error)
    E = _dense_vcycle_propagator(32, 5, 2.0 / 3.0, 2, 2)
    rho = float(max(abs(np.linalg.eigvals(E))))
    assert 0.30 < rho < 0.31
    h = _square(5, 5)
    r = mg.mg_solve(h, W.uniform_field(h.finest.mesh.nv, 13), 1e-13, 100)
    assert r.iters >= 21
    fac = (r.history[20] / r.history[15]) ** 0.2  # asymptotic rate: cycles 16-20, past the fast start
    assert abs(fac - rho) < 0.02, (fac, rho)

