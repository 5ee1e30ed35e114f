"""Pins of the oracle's adaptive Runge-Kutta integrator (oracle/rk.py, the Tsit5
method of Sec. 3.2.2) against Butcher's order conditions, convergence rates,
tolerance proportionality and exact fixed points."""
import itertools
import math

import numpy as np
import pytest

import workloads as W
from oracle import multigrid as omg, porous as por, rk


def _trees(order):
    """Rooted trees up to `order` as nested tuples of children (Butcher): a tree is the
    tuple of its root's subtrees, sorted so each unlabelled tree appears once."""
    by_order = {1: [()]}
    for n in range(2, order + 1):
        out = set()
        # the children of the root form a multiset of trees whose orders sum to n - 1
        def parts(rem, maxo, acc):
            if rem == 0:
                out.add(tuple(sorted(acc)))
                return
            for o in range(min(rem, maxo), 0, -1):
                for t in by_order[o]:
                    parts(rem - o, o, acc + [t])
        parts(n - 1, n - 1, [])
        by_order[n] = sorted(out)
    return by_order


def _order(t):
    return 1 + sum(_order(c) for c in t)


def _density(t):
    return _order(t) * math.prod(_density(c) for c in t)


def _phi(t, A):
    """Stage vector of the elementary weight: Phi_i(t) = prod over children c of sum_j a_ij Phi_j(c)."""
    v = np.ones(A.shape[0])
    for c in t:
        v = v * (A @ _phi(c, A))
    return v


def _residuals(w, A, order):
    trees = _trees(order)
    return [w @ _phi(t, A) - 1.0 / _density(t) for o in range(1, order + 1) for t in trees[o]]


def test_tree_counts():
    # 1, 1, 2, 4, 9 rooted trees of orders 1..5: 17 conditions for order 5, 8 for order 4
    tr = _trees(5)
    assert [len(tr[o]) for o in range(1, 6)] == [1, 1, 2, 4, 9]


def test_tableau_satisfies_the_order_conditions():
    assert np.max(np.abs(rk.A.sum(axis=1) - rk.C)) < 1e-15       # row-sum (node) condition
    assert np.allclose(rk.B, rk.A[6], rtol=0, atol=0) and rk.C[6] == 1.0  # first same as last
    r5 = _residuals(rk.B, rk.A, 5)
    # the published decimals (entries up to 13 in size) round near 1e-16: residuals stay near 1e-14,
    # while a wrong digit anywhere above the 13th place shows
    assert len(r5) == 17 and max(abs(x) for x in r5) < 1e-13
    bhat = rk.B - rk.E
    assert max(abs(x) for x in _residuals(bhat, rk.A, 4)) < 1e-13
    # the embedded solution is genuinely of order 4: some order-5 condition fails
    assert max(abs(x) for x in _residuals(bhat, rk.A, 5)) > 1e-4


def _osc(y):
    return np.array([y[1], -y[0]])


def test_fifth_order_global_convergence():
    y0 = np.array([1.0, 0.0])
    errs = []
    for n in (10, 20, 40):
        y, st = rk.integrate(_osc, y0, 2.0, 2.0 / n, 1.0, 1.0, fixed_step=True)
        assert st.naccept == n and st.nfev == 1 + 6 * n
        errs.append(np.max(np.abs(y - np.array([math.cos(2.0), -math.sin(2.0)]))))
    for e1, e2 in zip(errs, errs[1:]):
        assert 26.0 < e1 / e2 < 38.0  # 2^5 = 32


def test_error_estimate_is_fifth_power_of_dt():
    y0 = np.array([1.0, 0.0])
    est = []
    for dt in (0.2, 0.1, 0.05):
        _, _, err = rk.step(_osc, y0, _osc(y0), dt)
        est.append(np.max(np.abs(err)))
    for e1, e2 in zip(est, est[1:]):
        assert 26.0 < e1 / e2 < 38.0


def test_adaptive_error_follows_the_tolerance():
    y0 = np.array([1.0, 0.0])
    exact = np.array([math.cos(10.0), -math.sin(10.0)])
    errs, steps = [], []
    for tol in (1e-5, 1e-7, 1e-9):
        y, st = rk.integrate(_osc, y0, 10.0, 0.01, tol, tol)
        assert st.t == 10.0
        errs.append(np.max(np.abs(y - exact)))
        steps.append(st.naccept)
    assert errs[0] > 30 * errs[1] > 900 * errs[2] and errs[2] < 1e-7
    assert steps[0] < steps[1] < steps[2]


def test_fixed_point_is_kept_exactly():
    y0 = np.array([2.0, -3.0])
    y, st = rk.integrate(lambda y: np.zeros_like(y), y0, 5.0, 1e-3, 1e-9, 1e-9)
    assert np.array_equal(y, y0) and st.nreject == 0
    assert st.naccept <= 6  # the step grows tenfold each time from 1e-3 to the end


def _square(nsub):
    v, t = W.unit_square()
    lev = omg.build_hierarchy(v, t, nsub, 1, "gauge").finest
    y = lev.mesh.verts[:, 1]
    return lev, (y == 0.0) | (y == 1.0)


def test_porous_conductive_equilibrium_stays():
    lev, fixed = _square(3)
    prm = por.PorousParams()
    pot = por.potential(lev.mesh.verts, prm)
    T0 = 100.0 - 200.0 * lev.mesh.verts[:, 1]
    T, st = rk.integrate(por.tdot_fn(lev, pot, fixed, prm), T0, 0.01, 1e-5, 1e-9, 1e-6)
    assert np.max(np.abs(T - T0)) < 1e-9 * 100.0 and st.nreject == 0


def test_porous_adaptive_matches_fine_fixed_steps():
    # the paper's initial state (Gaussian, walls at -100 / +100) on the unit square x3
    lev, fixed = _square(3)
    prm = por.PorousParams()
    xy = lev.mesh.verts
    pot = por.potential(xy, prm)
    T0 = W.gaussian_initial_T(xy, (0.5, 0.5))
    T0 = np.where(xy[:, 1] == 1.0, -100.0, np.where(xy[:, 1] == 0.0, 100.0, T0))
    f = por.tdot_fn(lev, pot, fixed, prm)
    t_end = 2e-3
    Ta, sta = rk.integrate(f, T0, t_end, 1e-5, 1e-8, 1e-8)
    Tr, _ = rk.integrate(f, T0, t_end, t_end / 400, 1.0, 1.0, fixed_step=True)
    assert sta.t == t_end and sta.naccept > 3
    assert np.max(np.abs(Ta - Tr)) < 1e-5 * np.max(np.abs(T0))
    assert np.array_equal(Ta[fixed], T0[fixed])


def test_porous_adaptive_matches_an_independent_integrator():
    # the same porous right-hand side integrated by SciPy's DOP853 (Dormand-Prince 8(5,3)) at a
    # tolerance far below ours: the oracle's Tsit5 result agrees to its own tolerance
    integrate = pytest.importorskip("scipy.integrate")
    lev, fixed = _square(3)
    prm = por.PorousParams()
    xy = lev.mesh.verts
    pot = por.potential(xy, prm)
    T0 = W.gaussian_initial_T(xy, (0.5, 0.5))
    T0 = np.where(xy[:, 1] == 1.0, -100.0, np.where(xy[:, 1] == 0.0, 100.0, T0))
    f = por.tdot_fn(lev, pot, fixed, prm)
    t_end = 2e-3
    ref = integrate.solve_ivp(lambda t, y: f(y), (0.0, t_end), T0, method="DOP853", rtol=1e-12, atol=1e-10)
    assert ref.success
    for tol, bound in ((1e-6, 1e-4), (1e-9, 1e-7)):
        T, st = rk.integrate(f, T0, t_end, 1e-5, tol, tol)
        err = np.max(np.abs(T - ref.y[:, -1]))
        assert err < bound * np.max(np.abs(T0)), (tol, err)
