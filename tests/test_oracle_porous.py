"""Pins of the oracle's porous-convection step (Sec. 3.2) and its adjoint."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import multigrid as omg, porous as por


def _level(nsub):
    v, t = W.unit_square()
    h = omg.build_hierarchy(v, t, nsub, 1, "gauge")
    lev = h.finest
    y = lev.mesh.verts[:, 1]
    fixed = (y == 0.0) | (y == 1.0)
    return lev, fixed


def test_constants_of_sec322():
    prm = por.PorousParams()
    assert prm.alpha_rho0 * prm.g_norm == pytest.approx(1.0)
    # (1/Ra) g (1/g) k dT y_max / phi = 200 / (1000 * 0.1)
    assert prm.kappa == pytest.approx(2.0, rel=1e-15)
    # the paper's initial Gaussian peaks at about 127 (400 / (2 pi * 1/2))
    xy = np.array([[0.0, 0.0]])
    assert W.gaussian_initial_T(xy, (0.0, 0.0))[0] == pytest.approx(400.0 / math.pi, rel=1e-14)


def test_conductive_profile_is_a_discrete_equilibrium():
    lev, fixed = _level(4)
    prm = por.PorousParams()
    xy = lev.mesh.verts
    pot = por.potential(xy, prm)
    assert np.allclose(pot, -xy[:, 1], rtol=0, atol=1e-15)
    T = 100.0 - 200.0 * xy[:, 1]
    # w is the exact gradient of Phi = 100 (y^2 - y), so P = Phi + c and q = 0
    P = por.solve_pressure(lev, por.pressure_rhs(lev, T, pot))
    Phi = omg.project_mean_zero(lev, 100.0 * (xy[:, 1] ** 2 - xy[:, 1]))
    assert np.max(np.abs(P - Phi)) < 1e-10 * np.max(np.abs(Phi))
    q = por.darcy_flux(lev, P, T, pot, prm)
    assert np.max(np.abs(q)) < 1e-10
    rate = por.tdot(lev, T, P, pot, fixed, prm)
    scale = prm.kappa * np.max(np.abs(lev.L.diagonal())) * 100.0
    assert np.max(np.abs(rate)) < 1e-12 * scale


def test_lie_derivative_of_linear_field_is_q_dot_grad():
    lev, fixed = _level(3)
    xy = lev.mesh.verts
    T = 3.0 * xy[:, 0] - 2.0 * xy[:, 1] + 1.0
    qv = np.array([0.7, -0.4])
    lo, hi = lev.mesh.edges[:, 0], lev.mesh.edges[:, 1]
    q = (xy[hi] - xy[lo]) @ qv
    lq = por.lie_derivative(lev, T, q)
    inner = (xy[:, 0] > 0) & (xy[:, 0] < 1) & (xy[:, 1] > 0) & (xy[:, 1] < 1)
    assert np.allclose(lq[inner], 0.7 * 3.0 + (-0.4) * (-2.0), rtol=1e-13)


def test_rollout_adjoint_matches_central_differences():
    lev, fixed = _level(3)
    prm = por.PorousParams()
    h = 1.0 / 8
    prm.dt = 0.5 * h * h / (4 * prm.kappa)
    xy = lev.mesh.verts
    pot = por.potential(xy, prm)
    T0 = 100.0 - 200.0 * xy[:, 1] + 5.0 * W.uniform_field(lev.mesh.nv, 0) * ~fixed
    top = xy[:, 1] == 1.0
    nsteps = 4
    lam_N = por.top_flux_grad(lev, top, prm)
    lam_0 = por.rollout_adjoint(lev, T0, pot, fixed, prm, nsteps, lam_N)

    def F(T):
        return por.top_flux(lev, por.rollout(lev, T, pot, fixed, prm, nsteps)[-1], top, prm)

    rng = np.random.default_rng(2)
    for _ in range(3):
        d = rng.standard_normal(lev.mesh.nv)
        eps = 1e-4
        fd = (F(T0 + eps * d) - F(T0 - eps * d)) / (2 * eps)
        an = lam_0 @ d
        assert abs(fd - an) <= 1e-6 * abs(an), (fd, an)
    # the advection term is active: the flux is not just the diffusive response
    T1, P = por.step(lev, T0, pot, fixed, prm)
    assert np.max(np.abs(por.darcy_flux(lev, P, T0, pot, prm))) > 1e-3
