"""Adjoint of the Poisson solve: gradients with respect to b and to *1.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper has no adjoint; this restates the derivative of u = L^-1 b for
L = *0^-1 d0^T *1 d0 (Sec. 3.1.1, Eq. hodge0-laplacian).  Write A = d0^T *1 d0.

Dirichlet (unknowns = free vertices f): A_ff u_f = *0_f b_f, so for a loss
J(u) with g = dJ/du,
    dJ/db_f = *0_f A_ff^-1 g_f = *0_f mu_f   with   L_ff mu_f = *0_f^-1 g_f,
and dA = d0^T diag(d*1) d0 gives dJ = -mu^T dA u, i.e.
    dJ/d*1_e = -(d0 mu)_e (d0 u)_e        (mu, u zero on Dirichlet vertices).
Gauge (constants are the nullspace, m = *0): u solves (A + m m^T/S) u = Q b
with Q = diag(m) - m m^T / S, S = sum(m).  Then dJ/db = Q K^-1 g = *0 P(K^-1 g)
where P removes the *0-weighted mean, and P(K^-1 g) is exactly the
*0-mean-zero solution mu of L mu = *0^-1 g after that right-hand side is
itself projected to *0-mean zero.  The *1 derivative is the same edge formula
because d0 kills the constant part of K^-1 g.
So in both cases: mu = solve(*0^-1 g), dJ/db = *0 mu, dJ/d*1 = -(d0 mu)(d0 u).
"""
from __future__ import annotations

import numpy as np

from . import dec
from .mesh import d0_matrix
from .multigrid import Level, direct_solve, make_level


def level_with_star1(mesh, bc, star1):
    """A finest level whose operator uses the given *1 (per edge) instead of the geometric one."""
    lev = make_level(mesh, bc)
    lev.star1 = np.asarray(star1, dtype=np.float64)
    lev.A = dec.stiffness(mesh, lev.star1)
    lev.L = dec.laplacian(mesh, lev.star0, lev.star1)
    lev.diag = lev.L.diagonal() * lev.free
    return lev


class _One:
    """Minimal stand-in hierarchy (one level, direct solves) for the adjoint formulas."""

    def __init__(self, lev, bc):
        self.levels = [lev]
        self.bc = bc

    @property
    def finest(self):
        return self.levels[-1]


def solve(lev, bc, b):
    return direct_solve(_One(lev, bc), b)


def loss_star0(lev, u, u_target):
    """J = 1/2 (u - u_t)^T *0 (u - u_t) over the free vertices, and dJ/du."""
    d = (u - u_target) * lev.free
    return 0.5 * np.sum(lev.star0 * d * d), lev.star0 * d


def gradients(lev, bc, u, grad_u):
    """(dJ/db, dJ/d*1) from u = L^-1 b and g = dJ/du, by one adjoint solve."""
    mu = solve(lev, bc, grad_u / lev.star0)
    d0 = d0_matrix(lev.mesh).astype(np.float64)
    grad_b = lev.star0 * mu * lev.free
    grad_s1 = -(d0 @ mu) * (d0 @ u)
    return grad_b, grad_s1
