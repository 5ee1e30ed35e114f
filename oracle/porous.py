"""One explicit porous-convection step in the DEC, its rollout and its adjoint.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Sec. 3.2.1 (the Darcy law, divergence-free flux and heat equation in the
exterior calculus, and the Decapode diagram) with the constants of Sec. 3.2.2.
Readings (the paper leaves the discrete operators implicit):
  * buoyancy 1-form: w = alpha rho0 (g^flat wedge T), with the primal 0-1
    wedge (g^flat wedge T)_e = g^flat_e (T_lo + T_hi)/2 and g^flat_e =
    g . (x_hi - x_lo) exact for constant g; alpha rho0 = 1/|g|.  Writing the
    potential pot_v = alpha rho0 g . x_v gives w_e = (pot_hi - pot_lo)(T_lo + T_hi)/2;
  * pressure: Delta P = delta w with Delta = -L and delta = -*0^-1 d0^T *1,
    i.e. L P = *0^-1 d0^T *1 w, a pure-Neumann (constant-nullspace) problem;
  * Darcy flux q = -(k/eta)(d0 P - w);
  * Lie derivative (Sec. 3.2.1, computed as *0^-1((*1 d0 T) wedge q)):
    (L_q T)_v = (1/*0_v) sum_{e containing v} (1/2) *1_e (d0 T)_e q_e;
  * heat equation dT/dt = -(1/phi) L_q T + kappa Delta T = -(1/phi) L_q T - kappa L T,
    with the bc mask setting dT/dt = 0 on the top and bottom rows;
  * kappa = (1/Ra) g alpha rho0 k_eta dT y_max / phi (Sec. 3.2.2);
  * time stepping: forward Euler with a fixed dt here; the paper's adaptive
    Tsit5 integration of the same right-hand side (tdot_fn) is oracle/rk.py.
The adjoint restates reverse-mode differentiation of that step; its
derivation is in the docstring of `step_adjoint`.  Parity beyond the pins in
tests/test_oracle_porous.py (conductive equilibrium, linear-field Lie
derivative, finite differences) is unpinned by the paper.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .mesh import d0_matrix
from .multigrid import direct_solve


@dataclass
class PorousParams:
    Ra: float = 1000.0
    phi: float = 0.1
    k_eta: float = 1.0
    dT: float = 200.0
    g: tuple = (0.0, -9.81)
    y_max: float = 1.0
    dt: float = 0.0

    @property
    def g_norm(self):
        return float(np.sqrt(np.sum(np.square(self.g))))

    @property
    def alpha_rho0(self):
        return 1.0 / self.g_norm

    @property
    def kappa(self):
        return (1.0 / self.Ra) * self.g_norm * self.alpha_rho0 * self.k_eta * self.dT * self.y_max / self.phi


def potential(verts, prm):
    """pot_v = alpha rho0 g . x_v, so that g^flat_e alpha rho0 = pot_hi - pot_lo."""
    g = np.asarray(prm.g, dtype=np.float64)
    return prm.alpha_rho0 * (verts[:, : len(g)] @ g)


def buoyancy(lev, T, pot):
    """w_e = (pot_hi - pot_lo) (T_lo + T_hi) / 2 on every edge."""
    lo, hi = lev.mesh.edges[:, 0], lev.mesh.edges[:, 1]
    return (pot[hi] - pot[lo]) * 0.5 * (T[lo] + T[hi])


def pressure_rhs(lev, T, pot):
    """*0^-1 d0^T *1 w."""
    d0 = d0_matrix(lev.mesh).astype(np.float64)
    return (d0.T @ (lev.star1 * buoyancy(lev, T, pot))) / lev.star0


def darcy_flux(lev, P, T, pot, prm):
    d0 = d0_matrix(lev.mesh).astype(np.float64)
    return -prm.k_eta * (d0 @ P - buoyancy(lev, T, pot))


def lie_derivative(lev, T, q):
    """(L_q T)_v = (1/*0_v) sum_{e ni v} (1/2) *1_e (d0 T)_e q_e."""
    d0 = d0_matrix(lev.mesh).astype(np.float64)
    a = 0.5 * lev.star1 * (d0 @ T) * q
    s = np.zeros(lev.mesh.nv)
    np.add.at(s, lev.mesh.edges[:, 0], a)
    np.add.at(s, lev.mesh.edges[:, 1], a)
    return s / lev.star0


def tdot(lev, T, P, pot, fixed, prm):
    q = darcy_flux(lev, P, T, pot, prm)
    rate = -(1.0 / prm.phi) * lie_derivative(lev, T, q) - prm.kappa * (lev.L @ T)
    return np.where(fixed, 0.0, rate)


class _One:
    def __init__(self, lev):
        self.levels = [lev]
        self.bc = "gauge"

    @property
    def finest(self):
        return self.levels[-1]


def solve_pressure(lev, rhs):
    """*0-mean-zero solution of the pure-Neumann pressure problem (direct solve)."""
    return direct_solve(_One(lev), rhs)


def tdot_fn(lev, pot, fixed, prm):
    """f(T) = dT/dt of the method of lines (Sec. 3.2.1), the pressure solved directly:
    the right-hand side the adaptive integrator (oracle/rk.py) advances."""
    def f(T):
        P = solve_pressure(lev, pressure_rhs(lev, T, pot))
        return tdot(lev, T, P, pot, fixed, prm)
    return f


def step(lev, T, pot, fixed, prm):
    """One forward-Euler step; returns (T_next, P)."""
    P = solve_pressure(lev, pressure_rhs(lev, T, pot))
    return T + prm.dt * tdot(lev, T, P, pot, fixed, prm), P


def rollout(lev, T0, pot, fixed, prm, nsteps):
    T = T0.copy()
    traj = [T]
    for _ in range(nsteps):
        T, _ = step(lev, T, pot, fixed, prm)
        traj.append(T)
    return traj


def top_flux(lev, T, top, prm):
    """F = -kappa sum_{v on the top row} (A T)_v with A = d0^T *1 d0."""
    return -prm.kappa * np.sum((lev.A @ T)[top])


def top_flux_grad(lev, top, prm):
    """dF/dT = -kappa A 1_top."""
    return -prm.kappa * (lev.A @ top.astype(np.float64))


def step_adjoint(lev, T, pot, fixed, prm, lam):
    """lam_n = (dT_{n+1}/dT_n)^T lam_{n+1} for T_{n+1} = T_n + dt mask(tdot(T_n, P(T_n))).

    With mu = dt * mask * lam (the sensitivity of tdot) the pieces are
      diffusion:  -kappa L^T mu, where L^T mu = *0 L (mu / *0);
      advection:  tdot_v contains -(1/(phi *0_v)) sum_{e ni v} a_e with the
                  orientation-free a_e = (1/2) *1_e (T_u - T_v) q_{v->u};
                  so each edge gets abar_e = nu_lo + nu_hi, nu = -mu/(phi *0),
                  and passes abar_e da_e/dT and abar_e da_e/dP to its ends;
      pressure:   P = solve(rhs(T)) gives rhs_bar = *0 m with L m = *0^-1 P_bar
                  (gauge, as for the Poisson adjoint), and
                  sum_v rhs_bar_v rhs_v = sum_e *1_e w_e (d0 m)_e, so
                  T_bar_v += sum_{e ni v} *1_e (d0 m)_e (pot_hi - pot_lo)/2.
    """
    P = solve_pressure(lev, pressure_rhs(lev, T, pot))
    q = darcy_flux(lev, P, T, pot, prm)
    mu = prm.dt * np.where(fixed, 0.0, lam)
    out = lam - prm.kappa * (lev.star0 * (lev.L @ (mu / lev.star0)))
    lo, hi = lev.mesh.edges[:, 0], lev.mesh.edges[:, 1]
    nu = -mu / (prm.phi * lev.star0)
    abar = nu[lo] + nu[hi]
    dT = T[hi] - T[lo]
    dpot = pot[hi] - pot[lo]
    s1 = lev.star1
    k = prm.k_eta
    # a_e = 1/2 *1 dT q, q = -k (P_hi - P_lo) + k dpot (T_lo + T_hi)/2 (oriented lo -> hi)
    da_dThi = 0.5 * s1 * (q + dT * k * dpot * 0.5)
    da_dTlo = 0.5 * s1 * (-q + dT * k * dpot * 0.5)
    da_dPhi = 0.5 * s1 * dT * (-k)
    da_dPlo = 0.5 * s1 * dT * k
    np.add.at(out, hi, abar * da_dThi)
    np.add.at(out, lo, abar * da_dTlo)
    Pbar = np.zeros(lev.mesh.nv)
    np.add.at(Pbar, hi, abar * da_dPhi)
    np.add.at(Pbar, lo, abar * da_dPlo)
    m = solve_pressure(lev, Pbar / lev.star0)
    dm = m[hi] - m[lo]
    c = s1 * dm * dpot * 0.5
    np.add.at(out, lo, c)
    np.add.at(out, hi, c)
    return out


def rollout_adjoint(lev, T0, pot, fixed, prm, nsteps, lam_final):
    """dF/dT_0 given dF/dT_N, by storing the trajectory and stepping back."""
    traj = rollout(lev, T0, pot, fixed, prm, nsteps)
    lam = lam_final.copy()
    for n in range(nsteps - 1, -1, -1):
        lam = step_adjoint(lev, traj[n], pot, fixed, prm, lam)
    return lam
