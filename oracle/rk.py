"""Adaptive explicit Runge-Kutta time stepping: Tsitouras' 5(4) pair.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper integrates its porous-convection model with the adaptive explicit
"Tsit5" method (Sec. 3.2.2, relative tolerance 1e-9).  That is the embedded
Runge-Kutta pair of orders 5 and 4 published by Ch. Tsitouras, "Runge-Kutta
pairs of order 5(4) satisfying only the first column simplifying assumption",
Computers & Mathematics with Applications 62 (2011) 770-775.  Seven stages;
the last stage is evaluated at the new state and is the next step's first
stage (first same as last), so an accepted step costs six new evaluations.

Readings (the paper names the method and its relative tolerance only):
  * error norm: the root mean square over all components of
    err_i / (atol + rtol max(|y_i|, |y_new_i|)), err = dt sum_j E_j k_j
    (Hairer, Norsett & Wanner, Solving ODEs I, Sec. II.4);
  * step-size control: the integral controller of the same section,
    dt <- dt min(facmax, max(facmin, fac * en^(-1/5))) with fac = 0.9,
    facmin = 0.2, facmax = 10 (after a rejection facmax = 1); a step is
    accepted when en <= 1;
  * the last step is shortened (or lengthened by less than 1e-12 t_end) to
    end exactly at t_end, so rounding in the accumulated time adds no step.
Pins: tests/test_oracle_rk.py (the Butcher order conditions of both weight
vectors, fifth-order convergence, fourth-order local error estimate,
tolerance proportionality, an exact fixed point, and the porous model
integrated by an independent library integrator at a far tighter tolerance).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# nodes, coupling matrix (strictly lower), weights of the 5th-order solution
# (the last row of A: first same as last) and error weights E = b - b_hat
C = np.array([0.0, 0.161, 0.327, 0.9, 0.9800255409045097, 1.0, 1.0])
A = np.zeros((7, 7))
A[1, 0] = 0.161
A[2, :2] = [-0.008480655492356989, 0.335480655492357]
A[3, :3] = [2.897153057105493, -6.359448489975075, 4.3622954328695815]
A[4, :4] = [5.325864828439257, -11.748883564062828, 7.4955393428898365, -0.09249506636175525]
A[5, :5] = [5.86145544294642, -12.92096931784711, 8.159367898576159, -0.071584973281401, -0.028269050394068383]
A[6, :6] = [0.09646076681806523, 0.01, 0.4798896504144996, 1.379008574103742, -3.290069515436081, 2.324710524099774]
B = A[6].copy()
E = np.array([-0.00178001105222577714, -0.0008164344596567469, 0.007880878010261995, -0.1447110071732629,
              0.5823571654525552, -0.45808210592918697, 1.0 / 66.0])

FAC, FACMIN, FACMAX = 0.9, 0.2, 10.0


def step(f, y, k1, dt):
    """One step from y with k1 = f(y): returns (y_new, k7 = f(y_new), err = dt sum_j E_j k_j)."""
    k = [k1]
    for i in range(1, 7):
        yi = y + dt * sum(A[i, j] * k[j] for j in range(i))
        k.append(f(yi))
    y_new = y + dt * sum(B[j] * k[j] for j in range(7))
    err = dt * sum(E[j] * k[j] for j in range(7))
    return y_new, k[6], err


def error_norm(err, y, y_new, rtol, atol):
    sc = atol + rtol * np.maximum(np.abs(y), np.abs(y_new))
    return float(np.sqrt(np.mean(np.square(err / sc))))


@dataclass
class RKStats:
    naccept: int = 0
    nreject: int = 0
    nfev: int = 0
    t: float = 0.0
    dt: float = 0.0
    dts: list = field(default_factory=list)


def integrate(f, y0, t_end, dt0, rtol, atol, max_steps=1_000_000, fixed_step=False):
    """Integrate y' = f(y) from t = 0 to t_end.  fixed_step: dt0 every step, no error control."""
    y = np.array(y0, dtype=np.float64, copy=True)
    k1 = f(y)
    st = RKStats(nfev=1)
    t, dt = 0.0, float(dt0)
    rejected_last = False
    slack = 1e-12 * t_end
    while t < t_end and st.naccept + st.nreject < max_steps:
        last = dt >= t_end - t - slack
        h = t_end - t if last else dt
        y_new, k7, err = step(f, y, k1, h)
        st.nfev += 6
        en = error_norm(err, y, y_new, rtol, atol)
        if fixed_step or en <= 1.0:
            t = t_end if last else t + h
            y, k1 = y_new, k7
            st.naccept += 1
            st.dts.append(h)
            if fixed_step:
                continue
            grow = FACMAX if not rejected_last else 1.0
            dt = h * (grow if en == 0.0 else min(grow, max(FACMIN, FAC * en ** -0.2)))
            rejected_last = False
        else:
            st.nreject += 1
            dt = h * max(FACMIN, FAC * en ** -0.2)
            rejected_last = True
    st.t, st.dt = t, dt
    return y, st
