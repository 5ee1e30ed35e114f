"""GPU porous convection (Sec. 3.2): steps and the checkpointed adjoint against the oracle.

Pressure solves run in FP64 to tol 1e-12 (the oracle solves them directly),
so a trajectory of a few steps agrees to ~1e-10 relative; the bound used is
1e-8.  The full-size run follows the porous-convection workload: unit square
x9 (263,169 vertices), T0 = 100 - 200 y + 1e-3 U[-1,1] (seed 0), 2000 steps,
dt = h^2 / (8 kappa) with h = 1/512, checkpoints every 100 steps, gradient of
the top-boundary heat flux with respect to T0 checked by central differences.
"""
import numpy as np
import pytest

import workloads as W
from oracle import multigrid as omg, porous as por

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _setup(nsub, nlevels):
    # the adjoint pressure right-hand sides sit next to the top boundary, where the paper's
    # row-normalized restriction makes the V-cycle preconditioner far from symmetric; the
    # *0-adjoint restriction keeps MG-PCG convergent there
    import paper_2508_12501_gb300 as P
    v, t = W.unit_square()
    h = P.Hierarchy(P.Mesh(v, t), nsub, nlevels, bc="gauge", restriction="star0")
    xy = h.table(-1, "verts")
    fixed = (xy[:, 1] == 0.0) | (xy[:, 1] == 1.0)
    return h, xy, fixed


def _oracle_level(nsub):
    v, t = W.unit_square()
    return omg.build_hierarchy(v, t, nsub, 1, "gauge").finest


def test_steps_match_oracle():
    nsub = 4
    h, xy, fixed = _setup(nsub, 3)
    lev = _oracle_level(nsub)
    prm = por.PorousParams()
    hh = 1.0 / 2 ** nsub
    prm.dt = hh * hh / (8 * prm.kappa)
    T0 = 100.0 - 200.0 * xy[:, 1] + 5.0 * W.uniform_field(len(xy), 0) * ~fixed
    pot = por.potential(xy, prm)
    ref = por.rollout(lev, T0, pot, fixed, prm, 10)[-1]
    T = torch.as_tensor(T0, device="cuda")
    P = torch.zeros_like(T)
    fx = torch.as_tensor(fixed.astype(np.uint8), device="cuda")
    st = h.porous_step(T, P, fx, 10, prm.dt, tol=1e-12, mode="f64", maxit=200)
    assert st.rel_res <= 1e-12
    got = T.cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 1e-8 * np.max(np.abs(ref))
    assert np.array_equal(got[fixed], T0[fixed])
    assert np.max(np.abs(got - T0)) > 1e-3  # the state did move


def test_conductive_state_stays_put():
    h, xy, fixed = _setup(5, 4)
    T0 = 100.0 - 200.0 * xy[:, 1]
    T = torch.as_tensor(T0, device="cuda")
    P = torch.zeros_like(T)
    fx = torch.as_tensor(fixed.astype(np.uint8), device="cuda")
    dt = (1.0 / 32) ** 2 / 16
    h.porous_step(T, P, fx, 20, dt, tol=1e-11, mode="mixed")
    assert np.max(np.abs(T.cpu().numpy() - T0)) < 1e-7 * 100.0


def test_adjoint_matches_oracle():
    nsub = 4
    h, xy, fixed = _setup(nsub, 3)
    lev = _oracle_level(nsub)
    prm = por.PorousParams()
    hh = 1.0 / 2 ** nsub
    prm.dt = hh * hh / (8 * prm.kappa)
    pot = por.potential(xy, prm)
    T0 = 100.0 - 200.0 * xy[:, 1] + 5.0 * W.uniform_field(len(xy), 1) * ~fixed
    top = xy[:, 1] == 1.0
    lamN = por.top_flux_grad(lev, top, prm)
    ref = por.rollout_adjoint(lev, T0, pot, fixed, prm, 7, lamN)
    fx = torch.as_tensor(fixed.astype(np.uint8), device="cuda")
    Tt = torch.as_tensor(T0, device="cuda")
    g, st = h.porous_backward(Tt, torch.zeros_like(Tt), fx, 7, torch.as_tensor(lamN, device="cuda"), prm.dt,
                              ckpt_every=3, tol=1e-12, mode="f64", maxit=200)
    got = g.cpu().numpy()
    assert np.linalg.norm(got - ref) <= 1e-8 * np.linalg.norm(ref)


def test_full_size_rollout_and_flux_gradient():
    nsub = 9
    h, xy, fixed = _setup(nsub, 7)
    n = h.n
    assert n == 263169
    kappa = 2.0
    dt = 0.5 * (1.0 / 512) ** 2 / (4 * kappa)
    T0 = torch.as_tensor(W.porous_initial_T(xy, 0), device="cuda")
    fx = torch.as_tensor(fixed.astype(np.uint8), device="cuda")
    top = torch.as_tensor(xy[:, 1] == 1.0, device="cuda").double()
    s0 = torch.as_tensor(h.table(-1, "star0"), device="cuda")
    # dF/dT for F = -kappa sum_top (A T)_v = -kappa 1_top^T *0 L T  ->  -kappa L^T (*0 1_top) = -kappa *0 L 1_top
    gradF = -kappa * s0 * h.laplace0_apply(top)
    nsteps, ce = 2000, 100
    ck = torch.empty((nsteps // ce + 1) * n, dtype=torch.float64, device="cuda")
    T = T0.clone()
    P = torch.zeros_like(T)
    st = h.porous_step(T, P, fx, nsteps, dt, checkpoints=ck, ckpt_every=ce, tol=1e-12, mode="f64", maxit=200)
    assert torch.isfinite(T).all() and st.rel_res <= 1e-12
    assert torch.equal(ck[:n], T0) and torch.equal(ck[-n:], T)
    assert torch.equal(T[fx.bool()], T0[fx.bool()])

    def F(Tinit):
        Tr = Tinit.clone()
        Pr = torch.zeros_like(Tr)
        h.porous_step(Tr, Pr, fx, nsteps, dt, tol=1e-12, mode="f64", maxit=200)
        return float((gradF * Tr).sum())  # F is linear in T_N

    g0, stb = h.porous_backward(T0, torch.zeros_like(T0), fx, nsteps, gradF, dt, ckpt_every=ce, tol=1e-12,
                                mode="f64", maxit=200)
    rng = np.random.default_rng(3)
    for _ in range(2):
        d = torch.as_tensor(rng.standard_normal(n), device="cuda") * (1 - fx.double())
        eps = 1e-2
        fd = (F(T0 + eps * d) - F(T0 - eps * d)) / (2 * eps)
        an = float((g0 * d).sum())
        assert abs(fd - an) <= 1e-6 * abs(an), (fd, an)


def _paper_T0(xy):
    # the paper's initial state (Sec. 3.2.2): 400 x the Gaussian of mean the centre and covariance I/2,
    # top wall at -100 and bottom wall at +100
    T0 = W.gaussian_initial_T(xy, (0.5, 0.5))
    return np.where(xy[:, 1] == 1.0, -100.0, np.where(xy[:, 1] == 0.0, 100.0, T0))


def _rk_pair(nsub, nlevels):
    from oracle import rk  # noqa: F401  (imported for the callers)
    h, xy, fixed = _setup(nsub, nlevels)
    lev = _oracle_level(nsub)
    prm = por.PorousParams()
    pot = por.potential(xy, prm)
    return h, xy, fixed, lev, prm, pot


@pytest.mark.parametrize("nsub", [3, 4])
def test_rk_fixed_steps_match_oracle(nsub):
    from oracle import rk
    h, xy, fixed, lev, prm, pot = _rk_pair(nsub, 3)
    T0 = _paper_T0(xy)
    dt = 2e-4 if nsub == 3 else 5e-5
    ref, rst = rk.integrate(por.tdot_fn(lev, pot, fixed, prm), T0, 5 * dt, dt, 1.0, 1.0, fixed_step=True)
    T = torch.as_tensor(T0, device="cuda")
    P = torch.zeros_like(T)
    fx = torch.as_tensor(fixed.astype(np.uint8), device="cuda")
    st = h.porous_rk(T, P, fx, 5 * dt, dt, fixed_step=True, tol=1e-12, mode="f64", maxit=200)
    assert st["naccept"] == rst.naccept == 5 and st["nfev"] == rst.nfev == 31 and st["t"] == 5 * dt
    got = T.cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 1e-9 * np.max(np.abs(ref))
    assert np.array_equal(got[fixed], T0[fixed]) and np.max(np.abs(got - T0)) > 1e-3


@pytest.mark.parametrize("rtol", [1e-6, 1e-8])
def test_rk_adaptive_matches_oracle(rtol):
    # the same accepted and rejected steps as the oracle (pressure solved to 1e-12 against its direct
    # solve), from a first step far too large, so that the controller has to reject
    from oracle import rk
    h, xy, fixed, lev, prm, pot = _rk_pair(3, 3)
    T0 = _paper_T0(xy)
    t_end, dt0 = 2e-3, 1e-3
    ref, rst = rk.integrate(por.tdot_fn(lev, pot, fixed, prm), T0, t_end, dt0, rtol, rtol)
    T = torch.as_tensor(T0, device="cuda")
    P = torch.zeros_like(T)
    fx = torch.as_tensor(fixed.astype(np.uint8), device="cuda")
    st = h.porous_rk(T, P, fx, t_end, dt0, rtol=rtol, atol=rtol, tol=1e-12, mode="f64", maxit=200)
    assert rst.nreject > 0 and rst.naccept > 3
    assert (st["naccept"], st["nreject"], st["nfev"]) == (rst.naccept, rst.nreject, rst.nfev)
    # the error estimate is a difference of stage rates whose weights sum to zero: it amplifies the
    # pressure solves' 1e-12 relative error to ~1e-6 in the error norm, and the next step follows its
    # -1/5 power
    assert st["t"] == t_end and st["dt"] == pytest.approx(rst.dt, rel=1e-4)
    assert np.max(np.abs(T.cpu().numpy() - ref)) <= 1e-9 * np.max(np.abs(ref))


def test_rk_conductive_state_stays_put():
    h, xy, fixed = _setup(5, 4)
    T0 = 100.0 - 200.0 * xy[:, 1]
    T = torch.as_tensor(T0, device="cuda")
    P = torch.zeros_like(T)
    fx = torch.as_tensor(fixed.astype(np.uint8), device="cuda")
    # an equilibrium only to the pressure solves' accuracy: the step grows until the explicit method's
    # diffusion stability bound limits it (with rejections there), and the state stays put
    st = h.porous_rk(T, P, fx, 0.01, 1e-5, rtol=1e-9, atol=1e-6, tol=1e-11, mode="mixed")
    assert st["t"] == 0.01 and st["naccept"] >= 5
    assert np.max(np.abs(T.cpu().numpy() - T0)) < 1e-7 * 100.0


def test_rk_paper_setup_mg_against_fp64_pressure():
    # the paper's porous setup on its 16,641-vertex mesh (unit square x7), Tsit5 at rtol 1e-9:
    # float-float MG-PCG pressure solves to 1e-8 against FP64 ones to 1e-12 over the same interval
    h, xy, fixed = _setup(7, 6)
    assert h.n == 16641
    T0 = torch.as_tensor(_paper_T0(xy), device="cuda")
    fx = torch.as_tensor(fixed.astype(np.uint8), device="cuda")
    out = {}
    for key, kw in (("ref", dict(tol=1e-12, mode="f64", maxit=300)), ("mg", dict(tol=1e-8, mode="mixed_ff"))):
        T = T0.clone()
        P = torch.zeros_like(T)
        st = h.porous_rk(T, P, fx, 2e-4, 1e-6, rtol=1e-9, atol=1e-6, **kw)
        assert st["t"] == 2e-4 and st["naccept"] > 5 and st["pressure_rel_res"] <= kw["tol"] * 1.01
        out[key] = (T.cpu().numpy(), st)
    rmse = float(np.sqrt(np.mean((out["mg"][0] - out["ref"][0]) ** 2)))
    assert rmse < 1e-5, rmse
    assert abs(out["mg"][1]["naccept"] - out["ref"][1]["naccept"]) <= 1


def test_rk_argument_and_step_limit_errors():
    import paper_2508_12501_gb300 as P_
    h, xy, fixed = _setup(3, 3)
    T0 = _paper_T0(xy)
    T = torch.as_tensor(T0, device="cuda")
    P = torch.zeros_like(T)
    fx = torch.as_tensor(fixed.astype(np.uint8), device="cuda")
    with pytest.raises(P_.DecError):
        h.porous_rk(T, P, fx, 1e-3, 0.0)
    with pytest.raises(P_.DecError):
        h.porous_rk(T, P, fx, 1e-3, 1e-5, rtol=0.0, atol=0.0)
    with pytest.raises(P_.DecError) as ei:
        h.porous_rk(T, P, fx, 1.0, 1e-6, max_steps=3, mode="f64", tol=1e-12)
    assert ei.value.code == 5  # DEC_ERR_NOT_CONVERGED: T holds the state reached
    assert np.max(np.abs(T.cpu().numpy() - T0)) > 0.0
