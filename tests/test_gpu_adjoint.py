"""GPU adjoint: dec_solve_backward and the autograd function against the oracle and finite differences.

Gradients are compared in the relative 2-norm.  The forward and adjoint GPU
solves run to tol = 1e-11, so their solutions carry relative errors of order
kappa_eff * 1e-11 <= 1e-6 on these meshes; the bound used is 1e-6.  The
full-size check follows the differentiable-solve workload: unit square x10
(1,050,625 vertices), *1 scaled by exp(0.5 z), loss 1/2 |u - u_t|^2 in the *0
norm, 32 seeded directions, central differences with FP64 solves to 1e-13,
agreement within 1e-5 relative.
"""
import numpy as np
import pytest

import workloads as W
from oracle import adjoint as adj, dec, mesh as M

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _setup(which, nsub):
    import paper_2508_12501_gb300 as P
    if which == "square":
        v, t = W.unit_square(); bc, sph, nl = "dirichlet", False, 4
    else:
        v, t = W.icosahedron(); bc, sph, nl = "gauge", True, 3
    m = M.refine(v, t, nsub, sphere=sph)[0][-1]
    scale = W.lognormal_factors(m.ne, 2)
    h = P.Hierarchy(P.Mesh(v, t), nsub, nl, bc=bc, sphere=sph, star1_scale=scale)
    s1 = dec.hodge_star1(m) * scale
    return P, h, m, bc, s1


@pytest.mark.parametrize("which", ["square", "ico"])
@pytest.mark.parametrize("mode", ["f64", "mixed"])
def test_backward_matches_oracle(which, mode):
    P, h, m, bc, s1 = _setup(which, 5 if which == "square" else 4)
    b = W.uniform_field(m.nv, 3)
    ut = W.uniform_field(m.nv, 5)
    lev = adj.level_with_star1(m, bc, s1)
    u_ref = adj.solve(lev, bc, b)
    _, g = adj.loss_star0(lev, u_ref, ut)
    gb_ref, gs_ref = adj.gradients(lev, bc, u_ref, g)
    u, st = h.solve(torch.as_tensor(b, device="cuda"), mode=mode, tol=1e-11, maxit=200)
    assert _rel(u.cpu().numpy(), u_ref) < 1e-6
    gb, gs, st2 = h.solve_backward(u, torch.as_tensor(g, device="cuda"), mode=mode, tol=1e-11, maxit=200)
    assert st2.rel_res <= 1e-11
    assert _rel(gb.cpu().numpy(), gb_ref) < 1e-6
    assert _rel(gs.cpu().numpy(), gs_ref) < 1e-6


def test_set_star1_rebuilds_finest_weights():
    import paper_2508_12501_gb300 as P
    v, t = W.unit_square()
    m = M.refine(v, t, 4)[0][-1]
    s1 = dec.hodge_star1(m) * W.lognormal_factors(m.ne, 7)
    h = P.Hierarchy(P.Mesh(v, t), 4, 3, bc="dirichlet")
    h.set_star1(torch.as_tensor(s1, device="cuda"))
    lev = adj.level_with_star1(m, "dirichlet", s1)
    x = W.uniform_field(m.nv, 1)
    y = h.laplace0_apply(torch.as_tensor(x, device="cuda")).cpu().numpy()
    ref = np.where(lev.free, lev.L @ x, 0.0)
    bound = 16 * 2.0 ** -53 * (abs(lev.L) @ np.abs(x))
    assert np.all(np.abs(y - ref) <= bound + 1e-300)


def test_autograd_function_matches_oracle():
    P, h, m, bc, s1 = _setup("square", 4)
    b = torch.as_tensor(W.uniform_field(m.nv, 3), device="cuda").requires_grad_(True)
    star1 = torch.as_tensor(s1, device="cuda").requires_grad_(True)
    ut = torch.as_tensor(W.uniform_field(m.nv, 5), device="cuda")
    s0 = torch.as_tensor(h.table(-1, "star0"), device="cuda")
    free = torch.as_tensor(h.table(-1, "free"), device="cuda").double()
    u = P.poisson_solve(b, star1, hier=h, mode="f64", tol=1e-12, maxit=200)
    d = (u - ut) * free
    J = 0.5 * (s0 * d * d).sum()
    J.backward()
    lev = adj.level_with_star1(m, bc, s1)
    u_ref = adj.solve(lev, bc, b.detach().cpu().numpy())
    _, g = adj.loss_star0(lev, u_ref, ut.cpu().numpy())
    gb_ref, gs_ref = adj.gradients(lev, bc, u_ref, g)
    assert _rel(b.grad.cpu().numpy(), gb_ref) < 1e-7
    assert _rel(star1.grad.cpu().numpy(), gs_ref) < 1e-7


def test_differentiable_solve_full_size_finite_differences():
    import paper_2508_12501_gb300 as P
    v, t = W.unit_square()
    nsub = 10
    h = P.Hierarchy(P.Mesh(v, t), nsub, 8, bc="dirichlet")
    n, ne = h.n, h.ne[-1]
    assert n == 1050625 and ne == 3147776
    s1 = torch.as_tensor(h.table(-1, "star1") * W.lognormal_factors(ne, 2), device="cuda")
    b0 = torch.as_tensor(W.uniform_field(n, 3), device="cuda")
    xy = h.table(-1, "verts")
    ut = torch.as_tensor(W.u_target_square(xy), device="cuda")
    s0 = torch.as_tensor(h.table(-1, "star0"), device="cuda")
    free = torch.as_tensor(h.table(-1, "free"), device="cuda").double()

    def J(bv, sv, tol, mode, x0=None):
        h.set_star1(sv)
        u, st = h.solve(bv, x=x0, warm_start=x0 is not None, mode=mode, tol=tol, maxit=300)
        d = (u - ut) * free
        return float(0.5 * (s0 * d * d).sum()), u

    # adjoint gradient: mixed-precision forward and backward solves
    b = b0.clone().requires_grad_(True)
    star1 = s1.clone().requires_grad_(True)
    u = P.poisson_solve(b, star1, hier=h, mode="mixed", tol=1e-10, maxit=300)
    d = (u - ut) * free
    (0.5 * (s0 * d * d).sum()).backward()
    gb, gs = b.grad, star1.grad

    _, u_c = J(b0, s1, 1e-13, "f64")
    rng = np.random.default_rng(4)
    eps = 1e-3
    worst = 0.0
    for k in range(32):
        db = torch.as_tensor(rng.standard_normal(n), device="cuda") * free
        ds = s1 * torch.as_tensor(rng.standard_normal(ne), device="cuda")  # relative change of each *1
        jp, _ = J(b0 + eps * db, s1 + eps * ds, 1e-13, "f64", u_c)
        jm, _ = J(b0 - eps * db, s1 - eps * ds, 1e-13, "f64", u_c)
        fd = (jp - jm) / (2 * eps)
        an = float((gb * db).sum() + (gs * ds).sum())
        worst = max(worst, abs(fd - an) / abs(an))
    assert worst < 1e-5, worst
