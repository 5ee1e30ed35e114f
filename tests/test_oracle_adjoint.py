"""Pins of the oracle adjoint: brute-force finite differences and an explicit dense Jacobian."""
import numpy as np
import pytest

import workloads as W
from oracle import adjoint as adj, mesh as M, dec


def _case(which):
    if which == "square":
        v, t = W.unit_square()
        m = M.refine(v, t, 3)[0][-1]
        bc = "dirichlet"
    else:
        v, t = W.icosahedron()
        m = M.refine(v, t, 2, sphere=True)[0][-1]
        bc = "gauge"
    s1 = dec.hodge_star1(m) * W.lognormal_factors(m.ne, 2)
    return m, bc, s1


def _J(m, bc, b, s1, ut):
    lev = adj.level_with_star1(m, bc, s1)
    u = adj.solve(lev, bc, b)
    return adj.loss_star0(lev, u, ut)[0]


@pytest.mark.parametrize("which", ["square", "ico"])
def test_adjoint_matches_central_differences(which):
    m, bc, s1 = _case(which)
    b = W.uniform_field(m.nv, 3)
    ut = W.uniform_field(m.nv, 5)
    lev = adj.level_with_star1(m, bc, s1)
    u = adj.solve(lev, bc, b)
    J0, g = adj.loss_star0(lev, u, ut)
    gb, gs = adj.gradients(lev, bc, u, g)
    rng = np.random.default_rng(9)
    for _ in range(4):
        db = rng.standard_normal(m.nv)
        ds = s1 * rng.standard_normal(m.ne)  # multiplicative: zero weights stay zero
        eps = 1e-5
        fd = (_J(m, bc, b + eps * db, s1 + eps * ds, ut) - _J(m, bc, b - eps * db, s1 - eps * ds, ut)) / (2 * eps)
        an = gb @ db + gs @ ds
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-12 * J0), (fd, an)


def test_adjoint_rhs_gradient_is_dense_transpose_inverse():
    m, bc, s1 = _case("square")
    lev = adj.level_with_star1(m, bc, s1)
    idx = np.flatnonzero(lev.free)
    Lff = lev.L[idx][:, idx].toarray()
    g = W.uniform_field(m.nv, 11)
    b = W.uniform_field(m.nv, 12)
    u = adj.solve(lev, bc, b)
    gb, _ = adj.gradients(lev, bc, u, g)
    expect = np.zeros(m.nv)
    expect[idx] = np.linalg.solve(Lff.T, g[idx])
    assert np.allclose(gb, expect, rtol=1e-10, atol=1e-12 * np.abs(expect).max())
    assert np.all(gb[~lev.free] == 0.0)
