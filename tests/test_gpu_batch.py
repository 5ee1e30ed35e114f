"""Batched solves (many right-hand sides, uneven meshes) against the oracle.

Each right-hand side of a batch must reach its own relative residual
(recomputed in FP64 by the oracle's operator) and agree with the oracle's
direct solution in the *0 norm within the bound that tolerance implies.
The full-size case is the batched workload: 64 spherical-harmonic right-hand
sides on the icosphere x7 (163,842 vertices) plus 32 unit squares, 8 each at
subdivision levels 6-9 (4,225 ... 263,169 vertices), Dirichlet, U[-1,1].
"""
import numpy as np
import pytest

import workloads as W
from oracle import multigrid as omg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _mesh(kind, nsub, nl, restriction="rownorm"):
    import paper_2508_12501_gb300 as P
    if kind == "ico":
        v, t = W.icosahedron(); bc, sph = "gauge", True
    elif kind == "fan":
        v, t = W.heptagon_fan(); bc, sph = "dirichlet", False
    else:
        v, t = W.unit_square(); bc, sph = "dirichlet", False
    h = P.Hierarchy(P.Mesh(v, t), nsub, nl, bc=bc, sphere=sph, restriction=restriction)
    oh = omg.build_hierarchy(v, t, nsub, 1, bc, sphere=sph)
    return h, oh


def _rhs(n, k, seed):
    return np.stack([W.uniform_field(n, seed + j) for j in range(k)], axis=1)


def _check(oh, x, b, tol):
    lev = oh.finest
    for j in range(b.shape[1]):
        bj = omg.prepare_rhs(oh, b[:, j])
        xj = x[:, j]
        assert omg.rel_residual(lev, bj, xj) <= 4 * tol
        xs = omg.direct_solve(oh, b[:, j])
        assert omg.star0_norm(lev, xj - xs) / omg.star0_norm(lev, xs) < 1e-6


@pytest.mark.parametrize("solver", ["mgpcg", "mg"])
@pytest.mark.parametrize("kgroup", [0, 1, 2, 4, 8])
def test_uneven_batch_matches_oracle(kgroup, solver):
    import paper_2508_12501_gb300 as P
    cases = [("ico", 4, 3, 5), ("square", 5, 5, 1), ("square", 4, 3, 3), ("fan", 3, 3, 2)]
    hs, ohs, bs = [], [], []
    for i, (kind, nsub, nl, k) in enumerate(cases):
        h, oh = _mesh(kind, nsub, nl)
        hs.append(h); ohs.append(oh)
        bs.append(_rhs(h.n, k, 10 * i))
    B = P.Batch(hs, [c[3] for c in cases], kgroup=kgroup, nu=2, solver=solver)
    xs, st = B.solve([torch.as_tensor(b, device="cuda") for b in bs], tol=1e-10, maxit=100)
    assert st.status == 0 and st.max_rel_res <= 1e-10
    assert st.dof == sum(h.n * c[3] for h, c in zip(hs, cases))
    for oh, x, b in zip(ohs, xs, bs):
        _check(oh, x.reshape(len(b), -1).cpu().numpy(), b, 1e-10)


@pytest.mark.parametrize("smoother", ["jacobi", "chebyshev"])
@pytest.mark.parametrize("nu", [1, 3])
def test_batch_smoother_options(smoother, nu):
    import paper_2508_12501_gb300 as P
    h1, o1 = _mesh("square", 5, 4)
    h2, o2 = _mesh("ico", 3, 2)
    b1, b2 = _rhs(h1.n, 4, 1), _rhs(h2.n, 2, 2)
    B = P.Batch([h1, h2], [4, 2], nu=nu, smoother=smoother, block=128)
    xs, st = B.solve([torch.as_tensor(b1, device="cuda"), torch.as_tensor(b2, device="cuda")], tol=1e-10, maxit=200)
    assert st.max_rel_res <= 1e-10
    _check(o1, xs[0].cpu().numpy(), b1, 1e-10)
    _check(o2, xs[1].cpu().numpy(), b2, 1e-10)


def test_entries_sharing_a_hierarchy_are_one_group_and_match_the_oracle():
    # the same hierarchy passed three times (2 + 1 + 3 right-hand sides) and another once: the shared one's
    # six columns form one interleaved group of 8 (two padding columns); every column matches the oracle
    import paper_2508_12501_gb300 as P
    h1, o1 = _mesh("square", 5, 4)
    h2, o2 = _mesh("ico", 4, 3)
    ks = [2, 3, 1, 3]
    hs, ohs = [h1, h2, h1, h1], [o1, o2, o1, o1]
    bs = [_rhs(h.n, k, 40 + 10 * i) for i, (h, k) in enumerate(zip(hs, ks))]
    B = P.Batch(hs, ks)
    assert B.ngroups == 2 and B.total_rhs == 8 + 4
    xs, st = B.solve([torch.as_tensor(b.reshape(-1), device="cuda") for b in bs], tol=1e-10)
    assert st.max_rel_res <= 1e-10
    for oh, x, b, k in zip(ohs, xs, bs, ks):
        _check(oh, x.reshape(-1, k).cpu().numpy(), b, 1e-10)
    # bitwise reproducible: the per-right-hand-side sums have a fixed order
    xs2, _ = B.solve([torch.as_tensor(b.reshape(-1), device="cuda") for b in bs], tol=1e-10)
    assert all(torch.equal(a, c) for a, c in zip(xs, xs2))


@pytest.mark.parametrize("solver", ["mgpcg", "mg"])
def test_converged_groups_drop_out_without_changing_results(solver):
    # a quickly converging group (icosphere, gauge) beside slower ones (squares, Dirichlet): once a group
    # has converged its kernels return at once, so the batch gives every group exactly the bits of that
    # group solved on its own, and takes the slowest group's pass count
    import paper_2508_12501_gb300 as P
    h1, o1 = _mesh("ico", 5, 4)
    h2, o2 = _mesh("square", 7, 6)
    h3, o3 = _mesh("square", 6, 5)
    hs, ks = [h1, h2, h3], [8, 1, 2]
    bs = [torch.as_tensor(_rhs(h.n, k, 70 + 10 * i).reshape(-1), device="cuda")
          for i, (h, k) in enumerate(zip(hs, ks))]
    B = P.Batch(hs, ks, solver=solver)
    xs, st = B.solve(bs, tol=1e-9)
    iters = []
    for i, (h, k) in enumerate(zip(hs, ks)):
        Bi = P.Batch([h], [k], solver=solver)
        xi, sti = Bi.solve([bs[i]], tol=1e-9)
        assert torch.equal(xs[i], xi[0]), i
        iters.append(sti.iters)
    assert st.iters == max(iters) and min(iters) < max(iters), iters
    assert st.max_rel_res <= 1e-9
    for oh, x, b, k in zip((o1, o2, o3), xs, bs, ks):
        _check(oh, x.reshape(-1, k).cpu().numpy(), b.reshape(-1, k).cpu().numpy(), 1e-9)
    # the adjoint shares the loop: the same per-group bits
    us = [x.reshape(h.n, -1) for x, h in zip(xs, hs)]
    gb, gs, _ = B.solve_backward(us, us, tol=1e-9)
    for i, (h, k) in enumerate(zip(hs, ks)):
        Bi = P.Batch([h], [k], solver=solver)
        gbi, gsi, _ = Bi.solve_backward([us[i]], [us[i]], tol=1e-9)
        assert torch.equal(gb[i], gbi[0]) and torch.equal(gs[i], gsi[0]), i
    # the smoother timer after a solve sees every group again
    ms, by = B.time_smooth(2)
    assert ms > 0 and by > 0


@pytest.mark.parametrize("solver", ["mgpcg", "mg"])
def test_batched_adjoint_matches_oracle_gradients(solver):
    # dJ/db = *0 mu and dJ/d*1 = -(d0 mu)(d0 u) per right-hand side, mu = L^-1 (*0^-1 dJ/du), against the
    # oracle's adjoint formulas with its direct solves
    import paper_2508_12501_gb300 as P
    from oracle import adjoint as oadj
    h1, o1 = _mesh("square", 5, 4)
    h2, o2 = _mesh("ico", 4, 3)
    ks = [3, 2]
    bs = [_rhs(h1.n, 3, 61), _rhs(h2.n, 2, 62)]
    B = P.Batch([h1, h2], ks, solver=solver)
    xs, _ = B.solve([torch.as_tensor(b.reshape(-1), device="cuda") for b in bs], tol=1e-11, maxit=200)
    gus = [torch.as_tensor(_rhs(h1.n, 3, 71), device="cuda"), torch.as_tensor(_rhs(h2.n, 2, 72), device="cuda")]
    gbs, gss, st = B.solve_backward([x.reshape(h.n, -1) for x, h in zip(xs, (h1, h2))], gus, tol=1e-11, maxit=200)
    assert st.max_rel_res <= 1e-11
    for oh, x, gu, gb, gs, k in zip((o1, o2), xs, gus, gbs, gss, ks):
        lev = oh.finest
        bc = oh.bc
        for j in range(k):
            u = x.reshape(lev.mesh.nv, k)[:, j].cpu().numpy()
            g = gu[:, j].cpu().numpy()
            rb, rs = oadj.gradients(lev, bc, u, g)
            ab = gb.reshape(lev.mesh.nv, k)[:, j].cpu().numpy()
            as1 = gs.reshape(-1, k)[:, j].cpu().numpy()
            assert np.linalg.norm(ab - rb) <= 1e-8 * np.linalg.norm(rb), j
            assert np.linalg.norm(as1 - rs) <= 1e-8 * np.linalg.norm(rs), j


def test_batch_error_paths():
    import paper_2508_12501_gb300 as P
    h1, _ = _mesh("square", 4, 3)
    h2, _ = _mesh("square", 4, 3, restriction="star0")
    with pytest.raises(P.DecError):
        P.Batch([h1, h2], [1, 1])
    with pytest.raises(P.DecError):
        P.Batch([h1], [2], kgroup=3)
    B = P.Batch([h1], [2])
    b = torch.zeros(h1.n, 2, dtype=torch.float64, device="cuda")
    xy = h1.table(-1, "verts")
    free = np.flatnonzero((xy[:, 0] > 0) & (xy[:, 0] < 1) & (xy[:, 1] > 0) & (xy[:, 1] < 1))
    b[int(free[0]), 1] = float("nan")  # on a free row: fixed (Dirichlet) rows are masked out
    with pytest.raises(P.DecError) as ei:
        B.solve([b])
    assert ei.value.code == 6
    b = torch.as_tensor(_rhs(h1.n, 2, 3), device="cuda")
    xs, st = B.solve([b], tol=1e-12, maxit=1, raise_on_fail=False)
    assert st.status == 5 and st.iters == 1


def test_full_batched_workload():
    import paper_2508_12501_gb300 as P
    v, t = W.icosahedron()
    hi = P.Hierarchy(P.Mesh(v, t), 7, 6, bc="gauge", sphere=True)
    pos = hi.table(-1, "verts")
    b_ico = np.stack([W.sh_sum(pos, W.sh_coefficients(100 + j)) for j in range(64)], axis=1)
    hs, ks, bs = [hi], [64], [b_ico]
    seed = 200
    vs, ts = W.unit_square()
    for nsub in (6, 7, 8, 9):
        hq = P.Hierarchy(P.Mesh(vs, ts), nsub, nsub - 1, bc="dirichlet")
        for _ in range(8):
            hs.append(hq); ks.append(1)
            bs.append(W.uniform_field(hq.n, seed)[:, None]); seed += 1
    B = P.Batch(hs, ks)
    assert B.dof == 163842 * 64 + 8 * (4225 + 16641 + 66049 + 263169)
    xs, st = B.solve([torch.as_tensor(b.reshape(-1), device="cuda") for b in bs], tol=1e-8, maxit=100)
    assert st.max_rel_res <= 1e-8
    # every residual, recomputed in FP64 by the oracle operator
    done = {}
    for h, b, x in zip(hs, bs, xs):
        key = id(h)
        if key not in done:
            vv, tt = (v, t) if h is hi else (vs, ts)
            nsub = 7 if h is hi else int(round(np.log2(np.sqrt(h.n) - 1)))
            done[key] = omg.build_hierarchy(vv, tt, nsub, 1, "gauge" if h is hi else "dirichlet", sphere=h is hi)
        oh = done[key]
        xx = x.reshape(h.n, -1).cpu().numpy()
        for j in range(b.shape[1]):
            assert omg.rel_residual(oh.finest, omg.prepare_rhs(oh, b[:, j]), xx[:, j]) <= 2e-8
    # and a few right-hand sides agree with single solves
    for j in (0, 31, 63):
        xj, _ = hi.solve(torch.as_tensor(b_ico[:, j], device="cuda"), tol=1e-10)
        oh = done[id(hi)]
        a = xs[0][:, j].cpu().numpy()
        r = xj.cpu().numpy()
        assert omg.star0_norm(oh.finest, a - r) / omg.star0_norm(oh.finest, r) < 1e-6
    # sampled right-hand sides against the oracle's u*: its FP64 MG-PCG to 1e-13 on the full hierarchy,
    # *0-norm error <= 1e-6 (four of the 64 on the icosphere x7, one square per subdivision level)
    ohi = omg.build_hierarchy(v, t, 7, 6, "gauge", sphere=True)
    for j in (0, 21, 42, 63):
        ref = omg.pcg_solve(ohi, b_ico[:, j], 1e-13, 200)
        a = xs[0].reshape(hi.n, -1)[:, j].cpu().numpy()
        err = omg.star0_norm(ohi.finest, a - ref.x) / omg.star0_norm(ohi.finest, ref.x)
        print(f"batched icosphere x7 rhs {j}: *0 error vs oracle u* {err:.3e}")
        assert err <= 1e-6, (j, err)
    for m, nsub in zip((1, 9, 17, 25), (6, 7, 8, 9)):
        ohq = omg.build_hierarchy(vs, ts, nsub, nsub - 1, "dirichlet")
        ref = omg.pcg_solve(ohq, bs[m][:, 0], 1e-13, 200)
        a = xs[m].reshape(-1).cpu().numpy()
        err = omg.star0_norm(ohq.finest, a - ref.x) / omg.star0_norm(ohq.finest, ref.x)
        print(f"batched square x{nsub} (mesh {m}): *0 error vs oracle u* {err:.3e}")
        assert err <= 1e-6, (m, err)


def test_autotuner_picks_a_converging_setting():
    import paper_2508_12501_gb300 as P
    h1, o1 = _mesh("square", 6, 5)
    h2, o2 = _mesh("ico", 4, 3)
    b1, b2 = _rhs(h1.n, 8, 5), _rhs(h2.n, 4, 6)
    bs = [torch.as_tensor(b1.reshape(-1), device="cuda"), torch.as_tensor(b2.reshape(-1), device="cuda")]
    cands = [dict(block=128, kgroup=0, nu=2, smoother="chebyshev"), dict(block=256, kgroup=2, nu=1, smoother="jacobi"),
             dict(block=512, kgroup=8, nu=3, smoother="chebyshev"), dict(block=100, kgroup=0, nu=2, smoother="jacobi")]
    best, ms, table = P.tune_batch([h1, h2], [8, 4], bs, tol=1e-10, candidates=cands, reps=2)
    assert best["solver"] == "mgpcg"  # the candidates' default
    assert {k: v for k, v in best.items() if k != "solver"} in cands[:3] and ms > 0
    assert table[3][1] == -1.0  # an invalid candidate is reported, not chosen
    assert ms == min(t for _, t in table if t > 0)
    B = P.Batch([h1, h2], [8, 4], **best)
    xs, st = B.solve(bs, tol=1e-10)
    _check(o1, xs[0].cpu().numpy(), b1, 1e-10)
    ms2, by = B.time_smooth(5)
    assert ms2 > 0 and by > 0
