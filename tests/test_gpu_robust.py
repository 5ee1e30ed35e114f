"""Failure detection on the GPU without a fault: the bounded device-side wait.

The shared-memory coarse cycle waits on an mbarrier for the bulk copies of
its tables, with a bound on the try_wait rounds.  dec_mg_set_wait_limit(0)
makes that wait give up at once (a wait that runs out, not a fault): the
block records status 3, drains its copies with the default bound and
returns without writing; the rest of the solve is skipped and dec_solve
returns DEC_ERR_CUDA with x holding the iterate from before the failed
cycle.  The context stays usable: with the default bound restored the same
handle solves to the oracle's solution.
"""
import numpy as np
import pytest

import workloads as W
from oracle import multigrid as omg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _square():
    import paper_2508_12501_gb300 as P
    v, t = W.unit_square()
    h = P.Hierarchy(P.Mesh(v, t), 6, 5, bc="dirichlet", smoother="chebyshev")
    oh = omg.build_hierarchy(v, t, 6, 5, "dirichlet", opts=omg.MGOptions(smoother="chebyshev"))
    return h, oh


@pytest.mark.parametrize("mode", ["mixed", "mixed_f32dot"])
@pytest.mark.parametrize("host_loop", [False, True])
def test_coarse_wait_that_runs_out_fails_the_solve_and_keeps_x(mode, host_loop):
    import paper_2508_12501_gb300 as P
    h, oh = _square()
    b = torch.as_tensor(W.uniform_field(h.n, 5), device="cuda")
    x0 = torch.as_tensor(W.uniform_field(h.n, 6) * 1e-3, device="cuda")
    free = torch.as_tensor(oh.finest.free, device="cuda")
    x0 = torch.where(free, x0, torch.zeros_like(x0))  # a Dirichlet-compatible warm start
    x = x0.clone()
    h.set_wait_limit(0)
    with pytest.raises(P.DecError) as ei:
        h.solve(b, x, mode=mode, tol=1e-10, warm_start=True, host_loop=host_loop)
    assert ei.value.code == 3  # DEC_ERR_CUDA
    assert "device-side wait" in str(ei.value)
    torch.cuda.synchronize()
    assert torch.equal(x, x0)
    # the default bound again: the same handle solves, matching the oracle's direct solution
    h.set_wait_limit(-1)
    x, st = h.solve(b, x, mode=mode, tol=1e-10, warm_start=True, host_loop=host_loop)
    assert st.status == 0
    xs = omg.direct_solve(oh, b.cpu().numpy())
    lev = oh.finest
    assert omg.star0_norm(lev, x.cpu().numpy() - xs) / omg.star0_norm(lev, xs) < 1e-7


def test_wait_limit_arguments():
    h, _ = _square()
    h.set_wait_limit(1 << 30)  # clamped to the default bound
    h.set_wait_limit(-5)       # the default
    b = torch.as_tensor(W.uniform_field(h.n, 7), device="cuda")
    _, st = h.solve(b, mode="mixed_ff", tol=1e-8)
    assert st.status == 0
