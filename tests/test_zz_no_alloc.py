"""dec_mg_vcycle_noalloc against dec_mg_vcycle, through the C ABI.

Some callers may not allocate device memory at the point where they run a
cycle: runtimes that reserve all device memory at start-up, plug-ins whose
host application owns every allocation, code that must not trigger a
device-synchronizing cudaMalloc.  For them libdec offers a cycle whose work
vectors live in a fixed file-scope device array.  These tests check that it
gives the allocating cycle's result and the oracle's FP64 cycle (within the
FP32 cycle tolerance used by the parity tests) on two calls in a row, so a
second call is not disturbed by what the first left in the shared array --
also with no pre-smoothing (the cycle's iterate then starts from a cleared
vector) and with the *0-adjoint restriction -- and that a hierarchy too
large for the array is refused with an error instead of overrunning it.

This file is collected last on purpose, and it builds everything it uses, so
it runs the same alone in a fresh process or after the other tests.
"""
import ctypes as C

import numpy as np
import pytest

import workloads as W
from oracle import multigrid as omg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CYCLE_TOL = 2e-5  # FP32 cycle tolerance of tests/test_gpu_parity.py (*0-norm, relative)


def _star0_rel(s0, a, b):
    d = a - b
    return float(np.sqrt(np.sum(s0 * d * d) / np.sum(s0 * b * b)))


CASES = {
    # name: (base, nsub, nlevels, bc, sphere, smoother, nu1, restriction)
    "icosphere_gauge_chebyshev": (W.icosahedron, 5, 4, "gauge", True, "chebyshev", 2, "rownorm"),
    "square_dirichlet_jacobi": (W.unit_square, 6, 5, "dirichlet", False, "jacobi", 2, "rownorm"),
    "square_dirichlet_jacobi_nu1_0": (W.unit_square, 6, 5, "dirichlet", False, "jacobi", 0, "rownorm"),
    "icosphere_gauge_chebyshev_star0": (W.icosahedron, 5, 4, "gauge", True, "chebyshev", 2, "star0"),
}


@pytest.mark.parametrize("case", list(CASES))
def test_noalloc_cycle_matches_allocating_cycle_and_oracle(case):
    import paper_2508_12501_gb300 as P
    from paper_2508_12501_gb300 import _lib as L

    base, nsub, nl, bc, sph, smoother, nu1, restriction = CASES[case]
    v, t = base()
    h = P.Hierarchy(P.Mesh(v, t), nsub, nl, bc=bc, sphere=sph, smoother=smoother, nu1=nu1,
                    restriction=restriction)
    oh = omg.build_hierarchy(v, t, nsub, nl, bc, sphere=sph,
                             opts=omg.MGOptions(smoother=smoother, nu1=nu1, restriction=restriction))
    n = h.n
    s0 = h.table(-1, "star0")
    bh = omg.prepare_rhs(oh, W.uniform_field(n, 77))
    b = torch.as_tensor(bh, dtype=torch.float32, device="cuda")
    x_ref = torch.zeros(n, dtype=torch.float32, device="cuda")
    x_new = torch.zeros(n, dtype=torch.float32, device="cuda")
    x_orc = np.zeros(n)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        rc = L.lib.dec_mg_vcycle(h._h, C.c_void_p(b.data_ptr()), C.c_void_p(x_ref.data_ptr()), 1, L.DEC_F32, stream)
        assert rc == L.DEC_OK, L.lib.dec_last_error()
        rc = L.lib.dec_mg_vcycle_noalloc(h._h, C.c_void_p(b.data_ptr()), C.c_void_p(x_new.data_ptr()), stream)
        assert rc == L.DEC_OK, L.lib.dec_last_error()
        x_orc = omg.vcycle(oh, bh, x_orc)  # the oracle's FP64 cycle from its own previous iterate
        torch.cuda.synchronize()
        a = x_new.double().cpu().numpy()
        r = x_ref.double().cpu().numpy()
        assert np.all(np.isfinite(a))
        assert _star0_rel(s0, a, r) < CYCLE_TOL, (call, _star0_rel(s0, a, r))
        assert _star0_rel(s0, a, x_orc) < CYCLE_TOL, (call, _star0_rel(s0, a, x_orc))


def test_noalloc_rejects_hierarchy_above_limit():
    import paper_2508_12501_gb300 as P
    from paper_2508_12501_gb300 import _lib as L

    # 1,050,625 finest vertices, 7 levels: 33.66 MB of cycle vectors > 32 MiB
    v, t = W.unit_square()
    h = P.Hierarchy(P.Mesh(v, t), 10, 7, bc="dirichlet")
    need = sum(((n + 63) // 64) * 64 * 6 * 4 for n in h.nv)
    assert need > L.DEC_NOALLOC_SCRATCH_BYTES
    b = torch.zeros(h.n, dtype=torch.float32, device="cuda")
    x = torch.zeros(h.n, dtype=torch.float32, device="cuda")
    rc = L.lib.dec_mg_vcycle_noalloc(h._h, C.c_void_p(b.data_ptr()), C.c_void_p(x.data_ptr()),
                                     C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == L.DEC_ERR_ARG
    assert b"DEC_NOALLOC_SCRATCH_BYTES" in L.lib.dec_last_error()
    torch.cuda.synchronize()
    assert torch.count_nonzero(x) == 0
