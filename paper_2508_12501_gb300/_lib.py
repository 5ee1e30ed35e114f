"""ctypes declarations of libdec (include/dec.h).  Argument marshalling only.

Importing this module loads ``libdec.so`` from this package directory and
raises ImportError if it is missing: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdec.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"libdec.so not found at {LIB_PATH}; build it with "
        "`python -m paper_2508_12501_gb300.build` (needs nvcc with sm_103a)")

lib = C.CDLL(LIB_PATH)

# status codes and enums (mirror include/dec.h)
DEC_OK, DEC_ERR_ARG, DEC_ERR_MESH, DEC_ERR_CUDA, DEC_ERR_OOM, DEC_ERR_NOT_CONVERGED, DEC_ERR_NONFINITE = range(7)
DEC_SPHERE_PROJECT, DEC_HOST_ONLY, DEC_ORDER_MORTON, DEC_SUBDIV_CUBIC = 1, 2, 4, 8
DEC_NOALLOC_SCRATCH_BYTES = 32 << 20
DEC_BC_DIRICHLET, DEC_BC_GAUGE = 0, 1
DEC_F64, DEC_F32 = 0, 1
DEC_SMOOTH_JACOBI, DEC_SMOOTH_CHEBYSHEV, DEC_SMOOTH_MCGS = 0, 1, 2
DEC_RESTRICT_ROWNORM, DEC_RESTRICT_STAR0 = 0, 1
DEC_SOLVER_MG, DEC_SOLVER_MGPCG, DEC_SOLVER_CG = 0, 1, 2
DEC_MODE_F64, DEC_MODE_MIXED, DEC_MODE_MIXED_FF, DEC_MODE_MIXED_F32DOT = 0, 1, 2, 3
DEC_FUSE_SMOOTH01, DEC_FUSE_RESTRICT, DEC_FUSE_PROLONG, DEC_FUSE_RESTRICT0, DEC_FUSE_OUTER = 1, 2, 4, 8, 16
DEC_FUSE_COARSE = 32
DEC_FUSE_PATCH = 64
DEC_FUSE_ALL = 127
(DEC_TABLE_VERTS, DEC_TABLE_TRIS, DEC_TABLE_EDGES, DEC_TABLE_STAR0, DEC_TABLE_STAR1,
 DEC_TABLE_FREE, DEC_TABLE_PARENTS, DEC_TABLE_COLORS, DEC_TABLE_MAP_IDX, DEC_TABLE_MAP_W) = range(10)

STATUS_NAMES = {0: "DEC_OK", 1: "DEC_ERR_ARG", 2: "DEC_ERR_MESH", 3: "DEC_ERR_CUDA", 4: "DEC_ERR_OOM",
                5: "DEC_ERR_NOT_CONVERGED", 6: "DEC_ERR_NONFINITE"}


class dec_mg_opts(C.Structure):
    _fields_ = [("smoother", C.c_int), ("nu1", C.c_int), ("nu2", C.c_int), ("omega", C.c_double),
                ("cheby_lo", C.c_double), ("cheby_hi", C.c_double), ("power_iters", C.c_int), ("gamma", C.c_int),
                ("restriction", C.c_int), ("fcycle", C.c_int), ("coarse_max_rows", C.c_int), ("fuse", C.c_int),
                ("fuse_max_rows", C.c_int), ("patch_max_rows", C.c_int), ("patch_chunk", C.c_int),
                ("patch_threads", C.c_int)]


class dec_solve_opts(C.Structure):
    _fields_ = [("solver", C.c_int), ("mode", C.c_int), ("tol", C.c_double), ("maxit", C.c_int),
                ("warm_start", C.c_int), ("check_every", C.c_int), ("host_loop", C.c_int)]


class dec_stats(C.Structure):
    _fields_ = [("iters", C.c_int), ("rel_res", C.c_double), ("rel_res0", C.c_double), ("launches", C.c_int64)]


class dec_prof_entry(C.Structure):
    _fields_ = [("kind", C.c_int), ("level", C.c_int), ("launches", C.c_int64), ("total_ms", C.c_double),
                ("rows", C.c_int64)]


PROF_KINDS = ["smooth0", "smooth", "residual", "restrict", "prolong", "coarse", "spmv64", "update", "zdots",
              "pupd", "mgres", "add", "aux", "smooth01", "resrestrict", "prolsmooth",
              "smoothdots", "coarsecycle", "patchdown", "patchup"]


class dec_rk_stats(C.Structure):
    _fields_ = [("naccept", C.c_int64), ("nreject", C.c_int64), ("nfev", C.c_int64), ("t", C.c_double),
                ("dt", C.c_double), ("pressure_iters", C.c_int64), ("pressure_rel_res", C.c_double)]


class dec_porous_params(C.Structure):
    _fields_ = [("g", C.c_double * 3), ("alpha_rho0", C.c_double), ("phi", C.c_double), ("k_eta", C.c_double),
                ("kappa", C.c_double), ("dt", C.c_double), ("tol", C.c_double), ("mode", C.c_int),
                ("maxit", C.c_int)]


class dec_batch_opts(C.Structure):
    _fields_ = [("block", C.c_int), ("kgroup", C.c_int), ("nu", C.c_int), ("smoother", C.c_int),
                ("solver", C.c_int)]


class dec_batch_stats(C.Structure):
    _fields_ = [("iters", C.c_int), ("max_rel_res", C.c_double), ("launches", C.c_int64), ("dof", C.c_int64)]


class dec_mg_info_t(C.Structure):
    _fields_ = [("nlevels", C.c_int), ("nv", C.c_int64 * 16), ("ne", C.c_int64 * 16), ("nt", C.c_int64 * 16),
                ("ell_width", C.c_int * 16), ("lmax", C.c_double * 16), ("ncolors", C.c_int * 16),
                ("bc", C.c_int), ("dim", C.c_int), ("device_bytes", C.c_size_t), ("tiles", C.c_int * 16)]


_p = C.c_void_p
_i = C.c_int
_i64 = C.c_int64
_u32 = C.c_uint32

_SIGS = {
    "dec_last_error": (C.c_char_p, []),
    "dec_mg_default_opts": (None, [C.POINTER(dec_mg_opts)]),
    "dec_solve_default_opts": (None, [C.POINTER(dec_solve_opts)]),
    "dec_mesh_create": (_i, [_p, _i64, _i, _p, _i64, C.POINTER(_p)]),
    "dec_mesh_destroy": (None, [_p]),
    "dec_mesh_sizes": (_i, [_p, C.POINTER(_i64), C.POINTER(_i64), C.POINTER(_i64), C.POINTER(_i)]),
    "dec_mesh_refine": (_i, [_p, _i, _u32, C.POINTER(_p)]),
    "dec_mesh_copy_table": (_i, [_p, _i, _p]),
    "dec_mg_build": (_i, [_p, _i, _i, _i, _u32, _p, C.POINTER(dec_mg_opts), C.POINTER(_p)]),
    "dec_mg_build_maps": (_i, [C.POINTER(_p), _i, C.POINTER(_p), C.POINTER(_p), _i, _u32, _p,
                              C.POINTER(dec_mg_opts), C.POINTER(_p)]),
    "dec_mg_destroy": (None, [_p]),
    "dec_mg_info": (_i, [_p, C.POINTER(dec_mg_info_t)]),
    "dec_mg_copy_table": (_i, [_p, _i, _i, _p]),
    "dec_mg_set_star1": (_i, [_p, _p, _p]),
    "dec_laplace0_apply": (_i, [_p, _i, _p, _p, _i, _i, _p]),
    "dec_residual": (_i, [_p, _i, _p, _p, _p, _i, _i, _p]),
    "dec_mg_vcycle": (_i, [_p, _p, _p, _i, _i, _p]),
    "dec_solve": (_i, [_p, _p, _p, _i, C.POINTER(dec_solve_opts), C.POINTER(dec_stats), _p]),
    "dec_solve_host": (_i, [_p, _p, _p, _i, C.POINTER(dec_solve_opts), C.POINTER(dec_stats), _p]),
    "dec_solve_backward": (_i, [_p, _p, _p, _p, _p, C.POINTER(dec_solve_opts), C.POINTER(dec_stats), _p]),
    "dec_mg_profile": (_i, [_p, _i]),
    "dec_mg_set_wait_limit": (_i, [_p, _i]),
    "dec_mg_vcycle_noalloc": (_i, [_p, _p, _p, _p]),
    "dec_batch_default_opts": (None, [C.POINTER(dec_batch_opts)]),
    "dec_batch_create": (_i, [C.POINTER(_p), C.POINTER(_i), _i, C.POINTER(dec_batch_opts), C.POINTER(_p)]),
    "dec_batch_destroy": (None, [_p]),
    "dec_batch_solve": (_i, [_p, C.POINTER(_p), C.POINTER(_p), C.c_double, _i, C.POINTER(dec_batch_stats), _p]),
    "dec_batch_solve_backward": (_i, [_p, C.POINTER(_p), C.POINTER(_p), C.POINTER(_p), C.POINTER(_p), C.c_double, _i,
                                      C.POINTER(dec_batch_stats), _p]),
    "dec_batch_info": (_i, [_p, C.POINTER(_i), C.POINTER(_i), C.POINTER(_i64), C.POINTER(C.c_size_t)]),
    "dec_batch_tune": (_i, [C.POINTER(_p), C.POINTER(_i), _i, C.POINTER(_p), C.POINTER(_p), C.c_double, _i,
                            C.POINTER(dec_batch_opts), _i, _i, C.POINTER(dec_batch_opts), C.POINTER(C.c_double),
                            C.POINTER(C.c_double), _p]),
    "dec_batch_time_smooth": (_i, [_p, _i, C.POINTER(C.c_double), C.POINTER(C.c_double), _p]),
    "dec_porous_default_params": (None, [C.POINTER(dec_porous_params)]),
    "dec_porous_rk": (_i, [_p, _p, _p, _p, C.POINTER(dec_porous_params), C.c_double, C.c_double, C.c_double,
                           C.c_double, C.c_int64, _i, C.POINTER(dec_rk_stats), _p]),
    "dec_porous_step": (_i, [_p, _p, _p, _p, C.POINTER(dec_porous_params), _i, _p, _i, C.POINTER(dec_stats), _p]),
    "dec_porous_backward": (_i, [_p, _p, _p, _p, C.POINTER(dec_porous_params), _i, _i, _p, _p,
                                 C.POINTER(dec_stats), _p]),
    "dec_mg_profile_read": (_i, [_p, C.POINTER(dec_prof_entry), _i, C.POINTER(_i)]),
    "dec_mg_time_smooth": (_i, [_p, _i, _i, C.POINTER(C.c_double), C.POINTER(C.c_double), _p]),
    "dec_mg_time_kernel": (_i, [_p, _i, _i, _i, C.POINTER(C.c_double), C.POINTER(C.c_double), _p]),
}

for _name, (_res, _args) in _SIGS.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args


class DecError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        msg = lib.dec_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS_NAMES.get(code, code)}: {msg}")


def check(code, where):
    if code != DEC_OK:
        raise DecError(code, where)
    return code
