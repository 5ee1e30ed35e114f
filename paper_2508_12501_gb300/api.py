"""Python face of libdec: meshes, hierarchies, operator calls, solves, autograd.

Everything here is argument marshalling around the C ABI of include/dec.h:
shapes, dtypes, devices and the current CUDA stream are checked and passed
through; every arithmetic step runs inside libdec's CUDA kernels.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np

from . import _lib as L
from ._lib import check, lib

SMOOTHERS = {"jacobi": L.DEC_SMOOTH_JACOBI, "chebyshev": L.DEC_SMOOTH_CHEBYSHEV, "mcgs": L.DEC_SMOOTH_MCGS}
SOLVERS = {"mg": L.DEC_SOLVER_MG, "mgpcg": L.DEC_SOLVER_MGPCG, "cg": L.DEC_SOLVER_CG}
MODES = {"f64": L.DEC_MODE_F64, "mixed": L.DEC_MODE_MIXED, "mixed_ff": L.DEC_MODE_MIXED_FF,
         "mixed_f32dot": L.DEC_MODE_MIXED_F32DOT}
ORDERS = {"edge": 0, "morton": L.DEC_ORDER_MORTON}
SCHEMES = {"binary": 0, "cubic": L.DEC_SUBDIV_CUBIC}
BCS = {"dirichlet": L.DEC_BC_DIRICHLET, "gauge": L.DEC_BC_GAUGE}
RESTRICTIONS = {"rownorm": L.DEC_RESTRICT_ROWNORM, "star0": L.DEC_RESTRICT_STAR0}
TABLES = {"verts": L.DEC_TABLE_VERTS, "tris": L.DEC_TABLE_TRIS, "edges": L.DEC_TABLE_EDGES,
          "star0": L.DEC_TABLE_STAR0, "star1": L.DEC_TABLE_STAR1, "free": L.DEC_TABLE_FREE,
          "parents": L.DEC_TABLE_PARENTS, "colors": L.DEC_TABLE_COLORS, "map_idx": L.DEC_TABLE_MAP_IDX,
          "map_w": L.DEC_TABLE_MAP_W}


def _np_ptr(a):
    return C.c_void_p(a.ctypes.data)


class Mesh:
    """Host mesh (dec_mesh_*): validated triangles and canonical edges."""

    def __init__(self, verts=None, tris=None, _handle=None):
        if _handle is not None:
            self._h = _handle
        else:
            v = np.ascontiguousarray(verts, dtype=np.float64)
            t = np.ascontiguousarray(tris, dtype=np.int32)
            if v.ndim != 2 or t.ndim != 2 or t.shape[1] != 3:
                raise ValueError("verts must be [nv, dim], tris [nt, 3]")
            h = C.c_void_p()
            check(lib.dec_mesh_create(_np_ptr(v), v.shape[0], v.shape[1], _np_ptr(t), t.shape[0], C.byref(h)),
                  "dec_mesh_create")
            self._h = h
        nv, ne, nt, dim = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int()
        check(lib.dec_mesh_sizes(self._h, C.byref(nv), C.byref(ne), C.byref(nt), C.byref(dim)), "dec_mesh_sizes")
        self.nv, self.ne, self.nt, self.dim = nv.value, ne.value, nt.value, dim.value

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib.dec_mesh_destroy(h)
            self._h = None

    def refine(self, nsub, sphere=False, order="edge", scheme="binary"):
        """nsub subdivisions (scheme "binary": 1->4, "cubic": 1->9); order numbers each binary level's
        new vertices ("edge" or "morton")."""
        h = C.c_void_p()
        flags = (L.DEC_SPHERE_PROJECT if sphere else 0) | ORDERS[order] | SCHEMES[scheme]
        check(lib.dec_mesh_refine(self._h, int(nsub), flags, C.byref(h)), "dec_mesh_refine")
        return Mesh(_handle=h)

    def table(self, what):
        n = {"verts": self.nv * self.dim, "tris": self.nt * 3, "edges": self.ne * 2,
             "star0": self.nv, "star1": self.ne}[what]
        dt = np.float64 if what in ("verts", "star0", "star1") else np.int32
        out = np.empty(n, dtype=dt)
        check(lib.dec_mesh_copy_table(self._h, TABLES[what], _np_ptr(out)), "dec_mesh_copy_table")
        if what == "verts":
            return out.reshape(self.nv, self.dim)
        if what in ("tris", "edges"):
            return out.reshape(-1, 3 if what == "tris" else 2)
        return out


@dataclass
class SolveStats:
    iters: int
    rel_res: float
    rel_res0: float
    status: int
    launches: int = 0


def _torch():
    import torch
    return torch


class Hierarchy:
    """A multigrid hierarchy on the current CUDA device (dec_mg_*)."""

    def __init__(self, mesh, nsub, nlevels, bc="dirichlet", sphere=False, star1_scale=None, smoother="jacobi",
                 nu1=2, nu2=2, omega=2.0 / 3.0, cheby_lo=0.3, cheby_hi=1.1, power_iters=10, gamma=1,
                 restriction="rownorm", host_only=False, fuse=None, order="edge", coarse_max_rows=0,
                 fcycle=False, scheme="binary", fuse_max_rows=None, patch_max_rows=0, patch_chunk=0,
                 patch_threads=0):
        if not isinstance(mesh, Mesh):
            raise TypeError("mesh must be a Mesh")
        o = self._opts(smoother, nu1, nu2, omega, cheby_lo, cheby_hi, power_iters, gamma, restriction, fuse,
                       fuse_max_rows, coarse_max_rows, fcycle, patch_max_rows, patch_chunk, patch_threads)
        self.fuse = int(o.fuse)
        flags = ((L.DEC_SPHERE_PROJECT if sphere else 0) | (L.DEC_HOST_ONLY if host_only else 0) | ORDERS[order]
                 | SCHEMES[scheme])
        scale = None
        if star1_scale is not None:
            scale = np.ascontiguousarray(star1_scale, dtype=np.float64)
        h = C.c_void_p()
        self.device = None
        if not host_only:
            torch = _torch()
            self.device = torch.device("cuda", torch.cuda.current_device())
        check(lib.dec_mg_build(mesh._h, int(nsub), int(nlevels), BCS[bc], flags,
                               _np_ptr(scale) if scale is not None else None, C.byref(o), C.byref(h)),
              "dec_mg_build")
        self._finish(h, bc, host_only)

    @classmethod
    def from_maps(cls, meshes, maps_idx, maps_w, bc="dirichlet", star1_scale=None, host_only=False, smoother="jacobi",
                  nu1=2, nu2=2, omega=2.0 / 3.0, cheby_lo=0.3, cheby_hi=1.1, power_iters=10, gamma=1,
                  restriction="rownorm", fuse=None, fcycle=False, fuse_max_rows=None):
        """A hierarchy on given meshes (coarsest first) related by given geometric maps (dec_mg_build_maps):
        maps_idx[l], maps_w[l] are [nv(l+1), 3] arrays -- the coarse vertices of level l and barycentric
        weights of each vertex of level l+1."""
        self = cls.__new__(cls)
        if not all(isinstance(m, Mesh) for m in meshes):
            raise TypeError("meshes must be Mesh objects")
        nl = len(meshes)
        if len(maps_idx) != nl - 1 or len(maps_w) != nl - 1:
            raise ValueError("one map per pair of consecutive levels")
        o = self._opts(smoother, nu1, nu2, omega, cheby_lo, cheby_hi, power_iters, gamma, restriction, fuse,
                       fuse_max_rows, 0, fcycle)
        self.fuse = int(o.fuse)
        mi = [np.ascontiguousarray(a, dtype=np.int32).reshape(-1) for a in maps_idx]
        mw = [np.ascontiguousarray(a, dtype=np.float64).reshape(-1) for a in maps_w]
        for l, (a, w) in enumerate(zip(mi, mw)):
            if a.size != 3 * meshes[l + 1].nv or w.size != 3 * meshes[l + 1].nv:
                raise ValueError(f"map {l} must have 3 entries per vertex of level {l + 1}")
        hs = (C.c_void_p * nl)(*[m._h for m in meshes])
        pi = (C.c_void_p * max(1, nl - 1))(*[C.c_void_p(a.ctypes.data) for a in mi])
        pw = (C.c_void_p * max(1, nl - 1))(*[C.c_void_p(w.ctypes.data) for w in mw])
        scale = None if star1_scale is None else np.ascontiguousarray(star1_scale, dtype=np.float64)
        self.device = None
        if not host_only:
            torch = _torch()
            self.device = torch.device("cuda", torch.cuda.current_device())
        h = C.c_void_p()
        check(lib.dec_mg_build_maps(hs, nl, pi, pw, BCS[bc], L.DEC_HOST_ONLY if host_only else 0,
                                    _np_ptr(scale) if scale is not None else None, C.byref(o), C.byref(h)),
              "dec_mg_build_maps")
        self._finish(h, bc, host_only)
        return self

    @staticmethod
    def _opts(smoother, nu1, nu2, omega, cheby_lo, cheby_hi, power_iters, gamma, restriction, fuse, fuse_max_rows,
              coarse_max_rows, fcycle, patch_max_rows=0, patch_chunk=0, patch_threads=0):
        o = L.dec_mg_opts()
        lib.dec_mg_default_opts(C.byref(o))
        o.smoother = SMOOTHERS[smoother]
        o.nu1, o.nu2, o.omega = nu1, nu2, omega
        o.cheby_lo, o.cheby_hi = cheby_lo, cheby_hi
        o.power_iters, o.gamma = power_iters, gamma
        o.restriction = RESTRICTIONS[restriction]
        if fuse is not None:  # None keeps the library default (the row-local fusions)
            o.fuse = int(fuse) if not isinstance(fuse, bool) else (L.DEC_FUSE_ALL if fuse else 0)
        if fuse_max_rows is not None:  # None keeps the library default
            o.fuse_max_rows = int(fuse_max_rows)
        o.coarse_max_rows = int(coarse_max_rows)
        o.fcycle = 1 if fcycle else 0
        o.patch_max_rows = int(patch_max_rows)
        o.patch_chunk = int(patch_chunk)
        o.patch_threads = int(patch_threads)
        return o

    def _finish(self, h, bc, host_only):
        self._h = h
        self.bc = bc
        self.host_only = host_only
        info = L.dec_mg_info_t()
        check(lib.dec_mg_info(self._h, C.byref(info)), "dec_mg_info")
        self.nlevels = info.nlevels
        self.nv = [info.nv[i] for i in range(self.nlevels)]
        self.ne = [info.ne[i] for i in range(self.nlevels)]
        self.nt = [info.nt[i] for i in range(self.nlevels)]
        self.ell_width = [info.ell_width[i] for i in range(self.nlevels)]
        self.lmax = [info.lmax[i] for i in range(self.nlevels)]
        self.ncolors = [info.ncolors[i] for i in range(self.nlevels)]
        self.dim = info.dim
        self.device_bytes = info.device_bytes
        self.tiles = [info.tiles[i] for i in range(self.nlevels)]  # halo tiles per level (DEC_FUSE_PATCH)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib.dec_mg_destroy(h)
            self._h = None

    @property
    def n(self):
        return self.nv[-1]

    def table(self, level, what):
        level = level % self.nlevels
        nv, ne, nt = self.nv[level], self.ne[level], self.nt[level]
        nf = self.nv[level + 1] if level + 1 < self.nlevels else 0
        n = {"verts": nv * self.dim, "tris": nt * 3, "edges": ne * 2, "parents": ne * 2, "star0": nv,
             "star1": ne, "free": nv, "colors": nv, "map_idx": nf * 3, "map_w": nf * 3}[what]
        dt = np.float64 if what in ("verts", "star0", "star1", "map_w") else np.int32
        out = np.empty(n, dtype=dt)
        check(lib.dec_mg_copy_table(self._h, level, TABLES[what], _np_ptr(out)), "dec_mg_copy_table")
        if what == "verts":
            return out.reshape(nv, self.dim)
        if what == "tris":
            return out.reshape(nt, 3)
        if what in ("edges", "parents"):
            return out.reshape(ne, 2)
        if what in ("map_idx", "map_w"):
            return out.reshape(nf, 3)
        return out

    # ---- device calls ----------------------------------------------------
    def _vec(self, t, n, dtypes, name, device=None):
        torch = _torch()
        if not isinstance(t, torch.Tensor):
            raise TypeError(f"{name} must be a torch tensor")
        dev = self.device if device is None else device
        if t.device != dev:
            raise ValueError(f"{name} must live on {dev}")
        if t.dtype not in dtypes:
            raise TypeError(f"{name} has dtype {t.dtype}")
        if t.numel() != n or not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous with {n} entries")
        return C.c_void_p(t.data_ptr())

    def _stream(self):
        return C.c_void_p(_torch().cuda.current_stream(self.device).cuda_stream)

    def laplace0_apply(self, x, level=-1, out=None):
        torch = _torch()
        level = level % self.nlevels
        n = self.nv[level]
        prec = L.DEC_F64 if x.dtype == torch.float64 else L.DEC_F32
        px = self._vec(x, n, (torch.float64, torch.float32), "x")
        y = torch.empty_like(x) if out is None else out
        py = self._vec(y, n, (x.dtype,), "out")
        check(lib.dec_laplace0_apply(self._h, level, px, py, 1, prec, self._stream()), "dec_laplace0_apply")
        return y

    def residual(self, b, x, level=-1, out=None):
        torch = _torch()
        level = level % self.nlevels
        n = self.nv[level]
        prec = L.DEC_F64 if x.dtype == torch.float64 else L.DEC_F32
        pb = self._vec(b, n, (x.dtype,), "b")
        px = self._vec(x, n, (torch.float64, torch.float32), "x")
        r = torch.empty_like(x) if out is None else out
        pr = self._vec(r, n, (x.dtype,), "out")
        check(lib.dec_residual(self._h, level, pb, px, pr, 1, prec, self._stream()), "dec_residual")
        return r

    def vcycle(self, b, x):
        """x <- x + C(b - L x) in place (one multigrid cycle, precision of x)."""
        torch = _torch()
        prec = L.DEC_F64 if x.dtype == torch.float64 else L.DEC_F32
        pb = self._vec(b, self.n, (x.dtype,), "b")
        px = self._vec(x, self.n, (torch.float64, torch.float32), "x")
        check(lib.dec_mg_vcycle(self._h, pb, px, 1, prec, self._stream()), "dec_mg_vcycle")
        return x

    def _solve_opts(self, solver, mode, tol, maxit, warm_start, check_every, host_loop=False):
        o = L.dec_solve_opts()
        lib.dec_solve_default_opts(C.byref(o))
        o.solver = SOLVERS[solver]
        o.mode = MODES[mode]
        o.tol = float(tol)
        o.maxit = int(maxit)
        o.warm_start = 1 if warm_start else 0
        o.check_every = int(check_every)
        o.host_loop = 1 if host_loop else 0
        return o

    def solve(self, b, x=None, solver="mgpcg", mode="mixed", tol=1e-8, maxit=100, warm_start=False,
              check_every=1, raise_on_fail=True, host_loop=False):
        """Solve L x = b on the finest level; returns (x, SolveStats).

        b may be a CUDA or a CPU float64 tensor.  A CPU b goes through
        dec_solve_host: b is copied into the solver and the result into x, a
        CPU tensor (the one given, else a new one); pinned b and x make the
        copies DMA transfers.
        """
        torch = _torch()
        host = b.device.type == "cpu"
        cpu = torch.device("cpu")
        if x is None:
            x = torch.empty(self.n, dtype=torch.float64, device=cpu if host else self.device)
            warm_start = False
        pb = self._vec(b, self.n, (torch.float64,), "b", cpu if host else None)
        px = self._vec(x, self.n, (torch.float64,), "x", cpu if host else None)
        o = self._solve_opts(solver, mode, tol, maxit, warm_start, check_every, host_loop)
        st = L.dec_stats()
        fn = lib.dec_solve_host if host else lib.dec_solve
        rc = fn(self._h, pb, px, 1, C.byref(o), C.byref(st), self._stream())
        if rc not in (L.DEC_OK, L.DEC_ERR_NOT_CONVERGED) or (raise_on_fail and rc != L.DEC_OK):
            check(rc, "dec_solve_host" if host else "dec_solve")
        stats = SolveStats(st.iters, st.rel_res, st.rel_res0, rc, st.launches)
        return x, stats

    def solve_backward(self, u, grad_u, want_star1=True, solver="mgpcg", mode="mixed", tol=1e-8, maxit=100,
                       check_every=1):
        """Adjoint of x = L^-1 b: returns (dJ/db, dJ/d*1 or None, SolveStats)."""
        torch = _torch()
        pu = self._vec(u, self.n, (torch.float64,), "u")
        pg = self._vec(grad_u, self.n, (torch.float64,), "grad_u")
        gb = torch.empty_like(u)
        gs = torch.empty(self.ne[-1], dtype=torch.float64, device=self.device) if want_star1 else None
        o = self._solve_opts(solver, mode, tol, maxit, False, check_every)
        st = L.dec_stats()
        rc = lib.dec_solve_backward(self._h, pu, pg, C.c_void_p(gb.data_ptr()),
                                    C.c_void_p(gs.data_ptr()) if gs is not None else None,
                                    C.byref(o), C.byref(st), self._stream())
        check(rc, "dec_solve_backward")
        return gb, gs, SolveStats(st.iters, st.rel_res, st.rel_res0, rc, st.launches)

    def set_wait_limit(self, rounds=-1):
        """Bound (try_wait rounds) of the coarse cycle's device-side table-load wait; -1 restores the default,
        0 makes it give up at once (the solve then fails with DEC_ERR_CUDA and leaves x as it was)."""
        check(lib.dec_mg_set_wait_limit(self._h, int(rounds)), "dec_mg_set_wait_limit")

    def profile(self, enable=1):
        """Live CUDA-event timing of the solver's kernels (1: finest level, 2: all levels, 0: off)."""
        check(lib.dec_mg_profile(self._h, int(enable)), "dec_mg_profile")

    def profile_read(self):
        """List of dicts {kind, level, launches, total_ms, rows} accumulated since profile() was enabled."""
        buf = (L.dec_prof_entry * 256)()
        cnt = C.c_int()
        check(lib.dec_mg_profile_read(self._h, buf, 256, C.byref(cnt)), "dec_mg_profile_read")
        return [dict(kind=L.PROF_KINDS[e.kind], level=e.level, launches=e.launches, total_ms=e.total_ms,
                     rows=e.rows) for e in buf[: cnt.value]]

    def time_smooth(self, level=-1, reps=50):
        """(mean ms, algorithmic bytes) of one FP32 smoothing launch on `level`, back-to-back launches."""
        ms, by = C.c_double(), C.c_double()
        check(lib.dec_mg_time_smooth(self._h, int(level), int(reps), C.byref(ms), C.byref(by), self._stream()),
              "dec_mg_time_smooth")
        return ms.value, by.value

    def time_kernel(self, kind, level=-1, reps=50):
        """(mean ms, algorithmic bytes) of back-to-back launches of one kernel kind ("smooth", "smoothdots",
        "spmv64", "update"; all but "smooth" on the finest level)."""
        ms, by = C.c_double(), C.c_double()
        check(lib.dec_mg_time_kernel(self._h, L.PROF_KINDS.index(kind), int(level), int(reps), C.byref(ms),
                                     C.byref(by), self._stream()), "dec_mg_time_kernel")
        return ms.value, by.value

    # ---- porous convection (Sec. 3.2) ------------------------------------
    def _porous_params(self, dt, g=(0.0, -9.81, 0.0), alpha_rho0=0.0, phi=0.1, k_eta=1.0, kappa=2.0, tol=1e-8,
                       mode="mixed", maxit=100):
        p = L.dec_porous_params()
        lib.dec_porous_default_params(C.byref(p))
        for i in range(3):
            p.g[i] = float(g[i]) if i < len(g) else 0.0
        p.alpha_rho0, p.phi, p.k_eta, p.kappa, p.dt, p.tol = alpha_rho0, phi, k_eta, kappa, dt, tol
        p.mode, p.maxit = MODES[mode], maxit
        return p

    def porous_step(self, T, P, fixed, nsteps, dt, checkpoints=None, ckpt_every=100, **params):
        """Advance T (and the pressure P) by nsteps explicit porous-convection steps, in place."""
        torch = _torch()
        pT = self._vec(T, self.n, (torch.float64,), "T")
        pP = self._vec(P, self.n, (torch.float64,), "P")
        pf = self._vec(fixed, self.n, (torch.uint8,), "fixed")
        pc = None
        if checkpoints is not None:
            pc = self._vec(checkpoints, checkpoints.numel(), (torch.float64,), "checkpoints")
            if checkpoints.numel() < (nsteps // ckpt_every + 1) * self.n:
                raise ValueError("checkpoints too small")
        prm = self._porous_params(dt, **params)
        st = L.dec_stats()
        check(lib.dec_porous_step(self._h, pT, pP, pf, C.byref(prm), int(nsteps), pc, int(ckpt_every),
                                  C.byref(st), self._stream()), "dec_porous_step")
        return SolveStats(st.iters, st.rel_res, st.rel_res0, 0, st.launches)

    def porous_rk(self, T, P, fixed, t_end, dt0, rtol=1e-9, atol=1e-6, max_steps=10 ** 7, fixed_step=False,
                  **params):
        """Integrate the porous model adaptively (Tsit5, dec_porous_rk) from 0 to t_end, T and P in place.

        Returns a dict: naccept, nreject, nfev, t, dt, pressure_iters, pressure_rel_res."""
        torch = _torch()
        pT = self._vec(T, self.n, (torch.float64,), "T")
        pP = self._vec(P, self.n, (torch.float64,), "P")
        pf = self._vec(fixed, self.n, (torch.uint8,), "fixed")
        prm = self._porous_params(dt0, **params)
        st = L.dec_rk_stats()
        check(lib.dec_porous_rk(self._h, pT, pP, pf, C.byref(prm), float(t_end), float(dt0), float(rtol),
                                float(atol), int(max_steps), 1 if fixed_step else 0, C.byref(st), self._stream()),
              "dec_porous_rk")
        return {k: getattr(st, k) for k, _ in L.dec_rk_stats._fields_}

    def porous_backward(self, T0, P0, fixed, nsteps, grad_TN, dt, ckpt_every=100, **params):
        """dF/dT0 of T_N = step^N(T0) given dF/dT_N (checkpointed recomputation)."""
        torch = _torch()
        args = [self._vec(T0, self.n, (torch.float64,), "T0"), self._vec(P0, self.n, (torch.float64,), "P0"),
                self._vec(fixed, self.n, (torch.uint8,), "fixed")]
        pg = self._vec(grad_TN, self.n, (torch.float64,), "grad_TN")
        out = torch.empty_like(grad_TN)
        prm = self._porous_params(dt, **params)
        st = L.dec_stats()
        check(lib.dec_porous_backward(self._h, *args, C.byref(prm), int(nsteps), int(ckpt_every), pg,
                                      C.c_void_p(out.data_ptr()), C.byref(st), self._stream()),
              "dec_porous_backward")
        return out, SolveStats(st.iters, st.rel_res, st.rel_res0, 0, st.launches)

    def set_star1(self, star1):
        torch = _torch()
        p = self._vec(star1, self.ne[-1], (torch.float64,), "star1")
        check(lib.dec_mg_set_star1(self._h, p, self._stream()), "dec_mg_set_star1")


def _autograd_function():
    import torch

    class PoissonSolve(torch.autograd.Function):
        """u = L(*1)^-1 b with a hand-written backward: one adjoint solve on the same hierarchy.

        forward(b, star1): if star1 is given it becomes the finest-level *1 (dec_mg_set_star1);
        backward(dJ/du): dec_solve_backward returns dJ/db = *0 mu and dJ/d*1 = -(d0 mu)(d0 u),
        with L mu = *0^-1 dJ/du.
        """

        @staticmethod
        def forward(ctx, b, star1, hier, opts):
            if star1 is not None:
                hier.set_star1(star1.detach().contiguous())
            u, _ = hier.solve(b.detach().contiguous(), **opts)
            ctx.hier = hier
            ctx.opts = opts
            ctx.save_for_backward(u, star1 if star1 is not None else torch.empty(0, device=u.device))
            ctx.has_star1 = star1 is not None
            return u

        @staticmethod
        def backward(ctx, grad_u):
            u, star1 = ctx.saved_tensors
            hier = ctx.hier
            if ctx.has_star1:
                hier.set_star1(star1.contiguous())
            o = {k: v for k, v in ctx.opts.items() if k in ("solver", "mode", "tol", "maxit", "check_every")}
            want_s1 = ctx.has_star1 and ctx.needs_input_grad[1]
            gb, gs, _ = hier.solve_backward(u, grad_u.contiguous(), want_star1=want_s1, **o)
            return gb, (gs if want_s1 else None), None, None

    return PoissonSolve


_PS = None


def poisson_solve(b, star1=None, hier=None, **opts):
    """Differentiable solve of L(*1) u = b on `hier`'s finest level (torch.autograd.Function).

    b: float64 CUDA tensor [nv]; star1: optional float64 CUDA tensor [ne] of
    finest-level *1 values (differentiable); opts: solve options
    (solver, mode, tol, maxit).  Returns u.
    """
    global _PS
    if hier is None:
        raise ValueError("hier is required")
    if _PS is None:
        _PS = _autograd_function()
    return _PS.apply(b, star1, hier, opts)


@dataclass
class BatchStats:
    iters: int
    max_rel_res: float
    launches: int
    dof: int
    status: int


class Batch:
    """Many right-hand sides on many hierarchies, solved together (dec_batch_*).

    hierarchies: list of Hierarchy on the same device; nrhs: right-hand sides
    per hierarchy.  Vectors are given per mesh as float64 CUDA tensors of
    shape [nv, nrhs] (or flat [nv * nrhs]) in row-major order.
    """

    def __init__(self, hierarchies, nrhs, block=256, kgroup=0, nu=2, smoother="chebyshev", solver="mgpcg"):
        self.h = list(hierarchies)
        self.nrhs = [int(k) for k in nrhs]
        if len(self.h) != len(self.nrhs) or not self.h:
            raise ValueError("one right-hand-side count per hierarchy")
        if solver not in ("mg", "mgpcg"):
            raise ValueError("batched solver must be 'mg' or 'mgpcg'")
        o = L.dec_batch_opts()
        lib.dec_batch_default_opts(C.byref(o))
        o.block, o.kgroup, o.nu, o.smoother, o.solver = block, kgroup, nu, SMOOTHERS[smoother], SOLVERS[solver]
        self.opts = dict(block=block, kgroup=kgroup, nu=nu, smoother=smoother, solver=solver)
        arr = (C.c_void_p * len(self.h))(*[hh._h.value for hh in self.h])
        ks = (C.c_int * len(self.h))(*self.nrhs)
        bh = C.c_void_p()
        check(lib.dec_batch_create(arr, ks, len(self.h), C.byref(o), C.byref(bh)), "dec_batch_create")
        self._h = bh
        ng, nt, dof, nb = C.c_int(), C.c_int(), C.c_int64(), C.c_size_t()
        check(lib.dec_batch_info(self._h, C.byref(ng), C.byref(nt), C.byref(dof), C.byref(nb)), "dec_batch_info")
        self.ngroups, self.total_rhs, self.dof, self.device_bytes = ng.value, nt.value, dof.value, nb.value

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib.dec_batch_destroy(h)
            self._h = None

    def solve(self, bs, tol=1e-8, maxit=100, raise_on_fail=True):
        torch = _torch()
        xs, pb, px = [], [], []
        for hh, k, b in zip(self.h, self.nrhs, bs):
            pb.append(hh._vec(b.reshape(-1) if b.is_contiguous() else b, hh.n * k, (torch.float64,), "b"))
            x = torch.empty(hh.n, k, dtype=torch.float64, device=hh.device) if k > 1 else \
                torch.empty(hh.n, dtype=torch.float64, device=hh.device)
            xs.append(x)
            px.append(C.c_void_p(x.data_ptr()))
        ab = (C.c_void_p * len(pb))(*[p.value for p in pb])
        ax = (C.c_void_p * len(px))(*[p.value for p in px])
        st = L.dec_batch_stats()
        rc = lib.dec_batch_solve(self._h, ab, ax, float(tol), int(maxit), C.byref(st), self.h[0]._stream())
        if rc not in (L.DEC_OK, L.DEC_ERR_NOT_CONVERGED) or (raise_on_fail and rc != L.DEC_OK):
            check(rc, "dec_batch_solve")
        return xs, BatchStats(st.iters, st.max_rel_res, st.launches, st.dof, rc)

    def solve_backward(self, us, grad_us, want_star1=True, tol=1e-8, maxit=100, raise_on_fail=True):
        """Adjoint of every solve (dec_batch_solve_backward): per entry, the solutions u and dJ/du in the
        layout of solve(); returns (grad_b list, grad_star1 list or None, BatchStats)."""
        torch = _torch()
        gb, gs, pu, pg = [], [], [], []
        for hh, k, u, g in zip(self.h, self.nrhs, us, grad_us):
            pu.append(hh._vec(u.reshape(-1), hh.n * k, (torch.float64,), "u"))
            pg.append(hh._vec(g.reshape(-1), hh.n * k, (torch.float64,), "grad_u"))
            gb.append(torch.empty_like(u))
            if want_star1:
                ne = hh.ne[-1]
                gs.append(torch.empty(ne, k, dtype=torch.float64, device=hh.device) if k > 1 else
                          torch.empty(ne, dtype=torch.float64, device=hh.device))
        arr = lambda ps: (C.c_void_p * len(ps))(*[p.value for p in ps])  # noqa: E731
        pgb = [C.c_void_p(t.data_ptr()) for t in gb]
        pgs = arr([C.c_void_p(t.data_ptr()) for t in gs]) if want_star1 else None
        st = L.dec_batch_stats()
        rc = lib.dec_batch_solve_backward(self._h, arr(pu), arr(pg), arr(pgb), pgs, float(tol), int(maxit),
                                          C.byref(st), self.h[0]._stream())
        if rc not in (L.DEC_OK, L.DEC_ERR_NOT_CONVERGED) or (raise_on_fail and rc != L.DEC_OK):
            check(rc, "dec_batch_solve_backward")
        return gb, (gs if want_star1 else None), BatchStats(st.iters, st.max_rel_res, st.launches, st.dof, rc)

    def time_smooth(self, reps=20):
        """(mean ms, algorithmic bytes) of one batched finest-level smoothing launch."""
        ms, by = C.c_double(), C.c_double()
        check(lib.dec_batch_time_smooth(self._h, int(reps), C.byref(ms), C.byref(by), self.h[0]._stream()),
              "dec_batch_time_smooth")
        return ms.value, by.value


def tune_batch(hierarchies, nrhs, bs, tol=1e-8, maxit=100, candidates=None, reps=3):
    """Batch autotuner (dec_batch_tune): returns (best options dict, best ms, list of (options, ms))."""
    torch = _torch()
    hs = list(hierarchies)
    arr = (C.c_void_p * len(hs))(*[hh._h.value for hh in hs])
    ks = (C.c_int * len(hs))(*[int(k) for k in nrhs])
    xs = [torch.empty_like(b) for b in bs]
    ab = (C.c_void_p * len(bs))(*[b.data_ptr() for b in bs])
    ax = (C.c_void_p * len(xs))(*[x.data_ptr() for x in xs])
    inv = {v: k for k, v in SMOOTHERS.items()}
    if candidates is None:
        candidates = [dict(block=bl, kgroup=kg, nu=nu, smoother="chebyshev")
                      for bl in (128, 256, 512) for kg in (0, 8, 16, 32) for nu in (1, 2, 3)]
    cands = (L.dec_batch_opts * len(candidates))()
    for c, o in zip(cands, candidates):
        c.block, c.kgroup, c.nu, c.smoother = o["block"], o["kgroup"], o["nu"], SMOOTHERS[o["smoother"]]
        c.solver = SOLVERS[o.get("solver", "mgpcg")]
    times = (C.c_double * len(candidates))()
    best = L.dec_batch_opts()
    best_ms = C.c_double()
    check(lib.dec_batch_tune(arr, ks, len(hs), ab, ax, float(tol), int(maxit), cands, len(candidates), int(reps),
                             C.byref(best), C.byref(best_ms), times, hs[0]._stream()), "dec_batch_tune")
    inv_solver = {v: k for k, v in SOLVERS.items()}
    bo = dict(block=best.block, kgroup=best.kgroup, nu=best.nu, smoother=inv[best.smoother],
              solver=inv_solver[best.solver])
    return bo, best_ms.value, [(o, t) for o, t in zip(candidates, times)]
