"""Geometric multigrid for the DEC 0-form Laplacian on nested 1->4 subdivisions.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Paper passages followed:
  * interpolation is multiplication by the matrix M(f) of the geometric map
    whose column j holds the global barycentric coordinates of fine vertex j
    (Sec. 2.2, Def. of M(f); Sec. 2.2.1 interpolation example): a coarse
    vertex keeps its value, an edge midpoint gets the mean of its two parents;
  * restriction is the transpose of the row-normalization of M(f)
    (Sec. 2.2.1, Def. of the restriction operator and its 6x3 example),
    which preserves constants;
  * the operator is rediscretized on every level (Sec. 3.1.1, last paragraph)
    and V-cycles (or W-cycles) are layered between interpolation and
    restriction (Sec. 3.1.1, Sec. 3.1.2);
  * the stopping test is the relative residual ||L u - b||_2 / ||b||_2
    (Sec. 3.1.2); MG is used standalone and as the CG preconditioner
    (Sec. 3.1.2 cross-comparison).
Readings where the paper is silent:
  * smoothers: damped Jacobi (omega = 2/3), Chebyshev on [lo*lmax, hi*lmax]
    of D^-1 L with lmax from 10 power iterations, lexicographic Gauss-Seidel
    (the paper's), and multicolour Gauss-Seidel on a greedy colouring;
  * coarsest level: a dense direct solve -- interior block A_II under
    Dirichlet conditions, (A + m m^T / sum(*0)) under the constant-nullspace
    gauge, m = *0 1, followed by projection to *0-weighted mean zero;
  * CG: flexible (Polak-Ribiere) PCG in the *0 inner product, because the
    row-normalized restriction is not the *0-adjoint of interpolation and the
    V-cycle is therefore not exactly symmetric.
The paper prints no iterates or convergence factors, so the tests pin the
operators, the converged solutions (direct solves), the smoothers against
closed forms and library triangular solves, the greedy colouring against a
hand-worked fan, and the Jacobi V(2,2) rate against the spectral radius of
the cycle's error propagator assembled from plain dense matrices (0.3066 on
the unit square x5).  Individual iterates stay "parity unpinned".
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import dec
from .mesh import boundary_vertices, refine


@dataclass
class MGOptions:
    smoother: str = "jacobi"      # jacobi | chebyshev | gs | mcgs
    nu1: int = 2
    nu2: int = 2
    omega: float = 2.0 / 3.0
    cheby_lo: float = 0.3         # interval [cheby_lo * lmax, cheby_hi * lmax]
    cheby_hi: float = 1.1
    power_iters: int = 10
    gamma: int = 1                # 1: V-cycle, 2: W-cycle
    fcycle: bool = False          # F-cycle: coarse correction = an F-cycle then a V-cycle
    restriction: str = "rownorm"  # rownorm: the paper's; star0: *0-adjoint of interpolation


@dataclass
class Level:
    mesh: object
    star0: np.ndarray
    star1: np.ndarray
    A: sp.csr_matrix
    L: sp.csr_matrix
    free: np.ndarray              # bool: unknown (not a Dirichlet vertex)
    diag: np.ndarray              # diagonal of L (0 on Dirichlet rows)
    lmax: float = 0.0             # power-iteration estimate of lambda_max(D^-1 L)
    colors: np.ndarray = None     # greedy colouring of the stencil graph
    Lo: sp.csr_matrix = None      # lower triangle incl. diagonal (free rows/cols)
    Up: sp.csr_matrix = None      # strict upper triangle


@dataclass
class Hierarchy:
    levels: list                  # index 0 = coarsest used level
    P: list                       # P[l]: level l -> l+1 interpolation, n_{l+1} x n_l
    R: list                       # R[l]: level l+1 -> l restriction, n_l x n_{l+1}
    bc: str                       # "dirichlet" or "gauge"
    opts: MGOptions = field(default_factory=MGOptions)

    @property
    def finest(self):
        return self.levels[-1]


# ----------------------------------------------------------------------------
# transfers (Sec. 2.2.1)
# ----------------------------------------------------------------------------

def barycentric_matrix(nc, parents):
    """M(f): n_c x n_f, column j = global barycentric coordinates of fine vertex j."""
    E = len(parents)
    nf = nc + E
    rows = np.concatenate([np.arange(nc), parents[:, 0], parents[:, 1]])
    cols = np.concatenate([np.arange(nc), nc + np.arange(E), nc + np.arange(E)])
    vals = np.concatenate([np.ones(nc), np.full(E, 0.5), np.full(E, 0.5)])
    return sp.csr_matrix((vals, (rows, cols)), shape=(nc, nf))


def map_matrix_from_table(nc, idx, w):
    """M(f) (n_c x n_f) of a geometric map given per fine vertex j as up to three
    coarse vertices idx[j] and the barycentric coordinates w[j] of f(v_j) in
    their triangle (Sec. 2.2, Def. of M(f): column j holds the global
    barycentric coordinates of the image of fine vertex j)."""
    idx = np.asarray(idx).reshape(-1, 3)
    w = np.asarray(w, dtype=np.float64).reshape(-1, 3)
    nf = len(idx)
    cols = np.repeat(np.arange(nf), 3)
    return sp.csr_matrix((w.ravel(), (idx.ravel(), cols)), shape=(nc, nf))


def _map_matrix(nc, parents):
    """M(f) from a binary parent table or an explicit map matrix (cubic subdivision)."""
    return parents if sp.issparse(parents) else barycentric_matrix(nc, parents)


def interpolation(nc, parents):
    """Interpolation acting on column vectors: x_f = M(f)^T x_c."""
    return _map_matrix(nc, parents).T.tocsr()


def restriction(nc, parents):
    """Row-normalized M(f): r_c = rownorm(M(f)) r_f (the transpose of what acts on row vectors)."""
    M = _map_matrix(nc, parents)
    rs = np.asarray(M.sum(axis=1)).ravel()
    return (sp.diags(1.0 / rs) @ M).tocsr()


def restriction_star0(nc, parents, star0_c, star0_f):
    """*0-adjoint of interpolation: r_c = *0c^-1 M(f) *0f r_f, so <R r, e>_*0c = <r, P e>_*0f.

    Not the paper's operator (an option): with it the cycle is self-adjoint in
    the *0 inner product, as CG's preconditioner needs.
    """
    M = _map_matrix(nc, parents)
    return (sp.diags(1.0 / star0_c) @ M @ sp.diags(star0_f)).tocsr()


# ----------------------------------------------------------------------------
# hierarchy
# ----------------------------------------------------------------------------

def _hash_start(n):
    """Deterministic power-iteration start vector: (i * 2654435761 mod 2^32) / 2^32 - 1/2."""
    i = np.arange(n, dtype=np.uint64)
    return ((i * np.uint64(2654435761)) % np.uint64(2 ** 32)).astype(np.float64) / 2.0 ** 32 - 0.5


def power_lmax(L, diag, free, iters):
    """Estimate of lambda_max(D^-1 L) on the free vertices: ||w|| / ||v|| after `iters` steps."""
    inv = np.where(free, 1.0 / np.where(free, diag, 1.0), 0.0)
    v = _hash_start(L.shape[0]) * free
    lam = 0.0
    for _ in range(iters):
        w = inv * (L @ (v * free))
        lam = np.linalg.norm(w) / np.linalg.norm(v)
        v = w / np.linalg.norm(w)
    return lam


def greedy_colors(mesh):
    """Colour of v = smallest colour not taken by a lower-numbered neighbour (stencil graph)."""
    nv = mesh.nv
    nbrs = [[] for _ in range(nv)]
    for a, b in mesh.edges:
        nbrs[b].append(a)
        nbrs[a].append(b)
    col = np.full(nv, -1, dtype=np.int64)
    for v in range(nv):
        taken = {col[u] for u in nbrs[v] if u < v}
        c = 0
        while c in taken:
            c += 1
        col[v] = c
    return col


def make_level(mesh, bc, star1_scale=None, opts=None, with_gs=False):
    opts = opts or MGOptions()
    s0 = dec.hodge_star0(mesh)
    s1 = dec.hodge_star1(mesh, star1_scale)
    A = dec.stiffness(mesh, s1)
    L = dec.laplacian(mesh, s0, s1)
    if bc == "dirichlet":
        free = ~boundary_vertices(mesh)
    elif bc == "gauge":
        free = np.ones(mesh.nv, dtype=bool)
    else:
        raise ValueError(bc)
    diag = L.diagonal() * free
    lev = Level(mesh, s0, s1, A, L, free, diag)
    lev.lmax = power_lmax(L, diag, free, opts.power_iters)
    if with_gs:
        F = sp.diags(free.astype(np.float64))
        Lf = (F @ L @ F).tocsr() + sp.diags((~free).astype(np.float64))
        lev.Lo = sp.tril(Lf, k=0).tocsr()
        lev.Up = sp.triu(Lf, k=1).tocsr()
        lev.colors = greedy_colors(mesh)
    return lev


def build_hierarchy(verts, tris, nsub, nlevels, bc, sphere=False, star1_scale=None,
                    opts=None, meshes=None, parents=None, order="edge", scheme="binary"):
    """Subdivide nsub times and keep the finest nlevels meshes as the MG hierarchy.

    star1_scale (per finest edge) multiplies *1 on the finest level only;
    coarser levels are rediscretized from their own geometry.  order is the
    numbering of each level's new vertices (see oracle.mesh.subdivide);
    scheme is "binary" (1->4) or "cubic" (1->9, oracle.mesh.subdivide_cubic).
    """
    opts = opts or MGOptions()
    if meshes is None:
        meshes, parents = refine(verts, tris, nsub, sphere=sphere, order=order, scheme=scheme)
    if not 1 <= nlevels <= nsub + 1:
        raise ValueError("nlevels out of range")
    first = nsub + 1 - nlevels
    with_gs = opts.smoother in ("gs", "mcgs")
    levels = []
    for i in range(first, nsub + 1):
        scale = star1_scale if i == nsub else None
        levels.append(make_level(meshes[i], bc, scale, opts, with_gs))
    P, R = [], []
    for i in range(first, nsub):
        nc = meshes[i].nv
        P.append(interpolation(nc, parents[i]))
        if opts.restriction == "star0":
            lc, lf = levels[i - first], levels[i - first + 1]
            R.append(restriction_star0(nc, parents[i], lc.star0, lf.star0))
        else:
            R.append(restriction(nc, parents[i]))
    return Hierarchy(levels, P, R, bc, opts)


# ----------------------------------------------------------------------------
# smoothers
# ----------------------------------------------------------------------------

def residual(lev, b, x):
    """r = b - L x on free vertices, 0 on Dirichlet vertices."""
    return lev.free * (b - lev.L @ (lev.free * x))


def jacobi(lev, b, x, omega, nu):
    inv = np.where(lev.free, 1.0 / np.where(lev.free, lev.diag, 1.0), 0.0)
    for _ in range(nu):
        x = x + omega * inv * residual(lev, b, x)
    return x


def chebyshev_coefficients(lmax, lo, hi, nu):
    """(c_k, e_k): step k uses d_k = c_k d_{k-1} + e_k D^-1 (b - L x_k),  x_{k+1} = x_k + d_k.

    Chebyshev semi-iteration for D^-1 L on the interval [lo*lmax, hi*lmax].
    """
    a, b = lo * lmax, hi * lmax
    theta = 0.5 * (b + a)
    delta = 0.5 * (b - a)
    sigma = theta / delta
    coeffs = [(0.0, 1.0 / theta)]
    rho_prev = 1.0 / sigma
    for _ in range(1, nu):
        rho = 1.0 / (2.0 * sigma - rho_prev)
        coeffs.append((rho * rho_prev, 2.0 * rho / delta))
        rho_prev = rho
    return coeffs


def chebyshev(lev, b, x, nu, lo, hi):
    inv = np.where(lev.free, 1.0 / np.where(lev.free, lev.diag, 1.0), 0.0)
    d = np.zeros_like(x)
    for c, e in chebyshev_coefficients(lev.lmax, lo, hi, nu):
        d = c * d + e * inv * residual(lev, b, x)
        x = x + d
    return x


def gauss_seidel(lev, b, x, nu):
    """Forward lexicographic Gauss-Seidel: (D + lower) x_new = b - upper x_old."""
    bf = lev.free * b
    for _ in range(nu):
        x = spla.spsolve_triangular(lev.Lo, bf - lev.Up @ (lev.free * x), lower=True)
        x = lev.free * x
    return x


def mc_gauss_seidel(lev, b, x, nu):
    """Gauss-Seidel over the greedy colour classes in increasing colour order."""
    inv = np.where(lev.free, 1.0 / np.where(lev.free, lev.diag, 1.0), 0.0)
    ncol = int(lev.colors.max()) + 1
    for _ in range(nu):
        for c in range(ncol):
            sel = lev.colors == c
            r = residual(lev, b, x)
            x = np.where(sel, x + inv * r, x)
    return x


def smooth(h, lev, b, x, nu):
    o = h.opts
    if nu == 0:
        return x
    if o.smoother == "jacobi":
        return jacobi(lev, b, x, o.omega, nu)
    if o.smoother == "chebyshev":
        return chebyshev(lev, b, x, nu, o.cheby_lo, o.cheby_hi)
    if o.smoother == "gs":
        return gauss_seidel(lev, b, x, nu)
    if o.smoother == "mcgs":
        return mc_gauss_seidel(lev, b, x, nu)
    raise ValueError(o.smoother)


# ----------------------------------------------------------------------------
# coarse solve, gauge
# ----------------------------------------------------------------------------

def star0_mean(lev, x):
    """*0-weighted mean of x over the free vertices."""
    w = lev.star0 * lev.free
    return np.dot(w, x) / np.sum(w)


def project_mean_zero(lev, x):
    return lev.free * (x - star0_mean(lev, x))


def coarse_solve(h, lev, b):
    """Dense direct solve of L x = b on the coarsest level (LU with partial pivoting)."""
    if h.bc == "dirichlet":
        idx = np.flatnonzero(lev.free)
        Aii = lev.A[idx][:, idx].toarray()
        x = np.zeros(len(b))
        x[idx] = np.linalg.solve(Aii, lev.star0[idx] * b[idx])
        return x
    m = lev.star0
    K = lev.A.toarray() + np.outer(m, m) / np.sum(m)
    x = np.linalg.solve(K, lev.star0 * b)
    return project_mean_zero(lev, x)


# ----------------------------------------------------------------------------
# cycles and solvers
# ----------------------------------------------------------------------------

def vcycle(h, b, x, l=None, kind=None):
    """One cycle x <- x + C(b - L x) on level l (default: finest).

    kind "gamma": the coarse correction is gamma cycles of the same kind
    (gamma = 1: V-cycle, 2: W-cycle); "V": one V-cycle below; "F": the coarse
    correction is an F-cycle followed by a V-cycle.  Default: "F" if
    opts.fcycle else "gamma".  On the coarsest level the solve is exact.
    """
    if l is None:
        l = len(h.levels) - 1
    if kind is None:
        kind = "F" if h.opts.fcycle else "gamma"
    lev = h.levels[l]
    if l == 0:
        return x + coarse_solve(h, lev, residual(lev, b, x))
    x = smooth(h, lev, b, x, h.opts.nu1)
    r = residual(lev, b, x)
    clev = h.levels[l - 1]
    rc = clev.free * (h.R[l - 1] @ r)
    ec = np.zeros(clev.mesh.nv)
    if kind == "F":
        ec = vcycle(h, rc, ec, l - 1, "F")
        ec = vcycle(h, rc, ec, l - 1, "V")
    else:
        for _ in range(h.opts.gamma if kind == "gamma" else 1):
            ec = vcycle(h, rc, ec, l - 1, kind)
    x = x + lev.free * (h.P[l - 1] @ ec)
    x = smooth(h, lev, b, x, h.opts.nu2)
    return x


def rel_residual(lev, b, x):
    return np.linalg.norm(residual(lev, b, x)) / np.linalg.norm(lev.free * b)


@dataclass
class SolveResult:
    x: np.ndarray
    iters: int
    rel_res: float
    history: list


def prepare_rhs(h, b):
    lev = h.finest
    b = lev.free * np.asarray(b, dtype=np.float64)
    if h.bc == "gauge":
        b = project_mean_zero(lev, b)
    return b


def mg_solve(h, b, tol, maxit, x0=None):
    """Standalone multigrid: repeat cycles until the relative residual is <= tol."""
    lev = h.finest
    b = prepare_rhs(h, b)
    x = np.zeros_like(b) if x0 is None else lev.free * x0
    if h.bc == "gauge":
        x = project_mean_zero(lev, x)
    hist = [rel_residual(lev, b, x)]
    it = 0
    while hist[-1] > tol and it < maxit:
        x = vcycle(h, b, x)
        if h.bc == "gauge":
            x = project_mean_zero(lev, x)
        it += 1
        hist.append(rel_residual(lev, b, x))
    return SolveResult(x, it, hist[-1], hist)


def inner(lev, x, y):
    """The *0 inner product <x, y> = sum_v *0_v x_v y_v over the free vertices."""
    return np.sum(lev.star0 * lev.free * x * y)


def pcg_solve(h, b, tol, maxit, x0=None, precondition=True):
    """Flexible preconditioned CG in the *0 inner product, one cycle per preconditioner call."""
    lev = h.finest
    b = prepare_rhs(h, b)
    bn = np.linalg.norm(b)
    x = np.zeros_like(b) if x0 is None else lev.free * x0
    if h.bc == "gauge":
        x = project_mean_zero(lev, x)
    r = residual(lev, b, x)

    def M(r):
        z = vcycle(h, r, np.zeros_like(r)) if precondition else r.copy()
        return project_mean_zero(lev, z) if h.bc == "gauge" else z

    hist = [np.linalg.norm(r) / bn if bn > 0 else 0.0]
    if hist[-1] <= tol:
        return SolveResult(x, 0, hist[-1], hist)
    z = M(r)
    p = z.copy()
    rz = inner(lev, r, z)
    it = 0
    while it < maxit:
        q = lev.free * (lev.L @ p)
        alpha = rz / inner(lev, p, q)
        x = x + alpha * p
        r = r - alpha * q
        it += 1
        hist.append(np.linalg.norm(r) / bn)
        if hist[-1] <= tol:
            break
        z_new = M(r)
        rz_new = inner(lev, r, z_new)
        beta = (rz_new - inner(lev, r, z)) / rz
        p = z_new + beta * p
        z, rz = z_new, rz_new
    return SolveResult(x, it, hist[-1], hist)


def direct_solve(h, b):
    """u* = L^-1 b on the finest level by a sparse direct factorization (reference solution)."""
    lev = h.finest
    b = prepare_rhs(h, b)
    if h.bc == "dirichlet":
        idx = np.flatnonzero(lev.free)
        Aii = lev.A[idx][:, idx].tocsc()
        x = np.zeros(len(b))
        x[idx] = spla.spsolve(Aii, lev.star0[idx] * b[idx])
        return x
    # pin one vertex, solve, then move to the *0-mean-zero representative
    n = len(b)
    idx = np.arange(1, n)
    A = lev.A.tocsr()
    x = np.zeros(n)
    x[idx] = spla.spsolve(A[idx][:, idx].tocsc(), (lev.star0 * b)[idx])
    return project_mean_zero(lev, x)


def star0_norm(lev, x):
    return np.sqrt(inner(lev, x, x))


def convergence_factor(hist):
    """Geometric-mean residual reduction per cycle over the recorded history."""
    h = [v for v in hist if v > 0]
    if len(h) < 2:
        return 0.0
    return (h[-1] / h[0]) ** (1.0 / (len(h) - 1))
