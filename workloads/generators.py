"""Base meshes and seeded inputs for the workloads the solver is measured on.

Every random quantity is drawn from ``numpy.random.default_rng(seed)`` so the
CPU oracle and the GPU path see identical bytes.  Nothing here depends on the
subdivision, the Hodge stars or any solver step: functions that need vertex
positions of a refined mesh take them as an argument.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "unit_square",
    "grid_mesh",
    "icosahedron",
    "one_triangle",
    "rhs_sin_square",
    "u_sin_square",
    "u_target_square",
    "uniform_field",
    "sh_coefficients",
    "sh_sum",
    "lognormal_factors",
    "porous_initial_T",
    "gaussian_initial_T",
    "random_directions",
    "heptagon_fan",
    "jittered_square_levels",
    "WORKLOADS",
]


def unit_square():
    """Unit square [0,1]^2 split into two right triangles along (0,0)-(1,1).

    Returns (verts float64 [4,2], tris int32 [2,3]), counter-clockwise.
    """
    verts = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [0.0, 1.0]])
    tris = np.array([[0, 1, 2], [0, 2, 3]], dtype=np.int32)
    return verts, tris


def grid_mesh(nx, ny, x0=0.0, x1=1.0, y0=0.0, y1=1.0):
    """Structured nx-by-ny vertex grid, each cell split along its (i,j)-(i+1,j+1) diagonal.

    Vertex (i, j) (column i, row j) has id j*nx + i.  Triangles are
    counter-clockwise.  A 25x25 grid has the 625 vertices, 1,776 edges and
    1,152 triangles of the paper's cross-comparison base mesh (Sec. 3.1.2).
    """
    xs = np.linspace(x0, x1, nx)
    ys = np.linspace(y0, y1, ny)
    X, Y = np.meshgrid(xs, ys)
    verts = np.stack([X.ravel(), Y.ravel()], axis=1)
    tris = []
    for j in range(ny - 1):
        for i in range(nx - 1):
            v00 = j * nx + i
            v10 = v00 + 1
            v01 = v00 + nx
            v11 = v01 + 1
            tris.append((v00, v10, v11))
            tris.append((v00, v11, v01))
    return verts, np.array(tris, dtype=np.int32)


_ICO_RAW = np.array(
    [
        [-1.618033988749895, 0.0, -1.0],
        [-1.618033988749895, 0.0, 1.0],
        [-1.0, -1.618033988749895, 0.0],
        [-1.0, 1.618033988749895, 0.0],
        [0.0, -1.0, -1.618033988749895],
        [0.0, -1.0, 1.618033988749895],
        [0.0, 1.0, -1.618033988749895],
        [0.0, 1.0, 1.618033988749895],
        [1.0, -1.618033988749895, 0.0],
        [1.0, 1.618033988749895, 0.0],
        [1.618033988749895, 0.0, -1.0],
        [1.618033988749895, 0.0, 1.0],
    ]
)
_ICO_TRIS = np.array(
    [
        (0, 2, 1), (0, 1, 3), (0, 4, 2), (0, 3, 6), (0, 6, 4),
        (1, 2, 5), (1, 7, 3), (1, 5, 7), (2, 4, 8), (2, 8, 5),
        (3, 9, 6), (3, 7, 9), (4, 6, 10), (4, 10, 8), (5, 11, 7),
        (5, 8, 11), (6, 9, 10), (7, 11, 9), (8, 10, 11), (9, 11, 10),
    ],
    dtype=np.int32,
)


def icosahedron():
    """Regular icosahedron on the unit sphere, outward-oriented.

    Vertices are the cyclic permutations of (0, +-1, +-phi), divided by their
    norm sqrt(1 + phi^2); the 20 faces are listed explicitly.
    Returns (verts float64 [12,3], tris int32 [20,3]).
    """
    nrm = np.sqrt(1.0 + ((1.0 + 5.0 ** 0.5) / 2.0) ** 2)
    return _ICO_RAW / nrm, _ICO_TRIS.copy()


def one_triangle():
    """A single triangle (a, b, c) = ((0,0), (1,0), (0,1))."""
    return np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]]), np.array([[0, 1, 2]], dtype=np.int32)


# ----------------------------------------------------------------------------
# right-hand sides and fields
# ----------------------------------------------------------------------------

def rhs_sin_square(xy):
    """f = -Delta u for u = sin(pi x) sin(pi y):  2 pi^2 sin(pi x) sin(pi y)."""
    x, y = xy[:, 0], xy[:, 1]
    return 2.0 * math.pi ** 2 * np.sin(math.pi * x) * np.sin(math.pi * y)


def u_sin_square(xy):
    x, y = xy[:, 0], xy[:, 1]
    return np.sin(math.pi * x) * np.sin(math.pi * y)


def u_target_square(xy):
    """Target field sin(2 pi x) sin(pi y) of the differentiable-solve workload."""
    x, y = xy[:, 0], xy[:, 1]
    return np.sin(2.0 * math.pi * x) * np.sin(math.pi * y)


def uniform_field(n, seed, lo=-1.0, hi=1.0):
    return np.random.default_rng(seed).uniform(lo, hi, size=n)


def sh_coefficients(seed, lmax=16):
    """N(0,1) coefficients for the real spherical harmonics of degree 1..lmax.

    Ordered by degree l = 1..lmax, then order m = -l..l: (lmax+1)^2 - 1 values.
    """
    return np.random.default_rng(seed).standard_normal((lmax + 1) ** 2 - 1)


def _assoc_legendre(lmax, x):
    """P_l^m(x) for 0 <= m <= l <= lmax (Condon-Shortley phase), via the standard three-term recurrences."""
    P = {}
    s = np.sqrt(np.maximum(0.0, 1.0 - x * x))
    pmm = np.ones_like(x)
    for m in range(lmax + 1):
        if m > 0:
            pmm = -(2 * m - 1) * s * pmm
        P[(m, m)] = pmm
        if m + 1 <= lmax:
            P[(m + 1, m)] = x * (2 * m + 1) * pmm
        for l in range(m + 2, lmax + 1):
            P[(l, m)] = ((2 * l - 1) * x * P[(l - 1, m)] - (l + m - 1) * P[(l - 2, m)]) / (l - m)
    return P


def sh_sum(pos, coeffs, lmax=16):
    """Sum of orthonormal real spherical harmonics Y_lm(pos/|pos|) weighted by coeffs.

    pos: [n,3] points (projected to the unit sphere here).  Degree 0 is not
    included, so the continuous field has zero mean on the sphere.
    """
    r = np.sqrt(np.sum(pos * pos, axis=1))
    x, y, z = pos[:, 0] / r, pos[:, 1] / r, pos[:, 2] / r
    ph = np.arctan2(y, x)
    P = _assoc_legendre(lmax, z)
    out = np.zeros(len(pos))
    k = 0
    for l in range(1, lmax + 1):
        for m in range(-l, l + 1):
            am = abs(m)
            norm = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - am) / math.factorial(l + am))
            if m == 0:
                Y = norm * P[(l, 0)]
            elif m > 0:
                Y = math.sqrt(2.0) * norm * P[(l, am)] * np.cos(am * ph)
            else:
                Y = math.sqrt(2.0) * norm * P[(l, am)] * np.sin(am * ph)
            out += coeffs[k] * Y
            k += 1
    return out


def lognormal_factors(n, seed, sigma=0.5):
    """Per-edge multiplicative factors exp(sigma z), z ~ N(0,1)."""
    return np.exp(sigma * np.random.default_rng(seed).standard_normal(n))


def porous_initial_T(xy, seed, amp=1e-3):
    """Conductive profile T = 100 - 200 y plus amp*U[-1,1] noise away from the top and bottom rows."""
    y = xy[:, 1]
    T = 100.0 - 200.0 * y
    noise = np.random.default_rng(seed).uniform(-1.0, 1.0, size=len(y))
    inner = (y > 0.0) & (y < 1.0)
    return T + amp * noise * inner


def gaussian_initial_T(xy, center, cov=0.5, scale=400.0):
    """Scaled bivariate normal density with covariance cov*I (the paper's porous-convection start, Sec. 3.2.2)."""
    d2 = (xy[:, 0] - center[0]) ** 2 + (xy[:, 1] - center[1]) ** 2
    return scale * np.exp(-0.5 * d2 / cov) / (2.0 * math.pi * cov)


def random_directions(k, n, seed):
    """k seeded N(0,1) direction vectors of length n, each scaled to unit 2-norm."""
    D = np.random.default_rng(seed).standard_normal((k, n))
    return D / np.linalg.norm(D, axis=1, keepdims=True)


# Named workloads: sizes and seeds of the measured configurations.
WORKLOADS = {
    "square_l5_dirichlet": dict(base="unit_square", nsub=5, nlevels=5, bc="dirichlet",
                                 rhs="sin_square", tol=1e-10, solver="mg"),
    "icosphere_l8_mgpcg": dict(base="icosahedron", nsub=8, nlevels=7, bc="gauge",
                                rhs="sh16", rhs_seed=1, tol=1e-8, solver="mgpcg"),
    "square_l10_adjoint": dict(base="unit_square", nsub=10, bc="dirichlet", star1_seed=2,
                                rhs_seed=3, fd_seed=4, tol=1e-8),
    "square_l9_porous": dict(base="unit_square", nsub=9, bc="gauge", T0_seed=0, steps=2000),
}


def heptagon_fan():
    """A centre vertex joined to 7 points on the unit circle: valence 7 at the centre.

    After subdivision the centre keeps valence 7, so every level has 7
    stencil slots per row; used to exercise meshes whose valence is not 6.
    """
    ang = 2.0 * math.pi * np.arange(7) / 7.0
    verts = np.concatenate([[[0.0, 0.0]], np.stack([np.cos(ang), np.sin(ang)], axis=1)])
    tris = np.array([[0, 1 + k, 1 + (k + 1) % 7] for k in range(7)], dtype=np.int32)
    return verts, tris


def jittered_square_levels(nlevels, seed, base=2, amp=0.15):
    """Non-nested meshes of the unit square and the geometric maps between them.

    Level l (0 = coarsest) is the (2^(base+l) + 1)^2 grid_mesh with each interior
    vertex moved by amp * h * U[-1,1]^2 (h its grid spacing, seeded by seed + l),
    so no level's vertices lie on the next coarser mesh's edges: the levels are
    not related by subdivision.  The map from level l+1 to level l sends every
    vertex to its own position; it is described, as a caller of a geometric-map
    hierarchy supplies it, by the coarse triangle that contains the position and
    the position's barycentric coordinates there: maps_idx[l], maps_w[l] are
    [nv(l+1), 3] arrays (int32 coarse vertex ids, float64 weights).

    Returns (meshes, maps_idx, maps_w), meshes a list of (verts, tris).
    """
    meshes = []
    for lev in range(nlevels):
        n = 2 ** (base + lev) + 1
        v, t = grid_mesh(n, n)
        h = 1.0 / (n - 1)
        inner = (v[:, 0] > 0.0) & (v[:, 0] < 1.0) & (v[:, 1] > 0.0) & (v[:, 1] < 1.0)
        d = np.random.default_rng(seed + lev).uniform(-1.0, 1.0, size=v.shape) * (amp * h)
        meshes.append((v + d * inner[:, None], t))
    maps_idx, maps_w = [], []
    for lev in range(nlevels - 1):
        cv, ct = meshes[lev]
        fv, _ = meshes[lev + 1]
        nc = 2 ** (base + lev) + 1
        H = 1.0 / (nc - 1)
        idx = np.zeros((len(fv), 3), dtype=np.int32)
        wts = np.zeros((len(fv), 3))
        for j, p in enumerate(fv):
            ci = min(int(p[0] / H), nc - 2)
            cj = min(int(p[1] / H), nc - 2)
            best = None
            # the containing triangle lies in this grid cell or a neighbouring one (jitter < H / 2)
            for dj in (-1, 0, 1):
                for di in (-1, 0, 1):
                    i2, j2 = ci + di, cj + dj
                    if not (0 <= i2 < nc - 1 and 0 <= j2 < nc - 1):
                        continue
                    for tri in ct[2 * (j2 * (nc - 1) + i2): 2 * (j2 * (nc - 1) + i2) + 2]:
                        a, b, c = cv[tri[0]], cv[tri[1]], cv[tri[2]]
                        m = np.array([[b[0] - a[0], c[0] - a[0]], [b[1] - a[1], c[1] - a[1]]])
                        s, r = np.linalg.solve(m, p - a)
                        lam = np.array([1.0 - s - r, s, r])
                        if best is None or lam.min() > best[1].min():
                            best = (tri, lam)
            tri, lam = best
            lam = np.where(np.abs(lam) < 1e-14, 0.0, lam)
            idx[j] = tri
            wts[j] = lam / lam.sum()
        maps_idx.append(idx)
        maps_w.append(wts)
    return meshes, maps_idx, maps_w

