"""Embedded simplicial complexes, signed incidence and 1->4 midpoint subdivision.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Follows Sec. 2.1 (the definition of an embedded 2-simplicial complex: face
maps E->V and T->E, no duplicate simplices, every vertex and edge in some
triangle) and Sec. 3.1.1 (d0 and the boundary matrix d1, with d1 d0 = 0).
Readings, where the paper fixes no convention:
  * an edge is stored once as (lo, hi) with lo < hi; edges are numbered in
    lexicographic (lo, hi) order; (d0)_{e,lo} = -1, (d0)_{e,hi} = +1;
  * (d1)_{t,e} = +1 when the triangle's cyclic order v0->v1->v2->v0 traverses
    e from lo to hi, else -1;
  * subdivision keeps coarse vertex ids, numbers the midpoint of coarse edge e
    as n_coarse + e, and splits t = (a,b,c) into
    4t+0 = (a, m_ab, m_ca), 4t+1 = (m_ab, b, m_bc), 4t+2 = (m_ca, m_bc, c),
    4t+3 = (m_ab, m_bc, m_ca)   (Sec. 2.2.1, binary subdivision).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp


class MeshError(ValueError):
    pass


@dataclass
class Mesh:
    verts: np.ndarray       # [V, dim] float64, dim in {2, 3}
    tris: np.ndarray        # [T, 3] int64
    edges: np.ndarray       # [E, 2] int64, lo < hi, lexicographic
    tri_edges: np.ndarray   # [T, 3] edge ids of (v0v1, v1v2, v2v0)
    tri_signs: np.ndarray   # [T, 3] +-1 orientation of each triangle edge

    @property
    def nv(self):
        return len(self.verts)

    @property
    def ne(self):
        return len(self.edges)

    @property
    def nt(self):
        return len(self.tris)


def validate(nv, tris):
    """Reject complexes that break the definition of Sec. 2.1 (plus manifold edges).

    Checks: indices in range, three distinct vertices per triangle, no two
    triangles on the same vertex set, every vertex in some triangle, and each
    edge in at most two triangles.
    """
    tris = np.asarray(tris, dtype=np.int64)
    if tris.ndim != 2 or tris.shape[1] != 3 or len(tris) == 0:
        raise MeshError("triangles must be a non-empty [T,3] array")
    if tris.min() < 0 or tris.max() >= nv:
        raise MeshError("triangle vertex index out of range")
    a, b, c = tris[:, 0], tris[:, 1], tris[:, 2]
    if np.any((a == b) | (b == c) | (a == c)):
        raise MeshError("a triangle repeats a vertex")
    key = np.sort(tris, axis=1)
    key = (key[:, 0] * nv + key[:, 1]) * nv + key[:, 2]
    if len(np.unique(key)) != len(key):
        raise MeshError("two triangles share the same vertex set")
    used = np.zeros(nv, dtype=bool)
    used[tris.ravel()] = True
    if not used.all():
        raise MeshError("a vertex lies in no triangle")
    pairs = np.sort(np.concatenate([tris[:, [0, 1]], tris[:, [1, 2]], tris[:, [2, 0]]]), axis=1)
    _, counts = np.unique(pairs[:, 0] * nv + pairs[:, 1], return_counts=True)
    if counts.max() > 2:
        raise MeshError("an edge lies in more than two triangles")


def build_mesh(verts, tris):
    """Enumerate the canonical edges of a triangle list and the T->E face map."""
    verts = np.asarray(verts, dtype=np.float64)
    tris = np.asarray(tris, dtype=np.int64)
    validate(len(verts), tris)
    T = len(tris)
    # the three edges of each triangle in cyclic order: (v0,v1), (v1,v2), (v2,v0)
    src = np.stack([tris[:, 0], tris[:, 1], tris[:, 2]], axis=1)
    dst = np.stack([tris[:, 1], tris[:, 2], tris[:, 0]], axis=1)
    lo = np.minimum(src, dst)
    hi = np.maximum(src, dst)
    signs = np.where(src < dst, 1, -1).astype(np.int64)
    # lexicographic (lo, hi) order is the order of the key lo * V + hi
    nv = len(verts)
    key = lo.ravel() * nv + hi.ravel()
    ukey, inverse = np.unique(key, return_inverse=True)
    edges = np.stack([ukey // nv, ukey % nv], axis=1)
    tri_edges = inverse.reshape(T, 3).astype(np.int64)
    return Mesh(verts, tris, edges.astype(np.int64), tri_edges, signs)


def d0_matrix(mesh):
    """Signed E x V incidence: (d0 u)_e = u_hi - u_lo  (the discrete gradient)."""
    E = mesh.ne
    rows = np.repeat(np.arange(E), 2)
    cols = mesh.edges.ravel()
    vals = np.tile(np.array([-1, 1], dtype=np.int64), E)
    return sp.csr_matrix((vals, (rows, cols)), shape=(E, mesh.nv), dtype=np.int64)


def d1_matrix(mesh):
    """Signed T x E boundary matrix of the triangles (the discrete curl)."""
    T = mesh.nt
    rows = np.repeat(np.arange(T), 3)
    return sp.csr_matrix((mesh.tri_signs.ravel(), (rows, mesh.tri_edges.ravel())),
                         shape=(T, mesh.ne), dtype=np.int64)


def boundary_edges(mesh):
    """Boolean [E]: edges that lie in exactly one triangle."""
    cnt = np.bincount(mesh.tri_edges.ravel(), minlength=mesh.ne)
    return cnt == 1


def boundary_vertices(mesh):
    """Boolean [V]: endpoints of boundary edges."""
    bv = np.zeros(mesh.nv, dtype=bool)
    be = boundary_edges(mesh)
    bv[mesh.edges[be].ravel()] = True
    return bv


def morton_keys(verts):
    """Z-order keys of points: each coordinate quantized on the points' bounding box to
    B bits (B = 21 in 3-D, 31 in 2-D), q = floor((x - lo) * ((2^B - 1) / (hi - lo)))
    clamped to [0, 2^B - 1], and the bits interleaved (axis 0 in the lowest bit).
    Every step is an exact or IEEE-rounded float64 operation, so any implementation
    that performs the same operations gets the same keys."""
    dim = verts.shape[1]
    B = 21 if dim == 3 else 31
    top = float((1 << B) - 1)
    keys = np.zeros(len(verts), dtype=np.uint64)
    for d in range(dim):
        x = verts[:, d]
        lo, hi = float(x.min()), float(x.max())
        scale = top / (hi - lo) if hi > lo else 0.0
        q = np.floor((x - lo) * scale)
        q = np.clip(q, 0.0, top).astype(np.uint64)
        for b in range(B):
            keys |= ((q >> np.uint64(b)) & np.uint64(1)) << np.uint64(dim * b + d)
    return keys


def subdivide(mesh, sphere=False, order="edge"):
    """One 1->4 midpoint subdivision (Sec. 2.2.1, binary subdivision).

    Returns (fine Mesh, parents [E_coarse, 2]).  Coarse vertices keep their
    ids, so level-l vertices are a prefix of every finer level.  The new
    vertex n_c + k is the midpoint of coarse edge parents[k]:
      order="edge":   k = e, the canonical coarse edge order;
      order="morton": the midpoints sorted (stably) by the Morton key of their
                      coordinates, quantized on the new points' bounding box
                      (a space-filling-curve order that keeps neighbours close
                      in memory).
    With sphere=True each midpoint is pushed back onto the unit sphere
    (m / |m|); the transfer weights stay 1/2, 1/2.
    """
    nc = mesh.nv
    E = mesh.ne
    a_idx = mesh.edges[:, 0]
    b_idx = mesh.edges[:, 1]
    mid = (mesh.verts[a_idx] + mesh.verts[b_idx]) * 0.5
    if sphere:
        if mesh.verts.shape[1] != 3:
            raise MeshError("sphere projection needs 3-D vertices")
        nrm = np.sqrt(mid[:, 0] * mid[:, 0] + mid[:, 1] * mid[:, 1] + mid[:, 2] * mid[:, 2])
        mid = mid / nrm[:, None]
    if order == "morton":
        perm = np.argsort(morton_keys(mid), kind="stable")  # perm[k] = coarse edge of new vertex k
    elif order == "edge":
        perm = np.arange(E)
    else:
        raise ValueError(order)
    rank = np.empty(E, dtype=np.int64)
    rank[perm] = np.arange(E)
    fverts = np.concatenate([mesh.verts, mid[perm]], axis=0)
    a, b, c = mesh.tris[:, 0], mesh.tris[:, 1], mesh.tris[:, 2]
    m_ab = nc + rank[mesh.tri_edges[:, 0]]
    m_bc = nc + rank[mesh.tri_edges[:, 1]]
    m_ca = nc + rank[mesh.tri_edges[:, 2]]
    T = mesh.nt
    ftris = np.empty((4 * T, 3), dtype=np.int64)
    ftris[0::4] = np.stack([a, m_ab, m_ca], axis=1)
    ftris[1::4] = np.stack([m_ab, b, m_bc], axis=1)
    ftris[2::4] = np.stack([m_ca, m_bc, c], axis=1)
    ftris[3::4] = np.stack([m_ab, m_bc, m_ca], axis=1)
    fine = build_mesh(fverts, ftris)
    assert fine.nv == nc + E
    return fine, mesh.edges[perm].copy()


def subdivide_cubic(mesh, sphere=False):
    """One 1->9 subdivision (Sec. 2.2.1, cubic subdivision).

    Coarse vertices keep their ids.  Coarse edge e = (lo, hi) gets two new
    vertices, n_c + 2e at (2 x_lo + x_hi)/3 and n_c + 2e + 1 at (x_lo + 2 x_hi)/3;
    coarse triangle t = (a, b, c) gets its centroid n_c + 2E + t at
    ((x_a + x_b) + x_c)/3.  With lattice points (i, j, k)/3 of weights on
    (a, b, c), the triangle becomes the nine lattice triangles
      9t+0 (a, ab1, ca2)   9t+1 (ab1, ab2, m)   9t+2 (ab2, b, bc1)
      9t+3 (ca2, m, ca1)   9t+4 (m, bc1, bc2)   9t+5 (ca1, bc2, c)
      9t+6 (ab1, m, ca2)   9t+7 (ab2, bc1, m)   9t+8 (m, bc2, ca1)
    where xy1 is the point on edge xy next to x and xy2 the one next to y, and
    m the centroid; all keep the coarse orientation.  With sphere=True the new
    points are pushed to the unit sphere and the weights stay combinatorial.

    Returns (fine Mesh, M) with M = M(f), the n_c x n_f matrix whose column j
    holds the global barycentric coordinates of fine vertex j (Sec. 2.2.1):
    1 for a kept vertex, 2/3 and 1/3 for an edge point, 1/3 three times for a
    centroid.
    """
    nc, E, T = mesh.nv, mesh.ne, mesh.nt
    lo, hi = mesh.edges[:, 0], mesh.edges[:, 1]
    xl, xh = mesh.verts[lo], mesh.verts[hi]
    pts = np.empty((2 * E + T, mesh.verts.shape[1]))
    pts[0:2 * E:2] = (2.0 * xl + xh) / 3.0
    pts[1:2 * E:2] = (xl + 2.0 * xh) / 3.0
    a, b, c = mesh.tris[:, 0], mesh.tris[:, 1], mesh.tris[:, 2]
    pts[2 * E:] = ((mesh.verts[a] + mesh.verts[b]) + mesh.verts[c]) / 3.0
    if sphere:
        if mesh.verts.shape[1] != 3:
            raise MeshError("sphere projection needs 3-D vertices")
        nrm = np.sqrt(pts[:, 0] * pts[:, 0] + pts[:, 1] * pts[:, 1] + pts[:, 2] * pts[:, 2])
        pts = pts / nrm[:, None]
    fverts = np.concatenate([mesh.verts, pts], axis=0)

    def near(k, corner):
        e = mesh.tri_edges[:, k]
        return nc + 2 * e + (corner != lo[e])

    ab1, ab2 = near(0, a), near(0, b)
    bc1, bc2 = near(1, b), near(1, c)
    ca1, ca2 = near(2, c), near(2, a)
    m = nc + 2 * E + np.arange(T)
    ftris = np.empty((9 * T, 3), dtype=np.int64)
    for q, tri in enumerate(((a, ab1, ca2), (ab1, ab2, m), (ab2, b, bc1), (ca2, m, ca1), (m, bc1, bc2),
                             (ca1, bc2, c), (ab1, m, ca2), (ab2, bc1, m), (m, bc2, ca1))):
        ftris[q::9] = np.stack(tri, axis=1)
    fine = build_mesh(fverts, ftris)
    assert fine.nv == nc + 2 * E + T
    third, two_thirds = 1.0 / 3.0, 2.0 / 3.0
    ids = np.arange(E)
    rows = np.concatenate([np.arange(nc), lo, hi, lo, hi, a, b, c])
    cols = np.concatenate([np.arange(nc), nc + 2 * ids, nc + 2 * ids, nc + 2 * ids + 1, nc + 2 * ids + 1, m, m, m])
    vals = np.concatenate([np.ones(nc), np.full(E, two_thirds), np.full(E, third), np.full(E, third),
                           np.full(E, two_thirds), np.full(3 * T, third)])
    M = sp.csr_matrix((vals, (rows, cols)), shape=(nc, fine.nv))
    return fine, M


def refine(verts, tris, nsub, sphere=False, order="edge", scheme="binary"):
    """Apply nsub subdivisions; returns the list of meshes (coarsest first) and, per step,
    the parent table (binary: the coarse edge of each new vertex) or, for
    scheme="cubic", the geometric-map matrix M(f) of subdivide_cubic."""
    meshes = [build_mesh(verts, tris)]
    parents = []
    for _ in range(nsub):
        if scheme == "cubic":
            fine, par = subdivide_cubic(meshes[-1], sphere=sphere)
            meshes.append(fine)
            parents.append(par)
            continue
        fine, par = subdivide(meshes[-1], sphere=sphere, order=order)
        meshes.append(fine)
        parents.append(par)
    return meshes, parents
