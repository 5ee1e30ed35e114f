"""Circumcentric diagonal Hodge stars and the DEC 0-form Laplacian.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Sec. 3.1.1, Eq. (hodge0-laplacian): Delta_0 = *0^-1 d~1 *1 d0 with d~1 the
negated transpose of d0, *0 the dual-cell areas and *1 the ratio of dual to
primal edge length.  Readings:
  * sign: the library solves L u = b with the positive semidefinite
    L = *0^-1 d0^T *1 d0 = -Delta_0;
  * *1 is |dual edge| / |primal edge| of the circumcentric dual, computed as
    (1/2) sum over the triangles t containing e of cot(angle of t opposite e);
    the paper's sentence names the ratio the other way round, which would not
    give the cotangent Laplacian;
  * *0 is the signed circumcentric dual area,
    sum over t containing v of (1/8)(|vp|^2 cot(opp vp) + |vq|^2 cot(opp vq)).
Cotangents are dot(u, w) / |u x w| so that a right angle gives exactly 0.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .mesh import d0_matrix


def _cross_norm(u, w):
    if u.shape[1] == 2:
        return np.abs(u[:, 0] * w[:, 1] - u[:, 1] * w[:, 0])
    c = np.cross(u, w)
    return np.sqrt(np.sum(c * c, axis=1))


def opposite_cotangents(mesh):
    """[T,3] cot of the angle opposite triangle edge k (k=0: v0v1, 1: v1v2, 2: v2v0)."""
    P = mesh.verts[mesh.tris]  # [T,3,dim]
    out = np.empty((mesh.nt, 3))
    # edge k joins vertices k and k+1; the opposite vertex is k+2
    for k in range(3):
        o = P[:, (k + 2) % 3]
        u = P[:, k] - o
        w = P[:, (k + 1) % 3] - o
        out[:, k] = np.sum(u * w, axis=1) / _cross_norm(u, w)
    return out


def edge_lengths_sq(mesh):
    """[T,3] squared length of triangle edge k."""
    P = mesh.verts[mesh.tris]
    out = np.empty((mesh.nt, 3))
    for k in range(3):
        d = P[:, (k + 1) % 3] - P[:, k]
        out[:, k] = np.sum(d * d, axis=1)
    return out


def hodge_star1(mesh, scale=None):
    """Diagonal of *1 per edge: (1/2) sum of opposite cotangents, optionally times scale[e]."""
    cot = opposite_cotangents(mesh)
    s1 = np.zeros(mesh.ne)
    np.add.at(s1, mesh.tri_edges.ravel(), 0.5 * cot.ravel())
    if scale is not None:
        s1 = s1 * np.asarray(scale, dtype=np.float64)
    return s1


def hodge_star0(mesh):
    """Diagonal of *0 per vertex: circumcentric dual-cell area."""
    cot = opposite_cotangents(mesh)
    l2 = edge_lengths_sq(mesh)
    s0 = np.zeros(mesh.nv)
    for k in range(3):
        contrib = l2[:, k] * cot[:, k] / 8.0
        np.add.at(s0, mesh.tris[:, k], contrib)
        np.add.at(s0, mesh.tris[:, (k + 1) % 3], contrib)
    return s0


def triangle_areas(mesh):
    P = mesh.verts[mesh.tris]
    return 0.5 * _cross_norm(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0])


def stiffness(mesh, star1):
    """A = d0^T diag(*1) d0 (symmetric, positive semidefinite when *1 >= 0)."""
    d0 = d0_matrix(mesh).astype(np.float64)
    return (d0.T @ sp.diags(star1) @ d0).tocsr()


def laplacian(mesh, star0, star1):
    """L = *0^-1 d0^T *1 d0 as a CSR matrix (the negated Delta_0 of Eq. hodge0-laplacian)."""
    return (sp.diags(1.0 / star0) @ stiffness(mesh, star1)).tocsr()


def stencil_nnz(mesh):
    """Number of stored entries of the Laplacian stencil, zero-weight edges included."""
    d0 = abs(d0_matrix(mesh))
    return (d0.T @ d0).nnz
