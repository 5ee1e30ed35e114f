"""Pins of the oracle's mesh layer against what the paper and combinatorics fix.

Each test would fail under a plausible slip in oracle/mesh.py or the
transfer matrices: a wrong edge orientation breaks d1 d0 = 0, a wrong child
triangle breaks the counts or the ring example, a transposed or unnormalized
restriction breaks the Sec. 2.2.1 restriction example.
"""
import os

import numpy as np
import pytest

import workloads as W
from oracle import dec, mesh as M, multigrid as mg

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    return np.loadtxt(os.path.join(GOLDEN, name), comments="#")


def _counts_table():
    rows = {}
    with open(os.path.join(GOLDEN, "paper_mesh_counts.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, grid, nsub, V, E, T, nnz = line.split()
            conv = lambda s: None if s == "-" else int(s)
            nx, ny = map(int, grid.split("x"))
            rows[name] = dict(nx=nx, ny=ny, nsub=int(nsub), V=conv(V), E=conv(E), T=conv(T), nnz=conv(nnz))
    return rows


COUNTS = _counts_table()


@pytest.mark.parametrize("case", ["square", "ico", "grid", "perturbed"])
def test_d1_d0_is_zero(case):
    # dd = 0 (Sec. 1, the de Rham complex), exactly, in integer arithmetic
    if case == "square":
        v, t = W.unit_square(); meshes, _ = M.refine(v, t, 3)
    elif case == "ico":
        v, t = W.icosahedron(); meshes, _ = M.refine(v, t, 2, sphere=True)
    elif case == "grid":
        v, t = W.grid_mesh(5, 4); meshes, _ = M.refine(v, t, 1)
    else:
        v, t = W.grid_mesh(4, 4)
        # flip the orientation of every other triangle: d1 d0 = 0 must not care
        t = t.copy(); t[::2] = t[::2, ::-1]
        meshes, _ = M.refine(v, t, 1)
    for m in meshes:
        prod = M.d1_matrix(m) @ M.d0_matrix(m)
        assert prod.count_nonzero() == 0
        assert M.d0_matrix(m).dtype.kind == "i"


def test_edges_canonical_and_orientation():
    v, t = W.one_triangle()
    m = M.build_mesh(v, t)
    assert m.edges.tolist() == [[0, 1], [0, 2], [1, 2]]
    # triangle (0,1,2): v0v1 = +e0, v1v2 = +e2, v2v0 = -e1
    assert m.tri_edges.tolist() == [[0, 2, 1]]
    assert m.tri_signs.tolist() == [[1, 1, -1]]
    d0 = M.d0_matrix(m).toarray()
    assert d0.tolist() == [[-1, 1, 0], [-1, 0, 1], [0, -1, 1]]


@pytest.mark.parametrize("order", ["edge", "morton"])
@pytest.mark.parametrize("base", ["square", "ico", "grid"])
def test_subdivision_counting(base, order):
    # V' = V + E, E' = 2E + 3T, T' = 4T for 1->4 midpoint subdivision
    if base == "square":
        v, t = W.unit_square(); meshes, par = M.refine(v, t, 4, order=order)
    elif base == "ico":
        v, t = W.icosahedron(); meshes, par = M.refine(v, t, 3, sphere=True, order=order)
    else:
        v, t = W.grid_mesh(3, 5); meshes, par = M.refine(v, t, 3, order=order)
    for c, f, p in zip(meshes[:-1], meshes[1:], par):
        assert f.nv == c.nv + c.ne
        assert f.ne == 2 * c.ne + 3 * c.nt
        assert f.nt == 4 * c.nt
        if order == "edge":
            assert np.array_equal(p, c.edges)
        else:
            # a permutation of the coarse edges, in non-decreasing Morton key of the midpoints
            assert np.array_equal(np.sort(p[:, 0] * c.nv + p[:, 1]), c.edges[:, 0] * c.nv + c.edges[:, 1])
            keys = M.morton_keys(f.verts[c.nv:])
            assert np.all(keys[1:] >= keys[:-1])
        # coarse vertices keep their position, midpoints are at the mean (planar)
        assert np.array_equal(f.verts[: c.nv], c.verts)
        if base != "ico":
            assert np.array_equal(f.verts[c.nv:], 0.5 * (c.verts[p[:, 0]] + c.verts[p[:, 1]]))
    if base == "ico":
        for m in meshes:
            assert m.nv - m.ne + m.nt == 2
            assert np.allclose(np.linalg.norm(m.verts, axis=1), 1.0, atol=1e-15)


def test_paper_counts_porous_mesh():
    # porous-convection mesh (Sec. 3.2.2 captions): sizes and nnz of L
    for name in ("porous_finest", "porous_second"):
        row = COUNTS[name]
        v, t = W.unit_square()
        meshes, _ = M.refine(v, t, row["nsub"])
        m = meshes[-1]
        assert m.nv == row["V"]
        if row["E"] is not None:
            assert (m.ne, m.nt) == (row["E"], row["T"])
        assert dec.stencil_nnz(m) == row["nnz"] == m.nv + 2 * m.ne


def test_paper_counts_vcycle_mesh():
    row = COUNTS["vcycle_binary4"]
    v, t = W.grid_mesh(row["nx"], row["ny"])
    assert len(t) == 32 and len(v) == 25
    meshes, _ = M.refine(v, t, row["nsub"])
    assert meshes[-1].nv == row["V"]


@pytest.mark.slow
def test_paper_counts_crosscomparison_mesh():
    # Sec. 3.1.2 caption: 625/1,776/1,152 -> 2,362,369/7,080,960/4,718,592 after 6 subdivisions
    base = COUNTS["crosscomp_base"]
    fine = COUNTS["crosscomp_sub6"]
    v, t = W.grid_mesh(base["nx"], base["ny"])
    m = M.build_mesh(v, t)
    assert (m.nv, m.ne, m.nt) == (base["V"], base["E"], base["T"])
    for _ in range(fine["nsub"]):
        m, _ = M.subdivide(m)
    assert (m.nv, m.ne, m.nt) == (fine["V"], fine["E"], fine["T"])


def _ring_order():
    # one triangle (a,b,c) = (0,1,2); edges (0,1)=e0, (0,2)=e1, (1,2)=e2, midpoints 3,4,5
    # boundary ring a, m_ab, b, m_bc, c, m_ca
    return [0, 3, 1, 5, 2, 4]


def test_interpolation_example_sec221():
    v, t = W.one_triangle()
    meshes, par = M.refine(v, t, 1)
    P = mg.interpolation(3, par[0]).toarray()
    expect = _load("interpolation_one_triangle.txt")
    assert np.array_equal(P[_ring_order()], expect)
    # applying it to [a b c] gives [a, (a+b)/2, b, (b+c)/2, c, (c+a)/2]
    a, b, c = 2.0, -3.0, 7.0
    assert np.allclose(P[_ring_order()] @ [a, b, c], [a, (a + b) / 2, b, (b + c) / 2, c, (c + a) / 2])


def test_restriction_example_sec221():
    v, t = W.one_triangle()
    _, par = M.refine(v, t, 1)
    R = mg.restriction(3, par[0]).toarray()      # n_c x n_f acting on column vectors
    expect = _load("restriction_one_triangle.txt")  # printed n_f x n_c
    assert np.array_equal(R.T[_ring_order()], expect)


@pytest.mark.parametrize("base", ["square", "ico", "grid"])
def test_transfers_preserve_constants(base):
    if base == "square":
        v, t = W.unit_square(); meshes, par = M.refine(v, t, 3)
    elif base == "ico":
        v, t = W.icosahedron(); meshes, par = M.refine(v, t, 2, sphere=True)
    else:
        v, t = W.grid_mesh(4, 3); meshes, par = M.refine(v, t, 2)
    for i, p in enumerate(par):
        c, f = meshes[i], meshes[i + 1]
        P = mg.interpolation(c.nv, p)
        R = mg.restriction(c.nv, p)
        assert np.allclose(P @ np.ones(c.nv), 1.0, rtol=0, atol=0)
        assert np.allclose(R @ np.ones(P.shape[0]), 1.0, rtol=1e-15, atol=0)
        # interpolation reproduces linear functions exactly on planar meshes
        if base != "ico":
            lin = 3.0 * c.verts[:, 0] - 2.0 * c.verts[:, 1] + 0.5
            assert np.allclose(P @ lin, 3.0 * f.verts[:, 0] - 2.0 * f.verts[:, 1] + 0.5, atol=1e-14)


@pytest.mark.parametrize("bad", ["dup", "isolated", "nonmanifold", "repeat", "range"])
def test_validation_rejects(bad):
    v, t = W.grid_mesh(3, 3)
    if bad == "dup":
        t = np.concatenate([t, t[:1, [1, 2, 0]]])
    elif bad == "isolated":
        v = np.concatenate([v, [[5.0, 5.0]]])
    elif bad == "nonmanifold":
        v = np.concatenate([v, [[0.5, -1.0]]])
        t = np.concatenate([t, [[0, 1, len(v) - 1], [1, 0, 4]]])
    elif bad == "repeat":
        t = np.concatenate([t, [[0, 0, 1]]])
    else:
        t = np.concatenate([t, [[0, 1, 99]]])
    with pytest.raises(M.MeshError):
        M.build_mesh(v, t)


def _z_less(a, b):
    """Z-order comparison without interleaving (the most-significant-differing-bit rule):
    the axis whose coordinates differ in the highest bit decides."""
    best, axis = -1, 0
    for d in range(len(a)):
        x = int(a[d]) ^ int(b[d])
        if x and x.bit_length() > best:
            best, axis = x.bit_length(), d
        elif x and x.bit_length() == best and d > axis:
            axis = d  # equal top bits: the higher axis holds the higher interleaved bit
    return best >= 0 and int(a[axis]) < int(b[axis])


@pytest.mark.parametrize("dim", [2, 3])
def test_morton_keys_order_points_in_z_order(dim):
    rng = np.random.default_rng(dim)
    pts = rng.uniform(-1.0, 1.0, size=(60, dim))
    pts[0] = -1.0
    pts[1] = 1.0  # the bounding box is [-1, 1]^dim
    B = 21 if dim == 3 else 31
    q = np.clip(np.floor((pts + 1.0) * (float((1 << B) - 1) / 2.0)), 0, (1 << B) - 1).astype(np.int64)
    keys = M.morton_keys(pts)
    for i in range(len(pts)):
        for j in range(len(pts)):
            assert (keys[i] < keys[j]) == _z_less(q[i], q[j])


def test_morton_keys_of_corners():
    # corners of the unit square: q in {0, 2^31 - 1}; axis 0 takes the even bits, axis 1 the odd bits
    k = M.morton_keys(np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0], [1.0, 1.0]]))
    even = sum(1 << (2 * b) for b in range(31))
    assert k.tolist() == [0, even, even << 1, even | (even << 1)]


def _gather_sectors_per_row(m):
    """32-byte sectors of a float vector touched by the neighbour gathers of each warp of 32 rows, per row."""
    nb = [[] for _ in range(m.nv)]
    for a, b in m.edges:
        nb[a].append(b)
        nb[b].append(a)
    tot = 0
    for w in range(0, m.nv, 32):
        tot += len({j // 8 for i in range(w, min(m.nv, w + 32)) for j in nb[i]})
    return tot / m.nv


@pytest.mark.parametrize("base", ["square", "ico"])
def test_morton_order_keeps_neighbours_close(base):
    # the same vertices in both orders, and a warp's neighbour gathers touch fewer sectors in Z-order
    if base == "square":
        v, t = W.unit_square(); args = dict(nsub=6)
    else:
        v, t = W.icosahedron(); args = dict(nsub=5, sphere=True)
    sec = {}
    for order in ("edge", "morton"):
        m = M.refine(v, t, order=order, **args)[0][-1]
        sec[order] = _gather_sectors_per_row(m)
        ref = M.refine(v, t, order="edge", **args)[0][-1]
        assert np.array_equal(np.unique(m.verts, axis=0), np.unique(ref.verts, axis=0))
    assert sec["morton"] < 0.92 * sec["edge"], sec
