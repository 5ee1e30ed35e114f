"""CPU tests of the C ABI: the library loads, exports every declared symbol,
and its host-side setup matches the oracle bit for bit on integer tables."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import workloads as W
from oracle import dec as odec, mesh as omesh, multigrid as omg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

lib_mod = pytest.importorskip("paper_2508_12501_gb300._lib")
from paper_2508_12501_gb300 import Hierarchy, Mesh  # noqa: E402
from paper_2508_12501_gb300._lib import DecError  # noqa: E402


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "dec.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dec_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported():
    names = _declared_functions()
    assert "dec_solve" in names and "dec_mg_vcycle" in names and "dec_laplace0_apply" in names
    lib = C.CDLL(lib_mod.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    # and the binding declares a signature for each of them
    for n in names:
        assert n in lib_mod._SIGS, n


def _cases():
    yield "square", W.unit_square(), 4, False
    yield "ico", W.icosahedron(), 3, True
    yield "grid", W.grid_mesh(5, 4), 2, False
    v, t = W.grid_mesh(4, 4)
    t = t.copy()
    t[::2] = t[::2, ::-1]
    yield "mixed_orientation", (v, t), 2, False


@pytest.mark.parametrize("order", ["edge", "morton"])
@pytest.mark.parametrize("name,vt,nsub,sphere", list(_cases()), ids=[c[0] for c in _cases()])
def test_refined_tables_bit_exact(name, vt, nsub, sphere, order):
    v, t = vt
    meshes, _ = omesh.refine(v, t, nsub, sphere=sphere, order=order)
    m = Mesh(v, t)
    for k, om in enumerate(meshes):
        lm = m.refine(k, sphere=sphere, order=order) if k else m
        assert (lm.nv, lm.ne, lm.nt) == (om.nv, om.ne, om.nt)
        assert np.array_equal(lm.table("tris"), om.tris)
        assert np.array_equal(lm.table("edges"), om.edges)
        assert np.array_equal(lm.table("verts"), om.verts)  # same op order, no FMA contraction
        s0 = lm.table("star0")
        s1 = lm.table("star1")
        assert np.allclose(s0, odec.hodge_star0(om), rtol=1e-13, atol=1e-16)
        assert np.allclose(s1, odec.hodge_star1(om), rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("order", ["edge", "morton"])
@pytest.mark.parametrize("bc", ["dirichlet", "gauge"])
def test_hierarchy_host_tables(bc, order):
    if bc == "dirichlet":
        v, t = W.unit_square(); nsub, nl, sphere = 4, 3, False
    else:
        v, t = W.icosahedron(); nsub, nl, sphere = 3, 3, True
    h = Hierarchy(Mesh(v, t), nsub, nl, bc=bc, sphere=sphere, host_only=True, order=order)
    oh = omg.build_hierarchy(v, t, nsub, nl, bc, sphere=sphere, opts=omg.MGOptions(smoother="mcgs"), order=order)
    assert h.nlevels == nl
    for l in range(nl):
        ol = oh.levels[l]
        assert h.nv[l] == ol.mesh.nv
        assert np.array_equal(h.table(l, "free").astype(bool), ol.free)
        assert np.array_equal(h.table(l, "colors"), ol.colors)
        assert h.ncolors[l] == int(ol.colors.max()) + 1
        assert abs(h.lmax[l] - ol.lmax) <= 1e-12 * ol.lmax
        assert np.array_equal(h.table(l, "edges"), ol.mesh.edges)
        if l + 1 < nl:
            # parents of level l+1 midpoints: the level-l edges, in the chosen order of the new vertices
            par = oh.levels[l].mesh.edges
            if order == "morton":
                fine = oh.levels[l + 1].mesh
                mid = 0.5 * (ol.mesh.verts[par[:, 0]] + ol.mesh.verts[par[:, 1]])
                if sphere:
                    mid = mid / np.sqrt(mid[:, 0] * mid[:, 0] + mid[:, 1] * mid[:, 1] + mid[:, 2] * mid[:, 2])[:, None]
                par = par[np.argsort(omesh.morton_keys(mid), kind="stable")]
                assert np.array_equal(fine.verts[ol.mesh.nv:], mid[np.argsort(omesh.morton_keys(mid), kind="stable")])
            assert np.array_equal(h.table(l, "parents"), par)
    assert h.ell_width[-1] == 6


def test_star1_scale_applies_to_finest_only():
    v, t = W.unit_square()
    om = omesh.refine(v, t, 3)[0]
    scale = W.lognormal_factors(om[-1].ne, 2)
    h = Hierarchy(Mesh(v, t), 3, 2, bc="dirichlet", star1_scale=scale, host_only=True)
    assert np.allclose(h.table(-1, "star1"), odec.hodge_star1(om[-1], scale), rtol=1e-14, atol=1e-15)
    assert np.allclose(h.table(0, "star1"), odec.hodge_star1(om[-2]), rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("bad", ["dup", "isolated", "nonmanifold", "repeat", "range"])
def test_invalid_meshes_rejected_like_oracle(bad):
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
    with pytest.raises(omesh.MeshError):
        omesh.build_mesh(v, t)
    with pytest.raises(DecError) as ei:
        Mesh(v, t)
    assert ei.value.code == lib_mod.DEC_ERR_MESH


def test_bad_arguments():
    v, t = W.unit_square()
    m = Mesh(v, t)
    with pytest.raises(DecError) as ei:
        Hierarchy(m, 2, 5, host_only=True)  # more levels than meshes
    assert ei.value.code == lib_mod.DEC_ERR_ARG
    with pytest.raises(DecError):
        m.refine(2, sphere=True)  # 2-D vertices cannot be projected to the sphere
    h = Hierarchy(m, 2, 2, host_only=True)
    # compute calls on a host-only handle are rejected, not run
    rc = lib_mod.lib.dec_laplace0_apply(h._h, 0, C.c_void_p(8), C.c_void_p(16), 1, 0, None)
    assert rc == lib_mod.DEC_ERR_ARG


def test_coarse_limit_and_nan_free_setup():
    v, t = W.icosahedron()
    with pytest.raises(DecError) as ei:
        Hierarchy(Mesh(v, t), 5, 1, bc="gauge", sphere=True, host_only=True)  # 10,242-vertex coarsest level
    assert ei.value.code == lib_mod.DEC_ERR_MESH


@pytest.mark.parametrize("name,vt,nsub,sphere", [c for c in _cases() if c[0] != "grid"], ids=lambda c: str(c)[:12])
def test_cubic_refined_tables_bit_exact(name, vt, nsub, sphere):
    v, t = vt
    meshes, _ = omesh.refine(v, t, min(nsub, 2), sphere=sphere, scheme="cubic")
    m = Mesh(v, t)
    for k, om in enumerate(meshes):
        lm = m.refine(k, sphere=sphere, scheme="cubic") if k else m
        assert (lm.nv, lm.ne, lm.nt) == (om.nv, om.ne, om.nt)
        assert np.array_equal(lm.table("tris"), om.tris)
        assert np.array_equal(lm.table("edges"), om.edges)
        assert np.array_equal(lm.table("verts"), om.verts)


@pytest.mark.parametrize("bc", ["dirichlet", "gauge"])
def test_cubic_hierarchy_map_tables(bc):
    # the library's map from level l to l+1, as three (coarse vertex, weight) slots per fine vertex,
    # is the oracle's M(f) exactly
    if bc == "dirichlet":
        v, t = W.unit_square(); nsub, nl, sphere = 3, 3, False
    else:
        v, t = W.icosahedron(); nsub, nl, sphere = 2, 3, True
    h = Hierarchy(Mesh(v, t), nsub, nl, bc=bc, sphere=sphere, host_only=True, scheme="cubic")
    meshes, maps = omesh.refine(v, t, nsub, sphere=sphere, scheme="cubic")
    first = nsub + 1 - nl
    for l in range(nl - 1):
        idx, w = h.table(l, "map_idx"), h.table(l, "map_w")
        Mo = maps[first + l].toarray()
        Ml = np.zeros_like(Mo)
        for q in range(3):
            np.add.at(Ml, (idx[:, q], np.arange(len(idx))), w[:, q])
        assert np.array_equal(Ml, Mo)
    with pytest.raises(Exception):
        h.table(0, "parents")


def test_binary_map_tables_are_the_parents():
    v, t = W.unit_square()
    h = Hierarchy(Mesh(v, t), 3, 3, bc="dirichlet", host_only=True)
    oh = omg.build_hierarchy(v, t, 3, 3, "dirichlet")
    idx, w = h.table(0, "map_idx"), h.table(0, "map_w")
    Mo = omg.barycentric_matrix(oh.levels[0].mesh.nv, h.table(0, "parents")).toarray()
    Ml = np.zeros_like(Mo)
    for q in range(3):
        np.add.at(Ml, (idx[:, q], np.arange(len(idx))), w[:, q])
    assert np.array_equal(Ml, Mo)


def test_option_defaults_and_fuse_max_rows_validation():
    o = lib_mod.dec_mg_opts()
    lib_mod.lib.dec_mg_default_opts(C.byref(o))
    assert o.fuse == (lib_mod.DEC_FUSE_RESTRICT0 | lib_mod.DEC_FUSE_OUTER | lib_mod.DEC_FUSE_COARSE
                      | lib_mod.DEC_FUSE_PATCH)
    assert (o.patch_max_rows, o.patch_chunk, o.patch_threads) == (0, 0, 0)
    assert o.fuse_max_rows == 0 and o.coarse_max_rows == 0 and o.fcycle == 0
    v, t = W.unit_square()
    Hierarchy(Mesh(v, t), 3, 2, bc="dirichlet", host_only=True, fuse=63, fuse_max_rows=100)
    with pytest.raises(DecError) as ei:
        Hierarchy(Mesh(v, t), 3, 2, bc="dirichlet", host_only=True, fuse_max_rows=-1)
    assert ei.value.code == lib_mod.DEC_ERR_ARG
    # halo tiles: every fusion bit, block sizes in warps up to 256 threads, non-negative sizes
    Hierarchy(Mesh(v, t), 3, 2, bc="dirichlet", host_only=True, fuse=lib_mod.DEC_FUSE_ALL, patch_chunk=7,
              patch_threads=64, patch_max_rows=10)
    for kw in (dict(patch_threads=48), dict(patch_threads=288), dict(patch_chunk=-1), dict(patch_max_rows=-5),
               dict(fuse=lib_mod.DEC_FUSE_ALL + 1)):
        with pytest.raises(DecError) as ei:
            Hierarchy(Mesh(v, t), 3, 2, bc="dirichlet", host_only=True, **kw)
        assert ei.value.code == lib_mod.DEC_ERR_ARG


def test_host_only_handles_refuse_device_entry_points():
    # dec_solve_host, dec_porous_rk and the kernel timer check the handle before anything else
    v, t = W.icosahedron()
    h = Hierarchy(Mesh(v, t), 2, 2, bc="gauge", sphere=True, host_only=True)
    L = lib_mod
    st = L.dec_stats()
    assert L.lib.dec_solve_host(h._h, None, None, 1, None, C.byref(st), None) == L.DEC_ERR_ARG
    rk = L.dec_rk_stats()
    assert L.lib.dec_porous_rk(h._h, None, None, None, None, 1e-3, 1e-5, 1e-9, 1e-6, 10, 0, C.byref(rk),
                               None) == L.DEC_ERR_ARG
    ms, by = C.c_double(), C.c_double()
    assert L.lib.dec_mg_time_kernel(h._h, L.PROF_KINDS.index("spmv64"), -1, 5, C.byref(ms), C.byref(by),
                                    None) == L.DEC_ERR_ARG


def test_mapped_hierarchy_host_tables_and_refusals():
    # dec_mg_build_maps (host only): the caller's map comes back bit for bit and equals the oracle's M(f);
    # the per-level tables match the oracle's levels; malformed maps are refused before any device work
    ms, mi, mw = W.jittered_square_levels(3, 5)
    meshes = [Mesh(v, t) for v, t in ms]
    h = Hierarchy.from_maps(meshes, mi, mw, bc="dirichlet", host_only=True)
    assert h.nv == [len(v) for v, _ in ms]
    om = [omesh.build_mesh(v, t) for v, t in ms]
    for l in range(2):
        assert np.array_equal(h.table(l, "map_idx"), mi[l]) and np.array_equal(h.table(l, "map_w"), mw[l])
        Mo = omg.map_matrix_from_table(om[l].nv, mi[l], mw[l]).toarray()
        Ml = np.zeros_like(Mo)
        for q in range(3):
            np.add.at(Ml, (h.table(l, "map_idx")[:, q], np.arange(om[l + 1].nv)), h.table(l, "map_w")[:, q])
        assert np.array_equal(Ml, Mo)
    for l in range(3):
        assert np.array_equal(h.table(l, "edges"), om[l].edges)
        lev = omg.make_level(om[l], "dirichlet")
        assert np.array_equal(h.table(l, "free").astype(bool), lev.free)
    bad = [a.copy() for a in mi]
    bad[0][0, 0] = -1
    with pytest.raises(DecError) as ei:
        Hierarchy.from_maps(meshes, bad, mw, host_only=True)
    assert ei.value.code == lib_mod.DEC_ERR_ARG and "out of range" in str(ei.value)
    badw = [a.copy() for a in mw]
    badw[1][5, :] = [0.5, 0.5, 0.5]
    with pytest.raises(DecError) as ei:
        Hierarchy.from_maps(meshes, mi, badw, host_only=True)
    assert ei.value.code == lib_mod.DEC_ERR_ARG and "sum to 1" in str(ei.value)
    with pytest.raises(ValueError):
        Hierarchy.from_maps(meshes, mi[:1], mw[:1], host_only=True)
