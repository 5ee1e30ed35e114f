"""Halo tiles built on the host (host_patch.cpp), checked without a GPU.

tests/host_patch_check.cpp is compiled with the library's host sources and
run on a few meshes, tile sizes and smoothing depths.  It checks what the
tiled cycle kernels rely on: the tiles' owned vertices partition each level,
the down tiles' coarse vertices partition the coarser level, ring 0 is the
restriction's support (down) or the owned set (up), every ring is exactly the
neighbours of the rings inside it, and every local ELL slot names the local
copy of the level's column.  The GPU side (tests/test_gpu_patch.py) checks
that tiled cycles are bitwise those of the per-step kernels.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2508_12501_gb300", "csrc")
SOURCES = [os.path.join(ROOT, "tests", "host_patch_check.cpp")] + [
    os.path.join(CSRC, f) for f in ("host_patch.cpp", "host_hier.cpp", "host_mesh.cpp", "capi_host.cpp")]
BC = {"dirichlet": 0, "gauge": 1}


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no g++")
    exe = str(tmp_path_factory.mktemp("hpc") / "host_patch_check")
    subprocess.run([gxx, "-std=c++17", "-O1", "-I", os.path.join(ROOT, "include"), "-I", CSRC] + SOURCES +
                   ["-o", exe], check=True)
    return exe


def _run(exe, verts, tris, sphere, nsub, nlevels, bc, chunk, dd, du):
    verts = np.asarray(verts, dtype=np.float64)
    tris = np.asarray(tris, dtype=np.int64)
    head = f"{len(verts)} {verts.shape[1]} {len(tris)} {int(sphere)} {nsub} {nlevels} {BC[bc]} {chunk} {dd} {du}\n"
    body = " ".join(repr(float(x)) for x in verts.ravel()) + "\n" + " ".join(str(int(t)) for t in tris.ravel())
    out = subprocess.run([exe], input=head + body + "\n", capture_output=True, text=True)
    return out.returncode, out.stdout.strip()


@pytest.mark.parametrize("mesh", ["square", "ico", "fan"])
@pytest.mark.parametrize("chunk", [1, 5, 24, 10 ** 6])
@pytest.mark.parametrize("depth", [(1, 1), (2, 2), (3, 1), (2, 3)])
def test_tiles_partition_and_rings(checker, mesh, chunk, depth):
    if mesh == "square":
        (v, t), sph, nsub, nl, bc = W.unit_square(), False, 5, 4, "dirichlet"
    elif mesh == "ico":
        (v, t), sph, nsub, nl, bc = W.icosahedron(), True, 4, 4, "gauge"
    else:
        (v, t), sph, nsub, nl, bc = W.heptagon_fan(), False, 4, 4, "dirichlet"
    rc, out = _run(checker, v, t, sph, nsub, nl, bc, chunk, *depth)
    assert rc == 0 and out.startswith("ok"), out
    ntiles = [int(x) for x in out.split()[1:]]
    assert len(ntiles) == nl - 1 and all(n >= 1 for n in ntiles)
    if chunk == 1:
        # one coarse vertex per tile: the tile counts are the coarser levels' vertex counts, which grow
        assert all(a < b for a, b in zip(ntiles, ntiles[1:]))
    if chunk == 10 ** 6:
        assert ntiles == [1] * (nl - 1)


def test_bad_depths_are_refused(checker):
    v, t = W.unit_square()
    for dd, du in ((0, 2), (4, 2), (2, 0), (2, 4)):
        rc, out = _run(checker, v, t, False, 3, 3, "dirichlet", 24, dd, du)
        assert rc == 1 and "smoothing steps" in out, out
