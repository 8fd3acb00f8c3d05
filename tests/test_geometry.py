"""CPU tests of the host's choice of gather variant (geometry.h).  The paper-geometry kernels index
the atlas, the planes and the occupancy levels with 32-bit offsets, so the choice must exclude every
scene whose offsets could exceed 2^32: the largest voxel offset is n_blocks * 17^3 - 1 (16^3 blocks
plus the one-voxel apron) and the largest finest-level cell offset is N^3 - 1.  No GPU."""
import ctypes as ct
import os
import subprocess

import pytest

from paper_2302_12249_b300 import merf

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
GEO_RUNTIME, GEO_PAPER, GEO_GRID_ONLY = 0, 1, 2


@pytest.fixture(scope="module")
def geolib(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("geometry_host") / "libgeometry_host.so")
    subprocess.run(["g++", "-std=c++17", "-O1", "-shared", "-fPIC", "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(ROOT, "paper_2302_12249_b300", "csrc"),
                    os.path.join(HERE, "native", "geometry_host.cpp"), "-o", out], check=True)
    L = ct.CDLL(out)
    L.host_gather_geometry.argtypes = [ct.POINTER(merf.Desc)]
    L.host_gather_geometry.restype = ct.c_int
    L.host_paper_max_blocks.restype = ct.c_ulonglong
    return L


def paper_desc(n_blocks=15_000, occ=(128, 64, 32, 16)):
    d = merf.Desc()
    d.grid_res, d.block_size, d.plane_res, d.channels = 512, 16, 2048, 8
    d.n_blocks, d.n_occ_levels = n_blocks, len(occ)
    for i, r in enumerate(occ):
        d.occ_res[i] = r
    d.mlp_in, d.mlp_hidden, d.mlp_out = 34, 16, 3
    d.storage = merf.STORAGE_U8_SPARSE
    return d


def test_paper_scene_takes_the_paper_kernels(geolib):
    assert geolib.host_gather_geometry(ct.byref(paper_desc())) == GEO_PAPER


def test_block_limit_is_the_largest_32_bit_atlas(geolib):
    n = geolib.host_paper_max_blocks()
    assert n * 17 ** 3 - 1 <= 2 ** 32 - 1 < (n + 1) * 17 ** 3 - 1
    assert geolib.host_gather_geometry(ct.byref(paper_desc(n_blocks=n))) == GEO_PAPER
    assert geolib.host_gather_geometry(ct.byref(paper_desc(n_blocks=n + 1))) == GEO_RUNTIME


def test_occupancy_limit(geolib):
    assert geolib.host_gather_geometry(ct.byref(paper_desc(occ=(1024, 128, 16)))) == GEO_PAPER
    assert 1024 ** 3 - 1 < 2 ** 32
    assert geolib.host_gather_geometry(ct.byref(paper_desc(occ=(2048, 128, 16)))) == GEO_RUNTIME


def test_other_geometries(geolib):
    d = paper_desc()
    d.plane_res = 1024
    assert geolib.host_gather_geometry(ct.byref(d)) == GEO_RUNTIME
    d = paper_desc()
    d.plane_res = 0
    assert geolib.host_gather_geometry(ct.byref(d)) == GEO_GRID_ONLY
    d = paper_desc()
    d.block_size = 8
    assert geolib.host_gather_geometry(ct.byref(d)) == GEO_RUNTIME
    d = paper_desc()
    d.storage = merf.STORAGE_F32_DENSE
    assert geolib.host_gather_geometry(ct.byref(d)) == GEO_RUNTIME
