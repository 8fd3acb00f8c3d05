"""CPU tests of the host's choice of gather variant (geometry.h).  The paper-geometry and grid-only
kernels index the atlas, the planes and the occupancy levels with 32-bit offsets, so the choice must
send every scene whose offsets could exceed 2^32 elsewhere: the largest voxel offset is
n_blocks * (B + 1)^3 - 1 (B^3 blocks plus the one-voxel apron) and the largest finest-level cell
offset is N^3 - 1.  No GPU."""
import ctypes as ct
import os
import subprocess

import pytest

from paper_2302_12249_b300 import merf

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
GEO_RUNTIME, GEO_PAPER, GEO_GRID_ONLY, GEO_GRID_ONLY_WIDE, GEO_DENSE_32 = 0, 1, 2, 3, 4


@pytest.fixture(scope="module")
def geolib(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("geometry_host") / "libgeometry_host.so")
    subprocess.run(["g++", "-std=c++17", "-O1", "-shared", "-fPIC", "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(ROOT, "paper_2302_12249_b300", "csrc"),
                    os.path.join(HERE, "native", "geometry_host.cpp"), "-o", out], check=True)
    L = ct.CDLL(out)
    L.host_gather_geometry.argtypes = [ct.POINTER(merf.Desc)]
    L.host_gather_geometry.restype = ct.c_int
    L.host_offsets_fit_32.argtypes = [ct.POINTER(merf.Desc)]
    L.host_offsets_fit_32.restype = ct.c_int
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


def largest_32_bit_atlas(B):
    """Most blocks of (B + 1)^3 voxels whose every voxel offset is below 2^32 (by search, not by the
    formula the header uses)."""
    lo, hi = 0, 2 ** 31
    while lo < hi:
        mid = (lo + hi + 1) // 2
        if mid * (B + 1) ** 3 - 1 <= 2 ** 32 - 1:
            lo = mid
        else:
            hi = mid - 1
    return lo


@pytest.mark.parametrize("B", [8, 16, 32])
def test_offsets_fit_32_at_the_block_limit(geolib, B):
    n = largest_32_bit_atlas(B)
    d = paper_desc(n_blocks=n)
    d.block_size = B
    assert geolib.host_offsets_fit_32(ct.byref(d)) == 1
    d.n_blocks = n + 1
    assert geolib.host_offsets_fit_32(ct.byref(d)) == 0


def test_block_limit_of_the_paper_geometry(geolib):
    n = largest_32_bit_atlas(16)
    assert n == 874204
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
    assert geolib.host_gather_geometry(ct.byref(d)) == GEO_DENSE_32


def test_grid_only_scenes_take_32_bit_offsets_only_when_they_fit(geolib):
    d = paper_desc(occ=(256, 64, 16))
    d.grid_res, d.plane_res = 2048, 0
    assert geolib.host_gather_geometry(ct.byref(d)) == GEO_GRID_ONLY
    d.n_blocks = largest_32_bit_atlas(16) + 1
    assert geolib.host_gather_geometry(ct.byref(d)) == GEO_GRID_ONLY_WIDE
    d = paper_desc(occ=(2048, 64, 16))
    d.plane_res = 0
    assert geolib.host_gather_geometry(ct.byref(d)) == GEO_GRID_ONLY_WIDE


def test_dense_scenes_take_32_bit_offsets_only_when_they_fit(geolib):
    """Dense float scenes hold 8 floats per grid texel and per plane texel.  The 32-bit variant forms
    float4 offsets in the forward pass and float offsets (8 per texel) in the adjoint's gradient
    scatter, so the bound is on floats: 8 L^3 and 24 R^2 must stay below 2^31, which admits
    L <= 645 and R <= 9459.  (An earlier bound of 2 L^3 admitted L up to 1023, where texel key * 8
    wrapped a signed 32-bit value.)"""
    def dense(L, R, occ=(128, 64, 32, 16)):
        d = paper_desc(occ=occ)
        d.storage, d.grid_res, d.plane_res = merf.STORAGE_F32_DENSE, L, R
        return d
    assert geolib.host_gather_geometry(ct.byref(dense(128, 512))) == GEO_DENSE_32
    L = max(l for l in range(1, 2000) if 8 * l ** 3 <= 2 ** 31 - 1)
    assert L == 645
    # the largest float offset of the adjoint's grid scatter: last texel's last float
    assert (L ** 3 - 1) * 8 + 7 <= 2 ** 31 - 1 < ((L + 1) ** 3 - 1) * 8 + 7
    assert geolib.host_gather_geometry(ct.byref(dense(L, 512))) == GEO_DENSE_32
    assert geolib.host_gather_geometry(ct.byref(dense(L + 1, 512))) == GEO_RUNTIME
    assert geolib.host_gather_geometry(ct.byref(dense(1023, 512))) == GEO_RUNTIME
    R = max(r for r in range(1, 30000) if 24 * r * r <= 2 ** 31 - 1)
    assert R == 9459
    assert (3 * R * R - 1) * 8 + 7 <= 2 ** 31 - 1 < (3 * (R + 1) ** 2 - 1) * 8 + 7
    assert geolib.host_gather_geometry(ct.byref(dense(128, R))) == GEO_DENSE_32
    assert geolib.host_gather_geometry(ct.byref(dense(128, R + 1))) == GEO_RUNTIME
    assert geolib.host_gather_geometry(ct.byref(dense(128, 512, occ=(2048, 64)))) == GEO_RUNTIME


def test_adjoint_scatter_widens_the_float_offset():
    """The gradient scatter forms its float offset in 64 bits (key * 8 with a 32-bit key could wrap
    if the bound above were ever loosened); the source states it."""
    src = open(os.path.join(ROOT, "paper_2302_12249_b300", "csrc", "backward.cuh")).read()
    assert "base + (long long)key * 8" in src
    assert "base + key * 8" not in src
