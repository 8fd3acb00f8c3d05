"""Pins of the oracle's feature field t~ = V + P_x + P_y + P_z (Sec. 3.1, Eq. 3) and of the
dequantisation (Sec. 4.2) -- CPU only."""
import dataclasses

import numpy as np

import oracle
from paper_2302_12249_b300 import synth
from tests import scenes


def test_dequantisation_end_points():
    """byte 0 -> -m, byte 255 -> +m for every source; four sources are summed."""
    for b, sgn in ((0, -1.0), (255, 1.0)):
        sc = scenes.const_scene(dens_byte=b, app_byte=b)
        t, miss = oracle.OracleScene(sc).field([0.1, -0.3, 0.7])
        assert miss == 0
        np.testing.assert_allclose(t[0], sgn * 4 * 14.0, atol=1e-12)
        np.testing.assert_allclose(t[1:], sgn * 4 * 7.0, atol=1e-12)


def test_dequantisation_step():
    """One byte step is 2m/255."""
    a = oracle.OracleScene(scenes.const_scene(dens_byte=100, app_byte=37)).field([0.2, 0.2, 0.2])[0]
    b = oracle.OracleScene(scenes.const_scene(dens_byte=101, app_byte=38)).field([0.2, 0.2, 0.2])[0]
    np.testing.assert_allclose(b - a, [4 * 28 / 255] + [4 * 14 / 255] * 7, atol=1e-12)


def _affine_scene(L=16, B=4, R=32, coef=(3, 5, 7), plane_coef=(2, 9)):
    """Grid bytes affine in the voxel index, plane bytes affine in the texel index."""
    sc = scenes.const_scene(L=L, B=B, R=R, dens_byte=0, app_byte=0)
    nb = L // B
    for bz in range(nb):
        for by in range(nb):
            for bx in range(nb):
                bid = sc.index_grid[bz, by, bx]
                z, y, x = np.meshgrid(np.arange(B) + bz * B, np.arange(B) + by * B, np.arange(B) + bx * B,
                                      indexing="ij")
                v = 10 + coef[0] * x + coef[1] * y + coef[2] * z
                sc.atlas[bid, ..., 1] = np.clip(v, 0, 255)
    rows, cols = np.meshgrid(np.arange(R), np.arange(R), indexing="ij")
    for q in range(3):
        sc.planes[q, :, :, 2] = np.clip(20 + plane_coef[0] * cols // 4 + plane_coef[1] * rows // 4, 0, 255)
        sc.planes[q, :, :, 3] = (np.arange(R)[None, :] + 0 * rows)          # byte = column index
        sc.planes[q, :, :, 4] = (np.arange(R)[:, None] + 0 * cols)          # byte = row index
    return sc


def test_trilinear_reproduces_affine_grid():
    """Linear interpolation is exact on affine data (away from the clamped edge texels)."""
    L = 16
    sc = _affine_scene(L=L)
    osc = oracle.OracleScene(sc)
    rng = np.random.default_rng(0)
    for p in rng.uniform(-2 + 8 / L, 2 - 8 / L, size=(300, 3)):
        t, _ = osc.field(p)
        u = (p + 2) * L / 4 - 0.5          # continuous voxel index of p (texel centres)
        byte = 10 + 3 * u[0] + 5 * u[1] + 7 * u[2]
        want = scenes.dequant(byte, 7.0) + 3 * scenes.dequant(0, 7.0)
        np.testing.assert_allclose(t[1], want, atol=1e-10)


def test_plane_axes():
    """P_x is indexed by (y, z), P_y by (x, z), P_z by (x, y): columns then rows (Eq. 3)."""
    R = 32
    sc = _affine_scene(R=R)
    osc = oracle.OracleScene(sc)
    rng = np.random.default_rng(1)
    for p in rng.uniform(-2 + 8 / R, 2 - 8 / R, size=(200, 3)):
        t, _ = osc.field(p)
        u = (p + 2) * R / 4 - 0.5
        # channel 3 byte = column index: columns are y for P_x, x for P_y and P_z
        col_sum = u[1] + u[0] + u[0]
        row_sum = u[2] + u[2] + u[1]
        want3 = scenes.dequant(col_sum, 7.0) + 2 * scenes.dequant(0, 7.0) * 0 + 3 * 0
        # each plane contributes dequant(col) = 14 col / 255 - 7; the grid contributes dequant(0)
        want3 = 14.0 * col_sum / 255.0 - 3 * 7.0 + scenes.dequant(0, 7.0)
        want4 = 14.0 * row_sum / 255.0 - 3 * 7.0 + scenes.dequant(0, 7.0)
        np.testing.assert_allclose(t[3], want3, atol=1e-10)
        np.testing.assert_allclose(t[4], want4, atol=1e-10)


def test_clamp_to_edge():
    """Outside the outer texel centres the edge texel value is held."""
    R = 32
    sc = _affine_scene(R=R)
    osc = oracle.OracleScene(sc)
    t_edge, _ = osc.field([-1.999, -1.999, 0.0])
    # for P_z the column (x) and row (y) indices both clamp to 0; P_x column y clamps to 0
    t_c, _ = osc.field([-2 + 2.0 / R, -2 + 2.0 / R, 0.0])     # exactly the first texel centre
    np.testing.assert_allclose(t_edge[3], t_c[3], atol=1e-10)


def test_block_sparse_equals_dense_and_missing_is_zero():
    """The block-sparse lookup gives the dense logical grid; a voxel of a block that is not
    stored contributes nothing (Sec. 4.3 stores only occupied blocks)."""
    rng = np.random.default_rng(2)
    L, B, R = 16, 4, 16
    sc = scenes.const_scene(L=L, B=B, R=R)
    sc.atlas[...] = rng.integers(0, 256, size=sc.atlas.shape, dtype=np.uint8)
    sc.planes[...] = rng.integers(0, 256, size=sc.planes.shape, dtype=np.uint8)
    nb = L // B
    # dense float copy of the logical grid (dequantised) with one block removed
    dense = np.zeros((L, L, L, 8), np.float32)
    m = np.array([14.0] + [7.0] * 7)
    for bz in range(nb):
        for by in range(nb):
            for bx in range(nb):
                blk = sc.atlas[sc.index_grid[bz, by, bx]].astype(np.float64)
                dense[bz * B:(bz + 1) * B, by * B:(by + 1) * B, bx * B:(bx + 1) * B] = 2 * m * blk / 255 - m
    drop = (1, 2, 1)
    sc.index_grid[drop] = -1
    dense[drop[0] * B:(drop[0] + 1) * B, drop[1] * B:(drop[1] + 1) * B, drop[2] * B:(drop[2] + 1) * B] = 0.0
    planes_f = (2 * m * sc.planes.astype(np.float64) / 255 - m).astype(np.float32)
    cfg = synth.SceneConfig("dense", L=L, B=0, R=R, occ_res=(16,), n_blobs=0, inner_blobs=None,
                            step=1 / 64, peak_opacity=0, storage="f32")
    dsc = synth.Scene(cfg=cfg, seed=0, occ=sc.occ, mlp=sc.mlp, grid_f32=dense, planes_f32=planes_f)
    a, b = oracle.OracleScene(sc), oracle.OracleScene(dsc)
    misses = 0
    for p in rng.uniform(-2, 2, size=(2000, 3)):
        ta, miss = a.field(p)
        tb, _ = b.field(p)
        misses += miss
        np.testing.assert_allclose(ta, tb, atol=2e-5)       # dense copy is float32
    assert misses > 0


def test_grid_only_scene_is_the_grid_alone():
    """R = 0 (the grid-only baseline of Sec. 6): t~ is the trilinear grid alone.  On an affine
    grid the value is the dequantised affine byte with no plane terms, and a scene with planes
    differs from its grid-only copy by exactly the bilinear plane terms, computed here apart."""
    L = 16
    sc = _affine_scene(L=L)
    g = dataclasses.replace(sc, cfg=dataclasses.replace(sc.cfg, R=0, grid_only=True), planes=None)
    osc, ogc = oracle.OracleScene(sc), oracle.OracleScene(g)
    rng = np.random.default_rng(7)
    R = sc.cfg.R
    m = np.array([14.0] + [7.0] * 7)
    planes = 2 * m * sc.planes.astype(np.float64) / 255 - m
    for p in rng.uniform(-2 + 8 / L, 2 - 8 / L, size=(200, 3)):
        t, _ = osc.field(p)
        tg, _ = ogc.field(p)
        u = (p + 2) * L / 4 - 0.5
        np.testing.assert_allclose(tg[1], scenes.dequant(10 + 3 * u[0] + 5 * u[1] + 7 * u[2], 7.0), atol=1e-10)
        # plane q: columns along axis (1, 0, 0)[q], rows along axis (2, 2, 1)[q]
        want = np.zeros(8)
        for q, (ca, ra) in enumerate([(1, 2), (0, 2), (0, 1)]):
            uc, ur = (p[ca] + 2) * R / 4 - 0.5, (p[ra] + 2) * R / 4 - 0.5
            c0, r0 = int(np.floor(uc)), int(np.floor(ur))
            fc, fr = uc - c0, ur - r0
            cl = lambda i: min(max(i, 0), R - 1)
            want += ((1 - fc) * (1 - fr) * planes[q, cl(r0), cl(c0)] + fc * (1 - fr) * planes[q, cl(r0), cl(c0 + 1)]
                     + (1 - fc) * fr * planes[q, cl(r0 + 1), cl(c0)] + fc * fr * planes[q, cl(r0 + 1), cl(c0 + 1)])
        np.testing.assert_allclose(t - tg, want, atol=1e-9)
