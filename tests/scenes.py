"""Hand-built scenes for pin tests: every byte chosen by the test, no generator involved."""
import types

import numpy as np

from paper_2302_12249_b300 import synth


def const_scene(L=16, B=4, R=32, occ_N=16, dens_byte=128, app_byte=128, occ=None, mlp=None,
                all_blocks=True):
    """Block-sparse uint8 scene with every voxel / texel equal (density byte, appearance byte)."""
    cfg = synth.SceneConfig("const", L=L, B=B, R=R, occ_res=(occ_N,), n_blobs=0, inner_blobs=None,
                            step=1.0 / 64, peak_opacity=0.0)
    nb = L // B
    ids = np.arange(nb ** 3, dtype=np.int32).reshape(nb, nb, nb) if all_blocks else \
        np.full((nb, nb, nb), -1, np.int32)
    n = int((ids >= 0).sum())
    atlas = np.empty((n, B, B, B, 8), np.uint8)
    atlas[..., 0] = dens_byte
    atlas[..., 1:] = app_byte
    planes = np.empty((3, R, R, 8), np.uint8)
    planes[..., 0] = dens_byte
    planes[..., 1:] = app_byte
    if occ is None:
        occ = np.ones((occ_N,) * 3, np.uint8)
    if mlp is None:
        mlp = np.zeros(synth.MLP_PARAMS, np.float32)
    return synth.Scene(cfg=cfg, seed=0, occ=[occ], mlp=mlp, index_grid=ids, atlas=atlas, planes=planes)


def dequant(byte, m):
    return 2.0 * m * byte / 255.0 - m
