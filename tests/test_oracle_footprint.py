"""Pin of the oracle's footprint count (the distinct data read beside the bandwidth roofline,
Sec. 5's access pattern): recomputed here with Python sets from the oracle's own evaluated
samples (trace) and contracted positions -- CPU only."""
import math

import numpy as np

import oracle
from paper_2302_12249_b300 import synth


def _lin(p, N):
    u = (p + 2.0) * N / 4.0 - 0.5
    a = math.floor(u)
    return min(max(a, 0), N - 1), min(max(a + 1, 0), N - 1)


def test_footprint_equals_a_set_recount():
    sc = synth.make_scene("tiny")
    osc = oracle.OracleScene(sc)
    cams = synth.config_cameras("tiny", W=16, H=12, n=1)
    W, H, step = 16, 12, 1 / 64
    rng = np.random.default_rng(4)
    pix = np.stack([np.zeros(25, int), rng.integers(0, W, 25), rng.integers(0, H, 25)], 1).astype(np.int32)
    got = oracle.footprint(osc, cams, W, H, step, pix=pix, early_term=False)
    words = 16                      # >= the longest lattice (384 samples at step 1/64)
    mask, _, nlat = oracle.trace(osc, cams, W, H, step, words=words, pix=pix)
    L, B, R = sc.cfg.L, sc.cfg.B, sc.cfg.R
    nb = L // B
    grid, planes, index = set(), set(), set()
    for r, (c, i, j) in enumerate(pix):
        o, d = oracle.ray(cams[c], int(i), int(j))
        segs = oracle.Segments(o, d)
        for k in range(int(nlat[r])):
            if not (int(mask[r, k >> 5]) >> (k & 31)) & 1:
                continue
            p = segs.point_at((k + 0.5) * step)
            xs, ys, zs = _lin(p[0], L), _lin(p[1], L), _lin(p[2], L)
            index.add((zs[0] // B, ys[0] // B, xs[0] // B))
            for z in zs:
                for y in ys:
                    for x in xs:
                        if sc.index_grid[z // B, y // B, x // B] >= 0:
                            grid.add((z, y, x))
            for q, (ca, ra) in enumerate([(1, 2), (0, 2), (0, 1)]):
                for v in _lin(p[ra], R):
                    for u in _lin(p[ca], R):
                        planes.add((q, v, u))
    assert got["grid_voxels"] == len(grid)
    assert got["plane_texels"] == len(planes)
    assert got["index_entries"] == len(index)
    assert got["bytes"] == 8 * (len(grid) + len(planes)) + 4 * len(index)
