"""Pin of the oracle's adjoint: central finite differences of the FP64 forward on 64 parameters
of a dense float scene (grid, planes, MLP) -- CPU only."""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2302_12249_b300 import synth


def _scene():
    cfg = dataclasses.replace(synth.CONFIGS["dense128"], name="dense32", L=32, R=64, occ_res=(32, 8),
                              step=1.0 / 32)
    return synth.make_scene(cfg, seed=1234)


def _loss(osc, cams, pix, dl, step, early_term):
    out = oracle.render(osc, cams, 16, 16, step, pix=pix, early_term=early_term, decide_f32=False)
    return float((out[:, 0:3] * dl).sum())


@pytest.mark.parametrize("early_term", [False, True])
def test_adjoint_matches_central_differences(early_term):
    sc = _scene()
    osc = oracle.OracleScene(sc)
    cams = synth.sphere_cameras(2, 16, 16, radius=2.2, seed=17)
    rng = np.random.default_rng(5)
    pix = np.stack([rng.integers(0, 2, 40), rng.integers(0, 16, 40), rng.integers(0, 16, 40)], 1).astype(np.int32)
    dl = rng.normal(size=(40, 3))
    step = sc.cfg.step
    gg, gp, gm = oracle.render_grad(osc, cams, 16, 16, step, pix, dl, early_term=early_term, decide_f32=False)
    assert np.abs(gg).max() > 0 and np.abs(gp).max() > 0 and np.abs(gm).max() > 0
    picks = []
    for arr, g, n in ((sc.grid_f32, gg, 24), (sc.planes_f32, gp, 24), (sc.mlp, gm, 16)):
        flat = np.abs(g).ravel()
        top = np.argsort(flat)[-4 * n:]
        idx = rng.choice(top, size=n - 4, replace=False).tolist() + rng.integers(0, flat.size, 4).tolist()
        picks += [(arr, g, int(i)) for i in idx]
    assert len(picks) == 64
    worst = 0.0
    for arr, g, i in picks:
        a = arr.reshape(-1)
        p0 = a[i]
        h = np.float32(2.0 ** -12) * max(np.float32(1.0), abs(p0))
        a[i] = p0 + h
        hp = float(a[i]) - float(p0)
        lp = _loss(osc, cams, pix, dl, step, early_term)
        a[i] = p0 - h
        hm = float(p0) - float(a[i])
        lm = _loss(osc, cams, pix, dl, step, early_term)
        a[i] = p0
        fd = (lp - lm) / (hp + hm)
        an = float(g.reshape(-1)[i])
        err = abs(fd - an) / (1e-6 + abs(an) + 1e-3 * np.abs(g).max())
        worst = max(worst, err)
        assert abs(fd - an) <= 1e-6 + 2e-4 * abs(an) + 1e-5 * np.abs(g).max(), (i, fd, an)
    assert worst < 0.05
