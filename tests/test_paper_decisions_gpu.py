"""The kernel's traversal and colours against the FP64 definition at paper scale (Sec. 3.2, Sec. 5).

The other GPU parity tests take the oracle's lattice and occupancy decisions in FP32 (the
kernel's precision), so that sample sets are identical by construction.  Here the reference is
the definition itself: the oracle's FP64 decisions, which flag the samples whose outcome a move
of eps = 8e-6 contracted units could change (the FP32 rounding measured on these rays stays
below 1.6e-6; tests/test_oracle_paper_decisions.py).  Outside the flags the kernel's evaluated
sets must equal the definition's bit for bit, and on rays with no flag its colours must match the
FP64-decision oracle within the FP32 bar."""
import numpy as np
import pytest
import torch

import oracle
from paper_2302_12249_b300 import merf
from tests import parity
from tests.decision_cams import decision_cameras, random_pixels

pytestmark = pytest.mark.gpu

STEP = 1.0 / 256
EPS = 8e-6
WORDS = 64


@pytest.fixture(scope="module")
def paper(paper_scene):
    return merf.Scene(paper_scene), oracle.OracleScene(paper_scene)


def _compare(gmask, gnlat, m64, fl, n64):
    """Words of the kernel's sets against the FP64 sets: equal outside flagged samples."""
    assert int(n64.max()) < 32 * WORDS
    for r in np.nonzero(gnlat != n64)[0]:
        lo = min(int(gnlat[r]), int(n64[r]))
        assert abs(int(gnlat[r]) - int(n64[r])) == 1 and (fl[r, lo >> 5] >> (lo & 31)) & 1, r
    bad = (gmask ^ m64) & ~fl
    assert not bad.any(), np.argwhere(bad)[:10]
    return int(np.bitwise_count(gmask ^ m64).sum()), float(fl.any(axis=1).mean())


def test_traversal_equals_fp64_definition_full_images(paper):
    """Every ray of 24 cameras (ring, random orbits, shell looking outward) at 240 x 135."""
    gs, osc = paper
    W, H = 240, 135
    cams = decision_cameras(W, H)
    mask, nlat = merf.trace(gs, cams, W, H, STEP, words=WORDS)
    gmask = mask.cpu().numpy().view(np.uint32)
    m64, fl, n64 = oracle.trace(osc, cams, W, H, STEP, words=WORDS, decide_f32=False, eps=EPS, decisive=True)
    changed, flagged = _compare(gmask, nlat.cpu().numpy(), m64, fl, n64)
    print(f"\nFP64 definition, {gmask.shape[0]} rays: {changed} samples differ, all flagged; "
          f"{100 * flagged:.2f} % of rays carry a flag")
    assert flagged < 0.10


def test_traversal_equals_fp64_definition_bench_cameras(paper):
    """The benchmark's 8 ring cameras at 1920 x 1080 (its launch), 4000 sampled rays."""
    gs, osc = paper
    W, H = 1920, 1080
    cams = decision_cameras(W, H)[:8]
    mask, nlat = merf.trace(gs, cams, W, H, STEP, words=WORDS)
    pix = random_pixels(8, W, H, per_cam=500, seed=11)
    lin = torch.as_tensor((pix[:, 0].astype(np.int64) * H + pix[:, 2]) * W + pix[:, 1], device="cuda")
    gmask = mask[lin].cpu().numpy().view(np.uint32)
    gnlat = nlat[lin].cpu().numpy()
    del mask, nlat
    m64, fl, n64 = oracle.trace(osc, cams, W, H, STEP, words=WORDS, pix=pix, decide_f32=False, eps=EPS,
                                decisive=True)
    _compare(gmask, gnlat, m64, fl, n64)


def test_colours_match_fp64_decisions_on_unflagged_rays(paper):
    """RGB of the bench launch (8 x 1920 x 1080) against the oracle with FP64 decisions, on
    sampled rays none of whose lattice samples is flagged."""
    gs, osc = paper
    W, H = 1920, 1080
    cams = decision_cameras(W, H)[:8]
    rgb, _ = parity.gpu_render(gs, cams, W, H, STEP)
    pix = random_pixels(8, W, H, per_cam=250, seed=13)
    _, fl, _ = oracle.trace(osc, cams, W, H, STEP, words=WORDS, pix=pix, decide_f32=False, eps=EPS, decisive=True)
    keep = ~fl.any(axis=1)
    assert keep.mean() > 0.9
    pix = pix[keep]
    lin = (pix[:, 0].astype(np.int64) * H + pix[:, 2]) * W + pix[:, 1]
    lo, hi = parity.oracle_rgb(osc, cams, W, H, STEP, pix=pix, decide_f32=False)
    err = parity.max_err(rgb[lin], lo, hi)
    assert err.max() <= parity.RGB_TOL, (err.max(), pix[np.argmax(err)])
