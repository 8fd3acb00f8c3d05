"""merf_render_host_noalloc: rendering into host memory for callers that cannot allocate device
memory (an application whose allocator owns the whole device pool, or a frame loop that must
not call cudaMalloc).  Its output must match merf_render's, call after call, although every call
reuses the library's one fixed staging area.

Kept in a file of its own that pytest collects last."""
import ctypes as ct

import numpy as np
import pytest
import torch

from paper_2302_12249_b300 import merf, synth
from tests import parity

pytestmark = pytest.mark.gpu


def _noalloc(gs, cams, W, H, step, pinned=True):
    """Call the entry point through the C ABI; returns the host image as numpy.  pinned False: the
    output is ordinary pageable host memory, which the copy out of the staging area must also
    serve."""
    cams = merf.cameras(cams)
    host = torch.full((cams.shape[0], H, W, 3), float("nan"), dtype=torch.float32, pin_memory=pinned)
    o = merf.opts(step)
    st = merf.lib().merf_render_host_noalloc(gs.handle, cams.ctypes.data_as(ct.c_void_p), cams.shape[0], W, H,
                                             ct.c_void_p(host.data_ptr()), ct.byref(o),
                                             torch.cuda.current_stream().cuda_stream)
    assert st == merf.MERF_OK, merf.lib().merf_last_error().decode()
    return host.numpy().copy()


def test_noalloc_matches_render_on_consecutive_calls(tiny_scene):
    gs = merf.Scene(tiny_scene)
    step = tiny_scene.cfg.step
    # two calls in a row with different cameras and sizes: the second must not see the first
    for n, W, H, seed in ((3, 64, 48, 21), (2, 40, 30, 22)):
        cams = synth.sphere_cameras(n, W, H, radius=3.0, seed=seed)
        ref = merf.render(gs, cams, W, H, step).cpu().numpy()
        got = _noalloc(gs, cams, W, H, step)
        assert np.isfinite(got).all()
        assert np.abs(got - ref).max() <= parity.RGB_TOL
    gs.close()


def test_noalloc_pageable_output_on_consecutive_calls(tiny_scene):
    """The same with pageable host output (not page-locked)."""
    gs = merf.Scene(tiny_scene)
    step = tiny_scene.cfg.step
    for n, W, H, seed in ((2, 56, 40, 23), (3, 32, 24, 24)):
        cams = synth.sphere_cameras(n, W, H, radius=3.0, seed=seed)
        ref = merf.render(gs, cams, W, H, step).cpu().numpy()
        got = _noalloc(gs, cams, W, H, step, pinned=False)
        assert np.isfinite(got).all()
        assert np.abs(got - ref).max() <= parity.RGB_TOL
    gs.close()


def test_noalloc_rejects_images_larger_than_its_staging_area(tiny_scene):
    gs = merf.Scene(tiny_scene)
    cams = merf.cameras(synth.config_cameras("tiny", W=1920, H=1080, n=2))   # 49.8 MB > 32 MiB
    host = torch.empty((2, 1080, 1920, 3), dtype=torch.float32)
    o = merf.opts(tiny_scene.cfg.step)
    st = merf.lib().merf_render_host_noalloc(gs.handle, cams.ctypes.data_as(ct.c_void_p), 2, 1920, 1080,
                                             ct.c_void_p(host.data_ptr()), ct.byref(o), None)
    assert st == merf.ERR_INVALID_ARG
    assert "staging area" in merf.lib().merf_last_error().decode()
    gs.close()
