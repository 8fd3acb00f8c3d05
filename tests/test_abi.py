"""The C-ABI library builds, loads and exports every entry point of include/merf.h; host-side
argument checks reject bad input before touching a device -- CPU only (no compute calls)."""
import ctypes as ct
import os
import re

import numpy as np
import pytest

from paper_2302_12249_b300 import merf, synth

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "merf.h")


def _declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"\b(merf_[a-z_0-9]+)\s*\(", text)))


def test_header_declarations_are_exported():
    L = merf.lib()
    names = _declared()
    assert len(names) >= 10
    for name in names:
        assert hasattr(L, name), name
    assert set(names) == set(merf.EXPORTS)


def test_bounds_checked_library_exports_the_header_and_release_refuses_self_test():
    from paper_2302_12249_b300 import build as _b
    dbg = ct.CDLL(_b.build(debug=True))
    for name in merf.EXPORTS:
        assert hasattr(dbg, name), name
    dbg.merf_version.restype = ct.c_char_p
    assert b"bounds-checked" in dbg.merf_version()
    assert merf.lib().merf_check_device(None, 1) == merf.ERR_UNSUPPORTED
    assert merf.lib().merf_check_device(None, 3) == merf.ERR_INVALID_ARG
    assert merf.lib().merf_check_device(None, -1) == merf.ERR_INVALID_ARG


def test_version_string():
    assert "sm_103a" in merf.version()


def _desc(**kw):
    d = merf.Desc()
    d.grid_res, d.block_size, d.plane_res, d.channels, d.n_blocks = 16, 4, 32, 8, 0
    d.n_occ_levels = 1
    d.occ_res[0] = 16
    d.mlp_in, d.mlp_hidden, d.mlp_out = 34, 16, 3
    d.storage = 0
    for k, v in kw.items():
        setattr(d, k, v)
    return d


def _upload(d, ig=None, occ=None, mlp=None):
    L = merf.lib()
    nb = max(1, d.grid_res // max(1, d.block_size))
    ig = np.full(nb ** 3, -1, np.int32) if ig is None else ig
    planes = np.zeros(3 * d.plane_res * d.plane_res * 8, np.uint8)
    occ = [np.ones((d.occ_res[0],) * 3, np.uint8)] if occ is None else occ
    ptrs = (ct.c_void_p * 8)(*[o.ctypes.data for o in occ])
    mlp = np.zeros(883, np.float32) if mlp is None else mlp
    h = ct.c_void_p()
    st = L.merf_scene_upload(ct.byref(d), ig.ctypes.data, None, planes.ctypes.data, ct.cast(ptrs, ct.c_void_p),
                             mlp.ctypes.data, None, ct.byref(h))
    return st, L.merf_last_error().decode()


@pytest.mark.parametrize("field,value", [("channels", 4), ("grid_res", 15), ("block_size", 3),
                                         ("plane_res", 7), ("n_occ_levels", 0), ("n_occ_levels", 9),
                                         ("storage", 1), ("n_blocks", -1)])
def test_upload_rejects_bad_desc(field, value):
    st, msg = _upload(_desc(**{field: value}))
    assert st == merf.ERR_INVALID_ARG and msg


def test_grid_only_desc_passes_validation_and_dense_needs_planes():
    """plane_res 0 is a grid-only uint8 scene: it passes validation (the device budget then
    refuses it before anything is allocated); dense float storage still needs planes."""
    L = merf.lib()
    L.merf_set_device_budget(1)
    try:
        st, msg = _upload(_desc(plane_res=0))
        assert st == merf.ERR_OOM and "budget" in msg
    finally:
        L.merf_set_device_budget(0)
    d = _desc(plane_res=0, storage=1)
    h = ct.c_void_p()
    occ = [np.ones((16,) * 3, np.uint8)]
    ptrs = (ct.c_void_p * 8)(*[o.ctypes.data for o in occ])
    grid = np.zeros(16 ** 3 * 8, np.float32)
    mlp = np.zeros(883, np.float32)
    st = L.merf_scene_upload_dense(ct.byref(d), grid.ctypes.data, None, ct.cast(ptrs, ct.c_void_p),
                                   mlp.ctypes.data, None, ct.byref(h))
    assert st == merf.ERR_INVALID_ARG


def test_upload_rejects_unsupported_mlp():
    st, _ = _upload(_desc(mlp_hidden=32))
    assert st == merf.ERR_UNSUPPORTED


def test_upload_rejects_block_id_out_of_range():
    ig = np.full(64, -1, np.int32)
    ig[5] = 3                      # n_blocks = 0
    st, msg = _upload(_desc(), ig=ig)
    assert st == merf.ERR_INVALID_ARG and "index_grid" in msg


def test_upload_rejects_inconsistent_occupancy():
    d = _desc(n_occ_levels=2)
    d.occ_res[1] = 4
    fine = np.zeros((16, 16, 16), np.uint8)
    fine[3, 9, 12] = 1
    coarse = np.zeros((4, 4, 4), np.uint8)          # not a max-pool of `fine`
    st, msg = _upload(d, occ=[fine, coarse])
    assert st == merf.ERR_INVALID_ARG and "occupancy" in msg


def test_upload_rejects_non_finite_weights():
    mlp = np.zeros(883, np.float32)
    mlp[100] = np.nan
    st, _ = _upload(_desc(), mlp=mlp)
    assert st == merf.ERR_INVALID_ARG


def test_device_budget_refuses_before_allocating():
    merf.set_device_budget(1000)
    try:
        st, msg = _upload(_desc())
        assert st == merf.ERR_OOM and "budget" in msg
    finally:
        merf.set_device_budget(0)


def test_render_rejects_null_and_bad_sizes():
    L = merf.lib()
    o = merf.opts(1 / 64)
    cams = synth.config_cameras("tiny")
    assert L.merf_render(None, cams.ctypes.data, 1, 4, 4, None, ct.byref(o), None) == merf.ERR_INVALID_ARG
    fake = ct.c_void_p(1)          # never dereferenced: the size checks fail first
    assert L.merf_render(fake, cams.ctypes.data, 0, 4, 4, None, ct.byref(o), None) == merf.ERR_INVALID_ARG
    assert L.merf_render(fake, cams.ctypes.data, 1, 0, 4, None, ct.byref(o), None) == merf.ERR_INVALID_ARG
    assert L.merf_render(fake, None, 1, 4, 4, None, ct.byref(o), None) == merf.ERR_INVALID_ARG
    bad = cams.copy()
    bad[0, 12] = 0.0               # fx = 0
    assert L.merf_render(fake, bad.ctypes.data, 1, 4, 4, None, ct.byref(o), None) == merf.ERR_INVALID_ARG


def test_spherical_ablation_is_fp32_only():
    L = merf.lib()
    o = merf.opts(1 / 64, precision=merf.PREC_FP16, contraction=merf.CONTRACT_SPHERICAL)
    cams = synth.config_cameras("tiny")
    assert L.merf_render(ct.c_void_p(1), cams.ctypes.data, 1, 4, 4, ct.c_void_p(1), ct.byref(o), None) == \
        merf.ERR_UNSUPPORTED


@pytest.mark.parametrize("kw", [dict(step=0.0), dict(step=float("nan")), dict(t_term=1.5),
                                dict(early_term=2), dict(contraction=2), dict(contraction=-1)])
def test_render_rejects_bad_opts(kw):
    L = merf.lib()
    o = merf.opts(1 / 64)
    for k, v in kw.items():
        setattr(o, k, v)
    cams = synth.config_cameras("tiny")
    fake = ct.c_void_p(1)
    out = ct.c_void_p(1)
    assert L.merf_render(fake, cams.ctypes.data, 1, 4, 4, out, ct.byref(o), None) == merf.ERR_INVALID_ARG


def test_server_create_and_submit_reject_bad_arguments():
    L = merf.lib()
    o = merf.ServerOpts(pool_bytes=1 << 20, max_tiles_per_iter=128, precision=1, step=1 / 64, t_term=2e-4,
                        early_term=1, max_tiles_backlog=0)
    h = ct.c_void_p()
    assert L.merf_server_create(None, 1, ct.byref(o), ct.byref(h)) == merf.ERR_INVALID_ARG
    fake = (ct.c_void_p * 1)(1)
    assert L.merf_server_create(ct.cast(fake, ct.c_void_p), 0, ct.byref(o), ct.byref(h)) == merf.ERR_INVALID_ARG
    assert L.merf_server_create(ct.cast(fake, ct.c_void_p), 9, ct.byref(o), ct.byref(h)) == merf.ERR_INVALID_ARG
    for field, value in (("max_tiles_per_iter", 0), ("max_tiles_per_iter", 1 << 17), ("precision", 7),
                         ("max_tiles_backlog", 64), ("max_tiles_backlog", 1 << 17), ("pool_bytes", 16),
                         ("step", 0.0)):
        bad = merf.ServerOpts.from_buffer_copy(o)
        setattr(bad, field, value)
        assert L.merf_server_create(ct.cast(fake, ct.c_void_p), 1, ct.byref(bad), ct.byref(h)) == merf.ERR_INVALID_ARG
    rid = ct.c_uint64()
    cam = synth.config_cameras("tiny")
    assert L.merf_server_submit(None, 0, cam.ctypes.data, 4, 4, None, ct.byref(rid)) == merf.ERR_INVALID_ARG
    assert L.merf_server_wait(None, 1, 0.0, None) == merf.ERR_INVALID_ARG
    assert L.merf_server_cancel(None, 1, ct.byref(ct.c_int())) == merf.ERR_INVALID_ARG
    assert L.merf_server_get_stats(None, ct.byref(merf.ServerStats())) == merf.ERR_INVALID_ARG
