"""GPU parity of the spherical-contraction ablation (Sec. 3.2, Table 2 (c)): mip-NeRF 360's
contraction marched densely (no empty-space skipping), against the FP64 oracle, through the C ABI."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2302_12249_b300 import merf, synth
from tests import parity

pytestmark = pytest.mark.gpu
SPH = merf.CONTRACT_SPHERICAL


def _oracle(osc, cams, W, H, step, pix=None):
    lo = oracle.render(osc, cams, W, H, step, pix=pix, t_term=2e-4 * (1 - parity.TERM_BAND), contraction=1)
    hi = oracle.render(osc, cams, W, H, step, pix=pix, t_term=2e-4 * (1 + parity.TERM_BAND), contraction=1)
    return lo, hi


def _render(gs, cams, W, H, step):
    aux = torch.zeros((cams.shape[0], H, W, merf.AUX_SIZE), device="cuda")
    out = merf.render(gs, cams, W, H, step, aux=aux, contraction=SPH)
    torch.cuda.synchronize()
    return out.reshape(-1, 3).double().cpu().numpy(), aux.reshape(-1, merf.AUX_SIZE).double().cpu().numpy()


def test_tiny_full_image_and_sample_sets(tiny_scene):
    gs, osc = merf.Scene(tiny_scene), oracle.OracleScene(tiny_scene)
    cams = synth.config_cameras("tiny", W=48, H=40, n=2)
    rgb, aux = _render(gs, cams, 48, 40, 1 / 64)
    lo, hi = _oracle(osc, cams, 48, 40, 1 / 64)
    err = parity.max_err(rgb, lo, hi)
    assert err.max() <= parity.RGB_TOL, (err.max(), np.argmax(err))
    np.testing.assert_array_equal(aux[:, merf.AUX_NLAT], lo[:, oracle.ORC_NLAT])
    n = oracle.sph_count(1 / 64, f32=True)
    words = int(math.ceil(n / 32))
    mask, nlat = merf.trace(gs, cams, 48, 40, 1 / 64, words=words, contraction=SPH)
    m_o, _, n_o = oracle.trace(osc, cams, 48, 40, 1 / 64, words=words, decide_f32=True, contraction=1)
    np.testing.assert_array_equal(nlat.cpu().numpy(), n_o)
    np.testing.assert_array_equal(mask.cpu().numpy().view(np.uint32), m_o)


def test_paper_scale_sampled_pixels(paper_scene):
    """The paper-scale scene (kernel compiled for its geometry) and the benchmark's cameras."""
    gs, osc = merf.Scene(paper_scene), oracle.OracleScene(paper_scene)
    cams = synth.config_cameras("paper")
    W, H, step = 1920, 1080, 1 / 256
    out = merf.render(gs, cams, W, H, step, contraction=SPH)
    torch.cuda.synchronize()
    pix, lin = parity.pick_pixels(cams.shape[0], W, H, 1500, seed=8)
    rgb = out.reshape(-1, 3)[torch.from_numpy(lin).cuda()].double().cpu().numpy()
    lo, hi = _oracle(osc, cams, W, H, step, pix=pix)
    err = parity.max_err(rgb, lo, hi)
    assert err.max() <= parity.RGB_TOL, (err.max(), np.argmax(err))


def test_dense_float_and_grid_only_scenes():
    """The ablation over the other storage / gather variants (dense float, grid only)."""
    for name, W, H in (("dense128", 40, 32), ("tiny_grid", 40, 32)):
        sc = synth.make_scene(name)
        gs, osc = merf.Scene(sc), oracle.OracleScene(sc)
        cams = synth.sphere_cameras(2, W, H, radius=2.2, seed=41)
        rgb, _ = _render(gs, cams, W, H, sc.cfg.step)
        lo, hi = _oracle(osc, cams, W, H, sc.cfg.step)
        assert parity.max_err(rgb, lo, hi).max() <= parity.RGB_TOL, name


def test_adjoint_refuses_the_ablation():
    sc = synth.make_scene("dense128")
    gs = merf.Scene(sc)
    cams = synth.config_cameras("dense128", W=8, H=8, n=1)
    d_out = torch.zeros((1, 8, 8, 3), device="cuda")
    o = merf.opts(sc.cfg.step, contraction=SPH)
    import ctypes as ct
    g = torch.zeros(1, device="cuda")
    st = merf.lib().merf_render_backward(gs.handle, merf.cameras(cams).ctypes.data, 1, 8, 8,
                                         ct.c_void_p(d_out.data_ptr()), ct.c_void_p(g.data_ptr()),
                                         ct.c_void_p(g.data_ptr()), ct.c_void_p(g.data_ptr()), ct.byref(o), None)
    assert st == merf.ERR_UNSUPPORTED
