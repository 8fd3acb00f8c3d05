"""Pins of the oracle's quadrature (Eq. 1, Eq. 2), early termination (Sec. 5), pinhole rays
and the deferred MLP (Sec. 2, App. B) -- CPU only."""
import math

import numpy as np
import pytest

import oracle
from paper_2302_12249_b300 import synth
from tests import scenes


def _cam_along(o, d, W=1, H=1):
    up = np.array([0.0, 0.0, 1.0]) if abs(d[2]) < 0.9 else np.array([1.0, 0.0, 0.0])
    cam = synth.camera_record(synth.look_at(o, np.asarray(o) + np.asarray(d), up), W, H)
    cam[14], cam[15] = W / 2.0, H / 2.0
    return cam


def _sig(x):
    return 1.0 / (1.0 + math.exp(-x))


def test_pinhole_ray():
    cam = synth.camera_record(synth.look_at([3.0, 1.0, 0.5]), 64, 48)
    o, d = oracle.ray(cam, 31, 23)          # pixel centre (31.5, 23.5) vs principal point (32, 24)
    np.testing.assert_allclose(o, [3.0, 1.0, 0.5], atol=1e-6)
    assert abs(np.linalg.norm(d) - 1) < 1e-15
    R = cam[:12].reshape(3, 4)[:, :3].astype(np.float64)
    dc = np.array([(31.5 - cam[14]) / cam[12], (23.5 - cam[15]) / cam[13], 1.0])
    np.testing.assert_allclose(d, R @ dc / np.linalg.norm(R @ dc), atol=1e-15)


def test_homogeneous_medium_inside_unit_cube():
    """Constant field occupied only inside [-3/4, 3/4]^3, ray from the origin: every evaluated
    step lies inside the unit cube, where world and contracted lengths agree, so delta = step,
    T = exp(-tau n step) and C_d = (1 - T) sigmoid(c~) exactly (telescoping of Eq. 1)."""
    N = 16
    occ = np.zeros((N, N, N), np.uint8)
    occ[5:11, 5:11, 5:11] = 1                      # cells of [-3/4, 3/4]^3
    db, ab = 120, 150
    sc = scenes.const_scene(occ_N=N, occ=occ, dens_byte=db, app_byte=ab)
    tau = math.exp(4 * scenes.dequant(db, 14.0))
    c = _sig(4 * scenes.dequant(ab, 7.0))
    step = 1.0 / 64
    rng = np.random.default_rng(0)
    for _ in range(10):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        cam = _cam_along([0.0, 0.0, 0.0], d)
        out = oracle.render(oracle.OracleScene(sc), cam[None], 1, 1, step, early_term=False,
                            decide_f32=False, no_mlp=True)[0]
        o, dd = oracle.ray(cam, 0, 0)
        n_inside = math.floor(0.75 / np.abs(dd).max() / step - 0.5) + 1   # samples with s_k < exit
        assert out[oracle.ORC_NEVAL] == n_inside
        T = math.exp(-tau * n_inside * step)
        assert abs(out[oracle.ORC_T] - T) < 1e-12
        np.testing.assert_allclose(out[oracle.ORC_CD:oracle.ORC_CD + 3], (1 - T) * c, atol=1e-12)


def test_homogeneous_medium_unbounded():
    """All cells occupied, constant density: T after all samples = exp(-tau t_end) with t_end the
    world distance to the end of the last lattice interval (computed here by brute force)."""
    db = 60
    sc = scenes.const_scene(occ_N=16, dens_byte=db, app_byte=200)
    tau = math.exp(4 * scenes.dequant(db, 14.0))
    step = 1.0 / 32
    rng = np.random.default_rng(1)
    for _ in range(8):
        o = rng.uniform(-2.5, 2.5, size=3)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        cam = _cam_along(o, d)
        out = oracle.render(oracle.OracleScene(sc), cam[None], 1, 1, step, early_term=False,
                            decide_f32=False, no_mlp=True)[0]
        oo, dd = oracle.ray(cam, 0, 0)
        n = int(out[oracle.ORC_NLAT])
        assert out[oracle.ORC_NEVAL] == n
        # brute force: contracted arc length along dense world samples, find t at s = n step
        u = np.linspace(0, 1 - 1e-4, 2_000_000)
        t = u / (1 - u) ** 2
        x = oo[None] + t[:, None] * dd[None]
        ax = np.abs(x)
        j = np.argmax(ax, axis=1)
        m = ax[np.arange(len(x)), j]
        reg = np.where(m <= 1, 0, 1 + 2 * j + (x[np.arange(len(x)), j] < 0))
        p = x.copy()
        out_i = m > 1
        p[out_i] = x[out_i] / m[out_i, None]
        p[out_i, j[out_i]] = np.sign(x[out_i, j[out_i]]) * (2 - 1 / m[out_i])
        seg = np.linalg.norm(np.diff(p, axis=0), axis=1) * (reg[1:] == reg[:-1])
        s = np.concatenate([[0], np.cumsum(seg)])
        t_end = np.interp(n * step, s, t)
        T = math.exp(-tau * t_end)
        assert abs(out[oracle.ORC_T] - T) < 1e-5 * max(T, 1e-3)
        c = _sig(4 * scenes.dequant(200, 7.0))
        np.testing.assert_allclose(out[oracle.ORC_CD:oracle.ORC_CD + 3], (1 - out[oracle.ORC_T]) * c, atol=1e-12)


def test_weights_sum_to_one_minus_transmittance(tiny_scene, tiny_oscene):
    """sum_i w_i = 1 - T_final <= 1 (Eq. 1): read through a scene whose colours are all equal."""
    sc = synth.make_scene("tiny")
    sc.atlas[..., 1:] = 255
    sc.planes[..., 1:] = 255
    c = _sig(4 * 7.0)
    cams = synth.config_cameras("tiny", W=24, H=24)
    out = oracle.render(oracle.OracleScene(sc), cams, 24, 24, 1 / 64, early_term=False,
                        decide_f32=False, no_mlp=True)
    wsum = out[:, oracle.ORC_CD] / c
    np.testing.assert_allclose(wsum, 1 - out[:, oracle.ORC_T], atol=1e-12)
    assert wsum.max() <= 1.0 + 1e-12 and wsum.min() >= 0.0
    np.testing.assert_allclose(out[:, oracle.ORC_F:oracle.ORC_F + 4], np.repeat(wsum[:, None] * c, 4, 1),
                               atol=1e-12)


def test_single_opaque_sample_takes_its_colour():
    """One occupied cell with a very dense field: C_d equals the colour there, T ~ 0."""
    N = 16
    occ = np.zeros((N, N, N), np.uint8)
    occ[8, 8, 8] = 1                                 # cell [0, 0.25)^3
    sc = scenes.const_scene(occ_N=N, occ=occ, dens_byte=255, app_byte=180)
    cam = _cam_along([0.125, 0.125, -0.5], [0.0, 0.0, 1.0])
    out = oracle.render(oracle.OracleScene(sc), cam[None], 1, 1, 1 / 64, early_term=False,
                        decide_f32=False, no_mlp=True)[0]
    c = _sig(4 * scenes.dequant(180, 7.0))
    assert out[oracle.ORC_NEVAL] == 16
    assert out[oracle.ORC_T] < 1e-300 or out[oracle.ORC_T] == 0.0
    np.testing.assert_allclose(out[oracle.ORC_CD:oracle.ORC_CD + 3], c, atol=1e-12)


def test_early_termination_bound():
    """Stopping once T < 2e-4 changes C_d by at most T_stop * max colour <= 2e-4 (Sec. 5)."""
    sc = scenes.const_scene(occ_N=16, dens_byte=150, app_byte=220)
    rng = np.random.default_rng(3)
    for _ in range(10):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        cam = _cam_along(rng.uniform(-0.5, 0.5, size=3), d)
        a = oracle.render(oracle.OracleScene(sc), cam[None], 1, 1, 1 / 64, early_term=True,
                          decide_f32=False, no_mlp=True)[0]
        b = oracle.render(oracle.OracleScene(sc), cam[None], 1, 1, 1 / 64, early_term=False,
                          decide_f32=False, no_mlp=True)[0]
        assert a[oracle.ORC_TERM] == 1 and a[oracle.ORC_T] < 2e-4
        assert a[oracle.ORC_NEVAL] < b[oracle.ORC_NEVAL]
        diff = np.abs(a[oracle.ORC_CD:oracle.ORC_CD + 3] - b[oracle.ORC_CD:oracle.ORC_CD + 3]).max()
        assert diff <= a[oracle.ORC_T] * 1.0 + 1e-15


def _posenc(d):
    out = [d]
    for l in range(4):
        out += [np.sin(2.0 ** l * d), np.cos(2.0 ** l * d)]
    return np.concatenate(out)


def test_mlp_is_the_matmul_chain():
    """h = W2 relu(W1 relu(W0 x + b0) + b1) + b2 on x = [C_d, F, gamma(d)] (App. B: 3 layers,
    16 hidden units, 4 frequencies), evaluated with numpy float64 matmuls."""
    rng = np.random.default_rng(4)
    w = synth._mlp_weights(77).astype(np.float64)
    W0 = w[:544].reshape(34, 16); b0 = w[544:560]
    W1 = w[560:816].reshape(16, 16); b1 = w[816:832]
    W2 = w[832:880].reshape(16, 3); b2 = w[880:883]
    for _ in range(50):
        cd, f = rng.uniform(size=3), rng.uniform(size=4)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        x = np.concatenate([cd, f, _posenc(d)])
        h = np.maximum(np.maximum(x @ W0 + b0, 0) @ W1 + b1, 0) @ W2 + b2
        np.testing.assert_allclose(oracle.mlp(synth._mlp_weights(77), cd, f, d), h, atol=1e-12)


def test_mlp_bias_only():
    w = np.zeros(synth.MLP_PARAMS, np.float32)
    w[880:883] = [0.25, -0.5, 0.125]
    np.testing.assert_allclose(oracle.mlp(w, [0.3, 0.2, 0.1], [0.5] * 4, [0, 0, 1]), [0.25, -0.5, 0.125])


def test_final_colour_adds_mlp_to_diffuse(tiny_oscene):
    """C = C_d + h(C_d, F, d) (Sec. 2)."""
    cams = synth.config_cameras("tiny", W=16, H=16)
    out = oracle.render(tiny_oscene, cams, 16, 16, 1 / 64)
    for r in range(0, 256, 17):
        o, d = oracle.ray(cams[0], r % 16, r // 16)
        h = oracle.mlp(tiny_oscene.scene.mlp, out[r, 3:6], out[r, 6:10], d)
        np.testing.assert_allclose(out[r, 0:3], out[r, 3:6] + h, atol=1e-12)


def test_fp32_decisions_agree_with_fp64_except_near_faces(tiny_oscene):
    """The FP32 restatement of the kernel's lattice/cell decisions differs from FP64 decisions
    only for samples within a few float ulps of a cell face."""
    cams = synth.config_cameras("tiny", W=64, H=64)
    m32, _, n32 = oracle.trace(tiny_oscene, cams, 64, 64, 1 / 64, words=16, decide_f32=True)
    m64, fl, n64 = oracle.trace(tiny_oscene, cams, 64, 64, 1 / 64, words=16, decide_f32=False, eps=2e-6)
    assert np.abs(n32 - n64).max() <= 1
    diff = (m32 ^ m64) & ~fl
    # a lattice sample that exists in only one precision (the last one) is allowed to differ
    for r in np.nonzero(diff.any(axis=1))[0]:
        bits = [k for k in range(512) if diff[r, k >> 5] >> (k & 31) & 1]
        assert bits == [min(n32[r], n64[r])] or bits == [max(n32[r], n64[r]) - 1]
