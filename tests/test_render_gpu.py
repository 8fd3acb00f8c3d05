"""GPU parity of the FP32 render path against the FP64 oracle, through the C ABI."""
import dataclasses
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2302_12249_b300 import merf, synth
from tests import parity, scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tiny(tiny_scene):
    return merf.Scene(tiny_scene), oracle.OracleScene(tiny_scene)


@pytest.fixture(scope="module")
def paper(paper_scene):
    return merf.Scene(paper_scene), oracle.OracleScene(paper_scene)


def _words(nlat):
    return int(math.ceil(max(1, int(nlat.max())) / 32))


def test_tiny_full_image_parity(tiny):
    """Config: 64^3 grid in 8^3 blocks, 256^2 planes, 64x64 pixels, fov 60, radius 3, step 1/64."""
    gs, osc = tiny
    cams = synth.config_cameras("tiny")
    rgb, aux = parity.gpu_render(gs, cams, 64, 64, 1 / 64)
    lo, hi = parity.oracle_rgb(osc, cams, 64, 64, 1 / 64)
    err = parity.max_err(rgb, lo, hi)
    assert err.max() <= parity.RGB_TOL, err.max()
    np.testing.assert_array_equal(aux[:, merf.AUX_NLAT], lo[:, oracle.ORC_NLAT])
    assert (aux[:, merf.AUX_NEVAL] > 0).mean() > 0.2


@pytest.mark.parametrize("W,H", [(1, 1), (17, 9), (33, 70), (250, 131)])
def test_tiny_ragged_sizes(tiny, W, H):
    gs, osc = tiny
    cams = synth.config_cameras("tiny", W=W, H=H, n=2)
    rgb, _ = parity.gpu_render(gs, cams, W, H, 1 / 64)
    lo, hi = parity.oracle_rgb(osc, cams, W, H, 1 / 64)
    assert parity.max_err(rgb, lo, hi).max() <= parity.RGB_TOL


def test_tiny_without_termination(tiny):
    gs, osc = tiny
    cams = synth.config_cameras("tiny", W=48, H=40)
    rgb, aux = parity.gpu_render(gs, cams, 48, 40, 1 / 64, early_term=False)
    lo, _ = parity.oracle_rgb(osc, cams, 48, 40, 1 / 64, early_term=False)
    assert np.abs(rgb - lo[:, 0:3]).max() <= parity.RGB_TOL
    np.testing.assert_array_equal(aux[:, merf.AUX_NEVAL], lo[:, oracle.ORC_NEVAL])
    # transmittance carries the FP32 position noise times the steep log-density gradient of
    # small blobs on a 64^3 grid (~1e-4 relative); colour is the quantity held to 1e-4
    np.testing.assert_allclose(aux[:, merf.AUX_T], lo[:, oracle.ORC_T], atol=2e-4)


def test_tiny_traversal_bit_exact(tiny):
    """Evaluated lattice samples identical to the FP32 restatement of dense sampling."""
    gs, osc = tiny
    cams = synth.config_cameras("tiny", W=64, H=64, n=3)
    mask, nlat = merf.trace(gs, cams, 64, 64, 1 / 64, words=16)
    m_o, _, n_o = oracle.trace(osc, cams, 64, 64, 1 / 64, words=16, decide_f32=True)
    np.testing.assert_array_equal(nlat.cpu().numpy(), n_o)
    np.testing.assert_array_equal(mask.cpu().numpy().view(np.uint32), m_o)


def test_many_cameras_chunked_launches(tiny):
    """More cameras than one launch carries (32)."""
    gs, osc = tiny
    cams = synth.sphere_cameras(37, 8, 6, radius=2.5, seed=11)
    rgb, _ = parity.gpu_render(gs, cams, 8, 6, 1 / 64)
    lo, hi = parity.oracle_rgb(osc, cams, 8, 6, 1 / 64)
    assert parity.max_err(rgb, lo, hi).max() <= parity.RGB_TOL


def test_camera_inside_unit_cube_and_axis_aligned(tiny):
    """Rays starting inside the cube, and rays along the axes and diagonals (region ties)."""
    gs, osc = tiny
    recs = []
    for eye, tgt in [((0.1, 0.2, -0.3), (1, 0.2, -0.3)), ((0, 0, 0), (0, 0, 1)), ((0, 0, 0), (1, 1, 0)),
                     ((0.5, 0.5, 0.5), (2, 2, 2)), ((-3, 0, 0), (0, 0, 0))]:
        up = (0, 0, 1) if abs(np.subtract(tgt, eye)[2]) < 0.9 * np.linalg.norm(np.subtract(tgt, eye)) else (1, 0, 0)
        recs.append(synth.camera_record(synth.look_at(eye, tgt, up), 21, 21))
    cams = np.stack(recs)
    rgb, _ = parity.gpu_render(gs, cams, 21, 21, 1 / 64)
    lo, hi = parity.oracle_rgb(osc, cams, 21, 21, 1 / 64)
    assert parity.max_err(rgb, lo, hi).max() <= parity.RGB_TOL
    mask, nlat = merf.trace(gs, cams, 21, 21, 1 / 64, words=24)
    m_o, _, n_o = oracle.trace(osc, cams, 21, 21, 1 / 64, words=24, decide_f32=True)
    np.testing.assert_array_equal(mask.cpu().numpy().view(np.uint32), m_o)


def test_unusual_geometry_and_far_cameras():
    """Run-time gather geometry off the usual sizes (L = 96 in 32^3 blocks, R = 200 planes, two
    occupancy levels 32^3 / 8^3) and cameras far outside the scene (world distance 10 to 1000),
    whose rays start near the edge of contracted space."""
    cfg = synth.SceneConfig("odd", L=96, B=32, R=200, occ_res=(32, 8), n_blobs=24, inner_blobs=None,
                            step=1.0 / 64, peak_opacity=3.0)
    sc = synth.make_scene(cfg, seed=1234)
    gs, osc = merf.Scene(sc), oracle.OracleScene(sc)
    recs = [synth.camera_record(synth.look_at(np.array(e, float), (0, 0, 0)), 23, 17)
            for e in [(10.0, 0.3, 0.2), (-40.0, 25.0, 8.0), (0.5, -1000.0, 3.0), (2.2, 1.9, -1.7)]]
    cams = np.stack(recs)
    rgb, aux = parity.gpu_render(gs, cams, 23, 17, cfg.step)
    lo, hi = parity.oracle_rgb(osc, cams, 23, 17, cfg.step)
    assert parity.max_err(rgb, lo, hi).max() <= parity.RGB_TOL
    words = _words(aux[:, merf.AUX_NLAT])
    mask, nlat = merf.trace(gs, cams, 23, 17, cfg.step, words=words)
    m_o, _, n_o = oracle.trace(osc, cams, 23, 17, cfg.step, words=words, decide_f32=True)
    np.testing.assert_array_equal(nlat.cpu().numpy(), n_o)
    np.testing.assert_array_equal(mask.cpu().numpy().view(np.uint32), m_o)


def test_empty_and_full_occupancy():
    """No occupied cell: C = h(0, 0, d).  Every cell occupied: nothing is skipped."""
    for occ_val in (0, 1):
        sc = scenes.const_scene(L=16, B=4, R=32, occ_N=16, dens_byte=110, app_byte=90,
                                occ=np.full((16, 16, 16), occ_val, np.uint8), mlp=synth._mlp_weights(5))
        gs, osc = merf.Scene(sc), oracle.OracleScene(sc)
        cams = synth.sphere_cameras(2, 19, 11, radius=1.7, seed=3)
        rgb, aux = parity.gpu_render(gs, cams, 19, 11, 1 / 64)
        lo, hi = parity.oracle_rgb(osc, cams, 19, 11, 1 / 64)
        assert parity.max_err(rgb, lo, hi).max() <= parity.RGB_TOL
        if occ_val == 0:
            assert aux[:, merf.AUX_NEVAL].max() == 0


def test_missing_blocks_contribute_nothing():
    """A scene whose index grid drops occupied blocks: missing voxels add zero (both sides)."""
    rng = np.random.default_rng(9)
    sc = scenes.const_scene(L=16, B=4, R=32, occ_N=16, mlp=synth._mlp_weights(6))
    sc.atlas[...] = rng.integers(60, 200, size=sc.atlas.shape, dtype=np.uint8)
    sc.planes[...] = rng.integers(60, 200, size=sc.planes.shape, dtype=np.uint8)
    ig = sc.index_grid
    ig[rng.uniform(size=ig.shape) < 0.3] = -1
    gs, osc = merf.Scene(sc), oracle.OracleScene(sc)
    cams = synth.sphere_cameras(2, 32, 24, radius=2.2, seed=4)
    rgb, _ = parity.gpu_render(gs, cams, 32, 24, 1 / 64)
    lo, hi = parity.oracle_rgb(osc, cams, 32, 24, 1 / 64)
    assert parity.max_err(rgb, lo, hi).max() <= parity.RGB_TOL


def test_deterministic(tiny):
    gs, _ = tiny
    cams = synth.config_cameras("tiny")
    a = merf.render(gs, cams, 64, 64, 1 / 64)
    b = merf.render(gs, cams, 64, 64, 1 / 64)
    assert torch.equal(a, b)


def test_render_host_matches_device(tiny):
    """Page-locked output (written by the kernel directly, no staging) and pageable output
    (staged per camera and copied) both equal the device render."""
    gs, _ = tiny
    cams = synth.sphere_cameras(3, 50, 37, radius=2.8, seed=12)
    dev = merf.render(gs, cams, 50, 37, 1 / 64)
    pinned = torch.full(dev.shape, -1.0, dtype=torch.float32, pin_memory=True)
    merf.render_host(gs, cams, 50, 37, 1 / 64, None, pinned)
    assert torch.equal(pinned, dev.cpu())
    pageable = torch.full(dev.shape, -1.0, dtype=torch.float32)
    merf.render_host(gs, cams, 50, 37, 1 / 64, torch.empty_like(dev), pageable)
    assert torch.equal(pageable, dev.cpu())
    with pytest.raises(merf.MerfError):
        merf.render_host(gs, cams, 50, 37, 1 / 64, None, torch.empty(dev.shape, dtype=torch.float32))


def test_counters_match_aux(tiny):
    gs, _ = tiny
    cams = synth.config_cameras("tiny")
    aux = torch.zeros((1, 64, 64, merf.AUX_SIZE), device="cuda")
    cnt = torch.zeros(4, dtype=torch.int64, device="cuda")
    merf.render(gs, cams, 64, 64, 1 / 64, aux=aux, counters=cnt)
    a = aux.reshape(-1, merf.AUX_SIZE).double()
    c = cnt.cpu().tolist()
    assert c[merf.CNT_RAYS] == 64 * 64
    assert c[merf.CNT_LATTICE] == int(a[:, merf.AUX_NLAT].sum())
    assert c[merf.CNT_EVAL] == int(a[:, merf.AUX_NEVAL].sum())
    assert c[merf.CNT_APPEAR] == int(a[:, merf.AUX_NAPP].sum())


def test_dense_float_storage():
    """Dense float32 grid 128^3 and planes 512^2 (the differentiable variant's storage)."""
    sc = synth.make_scene("dense128")
    gs, osc = merf.Scene(sc), oracle.OracleScene(sc)
    cams = synth.config_cameras("dense128", W=64, H=48, n=2)
    rgb, _ = parity.gpu_render(gs, cams, 64, 48, sc.cfg.step)
    lo, hi = parity.oracle_rgb(osc, cams, 64, 48, sc.cfg.step)
    assert parity.max_err(rgb, lo, hi).max() <= parity.RGB_TOL


# ---------------------------------------------------------------------------------------------
# paper-scale scene (L = 512 in 16^3 blocks, R = 2048, four occupancy levels), 1920 x 1080,
# in the launch configuration the benchmark times; sampled pixels are checked one by one.

@pytest.mark.parametrize("W,H", [(1920, 1080), (1280, 720)])
def test_paper_scale_sampled_pixels(paper, W, H):
    """The 8 ring cameras at both of the workload's resolutions, each in one launch."""
    gs, osc = paper
    cams = synth.config_cameras("paper", W=W, H=H)          # 8 cameras
    step = 1 / 256
    out = merf.render(gs, cams, W, H, step)
    aux = torch.zeros((cams.shape[0], H, W, merf.AUX_SIZE), device="cuda")
    out2 = merf.render(gs, cams, W, H, step, aux=aux)
    torch.cuda.synchronize()
    assert torch.equal(out, out2)
    pix, lin = parity.pick_pixels(cams.shape[0], W, H, 3000, seed=0)
    rgb = out.reshape(-1, 3)[torch.from_numpy(lin).cuda()].double().cpu().numpy()
    lo, hi = parity.oracle_rgb(osc, cams, W, H, step, pix=pix)
    err = parity.max_err(rgb, lo, hi)
    assert err.max() <= parity.RGB_TOL, (err.max(), np.argmax(err))
    a = aux.reshape(-1, merf.AUX_SIZE)[torch.from_numpy(lin).cuda()].double().cpu().numpy()
    np.testing.assert_array_equal(a[:, merf.AUX_NLAT], lo[:, oracle.ORC_NLAT])
    assert np.isfinite(out.cpu().numpy()).all()


def test_paper_scale_traversal_bit_exact(paper):
    gs, osc = paper
    cams = synth.config_cameras("paper", W=480, H=270, n=2)
    mask, nlat = merf.trace(gs, cams, 480, 270, 1 / 256, words=64)
    m_o, _, n_o = oracle.trace(osc, cams, 480, 270, 1 / 256, words=64, decide_f32=True)
    np.testing.assert_array_equal(nlat.cpu().numpy(), n_o)
    np.testing.assert_array_equal(mask.cpu().numpy().view(np.uint32), m_o)


def test_paper_geometry_full_occupancy_reaches_the_edges(paper_scene):
    """Every occupancy cell set on the paper-scale scene: nothing is skipped, so rays that do not
    terminate are evaluated out to the limit point of contracted space, where the grid's
    clamp-to-edge and the planes' border texels are read (the kernel compiled for the paper's
    geometry).  Sampled pixels against the oracle, and the traversal bit for bit."""
    sc = dataclasses.replace(paper_scene, occ=[np.ones_like(o) for o in paper_scene.occ])
    gs, osc = merf.Scene(sc), oracle.OracleScene(sc)
    # cameras in the shell looking outward, one along an axis: rays cross the outer shell to
    # the limit point instead of ending in the central blobs
    eyes = [(1.2, 0.3, 0.2), (-0.4, 1.3, -0.3), (0.0, 0.0, 1.4)]
    cams = np.stack([synth.camera_record(synth.look_at(e, 3.0 * np.asarray(e), up=(0.3, 0.2, 1.0)), 240, 135)
                     for e in eyes])
    W, H, step = 240, 135, 1 / 256
    rgb, aux = parity.gpu_render(gs, cams, W, H, step)
    pix, lin = parity.pick_pixels(cams.shape[0], W, H, 1200, seed=5)
    lo, hi = parity.oracle_rgb(osc, cams, W, H, step, pix=pix)
    err = parity.max_err(rgb[lin], lo, hi)
    assert err.max() <= parity.RGB_TOL, (err.max(), np.argmax(err))
    a = aux[lin]
    reached = a[:, merf.AUX_NEVAL] == a[:, merf.AUX_NLAT]
    assert reached.sum() > 40                        # rays evaluated through to the far edge
    mask, nlat = merf.trace(gs, cams[:1], W, H, step, words=_words(aux[:, merf.AUX_NLAT]))
    m_o, _, n_o = oracle.trace(osc, cams[:1], W, H, step, words=mask.shape[-1], decide_f32=True)
    np.testing.assert_array_equal(nlat.cpu().numpy(), n_o)
    np.testing.assert_array_equal(mask.cpu().numpy().view(np.uint32), m_o)


def test_traversal_bit_exact_dense_scene_and_random_orbits():
    """Lattice counts and evaluated sets identical to the FP32 restatement for the dense scene's
    cameras and for random orbit cameras (radius 1.2 .. 3.5, every region of contracted space)."""
    sc = synth.make_scene("dense128")
    gs, osc = merf.Scene(sc), oracle.OracleScene(sc)
    sets = [synth.config_cameras("dense128", W=128, H=128, n=4)]
    rng = np.random.default_rng(21)
    sets.append(np.stack([synth.sphere_cameras(1, 96, 64, radius=float(r), seed=int(s))[0]
                          for r, s in zip(rng.uniform(1.2, 3.5, 12), rng.integers(0, 10 ** 6, 12))]))
    for cams in sets:
        W, H = (128, 128) if cams.shape[0] == 4 else (96, 64)
        mask, nlat = merf.trace(gs, cams, W, H, sc.cfg.step, words=40)
        m_o, _, n_o = oracle.trace(osc, cams, W, H, sc.cfg.step, words=40, decide_f32=True)
        np.testing.assert_array_equal(nlat.cpu().numpy(), n_o)
        np.testing.assert_array_equal(mask.cpu().numpy().view(np.uint32), m_o)


@pytest.mark.parametrize("prec", [merf.PREC_FP32, merf.PREC_FP16])
def test_render_is_graph_capturable(tiny, prec):
    """merf_render allocates nothing and does not synchronise: it captures into a CUDA graph, and
    a replay writes the same image as an eager call (the FP16 form includes the tcgen05 MLP)."""
    gs, _ = tiny
    cams = synth.config_cameras("tiny", W=40, H=24, n=3)
    ref = merf.render(gs, cams, 40, 24, 1 / 64, precision=prec)
    out = torch.zeros_like(ref)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        merf.render(gs, cams, 40, 24, 1 / 64, out=out, precision=prec)
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        merf.render(gs, cams, 40, 24, 1 / 64, out=out, precision=prec)
    out.zero_()
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    merf.check_device()


@pytest.mark.parametrize("n,W,H", [(1, 16384, 16), (1, 16, 16384), (32, 8192, 7629)])
def test_maximum_sizes(tiny, n, W, H):
    """The largest accepted images (16384 pixels on a side) and one call close to the 2e9-ray limit
    (32 cameras x 8192 x 7629 = 1.9999e9 rays, a 24 GB output): sampled pixels, including the
    corners of the last camera, against the oracle."""
    gs, osc = tiny
    cams = synth.sphere_cameras(n, W, H, radius=2.5, seed=71)
    out = merf.render(gs, cams, W, H, 1 / 64)
    torch.cuda.synchronize()
    pix, lin = parity.pick_pixels(n, W, H, 400, seed=72)
    last = np.array([[n - 1, 0, 0], [n - 1, W - 1, 0], [n - 1, 0, H - 1], [n - 1, W - 1, H - 1]], np.int32)
    pix = np.concatenate([pix, last]).astype(np.int32)
    lin = (pix[:, 0].astype(np.int64) * H + pix[:, 2]) * W + pix[:, 1]
    rgb = out.reshape(-1, 3)[torch.from_numpy(lin).cuda()].double().cpu().numpy()
    del out
    torch.cuda.empty_cache()
    lo, hi = parity.oracle_rgb(osc, cams, W, H, 1 / 64, pix=pix)
    assert parity.max_err(rgb, lo, hi).max() <= parity.RGB_TOL


def test_paper_sparsity_scene_sampled_pixels():
    """The paper-scale geometry at the paper's sparsity (blob radii U(0.01, 0.08): about 9 % of
    blocks stored, ~200 MB): sampled pixels of the bench cameras against the oracle."""
    sc = synth.make_scene("paper_sparse")
    assert 0.05 < sc.stats["block_fraction"] < 0.12
    gs, osc = merf.Scene(sc), oracle.OracleScene(sc)
    cams = synth.config_cameras("paper_sparse")
    W, H, step = 1920, 1080, 1 / 256
    rgb, aux = parity.gpu_render(gs, cams, W, H, step)
    pix, lin = parity.pick_pixels(cams.shape[0], W, H, 1500, seed=12)
    lo, hi = parity.oracle_rgb(osc, cams, W, H, step, pix=pix)
    err = parity.max_err(rgb[lin], lo, hi)
    assert err.max() <= parity.RGB_TOL, (err.max(), np.argmax(err))
    assert aux[lin, merf.AUX_NEVAL].mean() > 1.0          # the rays do meet the blobs


def test_device_layout_is_texel_pairs(tiny_scene):
    """The device layout the upload builds: every atlas voxel and plane texel stored as a 16-byte
    texel pair (with its +x / +u neighbour), atlas slots of (B+1)^3 pairs, planes bordered to
    (R+2)^2 pairs, plus the index grid, the occupancy levels and the 11,776-byte MLP block."""
    sc = tiny_scene
    gs = merf.Scene(sc)
    B, R = sc.cfg.B, sc.cfg.R
    want = (sc.n_blocks * (B + 1) ** 3 * 16 + 3 * (R + 2) ** 2 * 16 + sc.index_grid.nbytes
            + sum(o.nbytes for o in sc.occ) + 11776)
    assert gs.device_bytes == want
