"""GPU tests of the serving form: continuous batching of mixed requests over resident scenes."""
import numpy as np
import pytest
import torch

from paper_2302_12249_b300 import merf, synth
from tests import parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def scenes(tiny_scene):
    other = synth.make_scene("tiny", seed=1007, mlp_seed=3007)
    return [merf.Scene(tiny_scene), merf.Scene(other)]


def _host(W, H):
    return torch.empty((H, W, 3), dtype=torch.float32, pin_memory=True)


def _reference(scene, cam, W, H, prec):
    return merf.render(scene, cam[None], W, H, 1 / 64, precision=prec)[0].cpu()


@pytest.mark.parametrize("prec", [merf.PREC_FP16, merf.PREC_FP32])
def test_single_request_equals_render(scenes, prec):
    srv = merf.Server(scenes, pool_bytes=1 << 24, step=1 / 64, precision=prec)
    cam = synth.config_cameras("tiny", W=50, H=37)[0]
    out = _host(50, 37)
    rid = srv.submit(0, cam, 50, 37, out)
    lat = srv.wait(rid)
    srv.close()
    assert lat > 0
    assert (out - _reference(scenes[0], cam, 50, 37, prec)).abs().max().item() <= parity.RGB_TOL


@pytest.mark.parametrize("prec", [merf.PREC_FP16, merf.PREC_FP32])
def test_paper_geometry_request_equals_render(paper_scene, prec):
    """With every resident scene in the paper's geometry the server runs the persistent kernel
    compiled for it; a request's image is the one merf_render gives."""
    g = merf.Scene(paper_scene)
    cams = synth.config_cameras("paper", W=320, H=180, n=2)
    srv = merf.Server([g], pool_bytes=1 << 26, step=1 / 256, precision=prec)
    outs = [_host(320, 180) for _ in range(2)]
    ids = [srv.submit(0, cams[k], 320, 180, outs[k]) for k in range(2)]
    for rid in ids:
        srv.wait(rid)
    srv.close()
    for k in range(2):
        ref = merf.render(g, cams[k][None], 320, 180, 1 / 256, precision=prec)[0].cpu()
        assert (outs[k] - ref).abs().max().item() <= parity.RGB_TOL


def test_same_alone_and_in_the_mix(scenes):
    """A request's image does not depend on what shares its iterations."""
    cam = synth.sphere_cameras(1, 61, 45, radius=2.6, seed=51)[0]
    srv = merf.Server(scenes, pool_bytes=1 << 24, step=1 / 64, max_tiles_per_iter=40)
    alone = _host(61, 45)
    srv.wait(srv.submit(1, cam, 61, 45, alone))
    rng = np.random.default_rng(3)
    ids, outs = [], []
    sizes = [(16, 16), (64, 36), (33, 70), (128, 72), (7, 5)]
    for k in range(24):
        W, H = sizes[k % len(sizes)]
        c = synth.sphere_cameras(1, W, H, radius=rng.uniform(1.2, 3.0), seed=100 + k)[0]
        o = _host(W, H)
        ids.append(srv.submit(int(rng.integers(0, 2)), c, W, H, o))
        outs.append((o, int(0), c, W, H))
        if k == 11:
            mixed = _host(61, 45)
            target = srv.submit(1, cam, 61, 45, mixed)
    for rid in ids + [target]:
        srv.wait(rid)
    st = srv.stats()
    srv.close()
    assert st["completed"] == st["submitted"] == 26
    assert st["iterations"] > 3
    assert (mixed - alone).abs().max().item() <= parity.RGB_TOL
    assert (alone - _reference(scenes[1], cam, 61, 45, merf.PREC_FP16)).abs().max().item() <= parity.RGB_TOL


def test_admission_is_limited_by_pool_memory(scenes):
    W, H = 64, 48
    img = W * H * 3 * 4
    srv = merf.Server(scenes, pool_bytes=2 * img + 4096, step=1 / 64, max_tiles_per_iter=16)
    cams = synth.sphere_cameras(8, W, H, radius=2.5, seed=77)
    outs = [_host(W, H) for _ in range(8)]
    ids = [srv.submit(k % 2, cams[k], W, H, outs[k]) for k in range(8)]
    for rid in ids:
        srv.wait(rid)
    st = srv.stats()
    srv.close()
    assert st["completed"] == 8
    assert st["peak_admitted"] <= 2
    assert st["peak_pool_bytes"] <= st["pool_bytes"]
    for k in range(8):
        ref = _reference(scenes[k % 2], cams[k], W, H, merf.PREC_FP16)
        assert (outs[k] - ref).abs().max().item() <= parity.RGB_TOL


def test_request_larger_than_pool_is_refused(scenes):
    srv = merf.Server(scenes, pool_bytes=1 << 16, step=1 / 64)
    cam = synth.config_cameras("tiny", W=128, H=128)[0]
    with pytest.raises(merf.MerfError) as e:
        srv.submit(0, cam, 128, 128, _host(128, 128))
    srv.close()
    assert e.value.status == merf.ERR_OOM


def test_wait_timeout_then_completion(scenes):
    srv = merf.Server(scenes, pool_bytes=1 << 26, step=1 / 64, max_tiles_per_iter=4)
    cam = synth.config_cameras("tiny", W=640, H=480)[0]
    out = _host(640, 480)
    rid = srv.submit(0, cam, 640, 480, out)
    with pytest.raises(TimeoutError):
        srv.wait(rid, timeout=0.0)
    srv.wait(rid, timeout=120.0)
    srv.close()
    assert (out - _reference(scenes[0], cam, 640, 480, merf.PREC_FP16)).abs().max().item() <= parity.RGB_TOL


def test_cancellation(scenes):
    """Requests withdrawn while queued or rendering end with ERR_CANCELLED and leave their host
    buffers unwritten; the others complete with merf_render's images, and the pool is free again."""
    W, H, n = 128, 96, 16
    srv = merf.Server(scenes, pool_bytes=2 * W * H * 3 * 4 + 4096, step=1 / 64, max_tiles_per_iter=8)
    cams = synth.sphere_cameras(n, W, H, radius=2.5, seed=91)
    outs = [_host(W, H).fill_(float("nan")) for _ in range(n)]
    ids = [srv.submit(k % 2, cams[k], W, H, outs[k]) for k in range(n)]
    withdrawn = {k for k in range(1, n, 2) if srv.cancel(ids[k])}
    assert len(withdrawn) >= n // 2 - 2                 # all but those already on their way out
    for k in range(n):
        if k in withdrawn:
            with pytest.raises(merf.MerfError) as e:
                srv.wait(ids[k])
            assert e.value.status == merf.ERR_CANCELLED
            assert torch.isnan(outs[k]).all()
        else:
            srv.wait(ids[k])
            ref = _reference(scenes[k % 2], cams[k], W, H, merf.PREC_FP16)
            assert (outs[k] - ref).abs().max().item() <= parity.RGB_TOL
    st = srv.stats()
    srv.close()
    assert st["cancelled"] == len(withdrawn) and st["completed"] == n - len(withdrawn)
    assert (st["pool_used_bytes"], st["admitted"], st["queued"]) == (0, 0, 0)


def test_four_paper_scenes_mixed_resolutions_against_oracle(paper_scene):
    """The serving workload at full size: four resident paper-scale scenes (seeds 1000-1003), orbit
    cameras at 256x256, 640x360, 1280x720 and 1920x1080, all requests in flight together in FP16;
    sampled pixels of every image against the FP64 oracle within the precision form's bars
    (2e-3 per channel, PSNR > 50 dB)."""
    import math
    import oracle
    scs = [paper_scene] + [synth.make_scene("paper", seed=synth.SEED_SCENE + k) for k in (1, 2, 3)]
    srv = merf.Server([merf.Scene(s) for s in scs], pool_bytes=1 << 30, step=1 / 256, max_tiles_per_iter=16384,
                      precision=merf.PREC_FP16)
    rng = np.random.default_rng(5)
    reqs = []
    for k, (W, H) in enumerate([(256, 256), (640, 360), (1280, 720), (1920, 1080)] * 2):
        r, az, el = rng.uniform(1.2, 3.0), rng.uniform(0, 2 * math.pi), math.radians(rng.uniform(-30, 30))
        eye = [r * math.cos(el) * math.cos(az), r * math.cos(el) * math.sin(az), r * math.sin(el)]
        cam = synth.camera_record(synth.look_at(eye), W, H)
        out = _host(W, H).fill_(float("nan"))
        s = (3 * k + 1) % 4
        reqs.append((s, cam, W, H, out, srv.submit(s, cam, W, H, out)))
    for *_, rid in reqs:
        srv.wait(rid, timeout=300.0)
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(reqs) and st["peak_admitted"] >= 2
    oscs = {}
    for k, (s, cam, W, H, out, _) in enumerate(reqs):
        osc = oscs.setdefault(s, oracle.OracleScene(scs[s]))
        pix, lin = parity.pick_pixels(1, W, H, 250, seed=60 + k)
        rgb = out.reshape(-1, 3)[torch.from_numpy(lin)].double().numpy()
        lo, hi = parity.oracle_rgb(osc, cam[None], W, H, 1 / 256, pix=pix)
        closer = np.where((np.abs(rgb - lo[:, 0:3]).max(1) <= np.abs(rgb - hi[:, 0:3]).max(1))[:, None],
                          lo[:, 0:3], hi[:, 0:3])
        err = np.abs(rgb - closer)
        assert err.max() <= 2e-3, (k, W, H, err.max())
        assert 10 * math.log10(1.0 / max(float(np.mean(err ** 2)), 1e-30)) > 50.0


def test_latency_phases_through_the_cuda_backend(scenes):
    """merf_server_wait_timed on the CUDA backend: every phase non-negative, the four adding up to
    the latency merf_server_wait reports, render time present for every request, and a request
    that waits behind a one-image pool shows admission time; the images stay correct."""
    W, H = 48, 40
    cams = synth.sphere_cameras(4, W, H, radius=2.6, seed=61)
    srv = merf.Server(scenes, pool_bytes=W * H * 3 * 4 + 255, step=1 / 64, max_tiles_per_iter=8)
    outs = [_host(W, H) for _ in range(4)]
    ids = [srv.submit(k % 2, cams[k], W, H, outs[k]) for k in range(4)]
    times = [srv.wait_timed(rid) for rid in ids]
    srv.close()
    for k, t in enumerate(times):
        parts = [t["admit_s"], t["queue_s"], t["render_s"], t["copy_s"]]
        assert min(parts) >= 0.0 and t["render_s"] > 0.0
        assert abs(sum(parts) - t["total_s"]) < 1e-9
        ref = _reference(scenes[k % 2], cams[k], W, H, merf.PREC_FP16)
        assert (outs[k] - ref).abs().max().item() <= parity.RGB_TOL
    # the pool holds one image, so the later requests waited for the earlier ones to leave it
    assert times[3]["admit_s"] >= times[0]["render_s"]
