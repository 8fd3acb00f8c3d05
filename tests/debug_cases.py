"""Render cases run by both the release and the bounds-checked library (tests/test_debug_bounds_gpu.py):
every kernel variant -- uint8 FP32 / FP16, grid-only, dense float, the spherical ablation, the
trace kernel and the server's persistent kernel."""
import numpy as np
import torch

from paper_2302_12249_b300 import merf, synth


def _scene(name):
    return merf.Scene(synth.make_scene(name))


def _tiny(prec=merf.PREC_FP32, contraction=merf.CONTRACT_PI, name="tiny"):
    gs = _scene(name)
    cams = synth.sphere_cameras(2, 37, 29, radius=2.3, seed=5)
    out = merf.render(gs, cams, 37, 29, 1 / 64, precision=prec, contraction=contraction)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _dense():
    gs = _scene("dense128")
    cams = synth.config_cameras("dense128", W=40, H=32, n=2)
    out = merf.render(gs, cams, 40, 32, 1 / 128)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _trace():
    gs = _scene("tiny")
    cams = synth.sphere_cameras(1, 24, 20, radius=2.0, seed=6)
    mask, nlat = merf.trace(gs, cams, 24, 20, 1 / 64, words=16)
    torch.cuda.synchronize()
    return np.concatenate([mask.cpu().numpy().view(np.uint32).astype(np.float64).ravel(),
                           nlat.cpu().numpy().astype(np.float64)])


def _serve():
    gs = _scene("tiny")
    srv = merf.Server([gs], pool_bytes=1 << 24, step=1 / 64, precision=merf.PREC_FP16)
    cam = synth.sphere_cameras(1, 30, 22, radius=2.4, seed=7)[0]
    out = torch.empty((22, 30, 3), dtype=torch.float32, pin_memory=True)
    srv.wait(srv.submit(0, cam, 30, 22, out))
    srv.close()
    return out.numpy().copy()


CASES = {
    "u8_fp32": lambda: _tiny(),
    "u8_fp16": lambda: _tiny(merf.PREC_FP16),
    "grid_only": lambda: _tiny(name="tiny_grid"),
    "spherical": lambda: _tiny(contraction=merf.CONTRACT_SPHERICAL),
    "dense": _dense,
    "trace": _trace,
    "serve": _serve,
}
