"""Seeded camera sets for the FP32-vs-FP64 decision tests at paper scale: the benchmark's ring,
random orbits, and cameras in the contracted shell looking outward, whose rays run out to the
limit point of contracted space (|p|_inf -> 2), where FP32 contracted positions are coarsest."""
import numpy as np

from paper_2302_12249_b300 import synth


def decision_cameras(W=1920, H=1080, n_each=8, seed=2026):
    rng = np.random.default_rng(seed)
    cams = list(synth.ring_cameras(n_each, W, H))
    for _ in range(n_each):            # random orbit: radius U(1.2, 3), elevation U(-30, 30) deg
        r, az, el = rng.uniform(1.2, 3.0), rng.uniform(0, 2 * np.pi), np.radians(rng.uniform(-30, 30))
        eye = r * np.array([np.cos(el) * np.cos(az), np.cos(el) * np.sin(az), np.sin(el)])
        cams.append(synth.camera_record(synth.look_at(eye), W, H))
    for _ in range(n_each):            # in the shell, looking away from the origin
        r, az, el = rng.uniform(1.1, 1.9), rng.uniform(0, 2 * np.pi), np.radians(rng.uniform(-40, 40))
        eye = r * np.array([np.cos(el) * np.cos(az), np.cos(el) * np.sin(az), np.sin(el)])
        cams.append(synth.camera_record(synth.look_at(eye, target=2.0 * eye), W, H))
    return np.asarray(cams, np.float32)


def random_pixels(n_cams, W, H, per_cam, seed=7):
    rng = np.random.default_rng(seed)
    cam = np.repeat(np.arange(n_cams), per_cam)
    pix = np.stack([cam, rng.integers(0, W, cam.size), rng.integers(0, H, cam.size)], axis=1)
    return pix.astype(np.int32)


def bits(mask):
    """[n, words] uint32 bit sets -> [n, 32 * words] 0/1."""
    return np.unpackbits(np.ascontiguousarray(mask).view(np.uint8), bitorder="little").reshape(mask.shape[0], -1)
