"""Shared helpers of the GPU parity tests: run the CUDA path and the oracle on the same inputs
and compare.  The oracle takes its lattice and occupancy decisions in FP32 (the kernel's
precision), so the evaluated sample sets are identical; the early-termination decision
(T < t_term) is taken in each side's own arithmetic, so rays whose transmittance sits at the
threshold are accepted against either of two oracle runs with the threshold moved by
+-0.1 %."""
import numpy as np
import torch

import oracle
from paper_2302_12249_b300 import merf

RGB_TOL = 1e-4          # max |dRGB| per channel against the FP64 oracle (FP32 path)
TERM_BAND = 1e-3


def oracle_rgb(osc, cams, W, H, step, pix=None, early_term=True, t_term=2e-4, threads=None, decide_f32=True):
    """Two oracle renders (threshold moved down / up by TERM_BAND): [n, ORC_OUT] each.  decide_f32
    False: lattice and occupancy decisions of the FP64 definition itself."""
    lo = oracle.render(osc, cams, W, H, step, pix=pix, t_term=t_term * (1 - TERM_BAND), early_term=early_term,
                       decide_f32=decide_f32, threads=threads)
    if not early_term:
        return lo, lo
    hi = oracle.render(osc, cams, W, H, step, pix=pix, t_term=t_term * (1 + TERM_BAND), early_term=early_term,
                       decide_f32=decide_f32, threads=threads)
    return lo, hi


def gpu_render(scene, cams, W, H, step, early_term=True, t_term=2e-4):
    n = cams.shape[0]
    aux = torch.zeros((n, H, W, merf.AUX_SIZE), dtype=torch.float32, device="cuda")
    out = merf.render(scene, cams, W, H, step, early_term=early_term, t_term=t_term, aux=aux)
    torch.cuda.synchronize()
    return out.reshape(-1, 3).double().cpu().numpy(), aux.reshape(-1, merf.AUX_SIZE).double().cpu().numpy()


def max_err(gpu_rgb, lo, hi):
    """Per-pixel error against the closer of the two oracle variants."""
    e_lo = np.abs(gpu_rgb - lo[:, 0:3]).max(axis=1)
    e_hi = np.abs(gpu_rgb - hi[:, 0:3]).max(axis=1)
    return np.minimum(e_lo, e_hi)


def pick_pixels(n_cams, W, H, count, seed):
    rng = np.random.default_rng(seed)
    cam = rng.integers(0, n_cams, size=count)
    col = rng.integers(0, W, size=count)
    row = rng.integers(0, H, size=count)
    # always include the four corners of camera 0 (ragged tile edges)
    extra = np.array([[0, 0, 0], [0, W - 1, 0], [0, 0, H - 1], [0, W - 1, H - 1]])
    pix = np.concatenate([np.stack([cam, col, row], axis=1), extra]).astype(np.int32)
    lin = (pix[:, 0].astype(np.int64) * H + pix[:, 2]) * W + pix[:, 1]
    return pix, lin
