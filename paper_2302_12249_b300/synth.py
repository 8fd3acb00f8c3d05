"""Seeded synthetic inputs for the MERF renderer: baked scenes and pinhole cameras.

This module produces the *inputs* of the real-time renderer -- the arrays that the
paper's baking stage writes out (Sec. 4.3: a block-sparse uint8 3D grid, three uint8
feature planes, a max-pooled occupancy hierarchy, the deferred-MLP weights) -- plus
camera poses.  It holds none of the renderer's arithmetic: no contraction, no
interpolation, no dequantisation, no compositing.  Both the CUDA path and the
CPU oracle consume exactly the arrays returned here.

The fields are defined directly in contracted space p in [-2, 2]^3:

* density: tau(p) = A * sum_b exp(-|p - c_b|^2 / (2 s_b^2)) with s_b = r_b / 3 (a blob of
  radius r_b is its 3-sigma extent) and A * delta_s = `peak_opacity`; the grid stores
  log(tau) clipped to [-14, 14] (the density range m = 14 of Sec. 4.2);
* diffuse colour and features (7 channels): sums of seeded plane waves with
  wavelengths of at least 0.1 contracted units, split between the 3D grid and the
  three planes, in pre-sigmoid units clipped to [-7, 7] (m = 7 of Sec. 4.2);
* values are written as bytes with the rounding of Sec. 4.2, byte = floor(255 x + 1/2)
  with x = (v + m) / (2 m);
* the finest occupancy level marks a cell iff an upper bound of the opacity of one
  lattice step inside it exceeds 0.005 (the threshold of Sec. 4.3); outside the unit
  cube the step's world length is taken as delta_s / (2 - |p|_inf)^2 at the cell centre,
  capped at 16 delta_s; coarser levels are max-pools of the finest (Sec. 5);
* a 3D-grid block is stored iff some occupied finest cell can reach one of its voxels
  through trilinear interpolation, so the renderer never needs a missing voxel.

Gaussians and plane waves are separable along the axes, so every field is
evaluated with small tensor contractions (torch CPU) and full paper-size scenes
(L = 512, R = 2048) build in seconds.

Grid arrays are indexed [z][y][x] (x fastest), with C = 8 channels innermost:
channel 0 is density, 1..3 diffuse RGB, 4..7 the view-dependence feature.
Plane 0 is P_x(y, z) stored [z][y][c]; plane 1 is P_y(x, z) stored [z][x][c];
plane 2 is P_z(x, y) stored [y][x][c].  Texel i of a resolution-N array has its
centre at p = (i + 1/2) * 4 / N - 2.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional, Tuple

import numpy as np
import torch

C = 8                 # channels per texel (Sec. 3.1: C = 4 + K with K = 4)
M_DENSITY = 14.0      # dequantisation range of the density channel (Sec. 4.2)
M_APPEAR = 7.0        # dequantisation range of colour / feature channels (Sec. 4.2)
LOG_TAU_MIN = -14.0
MLP_IN, MLP_HIDDEN, MLP_OUT = 34, 16, 3
MLP_PARAMS = MLP_IN * MLP_HIDDEN + MLP_HIDDEN + MLP_HIDDEN * MLP_HIDDEN + MLP_HIDDEN + MLP_HIDDEN * MLP_OUT + MLP_OUT
OCC_ALPHA_THRESHOLD = 0.005  # Sec. 4.3

SEED_SCENE = 1000
SEED_CAMERA = 2000
SEED_MLP = 3000
SEED_ARRIVALS = 4000


@dataclasses.dataclass
class SceneConfig:
    name: str
    L: int                       # 3D grid resolution
    B: int                       # block edge (voxels); 0 = dense storage
    R: int                       # plane resolution
    occ_res: Tuple[int, ...]     # occupancy resolutions, finest first
    n_blobs: int
    inner_blobs: Optional[int]   # blobs inside the unit cube (rest in the shell); None = uniform
    step: float                  # lattice step delta_s in contracted arc length
    peak_opacity: float          # A * step: opacity scale of one step at a blob centre
    storage: str = "u8"          # "u8" (block-sparse bytes) or "f32" (dense float)
    radius_range: Tuple[float, float] = (0.05, 0.3)
    # grid only (R = 0): the SNeRG++-style baseline of the paper's Sec. 6 -- the same fields
    # (same seeded draws, planes included) sampled at the voxel centres of a finer 3D grid,
    # with no planes stored
    grid_only: bool = False


CONFIGS: Dict[str, SceneConfig] = {
    # 64^3 grid in 8^3 blocks, 256^2 planes, one 64^3 occupancy level, step 1/64.
    "tiny": SceneConfig("tiny", L=64, B=8, R=256, occ_res=(64,), n_blobs=32, inner_blobs=None,
                        step=1.0 / 64, peak_opacity=3.0),
    # Dense float grid 128^3 and planes 512^2 (the differentiable variant).
    "dense128": SceneConfig("dense128", L=128, B=0, R=512, occ_res=(128, 32), n_blobs=32,
                            inner_blobs=None, step=1.0 / 128, peak_opacity=3.0, storage="f32"),
    # Paper-scale: L = 512 in 16^3 blocks, R = 2048, occupancy at 1/16 .. 1/128 of R.
    "paper": SceneConfig("paper", L=512, B=16, R=2048, occ_res=(128, 64, 32, 16), n_blobs=256,
                         inner_blobs=128, step=1.0 / 256, peak_opacity=3.0),
    # Grid-only (SNeRG++-style) versions of the same contents: "tiny" at 64^3 and 128^3, and
    # the paper-scale scene at L = 512 / 1024 / 2048 with 16^3 blocks and no planes.
    "tiny_grid": SceneConfig("tiny_grid", L=64, B=8, R=0, occ_res=(64,), n_blobs=32, inner_blobs=None,
                             step=1.0 / 64, peak_opacity=3.0, grid_only=True),
    "tiny_grid128": SceneConfig("tiny_grid128", L=128, B=8, R=0, occ_res=(64,), n_blobs=32, inner_blobs=None,
                                step=1.0 / 64, peak_opacity=3.0, grid_only=True),
    "snerg512": SceneConfig("snerg512", L=512, B=16, R=0, occ_res=(128, 64, 32, 16), n_blobs=256,
                            inner_blobs=128, step=1.0 / 256, peak_opacity=3.0, grid_only=True),
    "snerg1024": SceneConfig("snerg1024", L=1024, B=16, R=0, occ_res=(128, 64, 32, 16), n_blobs=256,
                             inner_blobs=128, step=1.0 / 256, peak_opacity=3.0, grid_only=True),
    "snerg2048": SceneConfig("snerg2048", L=2048, B=16, R=0, occ_res=(128, 64, 32, 16), n_blobs=256,
                             inner_blobs=128, step=1.0 / 256, peak_opacity=3.0, grid_only=True),
    # The paper-scale configuration with smaller blobs (radii U(0.01, 0.08)): about 9 % of 16^3
    # blocks stored and about 200 MB of arrays, the sparsity and size of the paper's scenes
    # (Sec. 6: 198-233 MB each), beside its grid-only counterpart at SNeRG++'s default L = 2048.
    "paper_sparse": SceneConfig("paper_sparse", L=512, B=16, R=2048, occ_res=(128, 64, 32, 16), n_blobs=256,
                                inner_blobs=128, step=1.0 / 256, peak_opacity=3.0, radius_range=(0.01, 0.08)),
    "snerg2048_sparse": SceneConfig("snerg2048_sparse", L=2048, B=16, R=0, occ_res=(128, 64, 32, 16), n_blobs=256,
                                    inner_blobs=128, step=1.0 / 256, peak_opacity=3.0, radius_range=(0.01, 0.08),
                                    grid_only=True),
}

# the MERF configuration whose seeded draws a grid-only configuration shares
GRID_ONLY_BASE = {"tiny_grid": 256, "tiny_grid128": 256, "snerg512": 2048, "snerg1024": 2048, "snerg2048": 2048,
                  "snerg2048_sparse": 2048}


@dataclasses.dataclass
class Scene:
    cfg: SceneConfig
    seed: int
    occ: List[np.ndarray]                       # uint8 [N, N, N] per level, finest first
    mlp: np.ndarray                             # float32 [MLP_PARAMS]
    index_grid: Optional[np.ndarray] = None     # int32 [L/B]^3, block id or -1
    atlas: Optional[np.ndarray] = None          # uint8 [n_blocks, B, B, B, C]
    planes: Optional[np.ndarray] = None         # uint8 [3, R, R, C]
    grid_f32: Optional[np.ndarray] = None       # float32 [L, L, L, C] (dense storage)
    planes_f32: Optional[np.ndarray] = None     # float32 [3, R, R, C]
    stats: Dict[str, float] = dataclasses.field(default_factory=dict)

    @property
    def n_blocks(self) -> int:
        return 0 if self.atlas is None else int(self.atlas.shape[0])

    def baked_bytes(self) -> int:
        """Bytes of the baked arrays (8 bytes per texel, no apron or border): the representation's
        size, as a scene file stores it.  The library's device layout is larger
        (merf.Scene.device_bytes)."""
        n = sum(int(o.nbytes) for o in self.occ) + int(self.mlp.nbytes)
        for a in (self.index_grid, self.atlas, self.planes, self.grid_f32, self.planes_f32):
            if a is not None:
                n += int(a.nbytes) if isinstance(a, np.ndarray) else a.numel() * a.element_size()
        return n


# ----------------------------------------------------------------------------------------------
# field synthesis (separable factors)

def _centres(n: int, lo: float, hi: float) -> torch.Tensor:
    return (torch.arange(n, dtype=torch.float64) + 0.5) * ((hi - lo) / n) + lo


def _blobs(rng: np.random.Generator, cfg: SceneConfig):
    n = cfg.n_blobs
    if cfg.inner_blobs is None:
        c = rng.uniform(-2.0, 2.0, size=(n, 3))
    else:
        ni = cfg.inner_blobs
        inner = rng.uniform(-1.0, 1.0, size=(ni, 3))
        shell = []
        while len(shell) < n - ni:
            q = rng.uniform(-2.0, 2.0, size=(4 * (n - ni), 3))
            q = q[np.abs(q).max(axis=1) > 1.0]
            shell.extend(list(q))
        c = np.concatenate([inner, np.array(shell[: n - ni])], axis=0)
    r = rng.uniform(cfg.radius_range[0], cfg.radius_range[1], size=n)
    return torch.from_numpy(c), torch.from_numpy(r)


def _waves(rng: np.random.Generator, n_terms: int, dim: int, lam: Tuple[float, float], amp: float):
    """Plane waves a*sin(k.p + phi): random directions, wavelengths in `lam` (contracted units)."""
    v = rng.normal(size=(n_terms, dim))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    wl = rng.uniform(lam[0], lam[1], size=n_terms)
    k = v * (2.0 * math.pi / wl)[:, None]
    phi = rng.uniform(0.0, 2.0 * math.pi, size=n_terms)
    a = rng.normal(0.0, amp, size=n_terms)
    return torch.from_numpy(k), torch.from_numpy(phi), torch.from_numpy(a)


def _wave_factors(k: torch.Tensor, phi: torch.Tensor, a: torch.Tensor, axes: List[torch.Tensor]):
    """Complex separable factors: a*sin(k.p+phi) = Im(a e^{i phi} prod_d e^{i k_d p_d})."""
    coef = a.to(torch.complex128) * torch.exp(1j * phi.to(torch.complex128))
    facs = [torch.exp(1j * k[:, d:d + 1].to(torch.complex128) * ax[None, :].to(torch.complex128))
            for d, ax in enumerate(axes)]
    return coef, facs


def _quantise(v: torch.Tensor, m: float) -> torch.Tensor:
    """Byte code of a value in [-m, m] (the rounding of Sec. 4.2, eq. for q)."""
    x = (v.clamp(-m, m) + m) / (2.0 * m)
    return torch.floor(255.0 * x + 0.5).clamp(0, 255).to(torch.uint8)


def _mlp_weights(seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    w0 = rng.normal(0, math.sqrt(2.0 / MLP_IN), size=(MLP_IN, MLP_HIDDEN))
    b0 = rng.normal(0, 0.05, size=MLP_HIDDEN)
    w1 = rng.normal(0, math.sqrt(2.0 / MLP_HIDDEN), size=(MLP_HIDDEN, MLP_HIDDEN))
    b1 = rng.normal(0, 0.05, size=MLP_HIDDEN)
    w2 = rng.normal(0, 0.3 / math.sqrt(MLP_HIDDEN), size=(MLP_HIDDEN, MLP_OUT))
    b2 = rng.normal(0, 0.02, size=MLP_OUT)
    flat = np.concatenate([w0.ravel(), b0, w1.ravel(), b1, w2.ravel(), b2]).astype(np.float32)
    assert flat.size == MLP_PARAMS
    return flat


def make_scene(name_or_cfg, seed: Optional[int] = None, mlp_seed: int = SEED_MLP, device: str = "cpu") -> Scene:
    """Build a seeded baked scene.  `name_or_cfg` is a key of CONFIGS or a SceneConfig.  device
    "cuda" (uint8 grid-only scenes): the stored blocks are evaluated on the GPU and the atlas is
    returned as a CUDA tensor, for scenes whose atlas is too large to stage in host memory (the
    same fields and quantisation; values may differ from the CPU build in the last bits of FP64
    summation order, so a byte can differ where a value sits on a rounding boundary)."""
    cfg = CONFIGS[name_or_cfg] if isinstance(name_or_cfg, str) else name_or_cfg
    seed = SEED_SCENE if seed is None else seed
    rng = np.random.default_rng(seed)
    centres, radii = _blobs(rng, cfg)
    amp = cfg.peak_opacity / cfg.step
    # colour/feature waves: 3D part (long wavelengths) and one 2D set per plane
    vol_waves = [_waves(rng, 8, 3, (0.5, 2.0), 0.6) for _ in range(C - 1)]
    plane_waves = [[_waves(rng, 8, 2, (0.1, 0.5), 0.25) for _ in range(C - 1)] for _ in range(3)]
    plane_dens = [_waves(rng, 4, 2, (0.1, 0.5), 0.1) for _ in range(3)]

    L, R = cfg.L, cfg.R
    if cfg.grid_only:
        R = GRID_ONLY_BASE.get(cfg.name, 2048)     # only for evaluating the plane fields
    two_s2 = 2.0 * (radii / 3.0) ** 2

    def gauss(ax: torch.Tensor, d: int) -> torch.Tensor:          # [n_blobs, len(ax)]
        return torch.exp(-((ax[None, :] - centres[:, d:d + 1]) ** 2) / two_s2[:, None])

    # ---- occupancy: finest level by an opacity bound, coarser by max-pooling (Sec. 4.3, 5)
    nf = cfg.occ_res[0]
    edges = torch.linspace(-2.0, 2.0, nf + 1, dtype=torch.float64)
    lo, hi = edges[:-1], edges[1:]
    gb = []
    for d in range(3):
        c = centres[:, d:d + 1]
        dist = torch.clamp(lo[None, :] - c, min=0) + torch.clamp(c - hi[None, :], min=0)
        gb.append(torch.exp(-dist ** 2 / two_s2[:, None]))
    tau_max = amp * torch.einsum("bz,by,bx->zyx", gb[2], gb[1], gb[0])
    mid = _centres(nf, -2.0, 2.0)
    linf = torch.maximum(torch.maximum(mid.abs()[:, None, None], mid.abs()[None, :, None]),
                         mid.abs()[None, None, :])
    stretch = torch.where(linf <= 1.0, torch.ones_like(linf), (1.0 / (2.0 - linf) ** 2).clamp(max=16.0))
    alpha_max = 1.0 - torch.exp(-tau_max * cfg.step * stretch)
    finest = (alpha_max > OCC_ALPHA_THRESHOLD)
    occ = [finest.to(torch.uint8).numpy()]
    for n in cfg.occ_res[1:]:
        f = nf // n
        assert f * n == nf, "occupancy resolutions must divide the finest one"
        pooled = finest.reshape(n, f, n, f, n, f).any(dim=5).any(dim=3).any(dim=1)
        occ.append(pooled.to(torch.uint8).numpy())

    # ---- planes
    pax = _centres(R, -2.0, 2.0)
    # plane index -> (row axis, column axis) in world axes: P_x(y,z)[z][y], P_y(x,z)[z][x], P_z(x,y)[y][x]
    plane_axes = [(2, 1), (2, 0), (1, 0)]

    def plane_field(waves_list, m, ax=None) -> torch.Tensor:
        ax = pax if ax is None else ax
        out = []
        for (k, phi, a) in waves_list:
            coef, (fc, fr) = _wave_factors(k, phi, a, [ax, ax])   # k[:,0] -> column, k[:,1] -> row
            out.append(torch.einsum("t,tv,tu->vu", coef, fr, fc).imag)
        return out

    if cfg.grid_only:
        planes = None
    elif cfg.storage == "u8":
        planes = torch.empty((3, R, R, C), dtype=torch.uint8)
    else:
        planes = torch.empty((3, R, R, C), dtype=torch.float32)
    for pi in range(3 if planes is not None else 0):
        dens = plane_field([plane_dens[pi]], M_DENSITY)[0]
        app = plane_field(plane_waves[pi], M_APPEAR)
        if cfg.storage == "u8":
            planes[pi, :, :, 0] = _quantise(dens, M_DENSITY)
            for ch in range(C - 1):
                planes[pi, :, :, 1 + ch] = _quantise(app[ch], M_APPEAR)
        else:
            planes[pi, :, :, 0] = dens.to(torch.float32)
            for ch in range(C - 1):
                planes[pi, :, :, 1 + ch] = app[ch].clamp(-M_APPEAR, M_APPEAR).to(torch.float32)

    # ---- 3D grid values on a set of voxel boxes
    if device != "cpu" and not (cfg.grid_only and cfg.storage == "u8"):
        raise ValueError("device generation is for uint8 grid-only scenes")
    gax = _centres(L, -2.0, 2.0)
    gx, gy, gz = (gauss(gax, d).to(device) for d in range(3))
    vol_facs = [_wave_factors(k, phi, a, [gax, gax, gax]) for (k, phi, a) in vol_waves]
    vol_facs = [(coef.to(device), [f.to(device) for f in facs]) for coef, facs in vol_facs]
    # grid only: the plane fields evaluated at the grid's voxel centres, [3][C][L][L] (row, column)
    ptab = None
    if cfg.grid_only:
        ptab = torch.empty((3, C, L, L), dtype=torch.float64, device=device)
        for pi in range(3):
            ptab[pi, 0] = plane_field([plane_dens[pi]], M_DENSITY, gax)[0].to(device)
            for ch, v in enumerate(plane_field(plane_waves[pi], M_APPEAR, gax)):
                ptab[pi, 1 + ch] = v.to(device)

    def grid_values(z0: torch.Tensor, y0: torch.Tensor, x0: torch.Tensor, n: int) -> torch.Tensor:
        """Pre-quantisation values of boxes of n^3 voxels starting at (z0, y0, x0): [nb, n, n, n, C]."""
        ar = torch.arange(n, device=z0.device)
        iz, iy, ix = z0[:, None] + ar, y0[:, None] + ar, x0[:, None] + ar       # [nb, n]
        out = torch.empty((z0.shape[0], n, n, n, C), dtype=torch.float64, device=z0.device)
        tau = amp * torch.einsum("bkz,bky,bkx->bzyx", gz[:, iz].permute(1, 0, 2),
                                 gy[:, iy].permute(1, 0, 2), gx[:, ix].permute(1, 0, 2))
        out[..., 0] = torch.log(torch.clamp(tau, min=1e-30)).clamp(LOG_TAU_MIN, M_DENSITY)
        for ch in range(C - 1):
            coef, (fx, fy, fz) = vol_facs[ch]
            v = torch.einsum("t,bzt,byt,bxt->bzyx", coef, fz[:, iz].permute(1, 2, 0),
                             fy[:, iy].permute(1, 2, 0), fx[:, ix].permute(1, 2, 0)).imag
            out[..., 1 + ch] = v
        if ptab is not None:
            # + P_x(y, z)[z][y] + P_y(x, z)[z][x] + P_z(x, y)[y][x] at every voxel centre
            for c in range(C):
                out[..., c] += (ptab[0, c][iz[:, :, None], iy[:, None, :]][:, :, :, None]
                                + ptab[1, c][iz[:, :, None], ix[:, None, :]][:, :, None, :]
                                + ptab[2, c][iy[:, :, None], ix[:, None, :]][:, None, :, :])
        return out

    scene = Scene(cfg=cfg, seed=seed, occ=occ, mlp=_mlp_weights(mlp_seed))
    if cfg.storage == "u8":
        scene.planes = None if planes is None else planes.numpy()
        B = cfg.B
        nbx = L // B
        assert nbx * B == L
        # blocks reachable from occupied finest cells: a sample in cell c touches voxels
        # floor(u) and floor(u)+1 with u = (p+2)/4*L - 1/2 over the cell's extent.
        cells = torch.arange(nf, dtype=torch.float64)
        vlo = torch.floor(cells * (L / nf) - 0.5).clamp(0, L - 1).long()
        vhi = (torch.floor((cells + 1) * (L / nf) - 0.5) + 1).clamp(0, L - 1).long()
        blk = torch.arange(nbx)
        touch = ((vlo[:, None] // B <= blk[None, :]) & (vhi[:, None] // B >= blk[None, :])).to(torch.float32)
        need = torch.einsum("zyx,za,yb,xc->abc", finest.to(torch.float32), touch, touch, touch) > 0
        ids = torch.full((nbx, nbx, nbx), -1, dtype=torch.int32)
        bz, by, bx = torch.nonzero(need, as_tuple=True)
        nblk = int(bz.numel())
        ids[bz, by, bx] = torch.arange(nblk, dtype=torch.int32)
        atlas = torch.empty((nblk, B, B, B, C), dtype=torch.uint8, device=device)
        chunk = max(1, ((1 << 20) if device == "cpu" else (1 << 23)) // (B ** 3))
        bz, by, bx = bz.to(device), by.to(device), bx.to(device)
        for s in range(0, nblk, chunk):
            e = min(nblk, s + chunk)
            vals = grid_values(bz[s:e] * B, by[s:e] * B, bx[s:e] * B, B)
            atlas[s:e, ..., 0] = _quantise(vals[..., 0], M_DENSITY)
            for ch in range(1, C):
                atlas[s:e, ..., ch] = _quantise(vals[..., ch], M_APPEAR)
        scene.index_grid = ids.numpy()
        scene.atlas = atlas.numpy() if device == "cpu" else atlas
        scene.stats["block_fraction"] = nblk / float(nbx ** 3)
    else:
        z0 = torch.arange(0, L, 16)
        zz, yy, xx = torch.meshgrid(z0, z0, z0, indexing="ij")
        vals = grid_values(zz.reshape(-1), yy.reshape(-1), xx.reshape(-1), 16)
        nb = L // 16
        grid = vals.reshape(nb, nb, nb, 16, 16, 16, C).permute(0, 3, 1, 4, 2, 5, 6).reshape(L, L, L, C)
        grid[..., 1:] = grid[..., 1:].clamp(-M_APPEAR, M_APPEAR)
        scene.grid_f32 = grid.to(torch.float32).numpy()
        scene.planes_f32 = planes.numpy()
    scene.stats["occ_fraction"] = float(finest.float().mean())
    scene.stats["baked_mb"] = scene.baked_bytes() / 1e6
    return scene


# ----------------------------------------------------------------------------------------------
# cameras

def look_at(eye, target=(0.0, 0.0, 0.0), up=(0.0, 0.0, 1.0)) -> np.ndarray:
    """Camera-to-world 3x4 [R | t] with OpenCV axes (x right, y down, z forward)."""
    eye = np.asarray(eye, dtype=np.float64)
    f = np.asarray(target, dtype=np.float64) - eye
    f /= np.linalg.norm(f)
    r = np.cross(f, np.asarray(up, dtype=np.float64))
    r /= np.linalg.norm(r)
    dn = np.cross(f, r)
    m = np.zeros((3, 4))
    m[:, 0], m[:, 1], m[:, 2], m[:, 3] = r, dn, f, eye
    return m


def camera_record(c2w: np.ndarray, W: int, H: int, fov_y_deg: float = 60.0) -> np.ndarray:
    """One camera as 16 float32: c2w row-major 3x4, then fx, fy, cx, cy (pixels)."""
    fy = H / (2.0 * math.tan(math.radians(fov_y_deg) / 2.0))
    rec = np.concatenate([c2w.reshape(-1), [fy, fy, W / 2.0, H / 2.0]])
    return rec.astype(np.float32)


def sphere_cameras(n: int, W: int, H: int, radius: float, seed: int = SEED_CAMERA,
                   elev_deg: Tuple[float, float] = (-30.0, 30.0)) -> np.ndarray:
    """n cameras at `radius` with seeded azimuth/elevation, looking at the origin."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        az = rng.uniform(0.0, 2.0 * math.pi)
        el = math.radians(rng.uniform(*elev_deg))
        eye = radius * np.array([math.cos(el) * math.cos(az), math.cos(el) * math.sin(az), math.sin(el)])
        out.append(camera_record(look_at(eye), W, H))
    return np.stack(out)


def ring_cameras(n: int, W: int, H: int, radius: float = 1.5, seed: int = SEED_CAMERA) -> np.ndarray:
    """n cameras on a ring of `radius` in the z = 0 plane, +z up, looking at the origin."""
    rng = np.random.default_rng(seed)
    off = rng.uniform(0.0, 2.0 * math.pi / n)
    out = []
    for i in range(n):
        az = off + 2.0 * math.pi * i / n
        eye = radius * np.array([math.cos(az), math.sin(az), 0.0])
        out.append(camera_record(look_at(eye), W, H))
    return np.stack(out)


def config_cameras(name: str, W: Optional[int] = None, H: Optional[int] = None, n: Optional[int] = None):
    """The cameras each scene configuration is rendered from."""
    if name == "tiny":
        return sphere_cameras(n or 1, W or 64, H or 64, radius=3.0)
    if name == "dense128":
        return sphere_cameras(n or 4, W or 512, H or 512, radius=3.0)
    if name in ("paper", "paper_sparse"):
        return ring_cameras(n or 8, W or 1920, H or 1080, radius=1.5)
    raise KeyError(name)
