"""FP64 CPU oracle of the MERF real-time renderer -- TEST INFRASTRUCTURE ONLY.

Only tests, ``__graft_entry__.smoke()`` and ``bench.py``'s oracle leg (its CPU
baseline, the reference values the precision form is scored against, the footprint
count) and reference arm may import this package.  The product path (the CUDA library and its
binding) never imports, links or executes anything here, and this package imports
nothing from the product.

The arithmetic lives in ``merf_oracle.c`` (plain C, double precision, built with
``-O2 -fno-fast-math -ffp-contract=off``); this module compiles it and marshals
numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "merf_oracle.c")
_HDR = os.path.join(_HERE, "merf_oracle.h")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "liborc.so")

ORC_OUT = 16
ORC_RGB, ORC_CD, ORC_F, ORC_T, ORC_NLAT, ORC_NEVAL, ORC_NAPP, ORC_TERM, ORC_SEGS = 0, 3, 6, 10, 11, 12, 13, 14, 15
MAX_SEGS = 16


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liborc.so (gcc, FP64, no contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= newest:
        return _SO
    tmp = _SO + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fno-fast-math", "-ffp-contract=off", "-fPIC", "-shared",
           "-pthread", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


class _Scene(ct.Structure):
    _fields_ = [("L", ct.c_int), ("B", ct.c_int), ("R", ct.c_int), ("C", ct.c_int),
                ("n_occ", ct.c_int), ("occ_res", ct.c_int * 8), ("occ", ct.c_void_p * 8),
                ("storage", ct.c_int), ("index_grid", ct.c_void_p), ("atlas", ct.c_void_p),
                ("n_blocks", ct.c_int), ("planes", ct.c_void_p), ("grid_f32", ct.c_void_p),
                ("planes_f32", ct.c_void_p), ("mlp", ct.c_void_p)]


class _Opts(ct.Structure):
    _fields_ = [("step", ct.c_double), ("t_term", ct.c_double), ("early_term", ct.c_int),
                ("decide_f32", ct.c_int), ("no_mlp", ct.c_int), ("contraction", ct.c_int)]


class _Seg(ct.Structure):
    _fields_ = [("region", ct.c_int), ("t0", ct.c_double), ("t1", ct.c_double),
                ("a", ct.c_double * 3), ("b", ct.c_double * 3), ("len", ct.c_double), ("s0", ct.c_double)]


class _Segs32(ct.Structure):
    _fields_ = [("n", ct.c_int), ("region", ct.c_int * MAX_SEGS), ("a", (ct.c_float * 3) * MAX_SEGS),
                ("e", (ct.c_float * 3) * MAX_SEGS), ("s0", ct.c_float * (MAX_SEGS + 1))]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ct.CDLL(build())
        D3 = ct.POINTER(ct.c_double)
        L.orc_region.argtypes = [D3]
        L.orc_region.restype = ct.c_int
        L.orc_contract.argtypes = [D3, D3]
        L.orc_contract_in_region.argtypes = [ct.c_int, D3, D3]
        L.orc_uncontract.argtypes = [ct.c_int, D3, D3]
        L.orc_ray.argtypes = [ct.c_void_p, ct.c_int, ct.c_int, D3, D3]
        L.orc_segments.argtypes = [D3, D3, ct.POINTER(_Seg)]
        L.orc_segments.restype = ct.c_int
        L.orc_t_of_s.argtypes = [ct.POINTER(_Seg), ct.c_int, D3, D3, ct.c_double]
        L.orc_t_of_s.restype = ct.c_double
        L.orc_point_at.argtypes = [ct.POINTER(_Seg), ct.c_int, ct.c_double, D3]
        L.orc_field.argtypes = [ct.POINTER(_Scene), D3, D3, ct.POINTER(ct.c_int)]
        L.orc_mlp.argtypes = [ct.c_void_p, D3, D3, D3, D3]
        L.orc_render.argtypes = [ct.POINTER(_Scene), ct.c_void_p, ct.c_int, ct.c_int, ct.c_int,
                                 ct.c_void_p, ct.c_int, ct.POINTER(_Opts), ct.c_void_p, ct.c_int]
        L.orc_render.restype = ct.c_int
        L.orc_trace.argtypes = [ct.POINTER(_Scene), ct.c_void_p, ct.c_int, ct.c_int, ct.c_int,
                                ct.c_void_p, ct.c_int, ct.c_double, ct.c_int, ct.c_double,
                                ct.c_void_p, ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_int, ct.c_int]
        L.orc_trace.restype = ct.c_int
        L.orc_trace_flagged.argtypes = L.orc_trace.argtypes + [ct.c_int]
        L.orc_trace_flagged.restype = ct.c_int
        L.orc_footprint.argtypes = [ct.POINTER(_Scene), ct.c_void_p, ct.c_int, ct.c_int, ct.c_int,
                                    ct.c_void_p, ct.c_int, ct.POINTER(_Opts), ct.c_void_p, ct.c_int]
        L.orc_footprint.restype = ct.c_int
        L.orc_contract_sph.argtypes = [D3, D3]
        L.orc_sph_t_of_s.argtypes = [ct.c_double]
        L.orc_sph_t_of_s.restype = ct.c_double
        L.orc_sph_count.argtypes = [ct.c_double]
        L.orc_sph_count.restype = ct.c_int
        L.orc32_sph_count.argtypes = [ct.c_float]
        L.orc32_sph_count.restype = ct.c_int
        L.orc32_sph_point.argtypes = [ct.c_void_p, ct.c_void_p, ct.c_float, ct.c_int, ct.c_void_p]
        L.orc_render_grad.argtypes = [ct.POINTER(_Scene), ct.c_void_p, ct.c_int, ct.c_int, ct.c_int, ct.c_void_p,
                                      ct.c_int, ct.POINTER(_Opts), ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p]
        L.orc_render_grad.restype = ct.c_int
        L.orc32_ray.argtypes = [ct.c_void_p, ct.c_int, ct.c_int, ct.c_void_p, ct.c_void_p]
        L.orc32_segments.argtypes = [ct.c_void_p, ct.c_void_p, ct.POINTER(_Segs32)]
        L.orc32_lattice_count.argtypes = [ct.POINTER(_Segs32), ct.c_float]
        L.orc32_lattice_count.restype = ct.c_int
        L.orc32_sample_cell.argtypes = [ct.POINTER(_Segs32), ct.c_float, ct.c_int, ct.c_int, ct.c_void_p]
        L.orc32_sample_cell.restype = ct.c_int
        _lib = L
    return _lib


def _d3(v) -> ct.Array:
    a = (ct.c_double * 3)()
    for k in range(3):
        a[k] = float(v[k])
    return a


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ct.c_void_p)


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


# ----------------------------------------------------------------------------------------------
# scalar entry points (pins)

def region(x) -> int:
    return lib().orc_region(_d3(x))


def contract(x) -> np.ndarray:
    p = (ct.c_double * 3)()
    lib().orc_contract(_d3(x), p)
    return np.array(p[:])


def contract_sph(x) -> np.ndarray:
    """The spherical contraction of mip-NeRF 360 (the ablation of Sec. 3.2 / Table 2 (c))."""
    p = (ct.c_double * 3)()
    lib().orc_contract_sph(_d3(x), p)
    return np.array(p[:])


def sph_t_of_s(s: float) -> float:
    return lib().orc_sph_t_of_s(float(s))


def sph_count(step: float, f32: bool = False) -> int:
    return lib().orc32_sph_count(float(step)) if f32 else lib().orc_sph_count(float(step))


def sph_point32(o, d, step: float, k: int) -> np.ndarray:
    """FP32 position of dense-march sample k (the kernel's rounding sequence)."""
    o32 = np.ascontiguousarray(o, dtype=np.float32)
    d32 = np.ascontiguousarray(d, dtype=np.float32)
    p = np.zeros(3, np.float32)
    lib().orc32_sph_point(_ptr(o32), _ptr(d32), float(step), int(k), _ptr(p))
    return p


def contract_in_region(r: int, x) -> np.ndarray:
    p = (ct.c_double * 3)()
    lib().orc_contract_in_region(int(r), _d3(x), p)
    return np.array(p[:])


def uncontract(r: int, p) -> np.ndarray:
    x = (ct.c_double * 3)()
    lib().orc_uncontract(int(r), _d3(p), x)
    return np.array(x[:])


def ray(cam: np.ndarray, i: int, j: int):
    cam = np.ascontiguousarray(cam, dtype=np.float32)
    o, d = (ct.c_double * 3)(), (ct.c_double * 3)()
    lib().orc_ray(_ptr(cam), i, j, o, d)
    return np.array(o[:]), np.array(d[:])


class Segments:
    """FP64 contracted segments of one ray (with the ray kept for t(s))."""

    def __init__(self, o, d):
        self.o, self.d = _d3(o), _d3(d)
        self._segs = (_Seg * MAX_SEGS)()
        self.n = lib().orc_segments(self.o, self.d, self._segs)

    def __len__(self):
        return self.n

    def __getitem__(self, i):
        g = self._segs[i]
        return dict(region=g.region, t0=g.t0, t1=g.t1, a=np.array(g.a[:]), b=np.array(g.b[:]),
                    len=g.len, s0=g.s0)

    @property
    def total(self) -> float:
        g = self._segs[self.n - 1]
        return g.s0 + g.len

    def t_of_s(self, s: float) -> float:
        return lib().orc_t_of_s(self._segs, self.n, self.o, self.d, float(s))

    def point_at(self, s: float) -> np.ndarray:
        p = (ct.c_double * 3)()
        lib().orc_point_at(self._segs, self.n, float(s), p)
        return np.array(p[:])


def mlp(w: np.ndarray, cd, f, d) -> np.ndarray:
    w = np.ascontiguousarray(w, dtype=np.float32)
    out = (ct.c_double * 3)()
    f4 = (ct.c_double * 4)(*[float(v) for v in f])
    lib().orc_mlp(_ptr(w), _d3(cd), ct.cast(f4, ct.POINTER(ct.c_double)), _d3(d), out)
    return np.array(out[:])


def ray32(cam: np.ndarray, i: int, j: int):
    cam = np.ascontiguousarray(cam, dtype=np.float32)
    o, d = np.zeros(3, np.float32), np.zeros(3, np.float32)
    lib().orc32_ray(_ptr(cam), i, j, _ptr(o), _ptr(d))
    return o, d


class Segments32:
    """FP32 decision replica of the kernel's segments for one ray."""

    def __init__(self, o32: np.ndarray, d32: np.ndarray):
        o32 = np.ascontiguousarray(o32, dtype=np.float32)
        d32 = np.ascontiguousarray(d32, dtype=np.float32)
        self._s = _Segs32()
        lib().orc32_segments(_ptr(o32), _ptr(d32), ct.byref(self._s))
        self.n = self._s.n
        self.region = list(self._s.region[: self.n])
        self.s0 = np.array(self._s.s0[: self.n + 1], dtype=np.float32)

    def lattice_count(self, step: float) -> int:
        return lib().orc32_lattice_count(ct.byref(self._s), ct.c_float(step))

    def sample_cell(self, step: float, k: int, N: int):
        c = np.zeros(3, np.int32)
        ok = lib().orc32_sample_cell(ct.byref(self._s), ct.c_float(step), int(k), int(N), _ptr(c))
        return c if ok else None


# ----------------------------------------------------------------------------------------------
# whole scenes

class OracleScene:
    """ctypes view of a baked scene (keeps the numpy arrays alive)."""

    def __init__(self, scene):
        self.scene = scene
        s = _Scene()
        cfg = scene.cfg
        s.L, s.R, s.C = cfg.L, cfg.R, 8
        s.B = cfg.B if cfg.storage == "u8" else 0
        self._occ = [np.ascontiguousarray(o, dtype=np.uint8) for o in scene.occ]
        s.n_occ = len(self._occ)
        for i, o in enumerate(self._occ):
            s.occ_res[i] = o.shape[0]
            s.occ[i] = o.ctypes.data
        self._mlp = np.ascontiguousarray(scene.mlp, dtype=np.float32)
        s.mlp = self._mlp.ctypes.data
        if cfg.storage == "u8":
            s.storage = 0
            self._ig = np.ascontiguousarray(scene.index_grid, dtype=np.int32)
            self._atlas = np.ascontiguousarray(scene.atlas, dtype=np.uint8)
            s.index_grid, s.atlas = self._ig.ctypes.data, self._atlas.ctypes.data
            if scene.planes is not None:            # grid-only scenes (R = 0) have none
                self._planes = np.ascontiguousarray(scene.planes, dtype=np.uint8)
                s.planes = self._planes.ctypes.data
            s.n_blocks = scene.n_blocks
        else:
            s.storage = 1
            self._grid = np.ascontiguousarray(scene.grid_f32, dtype=np.float32)
            self._pf = np.ascontiguousarray(scene.planes_f32, dtype=np.float32)
            s.grid_f32, s.planes_f32 = self._grid.ctypes.data, self._pf.ctypes.data
        self.s = s

    def field(self, p) -> np.ndarray:
        out = (ct.c_double * 8)()
        miss = ct.c_int(0)
        lib().orc_field(ct.byref(self.s), _d3(p), out, ct.byref(miss))
        return np.array(out[:]), miss.value


def render(oscene: OracleScene, cams: np.ndarray, W: int, H: int, step: float,
           pix: Optional[np.ndarray] = None, t_term: float = 2e-4, early_term: bool = True,
           decide_f32: bool = True, no_mlp: bool = False, threads: Optional[int] = None,
           contraction: int = 0) -> np.ndarray:
    """Render every pixel (or the (cam, col, row) triples in `pix`); returns [n, ORC_OUT] doubles.
    contraction 1: the spherical-contraction ablation, marched densely."""
    cams = np.ascontiguousarray(cams, dtype=np.float32).reshape(-1, 16)
    if pix is not None:
        pix = np.ascontiguousarray(pix, dtype=np.int32).reshape(-1, 3)
        n = pix.shape[0]
    else:
        n = cams.shape[0] * W * H
    out = np.zeros((n, ORC_OUT), dtype=np.float64)
    op = _Opts(step=step, t_term=t_term, early_term=int(early_term), decide_f32=int(decide_f32),
               no_mlp=int(no_mlp), contraction=int(contraction))
    lib().orc_render(ct.byref(oscene.s), _ptr(cams), cams.shape[0], W, H, _ptr(pix),
                     0 if pix is None else n, ct.byref(op), _ptr(out), threads or default_threads())
    return out


def footprint(oscene: OracleScene, cams: np.ndarray, W: int, H: int, step: float,
              pix: Optional[np.ndarray] = None, t_term: float = 2e-4, early_term: bool = True,
              threads: Optional[int] = None) -> dict:
    """Distinct grid voxels, plane texels and index entries read by the evaluated samples of the
    listed rays (uint8 scenes); bytes = 8 per voxel or texel, 4 per index entry."""
    cams = np.ascontiguousarray(cams, dtype=np.float32).reshape(-1, 16)
    if pix is not None:
        pix = np.ascontiguousarray(pix, dtype=np.int32).reshape(-1, 3)
    op = _Opts(step=step, t_term=t_term, early_term=int(early_term), decide_f32=1, no_mlp=0, contraction=0)
    counts = np.zeros(3, np.uint64)
    st = lib().orc_footprint(ct.byref(oscene.s), _ptr(cams), cams.shape[0], W, H, _ptr(pix),
                             0 if pix is None else pix.shape[0], ct.byref(op), _ptr(counts),
                             threads or default_threads())
    if st != 0:
        raise ValueError("footprint needs a uint8 block-sparse scene")
    g, p, i = (int(v) for v in counts)
    return {"grid_voxels": g, "plane_texels": p, "index_entries": i, "bytes": 8 * (g + p) + 4 * i}


def trace(oscene: OracleScene, cams: np.ndarray, W: int, H: int, step: float, words: int,
          pix: Optional[np.ndarray] = None, decide_f32: bool = True, eps: float = 2e-6,
          threads: Optional[int] = None, contraction: int = 0, decisive: bool = False):
    """Evaluated lattice-sample sets (termination off) as bit masks [n, words] + FP64 flags: every
    sample within eps of a cell face, or (decisive) only the samples whose outcome a move of eps
    can change (orc_trace_flagged)."""
    cams = np.ascontiguousarray(cams, dtype=np.float32).reshape(-1, 16)
    if pix is not None:
        pix = np.ascontiguousarray(pix, dtype=np.int32).reshape(-1, 3)
        n = pix.shape[0]
    else:
        n = cams.shape[0] * W * H
    mask = np.zeros((n, words), dtype=np.uint32)
    flags = np.zeros((n, words), dtype=np.uint32)
    nlat = np.zeros(n, dtype=np.int32)
    lib().orc_trace_flagged(ct.byref(oscene.s), _ptr(cams), cams.shape[0], W, H, _ptr(pix),
                            0 if pix is None else n, float(step), int(decide_f32), float(eps),
                            _ptr(mask), _ptr(flags), words, _ptr(nlat), threads or default_threads(),
                            int(contraction), int(decisive))
    return mask, flags, nlat


def render_grad(oscene: OracleScene, cams: np.ndarray, W: int, H: int, step: float, pix: np.ndarray,
                dl_drgb: np.ndarray, t_term: float = 2e-4, early_term: bool = False, decide_f32: bool = True):
    """Gradient of sum_pixels dl_drgb . C (dense float scenes): (g_grid, g_planes, g_mlp) in FP64."""
    sc = oscene.scene
    if sc.cfg.storage != "f32":
        raise ValueError("the adjoint is defined for dense float storage")
    cams = np.ascontiguousarray(cams, dtype=np.float32).reshape(-1, 16)
    pix = np.ascontiguousarray(pix, dtype=np.int32).reshape(-1, 3)
    dl = np.ascontiguousarray(dl_drgb, dtype=np.float64).reshape(-1, 3)
    L, R = sc.cfg.L, sc.cfg.R
    g_grid = np.zeros((L, L, L, 8), np.float64)
    g_planes = np.zeros((3, R, R, 8), np.float64)
    g_mlp = np.zeros(883, np.float64)
    op = _Opts(step=step, t_term=t_term, early_term=int(early_term), decide_f32=int(decide_f32), no_mlp=0)
    rc = lib().orc_render_grad(ct.byref(oscene.s), _ptr(cams), cams.shape[0], W, H, _ptr(pix), pix.shape[0],
                               ct.byref(op), _ptr(dl), _ptr(g_grid), _ptr(g_planes), _ptr(g_mlp))
    if rc != 0:
        raise ValueError(f"orc_render_grad failed ({rc})")
    return g_grid, g_planes, g_mlp
