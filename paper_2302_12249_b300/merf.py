"""Python binding of the C-ABI renderer in libmerf.so (argument marshalling only).

Every step of rendering runs in the library's CUDA kernels; this module turns numpy arrays
and torch CUDA tensors into the plain pointers and structs of ``include/merf.h`` and turns
status codes into exceptions.  PyTorch supplies device memory and the current stream.
There is no CPU fallback: if the library cannot be built or loaded, every call raises.
"""
from __future__ import annotations

import ctypes as ct
import os
from typing import Optional, Sequence

import numpy as np
import torch

from . import build as _build

MERF_OK, ERR_INVALID_ARG, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_DEVICE_BOUNDS, ERR_UNSUPPORTED, ERR_CANCELLED = range(8)
STORAGE_U8_SPARSE, STORAGE_F32_DENSE = 0, 1
PREC_FP32, PREC_FP16, PREC_BF16 = 0, 1, 2
MAX_OCC_LEVELS = 8
AUX_SIZE = 12
NOALLOC_STAGING_BYTES = 32 << 20
AUX_CD, AUX_F, AUX_T, AUX_NLAT, AUX_NEVAL, AUX_NAPP, AUX_TERM = 0, 3, 7, 8, 9, 10, 11
CNT_RAYS, CNT_LATTICE, CNT_EVAL, CNT_APPEAR = 0, 1, 2, 3

EXPORTS = ("merf_scene_upload", "merf_scene_upload_dense", "merf_scene_upload_device", "merf_scene_load",
           "merf_scene_free",
           "merf_scene_device_bytes", "merf_render", "merf_render_aux", "merf_render_host", "merf_render_host_noalloc",
           "merf_trace", "merf_set_device_budget", "merf_scene_set_dense", "merf_scene_param_version",
           "merf_render_backward",
           "merf_render_backward_aux", "merf_server_create", "merf_server_submit", "merf_server_wait",
           "merf_server_wait_timed", "merf_server_cancel", "merf_server_get_stats", "merf_server_destroy",
           "merf_check_device",
           "merf_last_error", "merf_version")


class MerfError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"merf status {status}: {msg}")
        self.status = status


class Desc(ct.Structure):
    _fields_ = [("grid_res", ct.c_int32), ("block_size", ct.c_int32), ("plane_res", ct.c_int32),
                ("channels", ct.c_int32), ("n_blocks", ct.c_int32), ("n_occ_levels", ct.c_int32),
                ("occ_res", ct.c_int32 * MAX_OCC_LEVELS), ("mlp_in", ct.c_int32), ("mlp_hidden", ct.c_int32),
                ("mlp_out", ct.c_int32), ("storage", ct.c_int32)]


class Opts(ct.Structure):
    _fields_ = [("step", ct.c_float), ("t_term", ct.c_float), ("precision", ct.c_int32),
                ("early_term", ct.c_int32), ("contraction", ct.c_int32)]


class ServerOpts(ct.Structure):
    _fields_ = [("pool_bytes", ct.c_size_t), ("max_tiles_per_iter", ct.c_int32), ("precision", ct.c_int32),
                ("step", ct.c_float), ("t_term", ct.c_float), ("early_term", ct.c_int32),
                ("max_tiles_backlog", ct.c_int32)]


class ServerStats(ct.Structure):
    _fields_ = [("submitted", ct.c_ulonglong), ("completed", ct.c_ulonglong), ("rays", ct.c_ulonglong),
                ("iterations", ct.c_ulonglong), ("tiles", ct.c_ulonglong), ("cancelled", ct.c_ulonglong),
                ("pool_bytes", ct.c_size_t), ("peak_pool_bytes", ct.c_size_t), ("pool_used_bytes", ct.c_size_t),
                ("peak_admitted", ct.c_int32), ("admitted", ct.c_int32), ("queued", ct.c_int32),
                ("reserved", ct.c_int32)]


class RequestTiming(ct.Structure):
    _fields_ = [("total_s", ct.c_double), ("admit_s", ct.c_double), ("queue_s", ct.c_double),
                ("render_s", ct.c_double), ("copy_s", ct.c_double)]


_lib = None
_debug = False


def use_debug_build():
    """Load the bounds-checked library (libmerf_debug.so) instead of the release one; call before
    the first use of the library in this process."""
    global _debug
    if _lib is not None:
        raise RuntimeError("the library is already loaded")
    _debug = True


def lib():
    """Load libmerf.so, building it in-tree with nvcc first if it is missing or stale."""
    global _lib
    if _lib is None:
        path = _build.build(debug=True) if _debug else _build.build()
        L = ct.CDLL(path)
        vp, i32 = ct.c_void_p, ct.c_int
        L.merf_scene_upload.argtypes = [ct.POINTER(Desc), vp, vp, vp, vp, vp, vp, ct.POINTER(vp)]
        L.merf_scene_upload_dense.argtypes = [ct.POINTER(Desc), vp, vp, vp, vp, vp, ct.POINTER(vp)]
        L.merf_scene_upload_device.argtypes = [ct.POINTER(Desc), vp, vp, vp, vp, vp, vp, ct.POINTER(vp)]
        L.merf_scene_free.argtypes = [vp]
        L.merf_scene_free.restype = None
        L.merf_scene_device_bytes.argtypes = [vp]
        L.merf_scene_device_bytes.restype = ct.c_size_t
        L.merf_render.argtypes = [vp, vp, i32, i32, i32, vp, ct.POINTER(Opts), vp]
        L.merf_render_aux.argtypes = [vp, vp, i32, i32, i32, vp, vp, vp, ct.POINTER(Opts), vp]
        L.merf_render_host.argtypes = [vp, vp, i32, i32, i32, vp, vp, ct.POINTER(Opts), vp]
        L.merf_render_host_noalloc.argtypes = [vp, vp, i32, i32, i32, vp, ct.POINTER(Opts), vp]
        L.merf_trace.argtypes = [vp, vp, i32, i32, i32, vp, i32, vp, ct.POINTER(Opts), vp]
        L.merf_set_device_budget.argtypes = [ct.c_size_t]
        L.merf_set_device_budget.restype = None
        L.merf_scene_set_dense.argtypes = [vp, vp, vp, vp, vp]
        L.merf_scene_param_version.argtypes = [vp]
        L.merf_scene_param_version.restype = ct.c_ulonglong
        L.merf_render_backward.argtypes = [vp, vp, i32, i32, i32, vp, vp, vp, vp, ct.POINTER(Opts), vp]
        L.merf_render_backward_aux.argtypes = [vp, vp, i32, i32, i32, vp, vp, vp, vp, vp, ct.POINTER(Opts), vp]
        L.merf_render_backward_aux.restype = ct.c_int
        L.merf_check_device.argtypes = [vp, i32]
        L.merf_check_device.restype = ct.c_int
        L.merf_scene_set_dense.restype = ct.c_int
        L.merf_render_backward.restype = ct.c_int
        L.merf_server_create.argtypes = [vp, i32, ct.POINTER(ServerOpts), ct.POINTER(vp)]
        L.merf_server_submit.argtypes = [vp, i32, vp, i32, i32, vp, ct.POINTER(ct.c_uint64)]
        L.merf_server_wait.argtypes = [vp, ct.c_uint64, ct.c_double, ct.POINTER(ct.c_double)]
        L.merf_server_wait_timed.argtypes = [vp, ct.c_uint64, ct.c_double, ct.POINTER(ct.c_double),
                                             ct.POINTER(RequestTiming)]
        L.merf_server_get_stats.argtypes = [vp, ct.POINTER(ServerStats)]
        L.merf_server_cancel.argtypes = [vp, ct.c_uint64, ct.POINTER(ct.c_int)]
        L.merf_scene_load.argtypes = [ct.c_char_p, vp, ct.POINTER(vp)]
        L.merf_scene_load.restype = ct.c_int
        L.merf_server_destroy.argtypes = [vp]
        L.merf_server_destroy.restype = None
        for name in ("merf_server_create", "merf_server_submit", "merf_server_wait", "merf_server_wait_timed",
                     "merf_server_cancel",
                     "merf_server_get_stats"):
            getattr(L, name).restype = ct.c_int
        L.merf_last_error.restype = ct.c_char_p
        L.merf_version.restype = ct.c_char_p
        for name in ("merf_scene_upload", "merf_scene_upload_dense", "merf_scene_upload_device", "merf_render",
                     "merf_render_aux",
                     "merf_render_host", "merf_render_host_noalloc", "merf_trace"):
            getattr(L, name).restype = ct.c_int
        _lib = L
    return _lib


def _check(status: int):
    if status != MERF_OK:
        raise MerfError(status, lib().merf_last_error().decode())


def _stream(stream) -> Optional[int]:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _np_ptr(a: np.ndarray):
    return a.ctypes.data_as(ct.c_void_p)


def _dev_ptr(t: torch.Tensor, dtype, numel: int, name: str):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous() or t.numel() != numel:
        raise ValueError(f"{name} must be a contiguous {dtype} tensor of {numel} elements")
    return ct.c_void_p(t.data_ptr())


CONTRACT_PI, CONTRACT_SPHERICAL = 0, 1   # merf_render_opts.contraction


def opts(step: float, t_term: float = 2e-4, early_term: bool = True, precision: int = PREC_FP32,
         contraction: int = CONTRACT_PI) -> Opts:
    return Opts(step=step, t_term=t_term, precision=precision, early_term=int(early_term),
                contraction=int(contraction))


def cameras(cams: np.ndarray) -> np.ndarray:
    cams = np.ascontiguousarray(cams, dtype=np.float32).reshape(-1, 16)
    return cams


class Scene:
    """A baked scene resident on the current CUDA device (owns device memory)."""

    def __init__(self, scene, stream=None):
        cfg = scene.cfg
        d = Desc()
        d.grid_res, d.plane_res, d.channels = cfg.L, cfg.R, 8
        d.n_occ_levels = len(scene.occ)
        for i, o in enumerate(scene.occ):
            d.occ_res[i] = o.shape[0]
        d.mlp_in, d.mlp_hidden, d.mlp_out = 34, 16, 3
        self._occ = [np.ascontiguousarray(o, dtype=np.uint8) for o in scene.occ]
        occ_ptrs = (ct.c_void_p * MAX_OCC_LEVELS)(*[o.ctypes.data for o in self._occ])
        mlp = np.ascontiguousarray(scene.mlp, dtype=np.float32)
        handle = ct.c_void_p()
        s = _stream(stream)
        if cfg.storage == "u8" and torch.is_tensor(scene.atlas) and scene.atlas.is_cuda:
            # arrays already on the device (merf_scene_upload_device): small ones follow them there
            d.storage = STORAGE_U8_SPARSE
            d.block_size, d.n_blocks = cfg.B, int(scene.atlas.shape[0])
            dev = scene.atlas.device
            occ_d = [torch.as_tensor(np.ascontiguousarray(o, dtype=np.uint8)).to(dev) for o in scene.occ]
            ig = torch.as_tensor(scene.index_grid).to(device=dev, dtype=torch.int32).contiguous()
            atlas = scene.atlas.contiguous()
            planes = None if scene.planes is None else torch.as_tensor(scene.planes).to(dev).contiguous()
            mlp_d = torch.as_tensor(mlp).to(dev)
            dptrs = (ct.c_void_p * MAX_OCC_LEVELS)(*[o.data_ptr() for o in occ_d])
            _check(lib().merf_scene_upload_device(ct.byref(d), ct.c_void_p(ig.data_ptr()),
                                                  ct.c_void_p(atlas.data_ptr()),
                                                  None if planes is None else ct.c_void_p(planes.data_ptr()),
                                                  ct.cast(dptrs, ct.c_void_p), ct.c_void_p(mlp_d.data_ptr()), s,
                                                  ct.byref(handle)))
        elif cfg.storage == "u8":
            d.storage = STORAGE_U8_SPARSE
            d.block_size, d.n_blocks = cfg.B, scene.n_blocks
            ig = np.ascontiguousarray(scene.index_grid, dtype=np.int32)
            atlas = np.ascontiguousarray(scene.atlas, dtype=np.uint8)
            # a grid-only scene (R = 0) passes no planes
            planes = None if scene.planes is None else np.ascontiguousarray(scene.planes, dtype=np.uint8)
            _check(lib().merf_scene_upload(ct.byref(d), _np_ptr(ig), _np_ptr(atlas),
                                           None if planes is None else _np_ptr(planes),
                                           ct.cast(occ_ptrs, ct.c_void_p), _np_ptr(mlp), s, ct.byref(handle)))
        else:
            d.storage = STORAGE_F32_DENSE
            grid = np.ascontiguousarray(scene.grid_f32, dtype=np.float32)
            planes = np.ascontiguousarray(scene.planes_f32, dtype=np.float32)
            _check(lib().merf_scene_upload_dense(ct.byref(d), _np_ptr(grid), _np_ptr(planes),
                                                 ct.cast(occ_ptrs, ct.c_void_p), _np_ptr(mlp), s,
                                                 ct.byref(handle)))
        self.handle = handle
        self.desc = d
        self.source = scene

    @classmethod
    def load(cls, path: str, stream=None) -> "Scene":
        """Upload a scene file (merf_scene_load: the library maps, validates and uploads it)."""
        handle = ct.c_void_p()
        _check(lib().merf_scene_load(os.fsencode(path), _stream(stream), ct.byref(handle)))
        self = cls.__new__(cls)
        self.handle = handle
        with open(path, "rb") as f:
            head = f.read(64 + ct.sizeof(Desc))
        self.desc = Desc.from_buffer_copy(head[64:])
        self.source = None
        return self

    @property
    def device_bytes(self) -> int:
        return int(lib().merf_scene_device_bytes(self.handle))

    def close(self):
        if self.handle:
            lib().merf_scene_free(self.handle)
            self.handle = ct.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def render(scene: Scene, cams: np.ndarray, W: int, H: int, step: float, out: Optional[torch.Tensor] = None,
           t_term: float = 2e-4, early_term: bool = True, precision: int = PREC_FP32,
           aux: Optional[torch.Tensor] = None, counters: Optional[torch.Tensor] = None,
           stream=None, contraction: int = CONTRACT_PI) -> torch.Tensor:
    """Render n cameras into a CUDA float32 tensor [n, H, W, 3].  contraction CONTRACT_SPHERICAL
    selects the spherical-contraction ablation (dense march, FP32)."""
    cams = cameras(cams)
    n = cams.shape[0]
    if out is None:
        out = torch.empty((n, H, W, 3), dtype=torch.float32, device="cuda")
    o = opts(step, t_term, early_term, precision, contraction)
    op = _dev_ptr(out, torch.float32, n * H * W * 3, "out")
    ap = _dev_ptr(aux, torch.float32, n * H * W * AUX_SIZE, "aux") if aux is not None else None
    cp = _dev_ptr(counters, torch.int64, 4, "counters") if counters is not None else None
    if ap is None and cp is None:
        _check(lib().merf_render(scene.handle, _np_ptr(cams), n, W, H, op, ct.byref(o), _stream(stream)))
    else:
        _check(lib().merf_render_aux(scene.handle, _np_ptr(cams), n, W, H, op, ap, cp, ct.byref(o),
                                     _stream(stream)))
    return out


def render_host(scene: Scene, cams: np.ndarray, W: int, H: int, step: float, staging: Optional[torch.Tensor],
                host_out: torch.Tensor, t_term: float = 2e-4, early_term: bool = True,
                precision: int = PREC_FP32, stream=None) -> torch.Tensor:
    """Render into host memory through the library's host-output entry point (`staging` may be
    None when host_out is page-locked: the kernel then writes it directly)."""
    cams = cameras(cams)
    n = cams.shape[0]
    if host_out.is_cuda or host_out.dtype != torch.float32 or not host_out.is_contiguous() or \
            host_out.numel() != n * H * W * 3:
        raise ValueError("host_out must be a contiguous host float32 tensor [n, H, W, 3]")
    o = opts(step, t_term, early_term, precision)
    _check(lib().merf_render_host(scene.handle, _np_ptr(cams), n, W, H,
                                  None if staging is None else _dev_ptr(staging, torch.float32, n * H * W * 3,
                                                                        "staging"),
                                  ct.c_void_p(host_out.data_ptr()), ct.byref(o), _stream(stream)))
    return host_out


def render_host_noalloc(scene: Scene, cams: np.ndarray, W: int, H: int, step: float, host_out: torch.Tensor,
                        t_term: float = 2e-4, early_term: bool = True, precision: int = PREC_FP32,
                        stream=None) -> torch.Tensor:
    """Render into host memory through the library's fixed staging area (no device allocation
    by the caller or the library; at most NOALLOC_STAGING_BYTES of image per call)."""
    cams = cameras(cams)
    n = cams.shape[0]
    if host_out.is_cuda or host_out.dtype != torch.float32 or not host_out.is_contiguous() or \
            host_out.numel() != n * H * W * 3:
        raise ValueError("host_out must be a contiguous host float32 tensor [n, H, W, 3]")
    o = opts(step, t_term, early_term, precision)
    _check(lib().merf_render_host_noalloc(scene.handle, _np_ptr(cams), n, W, H, ct.c_void_p(host_out.data_ptr()),
                                          ct.byref(o), _stream(stream)))
    return host_out


def trace(scene: Scene, cams: np.ndarray, W: int, H: int, step: float, words: int, stream=None,
          contraction: int = CONTRACT_PI):
    """Evaluated lattice-sample bit masks [n*H*W, words] (uint32 as int32) and lattice counts."""
    cams = cameras(cams)
    n = cams.shape[0]
    mask = torch.empty((n * H * W, words), dtype=torch.int32, device="cuda")
    nlat = torch.empty((n * H * W,), dtype=torch.int32, device="cuda")
    o = opts(step, early_term=False, contraction=contraction)
    _check(lib().merf_trace(scene.handle, _np_ptr(cams), n, W, H, ct.c_void_p(mask.data_ptr()), words,
                            ct.c_void_p(nlat.data_ptr()), ct.byref(o), _stream(stream)))
    return mask, nlat


def set_dense(scene: Scene, grid: torch.Tensor, planes: torch.Tensor, mlp: torch.Tensor, stream=None):
    """Copy new parameter values (CUDA float32 tensors) into a dense float scene."""
    L, R = scene.desc.grid_res, scene.desc.plane_res
    _check(lib().merf_scene_set_dense(scene.handle, _dev_ptr(grid, torch.float32, L ** 3 * 8, "grid"),
                                      _dev_ptr(planes, torch.float32, 3 * R * R * 8, "planes"),
                                      _dev_ptr(mlp, torch.float32, 883, "mlp"), _stream(stream)))


def param_version(scene: Scene) -> int:
    """How many times set_dense has replaced the scene's parameters (merf_scene_param_version)."""
    return int(lib().merf_scene_param_version(scene.handle))


def render_backward(scene: Scene, cams: np.ndarray, W: int, H: int, step: float, d_out: torch.Tensor,
                    g_grid: torch.Tensor, g_planes: torch.Tensor, g_mlp: torch.Tensor, t_term: float = 2e-4,
                    early_term: bool = True, stream=None, aux: Optional[torch.Tensor] = None):
    """Accumulate dL/dgrid, dL/dplanes, dL/dmlp (zeroed by the caller) for dL/dC = d_out.  `aux`:
    the forward render's per-pixel record (render(..., aux=...)), which saves the recomputed march."""
    cams = cameras(cams)
    n = cams.shape[0]
    L, R = scene.desc.grid_res, scene.desc.plane_res
    o = opts(step, t_term, early_term, PREC_FP32)
    _check(lib().merf_render_backward_aux(scene.handle, _np_ptr(cams), n, W, H,
                                          _dev_ptr(d_out, torch.float32, n * H * W * 3, "d_out"),
                                          None if aux is None else _dev_ptr(aux, torch.float32,
                                                                            n * H * W * AUX_SIZE, "aux"),
                                          _dev_ptr(g_grid, torch.float32, L ** 3 * 8, "g_grid"),
                                          _dev_ptr(g_planes, torch.float32, 3 * R * R * 8, "g_planes"),
                                          _dev_ptr(g_mlp, torch.float32, 883, "g_mlp"), ct.byref(o),
                                          _stream(stream)))


class _RenderFn(torch.autograd.Function):
    """Forward: install the parameters in the scene and render.  Backward: the adjoint at the same
    parameters.  The scene holds one set of parameters, so the forward records the scene's
    parameter version and keeps its parameter tensors (autograd raises if they are modified in
    place before the backward); if another forward installed other values in between, the
    backward installs this forward's values again before running the adjoint."""

    @staticmethod
    def forward(ctx, grid, planes, mlp, scene, cams, W, H, step, t_term, early_term):
        set_dense(scene, grid.detach(), planes.detach(), mlp.detach())
        ctx.version = param_version(scene)
        ctx.save_for_backward(grid, planes, mlp)
        n = cams.shape[0]
        aux = torch.empty((n, H, W, AUX_SIZE), dtype=torch.float32, device="cuda")
        out = render(scene, cams, W, H, step, t_term=t_term, early_term=early_term, aux=aux)
        ctx.aux = aux        # C_d and F per pixel: the adjoint needs no second forward march
        ctx.scene, ctx.cams, ctx.args = scene, cams, (W, H, step, t_term, early_term)
        return out

    @staticmethod
    def backward(ctx, g_out):
        W, H, step, t_term, early_term = ctx.args
        grid, planes, mlp = ctx.saved_tensors
        if param_version(ctx.scene) != ctx.version:
            set_dense(ctx.scene, grid.detach(), planes.detach(), mlp.detach())
        g_grid = torch.zeros(grid.shape, dtype=torch.float32, device="cuda")
        g_planes = torch.zeros(planes.shape, dtype=torch.float32, device="cuda")
        g_mlp = torch.zeros(mlp.shape, dtype=torch.float32, device="cuda")
        render_backward(ctx.scene, ctx.cams, W, H, step, g_out.contiguous(), g_grid, g_planes, g_mlp, t_term,
                        early_term, aux=ctx.aux)
        ctx.aux = None
        return g_grid, g_planes, g_mlp, None, None, None, None, None, None, None


def render_differentiable(scene: Scene, grid: torch.Tensor, planes: torch.Tensor, mlp: torch.Tensor,
                          cams: np.ndarray, W: int, H: int, step: float, t_term: float = 2e-4,
                          early_term: bool = True) -> torch.Tensor:
    """Render a dense float scene whose grid, planes and MLP weights are the given CUDA tensors;
    the result is differentiable with respect to them through the library's adjoint kernel.
    The scene's device copy of the parameters is replaced by these values (and again by the
    backward pass if another forward on the same scene replaced them in between)."""
    return _RenderFn.apply(grid, planes, mlp, scene, cameras(cams), W, H, step, t_term, early_term)


def check_device(stream=None, self_test: int = 0):
    """Synchronise and raise MerfError if a kernel recorded a problem since the last check:
    ERR_DEVICE_BOUNDS for an out-of-range index (bounds-checked build), ERR_TIMEOUT for a bounded
    tensor-core wait that gave up (any build).  self_test 1 / 2 exercises those two reports."""
    _check(lib().merf_check_device(_stream(stream), int(self_test)))


def set_device_budget(nbytes: int):
    lib().merf_set_device_budget(int(nbytes))


def version() -> str:
    return lib().merf_version().decode()


class Server:
    """Continuous-batching render server over resident scenes (the library's server thread does
    admission, batching and launches; this class only marshals arguments)."""

    def __init__(self, scenes: Sequence[Scene], pool_bytes: int, step: float, max_tiles_per_iter: int = 16384,
                 precision: int = PREC_FP16, t_term: float = 2e-4, early_term: bool = True,
                 max_tiles_backlog: int = 0):
        self.scenes = list(scenes)
        arr = (ct.c_void_p * len(self.scenes))(*[sc.handle.value for sc in self.scenes])
        o = ServerOpts(pool_bytes=int(pool_bytes), max_tiles_per_iter=int(max_tiles_per_iter), precision=precision,
                       step=step, t_term=t_term, early_term=int(early_term),
                       max_tiles_backlog=int(max_tiles_backlog))
        h = ct.c_void_p()
        _check(lib().merf_server_create(ct.cast(arr, ct.c_void_p), len(self.scenes), ct.byref(o), ct.byref(h)))
        self.handle = h
        self._outs = {}

    def submit(self, scene: int, cam: np.ndarray, W: int, H: int, host_out: torch.Tensor) -> int:
        if host_out.is_cuda or host_out.dtype != torch.float32 or not host_out.is_contiguous() or \
                host_out.numel() != W * H * 3:
            raise ValueError("host_out must be a contiguous host float32 tensor of H*W*3 elements")
        cam = np.ascontiguousarray(cam, dtype=np.float32).reshape(16)
        rid = ct.c_uint64()
        _check(lib().merf_server_submit(self.handle, int(scene), _np_ptr(cam), W, H, ct.c_void_p(host_out.data_ptr()),
                                        ct.byref(rid)))
        self._outs[rid.value] = host_out
        return rid.value

    def wait(self, rid: int, timeout: float = 60.0) -> float:
        lat = ct.c_double()
        st = lib().merf_server_wait(self.handle, ct.c_uint64(rid), float(timeout), ct.byref(lat))
        if st == ERR_TIMEOUT:
            raise TimeoutError(lib().merf_last_error().decode())
        self._outs.pop(rid, None)
        _check(st)
        return lat.value

    def wait_timed(self, rid: int, timeout: float = 60.0) -> dict:
        """wait, returning where the latency went (merf_request_timing): total, admit, queue,
        render and copy seconds."""
        lat, t = ct.c_double(), RequestTiming()
        st = lib().merf_server_wait_timed(self.handle, ct.c_uint64(rid), float(timeout), ct.byref(lat), ct.byref(t))
        if st == ERR_TIMEOUT:
            raise TimeoutError(lib().merf_last_error().decode())
        self._outs.pop(rid, None)
        _check(st)
        return {k: getattr(t, k) for k, _ in RequestTiming._fields_}

    def cancel(self, rid: int) -> bool:
        """Withdraw a request (True) unless its image is already on its way out (False); either way
        it must still be waited for, and a withdrawn one raises MerfError(ERR_CANCELLED) there."""
        c = ct.c_int()
        _check(lib().merf_server_cancel(self.handle, ct.c_uint64(rid), ct.byref(c)))
        return bool(c.value)

    def stats(self) -> dict:
        s = ServerStats()
        _check(lib().merf_server_get_stats(self.handle, ct.byref(s)))
        return {k: getattr(s, k) for k, _ in ServerStats._fields_ if k != "reserved"}

    def close(self):
        if self.handle:
            lib().merf_server_destroy(self.handle)
            self.handle = ct.c_void_p()
            self._outs.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
