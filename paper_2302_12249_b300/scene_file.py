"""Raw binary scene files: a baked scene's arrays behind a 256-byte header, the format that
``merf_scene_load`` (declared in ``include/merf.h``) maps and uploads.

Little-endian.  Header: magic ``MERFSCN1``, uint32 version 1, uint32 header size 256, uint64
file size, float32 lattice step, int32 seed, 32-byte NUL-padded name, the 72-byte
``merf_scene_desc``, zeros to 256.  Then, each array starting at the next multiple of 64
bytes: for uint8 storage the index grid (int32 [(L/B)^3]), the atlas (uint8
[n_blocks][B][B][B][8]) and, unless R = 0, the planes (uint8 [3][R][R][8]); for float storage
the grid (float32 [L][L][L][8]) and the planes (float32 [3][R][R][8]); then the occupancy levels
(uint8 [N][N][N], finest first) and the MLP (float32 [883]).  Writing and reading are plain numpy;
``load`` maps the file, so a paper-scale scene opens without reading it all.
"""
from __future__ import annotations

import os
import struct
from typing import List, Tuple

import numpy as np

from . import synth

MAGIC = b"MERFSCN1"
VERSION = 1
HEADER_BYTES = 256
MAX_OCC_LEVELS = 8
STORAGE_U8_SPARSE, STORAGE_F32_DENSE = 0, 1
_DESC = struct.Struct("<6i8i4i")            # merf_scene_desc: 18 int32 = 72 bytes
_HEAD = struct.Struct("<8sIIQfi32s")        # the first 64 bytes


def _align(n: int) -> int:
    return (n + 63) & ~63


def _arrays(scene: synth.Scene) -> List[np.ndarray]:
    if scene.cfg.storage == "u8":
        out = [np.ascontiguousarray(scene.index_grid, np.int32), np.ascontiguousarray(scene.atlas, np.uint8)]
        if scene.cfg.R > 0:
            out.append(np.ascontiguousarray(scene.planes, np.uint8))
    else:
        out = [np.ascontiguousarray(scene.grid_f32, np.float32), np.ascontiguousarray(scene.planes_f32, np.float32)]
    out += [np.ascontiguousarray(o, np.uint8) for o in scene.occ]
    out.append(np.ascontiguousarray(scene.mlp, np.float32))
    return out


def _desc(scene: synth.Scene) -> Tuple[int, ...]:
    cfg = scene.cfg
    occ = [int(o.shape[0]) for o in scene.occ] + [0] * (MAX_OCC_LEVELS - len(scene.occ))
    u8 = cfg.storage == "u8"
    return (cfg.L, cfg.B if u8 else 0, cfg.R, synth.C, scene.n_blocks if u8 else 0, len(scene.occ), *occ,
            synth.MLP_IN, synth.MLP_HIDDEN, synth.MLP_OUT, STORAGE_U8_SPARSE if u8 else STORAGE_F32_DENSE)


def save(scene: synth.Scene, path: str) -> int:
    """Write `scene` to `path`; returns the file size in bytes."""
    arrays = _arrays(scene)
    offsets, at = [], HEADER_BYTES
    for a in arrays:
        at = _align(at)
        offsets.append(at)
        at += a.nbytes
    head = _HEAD.pack(MAGIC, VERSION, HEADER_BYTES, at, float(scene.cfg.step), int(scene.seed),
                      scene.cfg.name.encode()[:31])
    head += _DESC.pack(*_desc(scene))
    head += bytes(HEADER_BYTES - len(head))
    tmp = path + ".tmp"
    with open(tmp, "wb") as f:
        f.write(head)
        for off, a in zip(offsets, arrays):
            f.write(bytes(off - f.tell()))
            f.write(a.tobytes())
    os.replace(tmp, path)
    return at


def read_header(path: str) -> dict:
    with open(path, "rb") as f:
        raw = f.read(HEADER_BYTES)
    if len(raw) < HEADER_BYTES:
        raise ValueError(f"{path} is shorter than a scene file header")
    magic, version, hbytes, fbytes, step, seed, name = _HEAD.unpack_from(raw, 0)
    if magic != MAGIC or version != VERSION or hbytes != HEADER_BYTES:
        raise ValueError(f"{path} is not a version-{VERSION} MERF scene file")
    d = _DESC.unpack_from(raw, _HEAD.size)
    return dict(file_bytes=fbytes, step=step, seed=seed, name=name.rstrip(b"\0").decode(),
                L=d[0], B=d[1], R=d[2], channels=d[3], n_blocks=d[4], occ_res=tuple(d[6:6 + d[5]]),
                storage=d[17])


def load(path: str, mmap: bool = True) -> synth.Scene:
    """Read a scene file back into a synth.Scene (arrays mapped read-only unless mmap=False)."""
    h = read_header(path)
    L, B, R, nb = h["L"], h["B"], h["R"], h["n_blocks"]
    u8 = h["storage"] == STORAGE_U8_SPARSE
    if u8:
        shapes = [(np.int32, ((L // B),) * 3), (np.uint8, (nb, B, B, B, synth.C))]
        if R > 0:
            shapes.append((np.uint8, (3, R, R, synth.C)))
    else:
        shapes = [(np.float32, (L, L, L, synth.C)), (np.float32, (3, R, R, synth.C))]
    shapes += [(np.uint8, (n, n, n)) for n in h["occ_res"]]
    shapes.append((np.float32, (synth.MLP_PARAMS,)))
    data = np.memmap(path, dtype=np.uint8, mode="r") if mmap else np.fromfile(path, dtype=np.uint8)
    if data.size != h["file_bytes"]:
        raise ValueError(f"{path} holds {data.size} bytes, its header says {h['file_bytes']}")
    arrays, at = [], HEADER_BYTES
    for dt, shape in shapes:
        at = _align(at)
        n = int(np.prod(shape)) * np.dtype(dt).itemsize
        if at + n > data.size:
            raise ValueError(f"{path} is truncated")
        arrays.append(data[at:at + n].view(dt).reshape(shape))
        at += n
    if at != data.size:
        raise ValueError(f"{path}: {data.size} bytes, its descriptor needs {at}")
    cfg = synth.CONFIGS.get(h["name"])
    if cfg is None or (cfg.L, cfg.R, tuple(cfg.occ_res)) != (L, R, h["occ_res"]):
        cfg = synth.SceneConfig(h["name"] or "file", L=L, B=B, R=R, occ_res=h["occ_res"], n_blobs=0,
                                inner_blobs=None, step=h["step"], peak_opacity=0.0,
                                storage="u8" if u8 else "f32", grid_only=u8 and R == 0)
    nocc = len(h["occ_res"])
    k = len(arrays) - nocc - 1                  # grid (+ atlas) (+ planes) come first
    occ = arrays[k:k + nocc]
    mlp = arrays[k + nocc]
    if u8:
        return synth.Scene(cfg=cfg, seed=h["seed"], occ=occ, mlp=mlp, index_grid=arrays[0], atlas=arrays[1],
                           planes=arrays[2] if R > 0 else None)
    return synth.Scene(cfg=cfg, seed=h["seed"], occ=occ, mlp=mlp, grid_f32=arrays[0], planes_f32=arrays[1])
