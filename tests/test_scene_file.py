"""Scene files (raw binary, the format of merf_scene_load in include/merf.h): the Python writer and
reader round-trip every storage kind, and the C loader accepts what the writer makes and refuses
damaged files -- all on the CPU (a one-byte device budget stops a valid file at the upload's
budget check, after the loader and the upload's host-side validation have run)."""
import ctypes as ct
import os
import struct

import numpy as np
import pytest

from paper_2302_12249_b300 import merf, scene_file, synth

NAMES = ("tiny", "tiny_grid", "dense128")


@pytest.fixture(scope="module")
def files(tmp_path_factory):
    d = tmp_path_factory.mktemp("scenes")
    out = {}
    for name in NAMES:
        sc = synth.make_scene(name)
        p = str(d / f"{name}.merf")
        scene_file.save(sc, p)
        out[name] = (sc, p)
    return out


@pytest.fixture
def L():
    lib = merf.lib()
    yield lib
    lib.merf_set_device_budget(0)


def _c_load(L, path):
    h = ct.c_void_p()
    st = L.merf_scene_load(None if path is None else os.fsencode(path), None, ct.byref(h))
    return st, L.merf_last_error().decode()


@pytest.mark.parametrize("name", NAMES)
def test_round_trip(files, name):
    sc, p = files[name]
    back = scene_file.load(p)
    for f in ("index_grid", "atlas", "planes", "grid_f32", "planes_f32", "mlp"):
        a, b = getattr(sc, f), getattr(back, f)
        assert (a is None) == (b is None), f
        if a is not None:
            assert a.dtype == b.dtype and a.shape == b.shape and np.array_equal(a, b), f
    assert len(back.occ) == len(sc.occ) and all(np.array_equal(a, b) for a, b in zip(sc.occ, back.occ))
    assert back.cfg is synth.CONFIGS[name] and back.seed == sc.seed
    h = scene_file.read_header(p)
    assert h["file_bytes"] == os.path.getsize(p) and h["name"] == name and h["step"] == np.float32(sc.cfg.step)


def test_layout_alignment_and_size(files):
    """Arrays start on 64-byte boundaries right after the header; the file ends with the MLP."""
    sc, p = files["tiny"]
    raw = open(p, "rb").read()
    assert raw[:8] == b"MERFSCN1" and struct.unpack_from("<II", raw, 8) == (1, 256)
    assert all(b == 0 for b in raw[136:256])
    ig = sc.index_grid.astype(np.int32).tobytes()
    assert raw[256:256 + len(ig)] == ig
    mlp = sc.mlp.astype(np.float32).tobytes()
    assert raw[-len(mlp):] == mlp and (len(raw) - len(mlp)) % 64 == 0


@pytest.mark.parametrize("name", NAMES)
def test_c_loader_accepts_the_writers_files(files, L, name):
    _, p = files[name]
    L.merf_set_device_budget(1)
    st, msg = _c_load(L, p)
    assert st == merf.ERR_OOM and "budget" in msg, msg


def _damaged(src, dst, fn):
    raw = bytearray(open(src, "rb").read())
    raw = fn(raw)
    open(dst, "wb").write(bytes(raw))
    return dst


def _put(fmt, off, *vals):
    def f(raw):
        struct.pack_into(fmt, raw, off, *vals)
        return raw
    return f


DESC = 64                                    # offset of merf_scene_desc in the header
DAMAGE = {
    "magic": _put("<8s", 0, b"MERFSCN2"),
    "version": _put("<I", 8, 2),
    "header_size": _put("<I", 12, 255),
    "file_bytes": lambda raw: _put("<Q", 16, len(raw) + 64)(raw),
    "truncated": lambda raw: _put("<Q", 16, len(raw) - 1)(raw)[:-1],
    "extra_byte": lambda raw: _put("<Q", 16, len(raw) + 1)(raw) + b"\0",
    "channels": _put("<i", DESC + 12, 7),
    "storage": _put("<i", DESC + 68, 5),
    "blocks_beyond_index_grid": _put("<i", DESC + 16, 8 ** 3 + 1),
    "short_header": lambda raw: raw[:100],
}


@pytest.mark.parametrize("what", sorted(DAMAGE))
def test_damaged_files_are_refused(files, L, tmp_path, what):
    p = _damaged(files["tiny"][1], str(tmp_path / "bad.merf"), DAMAGE[what])
    L.merf_set_device_budget(1)                  # a file that got through would stop with OOM
    st, msg = _c_load(L, p)
    assert st == merf.ERR_INVALID_ARG, (what, st, msg)
    if what not in ("channels", "blocks_beyond_index_grid"):   # the Python reader checks the framing
        with pytest.raises(ValueError):
            scene_file.load(p)


def test_missing_file_and_null_arguments(L, tmp_path):
    assert _c_load(L, str(tmp_path / "none.merf"))[0] == merf.ERR_INVALID_ARG
    assert _c_load(L, None)[0] == merf.ERR_INVALID_ARG
    assert L.merf_scene_load(b"x", None, None) == merf.ERR_INVALID_ARG
