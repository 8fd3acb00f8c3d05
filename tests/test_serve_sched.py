"""CPU tests of the serving form's scheduler (admission by output-pool memory, continuous batching
of 16 x 8 tiles, completion, cancellation, device failure) -- the scheduler the CUDA server runs,
driven here by a host stand-in for the device (tests/native/serve_host.cpp) whose tiles are
rendered by the FP64 oracle.  No GPU."""
import ctypes as ct
import os
import subprocess
import threading
import time

import numpy as np
import pytest

import oracle
from paper_2302_12249_b300 import merf, synth

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "native", "serve_host.cpp")
STEP = 1 / 64
TILE_FN = ct.CFUNCTYPE(ct.c_int, ct.c_void_p, ct.c_int, ct.c_int, ct.c_int, ct.POINTER(ct.c_float), ct.c_int,
                       ct.c_int, ct.POINTER(ct.c_float))


@pytest.fixture(scope="module")
def hostlib(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("serve_host") / "libserve_host.so")
    subprocess.run(["g++", "-std=c++17", "-O1", "-shared", "-fPIC", "-pthread", "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(ROOT, "paper_2302_12249_b300", "csrc"), SRC, "-o", out], check=True)
    L = ct.CDLL(out)
    vp = ct.c_void_p
    L.host_server_create.argtypes = [ct.c_int, ct.c_size_t, ct.c_int, ct.c_int, TILE_FN, vp, ct.c_int]
    L.host_server_create.restype = vp
    L.host_server_submit.argtypes = [vp, ct.c_int, vp, ct.c_int, ct.c_int, vp, ct.POINTER(ct.c_uint64)]
    L.host_server_wait.argtypes = [vp, ct.c_uint64, ct.c_double, ct.POINTER(ct.c_double)]
    L.host_server_wait_timed.argtypes = [vp, ct.c_uint64, ct.c_double, ct.POINTER(ct.c_double),
                                         ct.POINTER(merf.RequestTiming)]
    L.host_server_cancel.argtypes = [vp, ct.c_uint64, ct.POINTER(ct.c_int)]
    L.host_server_stats.argtypes = [vp, ct.POINTER(merf.ServerStats)]
    L.host_server_hold.argtypes = [vp, ct.c_int]
    L.host_server_hold.restype = None
    L.host_server_destroy.argtypes = [vp]
    L.host_server_destroy.restype = None
    L.host_server_last_error.restype = ct.c_char_p
    L.host_stats_size.restype = ct.c_size_t
    assert L.host_stats_size() == ct.sizeof(merf.ServerStats)     # the binding's struct is merf.h's
    return L


@pytest.fixture(scope="module")
def scenes():
    return [oracle.OracleScene(synth.make_scene("tiny", seed=s)) for s in (0, 5)]


class Server:
    """The scheduler over the host device; tiles are rendered by the oracle (FP64, stored as
    float32 exactly as the oracle's full-image result would be)."""

    def __init__(self, L, oscenes, pool_bytes, max_tiles, workers=3, fail_scene=None, max_tiles_backlog=0):
        self.L, self.oscenes, self.fail_scene = L, oscenes, fail_scene
        self.calls = []                       # (scene, cam[15], x0, y0) per tile
        self.lock = threading.Lock()
        self.fn = TILE_FN(self._tile)         # kept alive for the server's lifetime
        self.h = L.host_server_create(len(oscenes), pool_bytes, max_tiles, workers, self.fn, None, max_tiles_backlog)
        self.bufs = {}

    def _tile(self, user, scene, W, H, cam, x0, y0, image):
        try:
            c = np.ctypeslib.as_array(cam, shape=(16,)).copy()
            with self.lock:
                self.calls.append((scene, float(c[15]), x0, y0))
            if scene == self.fail_scene:
                return 1
            ii, jj = np.meshgrid(np.arange(x0, min(x0 + 16, W)), np.arange(y0, min(y0 + 8, H)))
            pix = np.stack([np.zeros(ii.size, np.int32), ii.ravel(), jj.ravel()], 1).astype(np.int32)
            rgb = oracle.render(self.oscenes[scene], c[None], W, H, STEP, pix=pix, threads=1)[:, 0:3]
            img = np.ctypeslib.as_array(image, shape=(H * W, 3))
            img[pix[:, 2] * W + pix[:, 1]] = rgb.astype(np.float32)
            return 0
        except Exception:                     # a tile that cannot be rendered fails its iteration
            return 2

    def submit(self, scene, cam, W, H, fill=np.nan):
        out = np.full((H, W, 3), fill, np.float32)
        rid = ct.c_uint64()
        st = self.L.host_server_submit(self.h, scene, np.ascontiguousarray(cam, np.float32).ctypes.data, W, H,
                                       out.ctypes.data, ct.byref(rid))
        if st != merf.MERF_OK:
            return st, None
        self.bufs[rid.value] = out
        return st, rid.value

    def wait(self, rid, timeout=60.0):
        lat = ct.c_double()
        return self.L.host_server_wait(self.h, rid, timeout, ct.byref(lat))

    def wait_timed(self, rid, timeout=60.0):
        lat, t = ct.c_double(), merf.RequestTiming()
        st = self.L.host_server_wait_timed(self.h, rid, timeout, ct.byref(lat), ct.byref(t))
        return st, lat.value, {k: getattr(t, k) for k, _ in merf.RequestTiming._fields_}

    def cancel(self, rid):
        c = ct.c_int(-1)
        st = self.L.host_server_cancel(self.h, rid, ct.byref(c))
        return st, c.value

    def stats(self):
        s = merf.ServerStats()
        assert self.L.host_server_stats(self.h, ct.byref(s)) == merf.MERF_OK
        return s

    def hold(self, on):
        self.L.host_server_hold(self.h, int(on))

    def until(self, pred, timeout=30.0):
        t0 = time.time()
        while not pred(self.stats()):
            assert time.time() - t0 < timeout, "scheduler made no progress"
            time.sleep(0.002)

    def close(self):
        if self.h:
            self.L.host_server_destroy(self.h)
            self.h = None


def _cams(n, seed):
    cams = synth.sphere_cameras(n, 32, 32, radius=2.3, seed=seed).copy()
    cams[:, 15] = 15.5 + np.arange(n)          # cy: tags each request (the principal point moves)
    return cams


def _expected(oscene, cam, W, H):
    return oracle.render(oscene, cam[None], W, H, STEP, threads=1)[:, 0:3].astype(np.float32).reshape(H, W, 3)


def _tiles(W, H):
    return -(-W // 16) * -(-H // 8)


def test_mixed_scenes_and_resolutions(hostlib, scenes):
    """Requests of two scenes and ragged sizes through a pool that holds about two images and
    iterations of five tiles: every image equals the oracle's, every tile ran exactly once, and the
    counters add up."""
    sizes = [(37, 29), (16, 8), (1, 1), (50, 20), (8, 33), (17, 9), (40, 24), (3, 70), (33, 16), (20, 20)]
    cams = _cams(len(sizes), seed=11)
    pool = 2 * 50 * 24 * 3 * 4 + 4096
    srv = Server(hostlib, scenes, pool, max_tiles=5)
    try:
        rids = []
        for k, (W, H) in enumerate(sizes):
            st, rid = srv.submit(k % 2, cams[k], W, H)
            assert st == merf.MERF_OK
            rids.append(rid)
        for rid in rids:
            assert srv.wait(rid) == merf.MERF_OK, hostlib.host_server_last_error()
        for k, ((W, H), rid) in enumerate(zip(sizes, rids)):
            np.testing.assert_array_equal(srv.bufs[rid], _expected(scenes[k % 2], cams[k], W, H))
        keys = [(s, cy, x0, y0) for s, cy, x0, y0 in srv.calls]
        assert len(keys) == len(set(keys)) == sum(_tiles(W, H) for W, H in sizes)
        s = srv.stats()
        assert (s.submitted, s.completed, s.cancelled) == (len(sizes), len(sizes), 0)
        assert s.rays == sum(W * H for W, H in sizes)
        assert s.tiles == len(keys)
        assert s.iterations >= -(-s.tiles // 5)
        assert s.peak_pool_bytes <= s.pool_bytes <= pool and s.pool_used_bytes == 0
        assert s.peak_admitted >= 2
    finally:
        srv.close()


def test_admission_in_arrival_order(hostlib, scenes):
    """A pool that holds one image admits one request at a time, in submission order."""
    n, W, H = 6, 24, 16
    cams = _cams(n, seed=12)
    srv = Server(hostlib, scenes, W * H * 3 * 4 + 255, max_tiles=2)
    try:
        rids = [srv.submit(0, cams[k], W, H)[1] for k in range(n)]
        for rid in rids:
            assert srv.wait(rid) == merf.MERF_OK
        order = []
        for _, cy, _, _ in srv.calls:
            if not order or order[-1] != cy:
                order.append(cy)
        assert order == sorted(order) == [15.5 + k for k in range(n)]
        assert srv.stats().peak_admitted == 1
    finally:
        srv.close()


def test_latency_phases(hostlib, scenes):
    """merf_request_timing: the phases are ordered and add up to the latency; with a one-image
    pool the second request waits for admission while the first renders, and iterations held
    for 0.2 s show up as render time."""
    W, H = 24, 16
    cams = _cams(2, seed=17)
    srv = Server(hostlib, scenes, W * H * 3 * 4 + 255, max_tiles=64)
    try:
        srv.hold(True)
        r0 = srv.submit(0, cams[0], W, H)[1]
        r1 = srv.submit(1, cams[1], W, H)[1]
        srv.until(lambda s: s.iterations >= 1)
        time.sleep(0.2)
        srv.hold(False)
        res = [srv.wait_timed(r) for r in (r0, r1)]
        for st, lat, t in res:
            assert st == merf.MERF_OK
            parts = [t["admit_s"], t["queue_s"], t["render_s"], t["copy_s"]]
            assert min(parts) >= 0.0
            assert abs(sum(parts) - t["total_s"]) < 1e-9 and abs(t["total_s"] - lat) < 1e-9
        assert res[0][2]["render_s"] >= 0.19            # its iteration was held
        assert res[1][2]["admit_s"] >= 0.19             # the pool held only the first image
        assert res[0][2]["admit_s"] < 0.1
    finally:
        srv.close()


def test_iterations_grow_under_a_backlog(hostlib, scenes):
    """With max_tiles_backlog, iterations carry more tiles while more than twice max_tiles_per_iter
    tiles wait (and never more than max_tiles_backlog); without it they stay at the cap.  Images
    are the oracle's either way."""
    W, H = 64, 32                                   # 16 tiles per request
    cams = _cams(8, seed=19)
    counts = {}
    for backlog in (0, 48):
        srv = Server(hostlib, scenes, 1 << 22, max_tiles=8, max_tiles_backlog=backlog)
        try:
            srv.hold(True)
            rids = [srv.submit(k % 2, cams[k], W, H)[1] for k in range(8)]
            srv.until(lambda s: s.iterations >= 1)
            srv.hold(False)
            for k, rid in enumerate(rids):
                assert srv.wait(rid) == merf.MERF_OK
                np.testing.assert_array_equal(srv.bufs[rid], _expected(scenes[k % 2], cams[k], W, H))
            counts[backlog] = srv.stats().iterations
        finally:
            srv.close()
    assert counts[0] >= 16                          # 128 tiles, 8 per iteration
    assert counts[48] < counts[0]
    assert counts[48] >= 128 // 48


def test_requests_share_iterations(hostlib, scenes):
    """One-tile requests that arrive while both iteration slots are busy are batched into one
    iteration."""
    n = 12
    cams = _cams(n, seed=13)
    srv = Server(hostlib, scenes, 1 << 20, max_tiles=64)
    try:
        srv.hold(True)
        rids = [srv.submit(k % 2, cams[k], 16, 8)[1] for k in range(n)]
        srv.until(lambda s: s.iterations >= 1)
        time.sleep(0.05)
        srv.hold(False)                                 # two held iterations and at most one more
        for rid in rids:
            assert srv.wait(rid) == merf.MERF_OK
        s = srv.stats()
        assert s.tiles == n and s.iterations <= 3
        for k, rid in enumerate(rids):
            np.testing.assert_array_equal(srv.bufs[rid], _expected(scenes[k % 2], cams[k], 16, 8))
    finally:
        srv.close()


def test_cancel_pending_scheduled_and_completed(hostlib, scenes):
    W, H = 20, 12
    cams = _cams(6, seed=14)
    srv = Server(hostlib, scenes, 2 * W * H * 3 * 4 + 512, max_tiles=64)
    try:
        srv.hold(True)
        a = srv.submit(0, cams[0], W, H)[1]
        srv.until(lambda s: s.iterations == 1)          # a in flight (held)
        b = srv.submit(0, cams[1], W, H)[1]
        srv.until(lambda s: s.iterations == 2)          # b in flight (held)
        c, d = (srv.submit(0, cams[k], W, H)[1] for k in (2, 3))   # pending: the pool holds two
        assert srv.cancel(c) == (merf.MERF_OK, 1)       # never admitted
        assert srv.wait(c, timeout=5) == merf.ERR_CANCELLED
        assert srv.cancel(a) == (merf.MERF_OK, 1)       # its tiles are in a held iteration
        assert srv.wait(a, timeout=0.05) == merf.ERR_TIMEOUT
        s = srv.stats()                                 # a keeps its space until its iteration ends
        assert (s.admitted, s.queued, s.pool_used_bytes) == (2, 1, 2 * (-(-W * H * 3 // 64) * 64) * 4)
        srv.hold(False)
        assert srv.wait(a) == merf.ERR_CANCELLED
        for rid in (b, d):
            assert srv.wait(rid) == merf.MERF_OK
        assert np.isnan(srv.bufs[a]).all() and np.isnan(srv.bufs[c]).all()   # never written
        np.testing.assert_array_equal(srv.bufs[b], _expected(scenes[0], cams[1], W, H))
        np.testing.assert_array_equal(srv.bufs[d], _expected(scenes[0], cams[3], W, H))
        assert not any(cy == cams[2, 15] for _, cy, _, _ in srv.calls)          # c never rendered
        # complete but not yet waited for: left to finish
        e = srv.submit(1, cams[4], W, H)[1]
        srv.until(lambda s: s.completed == 3)
        assert srv.cancel(e) == (merf.MERF_OK, 0)
        assert srv.wait(e) == merf.MERF_OK
        # released requests are unknown
        assert srv.cancel(e)[0] == merf.ERR_INVALID_ARG
        assert srv.wait(e, timeout=0) == merf.ERR_INVALID_ARG
        s = srv.stats()
        assert (s.cancelled, s.completed, s.pool_used_bytes, s.admitted, s.queued) == (2, 3, 0, 0, 0)
    finally:
        srv.close()


def test_cancel_wakes_blocked_waiters(hostlib, scenes):
    """A client already blocked in wait() returns as soon as its request is cancelled (pending) or
    as soon as the iteration carrying its cancelled tiles ends, not at its timeout."""
    W, H = 16, 8
    cams = _cams(3, seed=19)
    srv = Server(hostlib, scenes, W * H * 3 * 4, max_tiles=64)
    try:
        srv.hold(True)
        a = srv.submit(0, cams[0], W, H)[1]
        srv.until(lambda s: s.iterations == 1)          # a in flight (held); the pool is full
        b = srv.submit(0, cams[1], W, H)[1]             # pending
        got = {}

        def waiter(rid):
            t0 = time.time()
            got[rid] = (srv.wait(rid, timeout=30), time.time() - t0)

        ts = [threading.Thread(target=waiter, args=(r,)) for r in (a, b)]
        for t in ts:
            t.start()
        time.sleep(0.1)
        assert srv.cancel(b) == (merf.MERF_OK, 1)
        assert srv.cancel(a) == (merf.MERF_OK, 1)
        time.sleep(0.1)
        srv.hold(False)
        for t in ts:
            t.join(timeout=60)
        assert got[a][0] == got[b][0] == merf.ERR_CANCELLED
        assert got[a][1] < 10 and got[b][1] < 10
    finally:
        srv.close()


def test_cancel_partly_scheduled_request(hostlib, scenes):
    """A request with tiles still to schedule and tiles in flight: no further tile is issued, and
    its pool space returns once the iterations carrying its tiles end."""
    W, H = 48, 16                                       # 3 x 2 = 6 tiles, 2 per iteration
    cams = _cams(2, seed=15)
    srv = Server(hostlib, scenes, 1 << 20, max_tiles=2)
    try:
        srv.hold(True)
        a = srv.submit(0, cams[0], W, H)[1]
        srv.until(lambda s: s.iterations == 2)          # 4 of its 6 tiles in held iterations
        assert srv.cancel(a) == (merf.MERF_OK, 1)
        srv.hold(False)
        assert srv.wait(a) == merf.ERR_CANCELLED
        assert np.isnan(srv.bufs[a]).all()
        assert len(srv.calls) == 4
        b = srv.submit(1, cams[1], 16, 8)[1]           # the server goes on serving
        assert srv.wait(b) == merf.MERF_OK
        np.testing.assert_array_equal(srv.bufs[b], _expected(scenes[1], cams[1], 16, 8))
        s = srv.stats()
        assert (s.tiles, s.cancelled, s.pool_used_bytes) == (5, 1, 0)
    finally:
        srv.close()


def test_device_failure_fails_outstanding_requests(hostlib, scenes):
    """A failed iteration (here a tile of scene 1) fails every request not yet complete with
    MERF_ERR_CUDA, and the server refuses further work."""
    cams = _cams(3, seed=16)
    srv = Server(hostlib, scenes, 1 << 20, max_tiles=64, fail_scene=1)
    try:
        srv.hold(True)
        r0 = srv.submit(0, cams[0], 32, 16)[1]
        r1 = srv.submit(1, cams[1], 32, 16)[1]
        srv.hold(False)
        assert srv.wait(r1) == merf.ERR_CUDA
        assert srv.wait(r0) in (merf.MERF_OK, merf.ERR_CUDA)
        assert srv.submit(0, cams[2], 16, 8)[0] == merf.ERR_CUDA
    finally:
        srv.close()


def test_argument_validation(hostlib, scenes):
    cam = _cams(1, seed=17)[0]
    srv = Server(hostlib, scenes, 64 * 64 * 3 * 4, max_tiles=8)
    try:
        assert srv.submit(2, cam, 8, 8)[0] == merf.ERR_INVALID_ARG       # scene out of range
        assert srv.submit(-1, cam, 8, 8)[0] == merf.ERR_INVALID_ARG
        assert srv.submit(0, cam, 0, 8)[0] == merf.ERR_INVALID_ARG
        assert srv.submit(0, cam, 8, 16385)[0] == merf.ERR_INVALID_ARG
        bad = cam.copy()
        bad[3] = np.nan
        assert srv.submit(0, bad, 8, 8)[0] == merf.ERR_INVALID_ARG
        bad = cam.copy()
        bad[12] = 0.0
        assert srv.submit(0, bad, 8, 8)[0] == merf.ERR_INVALID_ARG       # fx = 0
        assert srv.submit(0, cam, 65, 64)[0] == merf.ERR_OOM             # larger than the pool
        assert srv.wait(12345, timeout=0) == merf.ERR_INVALID_ARG
        assert srv.cancel(12345)[0] == merf.ERR_INVALID_ARG
        assert srv.stats().submitted == 0
    finally:
        srv.close()


def test_concurrent_clients(hostlib, scenes):
    """Four client threads submitting and waiting at once."""
    rng = np.random.default_rng(18)
    cams = _cams(24, seed=18)
    sizes = [(int(rng.integers(1, 40)), int(rng.integers(1, 30))) for _ in range(24)]
    srv = Server(hostlib, scenes, 3 * 40 * 30 * 3 * 4, max_tiles=6, workers=4)
    errors = []

    def client(ks):
        try:
            mine = [(k, srv.submit(k % 2, cams[k], *sizes[k])[1]) for k in ks]
            for k, rid in mine:
                assert srv.wait(rid) == merf.MERF_OK
                np.testing.assert_array_equal(srv.bufs[rid], _expected(scenes[k % 2], cams[k], *sizes[k]))
        except Exception as e:                      # noqa: BLE001 -- reported below
            errors.append(e)

    try:
        ts = [threading.Thread(target=client, args=(range(c, 24, 4),)) for c in range(4)]
        for t in ts:
            t.start()
        for t in ts:
            t.join(timeout=300)
        assert not errors, errors[0]
        s = srv.stats()
        assert s.completed == 24 and s.pool_used_bytes == 0
    finally:
        srv.close()
