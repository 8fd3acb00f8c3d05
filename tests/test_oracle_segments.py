"""Pins of the oracle's contracted-ray segments, arc length, t(s) and the sample lattice,
against brute-force dense sampling of the world ray (Sec. 3.2, Sec. 5) -- CPU only."""
import numpy as np
import pytest

import oracle
from tests import scenes


def _region_np(x):
    ax = np.abs(x)
    j = np.argmax(ax, axis=1)                 # first maximum = lowest index on ties
    m = ax[np.arange(len(x)), j]
    r = 1 + 2 * j + (x[np.arange(len(x)), j] < 0)
    return np.where(m <= 1.0, 0, r)


def _contract_np(x, r):
    """Region maps for brute force; the contraction itself is pinned in test_oracle_contract."""
    p = x.copy()
    out = r > 0
    j = (r[out] - 1) // 2
    idx = np.nonzero(out)[0]
    ax = np.abs(x[idx, j])
    p[idx] = x[idx] / ax[:, None]
    p[idx, j] = np.sign(x[idx, j]) * (2.0 - 1.0 / ax)
    return p


def _rays(n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        kind = k % 3
        if kind == 0:
            o = rng.uniform(-0.9, 0.9, size=3)            # inside the unit cube
        elif kind == 1:
            o = rng.uniform(-4, 4, size=3)                 # anywhere
        else:
            o = rng.normal(size=3)
            o *= rng.uniform(1.2, 3.0) / np.abs(o).max()   # outside, near
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        out.append((o, d))
    return out


def _dense(o, d, n=1_000_000):
    # t on [0, inf) through t = u / (1 - u) ** 2 -> dense near the camera, reaching t ~ 1e8
    u = np.linspace(0.0, 1.0 - 1e-4, n)
    t = u / (1.0 - u) ** 2
    x = o[None, :] + t[:, None] * d[None, :]
    r = _region_np(x)
    return t, x, r


@pytest.mark.parametrize("o,d", _rays(24, 0))
def test_segments_match_brute_force(o, d):
    sg = oracle.Segments(o, d)
    t, x, r = _dense(o, d)
    # region sequence
    change = np.nonzero(np.diff(r) != 0)[0]
    seq = [r[0]] + [r[i + 1] for i in change]
    assert [sg[i]["region"] for i in range(len(sg))] == seq
    # breakpoints: refine each dense change by bisection on the region function
    tb = []
    for i, c in enumerate(change):
        lo, hi = t[c], t[c + 1]
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if _region_np((o + mid * d)[None])[0] == r[c]:
                lo = mid
            else:
                hi = mid
        assert abs(sg[i + 1]["t0"] - lo) <= 1e-9 * max(1.0, lo)
        tb.append(lo)
    # straightness and end points of every segment
    p = _contract_np(x, r)
    for i in range(len(sg)):
        g = sg[i]
        sel = r == g["region"]
        q = p[sel]
        ab = g["b"] - g["a"]
        if g["len"] < 1e-9:
            continue
        e = ab / g["len"]
        rel = q - g["a"]
        perp = rel - np.outer(rel @ e, e)
        assert np.abs(perp).max() < 1e-9
        assert (rel @ e).min() > -1e-9 and (rel @ e).max() < g["len"] + 1e-9
    # total contracted arc length = polyline length within regions (jumps excluded)
    same = r[1:] == r[:-1]
    poly = np.linalg.norm(np.diff(p, axis=0), axis=1)[same].sum()
    # plus the two pieces on either side of each boundary, each in its own region's map
    for c, t_b in zip(change, tb):
        xb = (o + t_b * d)[None]
        poly += np.linalg.norm(_contract_np(xb, np.array([r[c]]))[0] - p[c])
        poly += np.linalg.norm(p[c + 1] - _contract_np(xb, np.array([r[c + 1]]))[0])
    # the dense grid stops at t ~ 1e8: add the exact remaining piece of the last segment
    last = sg[len(sg) - 1]
    tail = np.linalg.norm(last["b"] - p[-1])
    assert abs(poly + tail - sg.total) < 1e-9 * sg.total


@pytest.mark.parametrize("o,d", _rays(12, 1))
def test_t_of_s_lies_on_ray_and_is_monotone(o, d):
    sg = oracle.Segments(o, d)
    ss = np.linspace(0.0, sg.total * (1 - 1e-6), 400)
    ts = np.array([sg.t_of_s(s) for s in ss])
    assert ts[0] == 0.0
    assert np.all(np.diff(ts) > 0)
    for s, t in zip(ss[1:], ts[1:]):
        p = sg.point_at(s)
        # the world point at t contracts back to the point at arc length s
        xw = o + t * d
        np.testing.assert_allclose(oracle.contract(xw), p, atol=1e-9 * max(1, t))
    for i in range(1, len(sg)):
        g = sg[i]
        assert abs(sg.t_of_s(g["s0"]) - g["t0"]) <= 1e-9 * max(1.0, g["t0"])


def test_lattice_mask_matches_brute_force_on_tiny_grid():
    """The evaluated sample set equals dense sampling of the world ray: lattice sample k sits at
    contracted arc length (k + 1/2) step and is evaluated iff its finest occupancy cell is set."""
    rng = np.random.default_rng(5)
    N = 8
    occ = (rng.uniform(size=(N, N, N)) < 0.4).astype(np.uint8)
    sc = scenes.const_scene(L=8, B=4, R=8, occ_N=N, occ=occ)
    osc = oracle.OracleScene(sc)
    from paper_2302_12249_b300 import synth
    step = 1.0 / 16
    checked = 0
    for (o, d) in _rays(18, 2):
        # a camera looking along d from o: build the 3x4 with forward = d
        up = np.array([0.0, 0.0, 1.0]) if abs(d[2]) < 0.9 else np.array([1.0, 0.0, 0.0])
        c2w = synth.look_at(o, o + d, up)
        cam = synth.camera_record(c2w, 1, 1)
        cam[14] = 0.5
        cam[15] = 0.5                                    # principal point at the pixel centre
        mask, flags, nlat = oracle.trace(osc, cam[None], 1, 1, step, words=16, decide_f32=False, eps=5e-5)
        oo, dd = oracle.ray(cam, 0, 0)
        t, x, r = _dense(oo, dd, n=2_000_000)
        p = _contract_np(x, r)
        same = np.concatenate([[True], r[1:] == r[:-1]])
        seglen = np.linalg.norm(np.diff(p, axis=0), axis=1) * same[1:]
        s = np.concatenate([[0.0], np.cumsum(seglen)])
        for k in range(int(nlat[0])):
            sk = (k + 0.5) * step
            i = np.searchsorted(s, sk)
            f = (sk - s[i - 1]) / (s[i] - s[i - 1])
            pk = p[i - 1] + f * (p[i] - p[i - 1])
            cell = np.clip(np.floor((pk + 2) * N / 4).astype(int), 0, N - 1)
            want = bool(occ[cell[2], cell[1], cell[0]])
            got = bool(mask[0, k >> 5] >> (k & 31) & 1)
            flagged = bool(flags[0, k >> 5] >> (k & 31) & 1)
            assert got == want or flagged
            checked += 1
        # number of lattice samples: (k + 1) step < total arc length
        assert int(nlat[0]) == int(np.ceil(oracle.Segments(oo, dd).total / step)) - 1
    assert checked > 500
