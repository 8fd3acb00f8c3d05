"""Pins of the oracle's contraction (Sec. 3.2, equation for contract_pi) -- CPU only."""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "contract_vectors.txt")


def _golden():
    rows = []
    for line in open(GOLDEN):
        line = line.split("#")[0].strip()
        if not line:
            continue
        lhs, rhs = line.split("|")
        x = [float(Fraction(v)) for v in lhs.split()]
        p = [float(Fraction(v)) for v in rhs.split()]
        rows.append((x, p))
    return rows


@pytest.mark.parametrize("x,p", _golden())
def test_hand_derived_values(x, p):
    np.testing.assert_allclose(oracle.contract(x), p, rtol=0, atol=1e-15)


def test_identity_inside_unit_cube():
    rng = np.random.default_rng(0)
    for x in rng.uniform(-1, 1, size=(2000, 3)):
        assert oracle.region(x) == 0
        np.testing.assert_array_equal(oracle.contract(x), x)


def _far_points(rng, n):
    d = rng.normal(size=(n, 3))
    d /= np.abs(d).max(axis=1, keepdims=True)
    r = 10.0 ** rng.uniform(0.0, 6.0, size=n)
    return d * r[:, None] * 1.0000001


def test_range_is_open_box_of_radius_two():
    rng = np.random.default_rng(1)
    for x in _far_points(rng, 3000):
        p = oracle.contract(x)
        assert np.all(np.abs(p) < 2.0)
        assert np.abs(p).max() >= 1.0 - 1e-12
        # the largest coordinate stays the largest and keeps its sign
        j = int(np.argmax(np.abs(x)))
        assert np.sign(p[j]) == np.sign(x[j]) and abs(p[j]) >= np.abs(p).max() - 1e-12


def test_continuous_across_unit_cube_boundary():
    rng = np.random.default_rng(2)
    for _ in range(500):
        x = rng.uniform(-1, 1, size=3)
        j = rng.integers(3)
        x[j] = np.sign(rng.normal()) * 1.0        # on a face of the cube
        n = np.zeros(3)
        n[j] = np.sign(x[j])
        for eps in (1e-3, 1e-6):
            pin, pout = oracle.contract(x - eps * n), oracle.contract(x + eps * n)
            assert np.abs(pin - pout).max() < 4 * eps


def test_jump_across_diagonal_between_outer_regions():
    """Reading: the map is continuous within each region but not across |x_j| = |x_k| > 1."""
    eps = 1e-9
    np.testing.assert_allclose(oracle.contract([3, 3 - eps, 0]), [5 / 3, (3 - eps) / 3, 0], atol=1e-15)
    np.testing.assert_allclose(oracle.contract([3 - eps, 3, 0]), [(3 - eps) / 3, 5 / 3, 0], atol=1e-15)


def test_round_trip_with_region_inverse():
    rng = np.random.default_rng(3)
    pts = np.concatenate([rng.uniform(-1, 1, size=(200, 3)), _far_points(rng, 2000)])
    for x in pts:
        r = oracle.region(x)
        back = oracle.uncontract(r, oracle.contract(x))
        # 2 - |p_j| loses digits as |x_j| grows: the inverse is conditioned like |x|_inf
        rel = 1e-13 + 1e-15 * np.abs(x).max()
        np.testing.assert_allclose(back, x, rtol=rel, atol=1e-13)


def test_projective_within_region_preserves_lines():
    """Three collinear points of one region stay collinear after contraction (Sec. 3.2)."""
    rng = np.random.default_rng(4)
    hits = 0
    while hits < 300:
        a = _far_points(rng, 1)[0] * rng.uniform(1, 3)
        b = a + rng.normal(size=3) * rng.uniform(0.01, 2.0) * np.abs(a).max()
        ts = np.sort(rng.uniform(0, 1, size=3))
        xs = [a + t * (b - a) for t in ts]
        regs = {oracle.region(x) for x in xs}
        if len(regs) != 1 or 0 in regs:
            continue
        ps = [oracle.contract(x) for x in xs]
        u, v = ps[1] - ps[0], ps[2] - ps[0]
        assert np.linalg.norm(np.cross(u, v)) <= 1e-12 * (1 + np.linalg.norm(u) * np.linalg.norm(v)) + 1e-14
        # and the parametrisation is monotone along the line
        assert np.dot(u, v) >= 0
        hits += 1


def test_region_labels_and_ties():
    assert oracle.region([0.3, 0.2, -1.0]) == 0
    assert oracle.region([1.5, 0, 0]) == 1
    assert oracle.region([-1.5, 0, 0]) == 2
    assert oracle.region([0, 1.5, 0]) == 3
    assert oracle.region([0, -1.5, 0]) == 4
    assert oracle.region([0, 0, 1.5]) == 5
    assert oracle.region([0, 0, -1.5]) == 6
    assert oracle.region([2, -2, 2]) == 1          # tie: lowest axis index
    assert oracle.region([0, -2, 2]) == 4
