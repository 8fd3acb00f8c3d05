"""Pins of the oracle's spherical-contraction ablation (Sec. 3.2, Eq. contract360, Table 2 (c)):
the contraction, its sample spacing and the densely marched quadrature -- CPU only."""
import math

import numpy as np

import oracle
from paper_2302_12249_b300 import synth
from tests import scenes


def test_contraction_closed_forms():
    """Identity inside the unit ball; outside, the direction is kept and the radius becomes
    2 - 1/|x| (continuous at |x| = 1, tending to 2 at infinity)."""
    rng = np.random.default_rng(0)
    for _ in range(200):
        x = rng.normal(size=3)
        x *= rng.uniform(0.05, 0.99) / np.linalg.norm(x)
        np.testing.assert_allclose(oracle.contract_sph(x), x, rtol=0, atol=0)
    for _ in range(200):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        r = math.exp(rng.uniform(0.0, 12.0))
        p = oracle.contract_sph(r * d)
        np.testing.assert_allclose(np.linalg.norm(p), 2.0 - 1.0 / r, rtol=1e-14)
        np.testing.assert_allclose(p / np.linalg.norm(p), d, atol=1e-12)
    d = np.array([0.6, -0.8, 0.0])
    np.testing.assert_allclose(oracle.contract_sph((1 + 1e-12) * d), d, atol=1e-11)
    assert 2.0 - np.linalg.norm(oracle.contract_sph(1e15 * d)) < 1e-14


def test_contraction_bends_straight_lines():
    """Three collinear points in one outer region of contract_pi (largest coordinate +x) stay
    collinear under contract_pi and do not under the spherical contraction, so a contracted ray
    is no longer straight and an AABB exit cannot be taken along it."""
    a, b = np.array([3.0, -1.0, 0.5]), np.array([3.0, 1.0, 0.5])
    m = 0.5 * (a + b)
    assert oracle.region(a) == oracle.region(b) == oracle.region(m)

    def bend(f):
        pa, pb, pm = (f(v) for v in (a, b, m))
        u, v = pb - pa, pm - pa
        return np.linalg.norm(np.cross(u, v)) / (np.linalg.norm(u) * np.linalg.norm(v))

    assert bend(oracle.contract) < 1e-12
    assert bend(oracle.contract_sph) > 0.01


def test_spacing_function_and_sample_count():
    """t(s) = s up to 1 and 1/(2 - s) beyond: continuous at s = 1, the inverse of s = 2 - 1/t;
    samples (k + 1/2) step for (k + 1) step < 2."""
    assert oracle.sph_t_of_s(1.0) == 1.0
    for t in (1.5, 3.0, 40.0, 1e6):
        np.testing.assert_allclose(oracle.sph_t_of_s(2.0 - 1.0 / t), t, rtol=1e-9)
    for s in (0.0, 0.3, 0.999):
        assert oracle.sph_t_of_s(s) == s
    for step in (1 / 64, 1 / 256, 0.3):
        n = oracle.sph_count(step)
        assert (n + 1) * step >= 2.0 > n * step
        assert oracle.sph_count(step, f32=True) == n


def test_fp32_positions_follow_the_fp64_ones():
    rng = np.random.default_rng(3)
    for _ in range(50):
        o = rng.uniform(-2, 2, 3)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        for k in (0, 17, 100, 200, 250):
            t = oracle.sph_t_of_s((k + 0.5) / 128)
            p64 = oracle.contract_sph(o + t * d)
            p32 = oracle.sph_point32(o, d, 1 / 128, k)
            np.testing.assert_allclose(p32, p64, atol=2e-5 * max(1.0, np.abs(p64).max()))


def test_constant_field_quadrature_closed_form():
    """Constant density and colour, every cell occupied, no termination: the world steps telescope,
    so T = exp(-tau t(n step)) with n the sample count, and C_d = (1 - T) sigmoid(colour)."""
    sc = scenes.const_scene(L=16, B=4, R=32, occ_N=16, dens_byte=100, app_byte=150)
    osc = oracle.OracleScene(sc)
    cams = synth.sphere_cameras(2, 6, 5, radius=1.7, seed=2)
    step = 1 / 64
    out = oracle.render(osc, cams, 6, 5, step, early_term=False, no_mlp=True, contraction=1)
    # per-source dequantisation: grid weight 1 plus three planes
    tau = math.exp(4 * scenes.dequant(100, 14.0))
    colour = 1 / (1 + math.exp(-4 * scenes.dequant(150, 7.0)))
    n = oracle.sph_count(step, f32=True)
    T = math.exp(-tau * oracle.sph_t_of_s(n * step))
    np.testing.assert_allclose(out[:, oracle.ORC_T], T, rtol=1e-9, atol=1e-300)
    np.testing.assert_allclose(out[:, oracle.ORC_CD], (1 - T) * colour, rtol=1e-9)
    assert (out[:, oracle.ORC_NEVAL] == n).all() and (out[:, oracle.ORC_NLAT] == n).all()
