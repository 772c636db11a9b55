"""Pins for the oracle's stage-2 pre-processing (Beer-Lambert, Gaussian blur)
and stage-4 output mapping (HU window, uint16), Sec. V-A(c): closed forms,
the definitions' fixed points, and scipy's Gaussian filter as an independent
routine."""
import math

import numpy as np
import pytest

import oracle


def test_beer_lambert_inverts_the_attenuation_law():
    rng = np.random.default_rng(0)
    p = rng.uniform(0, 8, size=(5, 40))
    I0 = rng.uniform(1e3, 1e5, size=40)            # per-bin flat field
    I = I0 * np.exp(-p)
    np.testing.assert_allclose(oracle.beer_lambert(I, I0), p, rtol=0, atol=1e-12)
    np.testing.assert_allclose(oracle.beer_lambert(I, I0, mu_scale=256.0), 256.0 * p, atol=1e-9)
    # scalar flat field, and the counting floor
    assert oracle.beer_lambert(np.array([1e4 / math.e]), 1e4)[0] == pytest.approx(1.0, abs=1e-15)
    assert oracle.beer_lambert(np.array([0.0]), 100.0, floor=1.0)[0] == pytest.approx(math.log(100.0))
    assert oracle.beer_lambert(np.array([100.0]), 100.0)[0] == 0.0


@pytest.mark.parametrize("sigma", [0.3, 0.8, 1.0, 1.7, 3.0])
def test_gaussian_taps(sigma):
    w = oracle.gaussian_taps(sigma)
    r = int(4 * sigma + 0.5)
    assert len(w) == 2 * r + 1
    assert w.sum() == pytest.approx(1.0, abs=1e-15)
    np.testing.assert_array_equal(w, w[::-1])
    if r >= 1:
        assert w[r + 1] / w[r] == pytest.approx(math.exp(-1 / (2 * sigma * sigma)), rel=1e-13)
    np.testing.assert_array_equal(oracle.gaussian_taps(0.0), [1.0])


@pytest.mark.parametrize("sigma", [0.5, 1.0, 2.2])
def test_gaussian_blur_equals_scipy_gaussian_filter(sigma):
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(1)
    p = rng.standard_normal((3, 57))
    ref = ndimage.gaussian_filter1d(p, sigma, axis=-1, mode="constant", cval=0.0, truncate=4.0)
    np.testing.assert_allclose(oracle.gaussian_blur(p, sigma), ref, rtol=0, atol=1e-13)


def test_gaussian_blur_fixed_points():
    sigma = 1.3
    w = oracle.gaussian_taps(sigma)
    r = (len(w) - 1) // 2
    # a constant row stays constant away from the edges; a delta becomes the taps
    y = oracle.gaussian_blur(np.ones((1, 40)), sigma)[0]
    np.testing.assert_allclose(y[r:40 - r], 1.0, atol=1e-15)
    d = np.zeros(41)
    d[20] = 1.0
    np.testing.assert_allclose(oracle.gaussian_blur(d, sigma)[20 - r:21 + r], w, atol=1e-16)
    # a linear ramp stays linear in the interior (symmetric kernel)
    x = np.arange(60.0)
    yl = oracle.gaussian_blur(x, sigma)
    np.testing.assert_allclose(yl[r:60 - r], x[r:60 - r], atol=1e-12)
    # sigma = 0 is the identity
    z = np.random.default_rng(2).standard_normal(30)
    np.testing.assert_array_equal(oracle.gaussian_blur(z, 0.0), z)


def test_hu_definition_and_window():
    mw, ma = 0.0193, 0.0
    assert oracle.hu(mw, mw, ma) == 0.0
    assert oracle.hu(ma, mw, ma) == -1000.0
    assert oracle.hu(2 * mw, mw, ma) == pytest.approx(1000.0)
    lo, hi = -1000.0, 3000.0
    mu = np.array([ma, mw * (1 + hi / 1000.0), -0.01, 1.0, mw])
    c = oracle.hu_codes(mu, mw, ma, lo, hi)
    assert c.dtype == np.uint16
    assert c[0] == 0 and c[1] == 65535 and c[2] == 0 and c[3] == 65535
    assert c[4] == round(1000.0 / 4000.0 * 65535)
    xs = np.linspace(-0.01, 0.1, 1001)
    assert np.all(np.diff(oracle.hu_codes(xs, mw, ma, lo, hi).astype(int)) >= 0)


def test_hu_affine_and_fp32_form():
    mw, ma, lo, hi = 0.0193, 0.0002, -1200.0, 2800.0
    a, b = oracle.hu_affine(mw, ma, lo, hi)
    mu = np.linspace(-0.005, 0.08, 777)
    x = (oracle.hu(mu, mw, ma) - lo) / (hi - lo) * 65535.0
    np.testing.assert_allclose(a * mu + b, x, rtol=0, atol=1e-8)
    # the FP32 sequence agrees with the FP64 codes except within FP32 rounding of a tie
    mu32 = mu.astype(np.float32)
    c32 = oracle.hu_codes_f32(mu32, np.float32(a), np.float32(b))
    c64 = oracle.hu_codes(mu32.astype(np.float64), mw, ma, lo, hi)
    frac = np.abs((a * mu32.astype(np.float64) + b) % 1.0 - 0.5)
    away = frac > 1e-2
    np.testing.assert_array_equal(c32[away], c64[away])
    assert np.max(np.abs(c32.astype(int) - c64.astype(int))) <= 1


def test_beer_lambert_then_fbp_equals_fbp_of_line_integrals():
    """Counts simulated without noise from a disk's line integrals (pixel
    units, mu_scale = N) reproduce the FBP of those line integrals."""
    N, K = 33, 24
    g = oracle.Geometry(K, N, N)
    s = np.arange(N) - (N - 1) / 2
    R = 10.0
    p = np.tile(2 * np.sqrt(np.maximum(R * R - s * s, 0.0)), (K, 1))   # unit density disk
    I0 = 1e4
    I = I0 * np.exp(-p / N)
    q = oracle.preprocess(I, I0, mu_scale=N, floor=1e-30, sigma=0.0)
    np.testing.assert_allclose(q, p, atol=1e-10)
    np.testing.assert_allclose(oracle.fbp(q, g), oracle.fbp(p, g), atol=1e-9)
