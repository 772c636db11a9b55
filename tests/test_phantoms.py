"""Pins for the seeded input generator (CPU only).

The generator evaluates the closed-form line integrals of ellipses
(Kak & Slaney ch. 3).  Checks: each projection integrates to the ellipse's
mass rho*pi*A*B at every angle; point values match a brute-force numerical
line integral through the rasterised indicator; rasterised areas match pi*A*B;
the random fields obey their stated distributions; everything is reproducible
from its seed.
"""
import numpy as np
import pytest

from paper_2505_13955_gb300 import phantoms


def test_projection_mass_equals_rho_pi_ab_at_every_angle():
    N = 256
    R = N / 2
    ell = np.array([[0.1, -0.2, 0.5, 0.2, 0.7, 1.3]])
    K, D = 37, 1024
    # fine detector: spacing 0.25 px, so the Riemann sum converges
    p = phantoms.sinogram(ell, K, D, N, det_spacing=0.25, dtype=np.float64)
    mass = 1.3 * np.pi * (0.5 * R) * (0.2 * R)
    np.testing.assert_allclose(p.sum(axis=1) * 0.25, mass, rtol=2e-4)


def test_point_values_match_brute_force_line_integral():
    N = 64
    R = N / 2
    ell = np.array([[0.2, 0.1, 0.45, 0.25, 0.4, 0.9],
                    [-0.3, -0.2, 0.2, 0.3, 2.0, 0.5]])
    K, D = 6, 64
    p = phantoms.sinogram(ell, K, D, N, dtype=np.float64)
    t = np.linspace(-2 * R, 2 * R, 400001)
    dt = t[1] - t[0]
    for k in range(K):
        th = k * np.pi / K
        for j in (10, 25, 31, 40, 50):
            s = j - 0.5 * (D - 1)
            X = s * np.cos(th) - t * np.sin(th)
            Y = s * np.sin(th) + t * np.cos(th)
            acc = np.zeros_like(t)
            for x0, y0, A, B, phi, rho in ell:
                dx, dy = X - x0 * R, Y - y0 * R
                xa = dx * np.cos(phi) + dy * np.sin(phi)
                xb = -dx * np.sin(phi) + dy * np.cos(phi)
                acc += rho * ((xa / (A * R)) ** 2 + (xb / (B * R)) ** 2 <= 1.0)
            assert p[k, j] == pytest.approx(np.sum(acc) * dt, abs=2e-3 * max(1.0, p[k, j]))


def test_rasterised_area():
    N = 200
    R = N / 2
    ell = np.array([[0.0, 0.1, 0.6, 0.3, 0.3, 1.0]])
    img = phantoms.image(ell, N, supersample=4)
    assert img.sum() == pytest.approx(np.pi * 0.6 * R * 0.3 * R, rel=3e-3)


def test_shepp_logan_table_shape_and_values():
    t = phantoms.shepp_logan()
    assert t.shape == (10, 6)
    assert t[0, 5] == 2.0 and t[1, 5] == -0.98
    # outer ellipse: 0.69 wide (x), 0.92 tall (y) after the 90 degree rotation
    img = phantoms.image(t, 256)
    cols = np.nonzero(img[128] != 0)[0]
    rows = np.nonzero(img[:, 128] != 0)[0]
    assert (cols.max() - cols.min() + 1) / 128 == pytest.approx(2 * 0.69, abs=0.02)
    assert (rows.max() - rows.min() + 1) / 128 == pytest.approx(2 * 0.92, abs=0.02)


def test_random_ellipses_distribution_and_determinism():
    a = phantoms.random_ellipses(phantoms.rng_for(123))
    b = phantoms.random_ellipses(phantoms.rng_for(123))
    np.testing.assert_array_equal(a, b)
    assert 20 <= len(a) <= 50
    assert np.all((a[:, 2] >= 0.04) & (a[:, 2] <= 0.8))
    assert np.all((a[:, 3] >= 0.04) & (a[:, 3] <= 0.8))
    assert np.all((a[:, 4] >= 0) & (a[:, 4] < np.pi))
    assert np.all((a[:, 5] >= 0) & (a[:, 5] <= 1))
    assert np.all(np.hypot(a[:, 0], a[:, 1]) + np.maximum(a[:, 2], a[:, 3]) <= 0.95)


def test_poisson_noise_is_unbiased_at_high_counts():
    rng = phantoms.rng_for(5)
    p = np.full(200000, 100.0)
    n = 256
    noisy = phantoms.poisson_noise(p, n, 1e6, rng)
    assert np.mean(noisy) == pytest.approx(100.0, abs=0.05)
    # relative count noise 1/sqrt(I0 e^-mu) -> line-integral noise n / sqrt(counts)
    expected_sd = n / np.sqrt(1e6 * np.exp(-100.0 / n))
    assert np.std(noisy) == pytest.approx(expected_sd, rel=0.02)


def test_workload_slices_are_reproducible():
    w = phantoms.WORKLOADS["fbp_ragged_batch"]
    specs = [phantoms.slice_spec(w, i)[:2] for i in range(40)]
    assert specs == [phantoms.slice_spec(w, i)[:2] for i in range(40)]
    ns = {s[0] for s in specs}
    ks = {s[1] for s in specs}
    assert ns <= {512, 1024, 2048, 4096} and len(ns) > 1
    assert ks <= {720, 1800, 3600} and len(ks) > 1
    w1 = phantoms.WORKLOADS["fbp_single_n256"]
    s = phantoms.slice_sinogram(w1, 0)
    assert s.shape == (360, 256) and s.dtype == np.float32
    np.testing.assert_array_equal(s, phantoms.slice_sinogram(w1, 0))
