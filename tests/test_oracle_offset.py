"""Pins for the oracle's offset-scan weighting (Sec. V-A(b), offset scans):
the redundancy identity, the reduction of a full 360-degree centred scan to
the 180-degree FBP, and the reconstruction of a phantom wider than the
detector."""
import math

import numpy as np
import pytest

import oracle
from paper_2505_13955_gb300 import phantoms


@pytest.mark.parametrize("D,c,delta", [(64, 10.0, 6.0), (65, 50.5, 8.0), (101, 50.0, 20.0), (300, 31.5, 31.5)])
def test_offset_weights_redundancy(D, c, delta):
    n_v, c_v, off, w = oracle.offset_virtual(D, c, delta)
    assert n_v % 1 == 0 and c_v == (n_v - 1) / 2
    # physical bins land inside the virtual detector, the long side reaches its end
    assert off >= 0 and off + D <= n_v and (off + D == n_v or off == 0)
    long_positive = (D - 1 - c) >= c
    t = (np.arange(n_v) - c_v) * (1 if long_positive else -1)
    assert np.all(w[t > delta] == 1.0) and np.all(w[t < -delta] == 0.0)
    assert np.all((w >= 0) & (w <= 1))
    # w(t) + w(-t) = 1 for every virtual bin (bin i mirrors to n_v - 1 - i)
    np.testing.assert_allclose(w + w[::-1], 1.0, atol=1e-15)
    # every virtual bin with a nonzero weight is a physical bin
    phys = np.zeros(n_v, bool)
    phys[off:off + D] = True
    assert np.all(phys[w > 0])
    order = np.argsort(t)
    assert np.all(np.diff(w[order]) >= -1e-15)
    assert oracle.offset_weight(np.array([0.0]), 4.0)[0] == pytest.approx(0.5)


def test_full_circle_centred_scan_with_half_weight_is_the_half_circle_fbp():
    """360 degrees at a centred detector with w = 1/2 reproduces the 180-degree
    FBP: p(th + pi, -s) = p(th, s), and the angle grid 2 pi k / 2K contains
    the pi k / K grid twice."""
    N = K = 64
    ell = phantoms.random_ellipses(phantoms.rng_for(5), count_range=(4, 6))
    g180 = oracle.Geometry(K, N, N)
    g360 = oracle.Geometry(2 * K, N, N, angle_step=2 * math.pi / (2 * K))
    p180 = phantoms.sinogram(ell, K, N, N, dtype=np.float64)
    p360 = phantoms.sinogram(ell, 2 * K, N, N, angle_step=2 * math.pi / (2 * K), dtype=np.float64)
    f360 = oracle.fbp_weighted(p360, g360, np.full(N, 0.5))
    f180 = oracle.fbp(p180, g180)
    np.testing.assert_allclose(f360, f180, atol=1e-9 * np.abs(f180).max())


def test_offset_scan_equals_the_half_circle_fbp_on_the_virtual_detector():
    """A detector of D bins with the axis at c covers a field of view of
    radius D - 1 - c.  Embedded in the virtual detector and weighted, the
    360-degree FBP of the offset scan equals the 180-degree FBP of a centred
    detector that spans the same field of view (exactly: each line's two
    weights sum to 1, and the filter sees the whole weighted row)."""
    N = 128
    D, c, delta = 80, 15.5, 12.0                  # FoV radius 63.5
    K = 360
    ell = phantoms.random_ellipses(phantoms.rng_for(9), count_range=(6, 10))
    p_off = phantoms.sinogram(ell, K, D, N, angle_step=2 * math.pi / K, det_center=c, dtype=np.float64)
    n_v, c_v, off, w = oracle.offset_virtual(D, c, delta)
    assert n_v == 128 and off == 48
    g_v = oracle.Geometry(K, n_v, N, angle_step=2 * math.pi / K)
    f_off = oracle.fbp_weighted(oracle.embed_rows(p_off, n_v, off), g_v, w)
    f_ref = oracle.fbp(phantoms.sinogram(ell, K // 2, n_v, N, dtype=np.float64), oracle.Geometry(K // 2, n_v, N))
    np.testing.assert_allclose(f_off, f_ref, atol=1e-9 * np.abs(f_ref).max())
    # the axis on the other side: the same scan mirrored
    p_mir = phantoms.sinogram(ell, K, D, N, angle_step=2 * math.pi / K, det_center=D - 1 - c, dtype=np.float64)
    n_m, c_m, off_m, w_m = oracle.offset_virtual(D, D - 1 - c, delta)
    assert n_m == 128 and off_m == 0
    f_mir = oracle.fbp_weighted(oracle.embed_rows(p_mir, n_m, off_m), oracle.Geometry(K, n_m, N, angle_step=2 * math.pi / K), w_m)
    np.testing.assert_allclose(f_mir, f_ref, atol=1e-9 * np.abs(f_ref).max())
    # without the weights the overlap is counted twice; on the physical
    # detector alone the filtered row's spill past the short edge is lost
    X = np.arange(N) - (N - 1) / 2
    inside = np.hypot(*np.meshgrid(X, X)) <= 0.45 * N
    dr = f_ref.max() - f_ref.min()
    f_unw = oracle.fbp(oracle.embed_rows(p_off, n_v, off), g_v)
    assert np.abs(f_unw - f_ref)[inside].mean() > 0.05 * dr
    f_phys = oracle.fbp_weighted(p_off, oracle.Geometry(K, D, N, angle_step=2 * math.pi / K, det_center=c),
                                 oracle.offset_weight(np.arange(D) - c, delta))
    assert np.abs(f_phys - f_ref)[inside].mean() > 0.01 * dr


def test_offset_fold_of_analytic_rows_is_the_half_turn_sinogram():
    """Noise-free: the folded rows of a full-turn offset scan are the
    analytic half-turn sinogram of the centred virtual detector (each line's
    two weights sum to 1 and both samples are the same line integral)."""
    N = 96
    D, c, delta = 60, 12.5, 9.0                   # FoV radius 46.5
    K = 200
    ell = phantoms.random_ellipses(phantoms.rng_for(17), count_range=(5, 8))
    p_off = phantoms.sinogram(ell, K, D, N, angle_step=2 * math.pi / K, det_center=c, dtype=np.float64)
    n_v, c_v, off, w = oracle.offset_virtual(D, c, delta)
    assert n_v == 94 and off == 34
    r = oracle.offset_fold(oracle.embed_rows(p_off, n_v, off), w)
    assert r.shape == (K // 2, n_v)
    ref = phantoms.sinogram(ell, K // 2, n_v, N, dtype=np.float64)
    np.testing.assert_allclose(r, ref, atol=1e-10 * np.abs(ref).max())
    # a wrong mirror (no reversal) or one weight for both halves fails
    bad = oracle.embed_rows(p_off, n_v, off)[:K // 2] * w + oracle.embed_rows(p_off, n_v, off)[K // 2:] * w
    assert np.abs(bad - ref).max() > 1e-2 * np.abs(ref).max()


def test_offset_fold_then_half_turn_fbp_equals_the_full_turn_fbp():
    N = 128
    D, c, delta = 80, 15.5, 12.0
    K = 240
    ell = phantoms.random_ellipses(phantoms.rng_for(21), count_range=(6, 10))
    p_off = phantoms.sinogram(ell, K, D, N, angle_step=2 * math.pi / K, det_center=c, dtype=np.float64)
    n_v, c_v, off, w = oracle.offset_virtual(D, c, delta)
    pv = oracle.embed_rows(p_off, n_v, off)
    f360 = oracle.fbp_weighted(pv, oracle.Geometry(K, n_v, N, angle_step=2 * math.pi / K), w,
                               oracle.SHEPP_LOGAN)
    f180 = oracle.fbp(oracle.offset_fold(pv, w), oracle.Geometry(K // 2, n_v, N, angle_step=2 * math.pi / K),
                      oracle.SHEPP_LOGAN)
    np.testing.assert_allclose(f180, f360, atol=1e-10 * np.abs(f360).max())
    with pytest.raises(ValueError):
        oracle.offset_fold(pv[:-1], w)
