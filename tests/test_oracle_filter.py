"""Pins for the oracle's filtering step (CPU only).

The paper names the step ("filtering", Sec. IV-B and Sec. V-A(c) stage 2) and
cites Kak & Slaney ch. 3 for it, but prints no formula.  These tests tie the
oracle's taps and convolution to facts fixed by mathematics, not by the
oracle's own code:

* the DTFT of the band-limited Ram-Lak kernel is |f| on [-1/2, 1/2] and that
  of the Shepp-Logan kernel is |sin(pi f)| / pi, to within the truncation tail;
* the DC gain of the truncated Ram-Lak kernel equals its closed-form tail,
  written with the trigamma function;
* the convolution equals numpy's linear convolution;
* the oracle's FFT equals numpy's FFT, and its FFT filter equals its direct one;
* tau scaling and the one-bin special case.
"""
import numpy as np
import pytest
from scipy.special import polygamma

import oracle

RL, SL = oracle.RAMLAK, oracle.SHEPP_LOGAN


def dtft(h, f):
    D = (len(h) + 1) // 2
    n = np.arange(-(D - 1), D)
    return np.real(np.exp(-2j * np.pi * np.outer(f, n)) @ h)


@pytest.mark.parametrize("D", [16, 65, 256, 1024])
def test_ramlak_frequency_response_is_abs_f(D):
    h = oracle.taps(RL, D)
    f = np.linspace(-0.5, 0.5, 2001)
    # tail bound: sum_{|n| > D-1} |h[n]| = (2/pi^2) sum_{odd n > D-1} 1/n^2
    m = D // 2  # odd n >= 2m+1 are the ones beyond D-1 (D-1 >= 2m-1)
    tail = (2.0 / np.pi ** 2) * polygamma(1, m + 0.5) / 4.0
    err = np.max(np.abs(dtft(h, f) - np.abs(f)))
    assert err <= tail * (1 + 1e-9) + 1e-12
    # and the bound is not vacuous: it is well below the response scale
    assert tail < 0.05


@pytest.mark.parametrize("D", [16, 65, 256, 1024])
def test_shepp_logan_frequency_response(D):
    h = oracle.taps(SL, D)
    f = np.linspace(-0.5, 0.5, 2001)
    n = np.arange(D, 200000)
    tail = 2.0 * np.sum(2.0 / (np.pi ** 2 * (4.0 * n * n - 1.0)))
    tail += 1.0 / (np.pi ** 2 * 200000)  # both sides' remainder beyond the explicit sum
    err = np.max(np.abs(dtft(h, f) - np.abs(np.sin(np.pi * f)) / np.pi))
    assert err <= tail * (1 + 1e-6)


@pytest.mark.parametrize("D", [1, 2, 3, 8, 101, 2048])
def test_ramlak_dc_gain_equals_closed_form_tail(D):
    h = oracle.taps(RL, D)
    # odd n beyond D-1: n >= 2*ceil(D/2)... write n = 2i+1 > D-1  <=>  i >= floor(D/2)
    m = D // 2
    expected = (2.0 / np.pi ** 2) * polygamma(1, m + 0.5) / 4.0
    assert np.sum(h) == pytest.approx(expected, rel=1e-10, abs=1e-15)


def test_taps_known_values_and_symmetry():
    h = oracle.taps(RL, 5)
    assert h[4] == pytest.approx(0.25)
    assert h[5] == pytest.approx(-1 / np.pi ** 2)
    assert h[6] == 0.0
    assert h[7] == pytest.approx(-1 / (9 * np.pi ** 2))
    np.testing.assert_array_equal(h, h[::-1])
    s = oracle.taps(SL, 5)
    assert s[4] == pytest.approx(2 / np.pi ** 2)
    assert s[5] == pytest.approx(-2 / (3 * np.pi ** 2))
    np.testing.assert_array_equal(s, s[::-1])
    # tau scales the kernel by 1/tau^2
    np.testing.assert_allclose(oracle.taps(RL, 5, tau=0.5), 4.0 * h, rtol=1e-15)


@pytest.mark.parametrize("kind", [RL, SL])
@pytest.mark.parametrize("D", [1, 2, 7, 64, 129])
def test_direct_filter_equals_numpy_linear_convolution(kind, D):
    rng = np.random.default_rng(D + 10 * kind)
    K = 5
    p = rng.standard_normal((K, D))
    tau = 0.75
    h = oracle.taps(kind, D, tau)
    q = oracle.filter_direct(p, kind, tau)
    for k in range(K):
        full = np.convolve(p[k], h)          # length 3D-2, index (D-1)+j is lag j
        np.testing.assert_allclose(q[k], tau * full[D - 1:2 * D - 1], rtol=1e-12, atol=1e-13)


def test_tau_scaling_of_filter():
    rng = np.random.default_rng(3)
    p = rng.standard_normal((3, 40))
    q1 = oracle.filter_direct(p, RL, 1.0)
    q2 = oracle.filter_direct(p, RL, 2.5)
    np.testing.assert_allclose(q2, q1 / 2.5, rtol=1e-12, atol=1e-15)


def test_single_bin_filter():
    p = np.array([[3.0], [-2.0]])
    np.testing.assert_allclose(oracle.filter_direct(p, RL, 1.0), p / 4.0)
    np.testing.assert_allclose(oracle.filter_direct(p, SL, 1.0), p * 2 / np.pi ** 2)


@pytest.mark.parametrize("L", [1, 2, 8, 64, 1024])
def test_oracle_fft_equals_numpy(L):
    rng = np.random.default_rng(L)
    x = rng.standard_normal(L) + 1j * rng.standard_normal(L)
    np.testing.assert_allclose(oracle.fft(x, -1), np.fft.fft(x), rtol=1e-11, atol=1e-11)
    np.testing.assert_allclose(oracle.fft(x, +1), L * np.fft.ifft(x), rtol=1e-11, atol=1e-11)


def test_conv_length():
    assert oracle.conv_length(1) == 1
    assert oracle.conv_length(2) == 4
    assert oracle.conv_length(256) == 512
    assert oracle.conv_length(257) == 1024
    assert oracle.conv_length(8192) == 16384


@pytest.mark.parametrize("kind", [RL, SL])
@pytest.mark.parametrize("D", [1, 5, 256, 2048])
def test_fft_filter_equals_direct(kind, D):
    rng = np.random.default_rng(D)
    p = rng.standard_normal((3, D)) * 10
    qd = oracle.filter_direct(p, kind)
    qf = oracle.filter_fft(p, kind)
    scale = np.max(np.abs(qd))
    np.testing.assert_allclose(qf, qd, rtol=0, atol=1e-12 * scale * max(1, np.log2(D)))


def test_filter_dispatch_uses_fft_above_2048():
    rng = np.random.default_rng(1)
    p = rng.standard_normal((1, 2049))
    np.testing.assert_array_equal(oracle.filter(p), oracle.filter_fft(p))
    p = rng.standard_normal((1, 2048))
    np.testing.assert_array_equal(oracle.filter(p), oracle.filter_direct(p))
