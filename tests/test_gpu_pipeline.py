"""GPU parity for the steps fused on either side of the path (Sec. V-A(c)
stages 2 and 4): fbp_filter_counts (Beer-Lambert + Gaussian blur + ramp
filter) and fbp_backproject_u16 (HU window quantised to uint16), against
the oracle's FP64 pre-processing and the FP32 code sequence."""
import math

import numpy as np
import pytest

import oracle
from gpu_util import assert_within_dr, fbp_api, needs_gpu, to_gpu, to_np, torch
from paper_2505_13955_gb300 import phantoms

pytestmark = [pytest.mark.gpu, needs_gpu]


def counts_for(N, K, seed, photons=1e4, noise=True):
    ell = phantoms.random_ellipses(phantoms.rng_for(seed), count_range=(5, 12))
    p = phantoms.sinogram(ell, K, N, N, dtype=np.float64)
    if noise:
        return phantoms.poisson_counts(p, N, photons, phantoms.rng_for(seed + 1)), p
    return (photons * np.exp(-p / N)).astype(np.float32), p


@pytest.mark.parametrize("sigma", [0.0, 0.7, 1.5, 3.875])
@pytest.mark.parametrize("S,K,D", [(1, 5, 7), (2, 9, 64), (1, 12, 257), (2, 7, 1000), (1, 6, 2049),
                                   (1, 4, 8192)])
def test_filter_counts_matches_oracle(sigma, S, K, D):
    api = fbp_api()
    rng = np.random.default_rng(S * 100 + K + D)
    I0 = 1e4
    counts = rng.poisson(I0 * np.exp(-rng.uniform(0, 3, size=(S, K, D)))).astype(np.float32)
    counts[0, 0, : min(D, 5)] = 0.0                       # below the counting floor
    g = api.Geometry(K, D, D)
    pre = api.Preprocess(flat_value=I0, count_floor=1.0, mu_scale=float(D), blur_sigma=sigma)
    q, _ = api.filter_counts(to_gpu(counts), g, pre)
    p = oracle.preprocess(counts.astype(np.float64), I0, mu_scale=D, floor=1.0, sigma=sigma)
    ref = oracle.filter(p.reshape(S * K, D)).reshape(S, K, D)
    assert_within_dr(to_np(q), ref, 2e-5, f"counts sigma={sigma} {S}x{K}x{D}")


def test_filter_counts_per_bin_flat_field_and_16bit():
    api = fbp_api()
    rng = np.random.default_rng(7)
    K, D = 9, 300
    flat = rng.uniform(5e3, 2e4, size=D).astype(np.float32)
    counts = rng.poisson(flat * np.exp(-rng.uniform(0, 2, size=(K, D)))).astype(np.float32)
    counts[4] = flat                                       # I = I0 everywhere: p = 0 -> zero row
    g = api.Geometry(K, D, D)
    pre = api.Preprocess(flat=to_gpu(flat), mu_scale=128.0, blur_sigma=1.2)
    q, _ = api.filter_counts(to_gpu(counts), g, pre)
    ref = oracle.filter(oracle.preprocess(counts, flat.astype(np.float64), 128.0, 1.0, 1.2))
    assert_within_dr(to_np(q), ref, 2e-5, "per-bin flat")
    assert np.all(to_np(q)[4] == 0.0)
    q16, rs = api.filter_counts(to_gpu(counts), g, pre, dtype=torch.float16)
    deq = to_np(q16) * to_np(rs)[:, None]
    assert np.max(np.abs(deq - ref)) <= 2.0 ** -11 * np.abs(ref).max() + 2e-5 * (ref.max() - ref.min())
    assert to_np(rs)[4] == 1.0


def test_fbp_counts_matches_oracle_and_batched_flat():
    """Counts -> FBP image, noise-free and Poisson, vs the oracle's FP64 chain."""
    api = fbp_api()
    N, K = 128, 180
    g, go = api.Geometry(K, N, N), oracle.Geometry(K, N, N)
    for noise in (False, True):
        counts, _ = counts_for(N, K, 31 if noise else 30, noise=noise)
        pre = api.Preprocess(flat_value=1e4, mu_scale=float(N), blur_sigma=1.0)
        f = to_np(api.fbp_counts(to_gpu(counts), g, pre))
        ref = oracle.fbp(oracle.preprocess(counts, 1e4, N, 1.0, 1.0), go)
        assert_within_dr(f, ref, 1e-4, f"fbp_counts noise={noise}")


@pytest.mark.parametrize("variant", [-1, 0, 5, 7, 8])
@pytest.mark.parametrize("dtype", [torch.float32, torch.float16])
def test_backproject_u16_codes(variant, dtype):
    """Codes equal the FP32 code sequence applied to the same kernel's FP32
    image (bit-exact), and lie within the FBP tolerance of the FP64 oracle's
    codes."""
    api = fbp_api()
    N, K = 256, 360
    g, go = api.Geometry(K, N, N), oracle.Geometry(K, N, N)
    if variant >= 0 and not api.variant_supports(variant, g, dtype):
        pytest.skip("variant not eligible")
    counts, _ = counts_for(N, K, 40)
    win = api.HuWindow(**{k: phantoms.PIPELINE[k] for k in ("mu_water", "mu_air", "hu_min", "hu_max")})
    pre = api.Preprocess(flat_value=1e4, mu_scale=float(N), blur_sigma=phantoms.PIPELINE["blur_sigma"])
    filt, rs = api.filter_counts(to_gpu(counts), g, pre, dtype=dtype)
    f32 = to_np(api.backproject(filt, g, row_scale=rs, variant=variant))
    codes = api.backproject_u16(filt, g, win, row_scale=rs, variant=variant).cpu().numpy().view(np.uint16)
    a, b = api.hu_coefficients(win)
    np.testing.assert_array_equal(codes, oracle.hu_codes_f32(f32, a, b))
    # the library's coefficients are the definition's, rounded once to FP32
    a64, b64 = oracle.hu_affine(win.mu_water, win.mu_air, win.hu_min, win.hu_max)
    assert a == np.float32(a64) and b == np.float32(b64)
    # against the FP64 chain: |code difference| <= a * (tolerance x DR) + 1
    ref = oracle.fbp(oracle.preprocess(counts, 1e4, N, 1.0, phantoms.PIPELINE["blur_sigma"]), go)
    tol = 1e-4 if dtype == torch.float32 else 2e-3
    c64 = oracle.hu_codes(ref, win.mu_water, win.mu_air, win.hu_min, win.hu_max)
    bound = math.ceil(a64 * tol * (ref.max() - ref.min())) + 1
    assert np.max(np.abs(codes.astype(int) - c64.astype(int))) <= bound
    assert codes.min() >= 0 and codes.max() <= 65535


def test_u16_clamps_and_rejects():
    api = fbp_api()
    N, K = 64, 32
    g = api.Geometry(K, N, N)
    q = torch.full((K, N), 0.5, device="cuda")
    # every pixel's value lies in [0, pi/2], so HU = 1000 (mu - 0.5) / 0.5 lies in [-1000, 2142]
    lo = api.backproject_u16(q, g, api.HuWindow(mu_water=0.5, hu_min=1e5, hu_max=1e5 + 1.0))
    hi = api.backproject_u16(q, g, api.HuWindow(mu_water=0.5, hu_min=-1e5, hu_max=-1e5 + 1.0))
    assert np.all(lo.cpu().numpy().view(np.uint16) == 0)
    assert np.all(hi.cpu().numpy().view(np.uint16) == 65535)
    for w in (api.HuWindow(mu_water=0.5, mu_air=0.5), api.HuWindow(mu_water=0.5, hu_min=10.0, hu_max=10.0)):
        with pytest.raises(api.FbpError, match="INVALID_ARG"):
            api.backproject_u16(q, g, w)
    with pytest.raises(api.FbpError, match="INVALID_ARG"):
        api.filter_counts(torch.ones((K, N), device="cuda"), g, api.Preprocess(blur_sigma=4.0))
