"""GPU parity: fbp_filter (K1, shared-memory FFT convolution) vs the FP64
oracle's direct/FFT linear convolution, element by element."""
import numpy as np
import pytest

import oracle
from gpu_util import assert_within_dr, fbp_api, needs_gpu, to_gpu, to_np, torch

pytestmark = [pytest.mark.gpu, needs_gpu]

KINDS = {"ramlak": oracle.RAMLAK, "shepp_logan": oracle.SHEPP_LOGAN}


@pytest.mark.parametrize("kind", ["ramlak", "shepp_logan"])
@pytest.mark.parametrize("S,K,D", [
    (1, 1, 1), (1, 3, 2), (1, 5, 7), (2, 3, 64), (1, 7, 255), (3, 5, 256), (1, 9, 257),
    (1, 4, 300), (1, 5, 512), (2, 33, 1000), (1, 4, 1024), (1, 17, 2048), (1, 6, 2049), (1, 5, 4096),
    (1, 3, 8192)])
def test_filter_f32_matches_oracle(kind, S, K, D):
    """Every transform length, with D = L / 2 at each of them (the one case
    where the difference at n = D falls in the R / 2-th column of step 1)."""
    api = fbp_api()
    rng = np.random.default_rng(S * 1000 + K * 10 + D)
    p = rng.standard_normal((S, K, D)).astype(np.float32) * 50.0
    g = api.Geometry(K, D, D)
    q, rs = api.filter(to_gpu(p), g, kind=kind)
    assert rs is None
    ref = oracle.filter(p.reshape(S * K, D).astype(np.float64), KINDS[kind]).reshape(S, K, D)
    assert_within_dr(to_np(q), ref, 2e-5, f"filter {kind} {S}x{K}x{D}")


@pytest.mark.parametrize("tau", [0.5, 1.7])
def test_filter_detector_spacing_scaling(tau):
    api = fbp_api()
    rng = np.random.default_rng(4)
    p = rng.standard_normal((6, 300)).astype(np.float32)
    g = api.Geometry(6, 300, 300, det_spacing=tau)
    q, _ = api.filter(to_gpu(p), g)
    ref = oracle.filter(p.astype(np.float64), oracle.RAMLAK, tau)
    assert_within_dr(to_np(q), ref, 2e-5, "tau")


def test_filter_phantom_rows_and_zero_rows():
    api = fbp_api()
    from paper_2505_13955_gb300 import phantoms
    p = phantoms.sinogram(phantoms.shepp_logan(), 36, 256, 256)
    p[5] = 0.0
    g = api.Geometry(36, 256, 256)
    q, _ = api.filter(to_gpu(p), g)
    ref = oracle.filter(p.astype(np.float64))
    assert_within_dr(to_np(q), ref, 2e-5, "phantom")
    assert np.all(to_np(q)[5] == 0.0)


@pytest.mark.parametrize("dtype,rel", [(torch.float16, 2.0 ** -11), (torch.bfloat16, 2.0 ** -8)])
@pytest.mark.parametrize("D", [256, 2048, 8192])
def test_filter_16bit_per_row_scale(dtype, rel, D):
    api = fbp_api()
    rng = np.random.default_rng(D)
    K = 9
    p = rng.standard_normal((K, D)).astype(np.float32) * 30
    p[3] = 0.0
    g = api.Geometry(K, D, D)
    q16, rs = api.filter(to_gpu(p), g, dtype=dtype)
    q32, _ = api.filter(to_gpu(p), g)
    assert q16.dtype == dtype and rs.shape == (K,)
    ref = oracle.filter(p.astype(np.float64))
    amax = np.max(np.abs(to_np(q32)), axis=1)
    expect_scale = np.where(amax > 0, amax, 1.0)
    np.testing.assert_allclose(to_np(rs), expect_scale, rtol=0, atol=0)
    deq = to_np(q16) * to_np(rs)[:, None]
    # each stored value is RNE(q/s): error <= s * ulp/2 of the 16-bit type, plus FP32 error
    err = np.abs(deq - ref)
    bound = expect_scale[:, None] * rel + 2e-5 * (ref.max() - ref.min())
    assert np.all(err <= bound)
    # stored values lie in [-1, 1]
    assert float(q16.float().abs().max()) <= 1.0
    # and each is the 16-bit rounding of the correctly rounded FP32 quotient
    # of the FP32 row (same transform arithmetic before the store)
    quot = (to_np(q32) / expect_scale[:, None].astype(np.float32)).astype(np.float32)
    want = torch.from_numpy(quot).to(dtype)
    assert torch.equal(q16.cpu().view(torch.int16), want.view(torch.int16))
    assert np.all(to_np(q16)[3] == 0.0) and to_np(rs)[3] == 1.0


def test_filter_empty_and_noncontiguous_rejected():
    api = fbp_api()
    g = api.Geometry(4, 16, 16)
    out, _ = api.filter(torch.zeros((0, 4, 16), device="cuda"), g)
    assert out.shape == (0, 4, 16)
    x = torch.zeros((16, 4), device="cuda").t()
    with pytest.raises(ValueError):
        api.filter(x, g)
    with pytest.raises(api.FbpError):
        api.filter(torch.zeros((4, 9000), device="cuda"), api.Geometry(4, 9000, 16))


@pytest.mark.parametrize("D,K", [(8192, 6), (2048, 8)])
def test_filter_large_line_integrals_difference_form(D, K):
    """Full-size phantom rows: line integrals reach ~1e4-1e5 (density x
    pixels) while the filtered rows are O(10).  The difference form keeps the
    FP32 transform's error relative to the row differences, so the filtered
    rows match the FP64 oracle to ~1e-7 of their magnitude (the direct
    spectrum would leave ~1e-4)."""
    api = fbp_api()
    from paper_2505_13955_gb300 import phantoms
    w = phantoms.WORKLOADS["fbp_precision_n8192" if D == 8192 else "fbp_stack_n2048"]
    p = phantoms.slice_sinogram(w, 0)[:: max(1, w.n_angles // K)][:K]
    p = np.ascontiguousarray(p)
    assert np.abs(p).max() > 1e4
    g = api.Geometry(K, D, D)
    q, _ = api.filter(to_gpu(p), g)
    ref = oracle.filter(p.astype(np.float64))
    err = np.max(np.abs(to_np(q) - ref)) / np.max(np.abs(ref))
    assert err <= 1e-5, err


@pytest.mark.parametrize("D", [8192, 4096, 3000])
@pytest.mark.parametrize("rows", [1, 7, 610])
def test_streamed_filter_equals_the_plain_kernel(D, rows):
    """At the one-pair-per-block lengths the library streams 16-byte aligned
    rows through the bulk-copy engine (filter_stream_kernel); rows that are
    not 16-byte aligned take the plain kernel.  Both compute the same
    arithmetic in the same order, so the results are bit-identical, and both
    match the oracle."""
    api = fbp_api()
    rng = np.random.default_rng(D + rows)
    p = (rng.standard_normal((rows, D)) * 40).astype(np.float32)
    g = api.Geometry(rows, D, D)
    aligned = to_gpu(p)
    buf = torch.empty(rows * D + 1, device="cuda")
    buf[1:] = aligned.reshape(-1)
    shifted = buf[1:].view(rows, D)                       # 4 bytes past an aligned address
    assert aligned.data_ptr() % 16 == 0 and shifted.data_ptr() % 16 == 4
    q1, _ = api.filter(aligned, g)
    q2, _ = api.filter(shifted, g)
    assert torch.equal(q1, q2)
    assert api.device_status() == 0
    if rows <= 7:
        ref = oracle.filter(p.astype(np.float64))
        assert_within_dr(to_np(q1), ref, 2e-5, "streamed filter")
    for dt in (torch.float16, torch.bfloat16):
        a1, s1 = api.filter(aligned, g, dtype=dt)
        a2, s2 = api.filter(shifted, g, dtype=dt)
        assert torch.equal(a1, a2) and torch.equal(s1, s2)


def test_streamed_filter_wait_runs_out_and_reports(monkeypatch):
    """Failure detection without a fault: with FBP_TEST_STREAM_NO_COPY=1 the
    streamed filter issues no row copy, so each block's capped wait on its
    mbarrier runs out; the kernel records code 6 in the device status word
    and returns.  The context stays usable: the next call is correct."""
    api = fbp_api()
    rng = np.random.default_rng(6)
    p = rng.standard_normal((8, 8192)).astype(np.float32)
    g = api.Geometry(8, 8192, 8192)
    x = to_gpu(p)
    assert api.device_status() == 0
    monkeypatch.setenv("FBP_TEST_STREAM_NO_COPY", "1")
    api.filter(x, g)
    assert api.device_status() == 6
    monkeypatch.delenv("FBP_TEST_STREAM_NO_COPY")
    q, _ = api.filter(x, g)
    assert api.device_status() == 0
    assert_within_dr(to_np(q), oracle.filter(p.astype(np.float64)), 2e-5, "after the timeout")
