"""The texture-unit backprojection (the measured alternative to staged
tables): its interpolation weight is quantised by the texture unit, so it is
held to the 16-bit staging bar (2e-3 of the dynamic range) rather than the
FP32 one, and its measured error is recorded; it refuses what it cannot
bind as a texture."""
import numpy as np
import pytest

import oracle
from gpu_util import assert_within_dr, fbp_api, needs_gpu, to_gpu, to_np, torch
from paper_2505_13955_gb300 import phantoms
from test_gpu_workloads import record, sample_pixels

pytestmark = [pytest.mark.gpu, needs_gpu]


def texture_variant(api):
    (v,) = [s["variant"] for s in api.bp_variants() if s["texture"]]
    return v


@pytest.mark.parametrize("N,K,D,kw", [(256, 180, 256, {}), (200, 90, 240, dict(det_center=120.25)),
                                      (128, 64, 184, dict(pixel_size=1.3, angle_start=0.3))])
def test_texture_variant_matches_oracle_within_the_16bit_bar(N, K, D, kw):
    api = fbp_api()
    v = texture_variant(api)
    g = api.Geometry(K, D, N, **kw)
    go = oracle.Geometry(K, D, N, **kw)
    assert api.variant_supports(v, g)
    rng = np.random.default_rng(N + K)
    q = rng.standard_normal((2, K, D)).astype(np.float32)
    f = to_np(api.backproject(to_gpu(q), g, variant=v))
    for s in range(2):
        ref = oracle.backproject(q[s].astype(np.float64), go)
        err = assert_within_dr(f[s], ref, 2e-3, f"texture slice {s}")
        record(f"texture/N{N}_K{K}_D{D}/slice{s}", err)


def test_texture_variant_fbp_of_a_phantom():
    api = fbp_api()
    v = texture_variant(api)
    N, K = 256, 360
    p = phantoms.sinogram(phantoms.shepp_logan(), K, N, N)
    g = api.Geometry(K, N, N)
    f = to_np(api.fbp(to_gpu(p), g, variant=v))
    ref = oracle.fbp(p.astype(np.float64), oracle.Geometry(K, N, N))
    err = assert_within_dr(f, ref, 2e-3, "texture FBP")
    record("texture/shepp_logan_n256", err)
    # the table kernel on the same rows meets the FP32 bar
    f32 = to_np(api.fbp(to_gpu(p), g))
    assert_within_dr(f32, ref, 1e-4, "table FBP")


def test_texture_variant_refusals():
    api = fbp_api()
    v = texture_variant(api)
    g = api.Geometry(36, 100, 64)                  # 100 bins: row pitch not a multiple of 32 bytes
    assert not api.variant_supports(v, g)
    with pytest.raises(api.FbpError):
        api.backproject(torch.zeros((36, 100), device="cuda"), g, variant=v)
    g = api.Geometry(36, 64, 64)
    assert not api.variant_supports(v, g, torch.float16)
    q = torch.zeros((36, 64), device="cuda")
    api.prepare(g)
    api.backproject(q, g, variant=v)               # tables exist before capture
    stream = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with pytest.raises(api.FbpError):
        with torch.cuda.graph(graph, stream=stream):
            api.backproject(q, g, variant=v)
    torch.cuda.synchronize()
    with pytest.raises(api.FbpError):              # never in a ragged batch
        api.fbp_batched([q], [g], variant=v)
    assert api.device_status() == 0


def test_texture_variant_full_size_sampled():
    """N = 8192, K = 4096 (the precision workload's geometry), 1 slice,
    sampled pixels against the oracle."""
    api = fbp_api()
    v = texture_variant(api)
    w = phantoms.WORKLOADS["fbp_precision_n8192"]
    sino = phantoms.slice_sinogram(w, 0)
    g = api.Geometry(4096, 8192, 8192)
    f = api.fbp(to_gpu(sino[None]), g, variant=v)
    rows, cols = sample_pixels(8192, 1500, 10)
    q = oracle.filter(sino.astype(np.float64))
    ref = oracle.backproject_pixels(q, oracle.Geometry(4096, 8192, 8192), rows, cols)
    got = to_np(f[0][torch.from_numpy(rows).cuda(), torch.from_numpy(cols).cuda()])
    err = assert_within_dr(got, ref, 2e-3, "texture N=8192")
    record("texture/fbp_precision_n8192/slice0", err)
