"""GPU parity of fbp_backproject_staged (16-bit rows; the backprojection
tables written once per slice and moved into shared memory by bulk-tensor
copies): bit-identical to the packed orbit kernel with the same tile (10 for
the 64 x 64 shapes, 11 for the 32 x 32 ones) on every shape, several
geometries, a workspace smaller than the stack and accumulation; within the
16-bit bar of the FP64 oracle; refusals before anything runs."""
import ctypes

import numpy as np
import pytest

import oracle
from gpu_util import assert_within_dr, fbp_api, needs_gpu, to_np, torch

pytestmark = [pytest.mark.gpu, needs_gpu]

GEOMS = [dict(K=64, D=128, N=128), dict(K=90, D=230, N=256, pixel_size=0.9), dict(K=36, D=64, N=128, pixel_size=1.7)]


def orbit_variant(shape):
    return 10 if shape in (0, 1) else 11


def rows_for(api, G, S, dtype, seed):
    g = api.Geometry(G["K"], G["D"], G["N"], pixel_size=G.get("pixel_size", 1.0))
    gen = torch.Generator(device="cuda").manual_seed(seed)
    x = torch.randn((S, G["K"], G["D"]), device="cuda", generator=gen) * 50
    filt, rs = api.filter(x, g, dtype=dtype)
    return g, x, filt, rs


@pytest.mark.parametrize("dtype", [torch.float16, torch.bfloat16])
@pytest.mark.parametrize("shape", range(6))
def test_staged_bit_identical_to_orbit_kernel(dtype, shape):
    api = fbp_api()
    for i, G in enumerate(GEOMS):
        g, x, filt, rs = rows_for(api, G, 3, dtype, 10 * shape + i)
        ref = api.backproject(filt, g, row_scale=rs, variant=orbit_variant(shape))
        got = api.backproject_staged(filt, g, rs, shape=shape, chunk=2)     # two passes through the workspace
        assert torch.equal(got, ref), f"shape {shape} {G}"
        # accumulate onto an image already there
        acc = torch.ones_like(ref)
        api.backproject_staged(filt, g, rs, out=acc, accumulate=True, shape=shape, chunk=3)
        ref2 = torch.ones_like(ref)
        api.backproject(filt, g, row_scale=rs, out=ref2, accumulate=True, variant=orbit_variant(shape))
        assert torch.equal(acc, ref2)
    assert api.device_status() == 0


@pytest.mark.parametrize("dtype", [torch.float16, torch.bfloat16])
def test_staged_matches_oracle(dtype):
    api = fbp_api()
    G = GEOMS[1]
    g, x, filt, rs = rows_for(api, G, 2, dtype, 77)
    q = to_np(api.filter(x, g)[0])
    got = api.backproject_staged(filt, g, rs)
    go = oracle.Geometry(G["K"], G["D"], G["N"], pixel_size=G["pixel_size"])
    for s in range(2):
        assert_within_dr(to_np(got[s]), oracle.backproject(q[s], go), 2e-3, f"staged {dtype} slice {s}")


def test_staged_refusals():
    api = fbp_api()
    g = api.Geometry(64, 128, 128)
    x = torch.randn((1, 64, 128), device="cuda")
    f16, rs = api.filter(x, g, dtype=torch.float16)
    f32, _ = api.filter(x, g)
    out = torch.full((1, 128, 128), 5.0, device="cuda")
    # FP32 rows: the C call refuses them (the binding checks the dtype first)
    L = api.lib()
    ws = torch.empty(api.backproject_staged_workspace_bytes(g, torch.float16), dtype=torch.uint8, device="cuda")
    gc = g.c()
    # 16-bit rows without their row scale
    st = L.fbp_backproject_staged(ctypes.c_void_p(f16.data_ptr()), None, 1, ctypes.c_void_p(out.data_ptr()),
                                  ctypes.byref(gc), 1, 1.0, 0, -1, ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                  None)
    assert st == -1                                   # FBP_ERR_INVALID_ARG
    with pytest.raises(ValueError):
        api.backproject_staged(f16, g)
    odd = api.Geometry(63, 128, 128)                  # K odd: no 90-degree pairs
    with pytest.raises(api.FbpError, match="UNSUPPORTED"):
        f, r = api.filter(torch.zeros((1, 63, 128), device="cuda"), odd, dtype=torch.float16)
        api.backproject_staged(f, odd, r)
    small = torch.empty(api.backproject_staged_workspace_bytes(g, torch.float16) - 16, dtype=torch.uint8,
                        device="cuda")
    with pytest.raises(api.FbpError, match="WORKSPACE"):
        api.backproject_staged(f16, g, rs, out=out, workspace=small)
    torch.cuda.synchronize()
    assert float(out.min()) == float(out.max()) == 5.0


@pytest.mark.parametrize("shape", range(4))
def test_staged_f32_matches_oracle_and_orbit_kernel(shape):
    """FP32 rows: midpoint/slope entries; within the FP32 bar of the oracle
    and within FP32 rounding of the orbit kernel of the same tile."""
    api = fbp_api()
    tile64 = shape == 3
    for i, G in enumerate(GEOMS):
        g, x, filt, _ = rows_for(api, G, 3, torch.float32, 100 + 10 * shape + i)
        got = api.backproject_staged(filt, g, shape=shape, chunk=2)
        ref_gpu = api.backproject(filt, g, variant=8 if tile64 else 7)
        assert_within_dr(to_np(got), to_np(ref_gpu), 1e-5, f"FP32 staged shape {shape} vs orbit {G}")
        go = oracle.Geometry(G["K"], G["D"], G["N"], pixel_size=G.get("pixel_size", 1.0))
        q = to_np(filt)
        for s in range(3):
            assert_within_dr(to_np(got[s]), oracle.backproject(q[s], go), 1e-4, f"FP32 staged {G} slice {s}")
        acc = torch.ones_like(got)
        api.backproject_staged(filt, g, out=acc, accumulate=True, shape=shape)
        assert torch.allclose(acc, got + 1.0, rtol=0, atol=1e-5 * float(got.abs().max()))
    assert api.device_status() == 0


@pytest.mark.parametrize("dtype", [torch.float32, torch.float16])
def test_staged_u16_codes_equal_the_fp32_sequence_on_the_staged_image(dtype):
    """The code epilogue takes the staged image's FP32 value through
    RN(RN(a mu) + b), rounds to nearest even and clamps: applied in numpy
    float32 to fbp_backproject_staged's FP32 image it gives the same codes
    bit for bit."""
    api = fbp_api()
    G = GEOMS[1]
    g, x, filt, rs = rows_for(api, G, 2, dtype, 55)
    win = api.HuWindow(0.5, 0.0, -1000.0, 3000.0)
    a, b = api.hu_coefficients(win)
    mu = api.backproject_staged(filt, g, rs)
    codes = api.backproject_staged_u16(filt, g, win, row_scale=rs, chunk=1)
    want = oracle.hu_codes_f32(mu.cpu().numpy(), np.float32(a), np.float32(b))
    assert np.array_equal(codes.cpu().numpy().view(np.uint16), want)
    assert api.device_status() == 0


def test_staged_offset_scan_matches_the_orbit_path():
    """A folded full-turn offset scan is a centred half turn: fbp_offset takes
    the staged path (n >= 1024) and agrees with the orbit kernel's image to
    FP32 rounding."""
    import math
    api = fbp_api()
    from paper_2505_13955_gb300 import phantoms
    n, k = 1024, 360
    d, c, ov = 9 * n // 16, n / 16 - 0.5, n / 32
    ell = phantoms.random_ellipses(phantoms.rng_for(3), count_range=(5, 10))
    p = phantoms.sinogram(ell, 2 * k, d, n, angle_step=2 * math.pi / (2 * k), det_center=c)
    g = api.Geometry(2 * k, d, n, angle_step=2 * math.pi / (2 * k), det_center=c)
    x = torch.from_numpy(p).cuda()
    staged = api.fbp_offset(x, g, ov, fold=True)
    gv, _ = api.offset_geometry(g, ov, True)
    assert api.staged_preferred(gv)
    orbit = api.fbp_offset(x, g, ov, fold=True, variant=7)
    dr = (orbit.max() - orbit.min()).item()
    assert (staged - orbit).abs().max().item() <= 1e-5 * dr
