"""GPU: the default backprojection of small slices, whose angle pairs are
shared among the blocks of a thread-block cluster (one orbit per cluster,
partial sums added in rank order through distributed shared memory).

Checked against the FP64 oracle, against the unsplit variant 7 (the same
per-pair arithmetic on 32 x 32 or 16 x 16 tiles, sums grouped differently:
within a few float ulps of the image), for run-to-run determinism, for independence from
the number of slices in the call, with accumulate, and for uint16 codes
(bit-identical to the quantisation of the FP32 default image)."""
import numpy as np
import pytest

import oracle
from gpu_util import assert_within_dr, fbp_api, needs_gpu, to_np, torch

pytestmark = [pytest.mark.gpu, needs_gpu]

TOL = 1e-4
TOL16 = 2e-3
# (K, N): the config-1 slice and neighbours; all have the orbit symmetry and
# few enough orbits per slice for the split.  (360, 256), (360, 192) and
# (180, 128) take the 16 x 16 orbits (at least 8 blocks per orbit); the
# others the 32 x 32 ones
SMALL = [(360, 256), (64, 128), (720, 512), (90, 192), (360, 192), (180, 128)]


def oracle_bp(q, g):
    go = oracle.Geometry(g.n_angles, g.n_det, g.n)
    return oracle.backproject(q.astype(np.float64), go)


@pytest.mark.parametrize("K,N", SMALL)
def test_split_default_matches_oracle_and_unsplit_kernel(K, N):
    api = fbp_api()
    g = api.Geometry(K, N, N)
    gen = torch.Generator(device="cuda").manual_seed(K + N)
    q = torch.randn((2, K, N), device="cuda", generator=gen)
    got = api.backproject(q, g)                               # default: split (16 x 16 orbits where N is small)
    unsplit = api.backproject(q, g, variant=7)
    torch.cuda.synchronize()
    assert_within_dr(to_np(got), to_np(unsplit), 1e-6, "split vs unsplit v7")
    for s in range(2):
        assert_within_dr(to_np(got[s]), oracle_bp(to_np(q[s]), g), TOL, f"split vs oracle K={K} N={N}")
    assert api.device_status() == 0


def test_split_is_deterministic_and_independent_of_the_slice_count():
    api = fbp_api()
    K, N = 360, 256
    g = api.Geometry(K, N, N)
    q = torch.randn((3, K, N), device="cuda", generator=torch.Generator(device="cuda").manual_seed(3))
    a = api.backproject(q, g)
    b = api.backproject(q, g)
    assert torch.equal(a, b)
    for s in range(3):
        assert torch.equal(api.backproject(q[s], g), a[s])


def test_split_accumulates():
    api = fbp_api()
    K, N = 180, 256
    g = api.Geometry(K, N, N)
    q = torch.randn((K, N), device="cuda", generator=torch.Generator(device="cuda").manual_seed(4))
    base = torch.randn((N, N), device="cuda", generator=torch.Generator(device="cuda").manual_seed(5))
    once = api.backproject(q, g)
    out = base.clone()
    api.backproject(q, g, out=out, accumulate=True)
    torch.cuda.synchronize()
    assert torch.allclose(out, base + once, rtol=0, atol=1e-5 * float(once.abs().max()))


@pytest.mark.parametrize("dtype", [torch.float16, torch.bfloat16])
def test_split_16bit_rows(dtype):
    """16-bit rows: the default packed 64 x 64 orbit, split over clusters."""
    api = fbp_api()
    K, N = 360, 256
    g = api.Geometry(K, N, N)
    rows = torch.randn((K, N), device="cuda", generator=torch.Generator(device="cuda").manual_seed(6))
    filt, rs = api.filter(rows, g, dtype=dtype)
    got = api.backproject(filt, g, row_scale=rs)
    unsplit = api.backproject(filt, g, row_scale=rs, variant=10)
    torch.cuda.synchronize()
    assert_within_dr(to_np(got), to_np(unsplit), 1e-6, "split vs unsplit v10")
    q = to_np(api.filter(rows, g)[0])
    assert_within_dr(to_np(got), oracle_bp(q, g), TOL16, f"{dtype} split vs oracle")


def test_split_codes_equal_the_quantised_default_image():
    api = fbp_api()
    K, N = 360, 256
    g = api.Geometry(K, N, N)
    rows = torch.randn((K, N), device="cuda", generator=torch.Generator(device="cuda").manual_seed(7)) * 50
    filt, _ = api.filter(rows, g)
    win = api.HuWindow(10.0, 0.0, -1000.0, 3000.0)     # mu of a few tens: codes across the window
    codes = api.backproject_u16(filt, g, win)
    f32 = api.backproject(filt, g)
    a, b = api.hu_coefficients(win)
    want = oracle.hu_codes_f32(to_np(f32).astype(np.float32), a, b)
    assert np.array_equal(codes.cpu().numpy().view(np.uint16), want)
