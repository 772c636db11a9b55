"""fbp_backproject_noalloc, called through the C ABI, against fbp_backproject
and the FP64 oracle.

Callers that cannot allocate device memory (a framework owning all of it in a
pool, memory fixed up front) use this entry point: its angle table lives in a
static device array instead of a cudaMalloc'd cache.  Two calls in a row with
different angle counts and geometries check that each call rebuilds the
shared table before reading it; FP16 and BF16 rows take the packed 16-bit
kernel; the free device memory is unchanged across a call for a geometry the
library has never seen; invalid calls are refused before anything runs.
This file sorts last so that a run stopping at the first failure has already
run every other test.
"""
import ctypes

import numpy as np
import pytest

import oracle
from gpu_util import assert_within_dr, fbp_api, needs_gpu, to_np, torch

pytestmark = [pytest.mark.gpu, needs_gpu]

TOL = 1e-4     # the FP32 backprojection tolerance used throughout the GPU tests
TOL16 = 2e-3   # the 16-bit staged-row tolerance
DTYPE_ID = {torch.float32: 0, torch.float16: 1, torch.bfloat16: 2}


def call_noalloc(L, q, g, out, scale, row_scale=None, accumulate=0):
    gc = g.c()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rs = None if row_scale is None else ctypes.c_void_p(row_scale.data_ptr())
    return L.fbp_backproject_noalloc(ctypes.c_void_p(q.data_ptr()), rs, DTYPE_ID[q.dtype],
                                     ctypes.c_void_p(out.data_ptr()), ctypes.byref(gc),
                                     q.shape[0] if q.dim() == 3 else 1, float(scale),
                                     accumulate, stream)


def oracle_bp(q, g):
    go = oracle.Geometry(g.n_angles, g.n_det, g.n, angle_start=g.angle_start, angle_step=g.angle_step,
                         det_center=g.det_center)
    return oracle.backproject(q.astype(np.float64), go)


CASES = [
    (dict(n_angles=360, n_det=256, n=256), 2),
    (dict(n_angles=97, n_det=300, n=200, det_center=151.25, angle_start=0.3), 1),
]


def test_noalloc_matches_fbp_backproject_and_the_oracle_on_two_calls_in_a_row():
    api = fbp_api()
    L = api.lib()
    gen = torch.Generator(device="cuda").manual_seed(5)
    for kw, S in CASES:
        g = api.Geometry(**kw)
        q = torch.randn((S, g.n_angles, g.n_det), device="cuda", generator=gen)
        expected = api.backproject(q, g)
        got = torch.full_like(expected, float("nan"))
        st = call_noalloc(L, q, g, got, g.angle_step)
        assert st == 0, L.fbp_last_error_message().decode()
        torch.cuda.synchronize()
        assert_within_dr(to_np(got), to_np(expected), TOL, f"noalloc vs fbp_backproject K={g.n_angles}")
        qn = to_np(q)
        for s in range(S):
            assert_within_dr(to_np(got[s]), oracle_bp(qn[s], g), TOL, f"noalloc vs oracle K={g.n_angles}")


@pytest.mark.parametrize("dtype", [torch.float16, torch.bfloat16])
def test_noalloc_16bit_rows_with_row_scale(dtype):
    """16-bit rows with their per-row scale (the default packed 16-bit kernel
    of fbp_backproject) on two calls in a row."""
    api = fbp_api()
    L = api.lib()
    gen = torch.Generator(device="cuda").manual_seed(7)
    for kw, S in CASES:
        g = api.Geometry(**kw)
        rows = torch.randn((S, g.n_angles, g.n_det), device="cuda", generator=gen)
        filt, rs = api.filter(rows, g, dtype=dtype)
        expected = api.backproject(filt, g, row_scale=rs)
        got = torch.full_like(expected, float("nan"))
        st = call_noalloc(L, filt, g, got, g.angle_step, row_scale=rs)
        assert st == 0, L.fbp_last_error_message().decode()
        torch.cuda.synchronize()
        assert_within_dr(to_np(got), to_np(expected), TOL16, f"noalloc {dtype} vs fbp_backproject")
        q = to_np(api.filter(rows, g)[0])           # the FP32 filtered rows the 16-bit ones store
        for s in range(S):
            assert_within_dr(to_np(got[s]), oracle_bp(q[s], g), TOL16, f"noalloc {dtype} vs oracle")


def test_noalloc_leaves_free_device_memory_unchanged():
    """A geometry the library has never seen would make fbp_backproject
    allocate its angle table; the no-alloc entry point does not: the free
    device memory is the same before and after the call.  A first call with
    the same kernel shape loads the kernel and looks up the static array."""
    api = fbp_api()
    L = api.lib()
    g0 = api.Geometry(4000, 256, 256)
    g1 = api.Geometry(4002, 256, 256, angle_start=0.0137)     # not seen before, same kernel shape
    q = torch.randn((1, g1.n_angles, g1.n_det), device="cuda")
    out = torch.empty((1, 256, 256), device="cuda")
    assert call_noalloc(L, q[:, :g0.n_angles], g0, out, g0.angle_step) == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    assert call_noalloc(L, q, g1, out, g1.angle_step) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert_within_dr(to_np(out[0]), oracle_bp(to_np(q[0]), g1), TOL, "noalloc new geometry vs oracle")


def test_noalloc_refusals_enqueue_nothing():
    api = fbp_api()
    L = api.lib()
    g = api.Geometry(64, 64, 64)
    # more angles than the static table holds
    big = api.Geometry(16385, 64, 64)
    q = torch.zeros((1, 8, 8), device="cuda")            # never read: rejected first
    out = torch.full((64, 64), 3.0, device="cuda")
    assert call_noalloc(L, q, big, out, 1.0) == -2       # FBP_ERR_UNSUPPORTED
    assert "16384" in L.fbp_last_error_message().decode()
    # 16-bit rows without their row scale
    q16 = torch.zeros((1, 64, 64), dtype=torch.float16, device="cuda")
    assert call_noalloc(L, q16, g, out, 1.0) == -1       # FBP_ERR_INVALID_ARG
    assert "row_scale" in L.fbp_last_error_message().decode()
    # rows and slice overlapping (the slice is written over the rows)
    buf = torch.zeros(64 * 64 * 2, device="cuda")
    rows, alias = buf[:64 * 64].view(1, 64, 64), buf[64 * 32:64 * 96].view(1, 64, 64)
    assert call_noalloc(L, rows, g, alias, 1.0) == -1
    assert "overlaps" in L.fbp_last_error_message().decode()
    torch.cuda.synchronize()
    assert float(out.min()) == float(out.max()) == 3.0  # nothing ran
    assert float(buf.abs().max()) == 0.0
