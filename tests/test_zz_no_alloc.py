"""fbp_backproject_noalloc, called through the C ABI, against fbp_backproject.

Callers that cannot allocate device memory (a framework owning all of it in a
pool, memory fixed up front, work enqueued inside stream capture) use this
entry point: its angle table lives in a static device array instead of a
cudaMalloc'd cache.  Two calls in a row with different angle counts and
geometries check that each call rebuilds the shared table before reading it.
This file sorts last so that a run stopping at the first failure has already
run every other test.
"""
import ctypes

import numpy as np
import pytest

from gpu_util import assert_within_dr, fbp_api, needs_gpu, to_np, torch

pytestmark = [pytest.mark.gpu, needs_gpu]

TOL = 1e-4   # the FP32 backprojection tolerance used throughout the GPU tests


def call_noalloc(L, q, g, out, scale, accumulate=0):
    gc = g.c()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return L.fbp_backproject_noalloc(ctypes.c_void_p(q.data_ptr()), None, 0,
                                     ctypes.c_void_p(out.data_ptr()), ctypes.byref(gc),
                                     q.shape[0] if q.dim() == 3 else 1, float(scale),
                                     accumulate, stream)


def test_noalloc_matches_fbp_backproject_on_two_calls_in_a_row():
    api = fbp_api()
    L = api.lib()
    cases = [
        (api.Geometry(360, 256, 256), 2),
        (api.Geometry(97, 300, 200, det_center=151.25, angle_start=0.3), 1),
    ]
    gen = torch.Generator(device="cuda").manual_seed(5)
    for g, S in cases:
        q = torch.randn((S, g.n_angles, g.n_det), device="cuda", generator=gen)
        expected = api.backproject(q, g)
        got = torch.full_like(expected, float("nan"))
        st = call_noalloc(L, q, g, got, g.angle_step)
        assert st == 0, L.fbp_last_error_message().decode()
        torch.cuda.synchronize()
        assert_within_dr(to_np(got), to_np(expected), TOL, f"noalloc K={g.n_angles}")


def test_noalloc_rejects_more_angles_than_its_table():
    api = fbp_api()
    L = api.lib()
    g = api.Geometry(16385, 64, 64)
    q = torch.zeros((1, 8, 8), device="cuda")       # never read: rejected first
    out = torch.zeros((64, 64), device="cuda")
    st = call_noalloc(L, q, g, out, 1.0)
    assert st == -2   # FBP_ERR_UNSUPPORTED
    assert "16384" in L.fbp_last_error_message().decode()
