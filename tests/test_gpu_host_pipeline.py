"""fbp_host (the C call that reconstructs a stack held in host memory, with
the copies of one chunk overlapping another chunk's kernels): its slices equal
the device calls' bit for bit -- FP32 and 16-bit rows, counts in and uint16
codes out, chunks that do not divide the stack -- and it refuses device
pointers and short workspaces before enqueueing anything."""
import ctypes

import numpy as np
import pytest

from gpu_util import fbp_api, needs_gpu, torch

pytestmark = [pytest.mark.gpu, needs_gpu]


@pytest.mark.parametrize("dtype", [torch.float32, torch.float16, torch.bfloat16])
@pytest.mark.parametrize("chunk,n_streams", [(2, 3), (3, 2), (7, 1)])
def test_fbp_host_equals_device_fbp(dtype, chunk, n_streams):
    api = fbp_api()
    rng = np.random.default_rng(9)
    S, K, N = 7, 64, 128          # K even: the filter's row pairs never straddle two slices
    host = torch.from_numpy(rng.standard_normal((S, K, N)).astype(np.float32) * 100).pin_memory()
    g = api.Geometry(K, N, N)
    out = api.fbp_host(host, g, dtype=dtype, chunk=chunk, n_streams=n_streams)
    assert not out.is_cuda and out.shape == (S, N, N)
    ref = api.fbp(host.cuda(), g, dtype=dtype).cpu()
    assert torch.equal(out, ref)


def test_fbp_host_counts_to_codes_equals_device_calls():
    api = fbp_api()
    rng = np.random.default_rng(11)
    S, K, N = 5, 90, 96
    counts = torch.from_numpy(rng.poisson(5e3, (S, K, N)).astype(np.float32)).pin_memory()
    g = api.Geometry(K, N, N)
    pre = api.Preprocess(flat_value=1e4, count_floor=1.0, mu_scale=float(N), blur_sigma=1.0)
    win = api.HuWindow(0.5, 0.0, -1000.0, 3000.0)
    out = api.fbp_host(counts, g, pre=pre, window=win, chunk=2, n_streams=2)
    assert out.dtype == torch.int16 and out.shape == (S, N, N)
    filt, _ = api.filter_counts(counts.cuda(), g, pre)
    ref = api.backproject_u16(filt, g, win).cpu()
    assert torch.equal(out, ref)


def test_fbp_host_staged_codes_equal_the_device_path():
    """n >= 1024 with the orbit symmetry: fbp_host takes the staged kernel
    for codes as for FP32 slices, as the device path (fbp_counts) does."""
    api = fbp_api()
    rng = np.random.default_rng(13)
    S, K, N = 3, 90, 1024
    counts = torch.from_numpy(rng.poisson(5e3, (S, K, N)).astype(np.float32)).pin_memory()
    g = api.Geometry(K, N, N)
    pre = api.Preprocess(flat_value=1e4, count_floor=1.0, mu_scale=float(N), blur_sigma=1.0)
    win = api.HuWindow(0.5, 0.0, -1000.0, 3000.0)
    assert api.staged_preferred(g)
    out = api.fbp_host(counts, g, pre=pre, window=win, chunk=2, n_streams=2)
    ref = api.fbp_counts(counts.cuda(), g, pre, window=win).cpu()
    assert torch.equal(out, ref)
    # and again: the pooled internal streams give the same result
    assert torch.equal(api.fbp_host(counts, g, pre=pre, window=win, chunk=1, n_streams=3), ref)


def test_fbp_host_refusals():
    api = fbp_api()
    L = api.lib()
    g = api.Geometry(32, 64, 64)
    gc = g.c()
    host_in = torch.zeros((2, 32, 64)).pin_memory()
    host_out = torch.zeros((2, 64, 64)).pin_memory()
    dev = torch.zeros((2, 32, 64), device="cuda")
    need = api.host_workspace_bytes(g, chunk=1, n_streams=2)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    def call(src, dst, nbytes, n_streams=2):
        return L.fbp_host(ctypes.c_void_p(src.data_ptr()), ctypes.c_void_p(dst.data_ptr()), ctypes.byref(gc), 2,
                          0, 0, -1, None, None, 1, n_streams, ctypes.c_void_p(ws.data_ptr()), nbytes, stream)

    assert call(dev, host_out, need) == -1                     # device pointer as the host input
    assert "host memory" in L.fbp_last_error_message().decode()
    assert call(host_in, host_out, need - 1) == -3             # workspace too small
    assert call(host_in, host_out, need, n_streams=17) == -1   # too many streams
    assert float(host_out.abs().max()) == 0.0
    assert call(host_in, host_out, need) == 0                  # and the valid call runs
