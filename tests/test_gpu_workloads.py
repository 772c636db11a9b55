"""GPU parity at the workloads' full sizes, in the launch configuration the
benchmark times, on outputs the oracle can compute one by one (sampled
pixels, all angles):

* FBP stack, N = 2048, 1800 angles, Shepp-Logan filter, Poisson 1e4 (2 slices);
* precision, N = 8192, 4096 angles: FP32, FP16 and BF16 staged rows
  (2 slices), the 16-bit forms also against the FP32 GPU image.
"""
import json
import os

import numpy as np
import pytest

import oracle
from gpu_util import fbp_api, needs_gpu, to_gpu, to_np, torch
from paper_2505_13955_gb300 import phantoms

pytestmark = [pytest.mark.gpu, needs_gpu]


def record(key, value):
    """Append a measured error to the JSON file named by FBP_ACCURACY_OUT."""
    path = os.environ.get("FBP_ACCURACY_OUT")
    if not path:
        return
    data = {}
    if os.path.exists(path):
        with open(path) as f:
            data = json.load(f)
    data[key] = value
    with open(path, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)


def sample_pixels(N, n, seed):
    rng = np.random.default_rng(seed)
    rows = rng.integers(0, N, n)
    cols = rng.integers(0, N, n)
    edge = np.array([0, N - 1, N // 2, N // 2 - 1, 1, N - 2])
    rr, cc = np.meshgrid(edge, edge)
    return np.concatenate([rows, rr.ravel()]), np.concatenate([cols, cc.ravel()])


def test_stack_n2048_sampled():
    api = fbp_api()
    w = phantoms.WORKLOADS["fbp_stack_n2048"]
    N, K = 2048, 1800
    sinos = np.stack([phantoms.slice_sinogram(w, i) for i in range(2)])
    g = api.Geometry(K, N, N)
    f = to_np(api.fbp(to_gpu(sinos), g, kind="shepp_logan"))
    go = oracle.Geometry(K, N, N)
    for s in range(2):
        q = oracle.filter(sinos[s].astype(np.float64), oracle.SHEPP_LOGAN)
        rows, cols = sample_pixels(N, 2000, s)
        ref = oracle.backproject_pixels(q, go, rows, cols)
        dr = ref.max() - ref.min()
        err = np.max(np.abs(f[s][rows, cols] - ref)) / dr
        record(f"fbp_stack_n2048/f32/slice{s}", err)
        assert err <= 1e-4


@pytest.fixture(scope="module")
def n8192():
    api = fbp_api()
    w = phantoms.WORKLOADS["fbp_precision_n8192"]
    N, K = 8192, 4096
    sinos = np.stack([phantoms.slice_sinogram(w, i) for i in range(2)])
    go = oracle.Geometry(K, N, N)
    refs = []
    for s in range(2):
        q = oracle.filter(sinos[s].astype(np.float64))
        rows, cols = sample_pixels(N, 1500, 10 + s)
        refs.append((rows, cols, oracle.backproject_pixels(q, go, rows, cols)))
    return api, sinos, refs


def test_precision_n8192_f32_sampled(n8192):
    api, sinos, refs = n8192
    g = api.Geometry(4096, 8192, 8192)
    f = api.fbp(to_gpu(sinos), g)
    for s, (rows, cols, ref) in enumerate(refs):
        got = to_np(f[s][torch.from_numpy(rows).cuda(), torch.from_numpy(cols).cuda()])
        dr = ref.max() - ref.min()
        err = np.max(np.abs(got - ref)) / dr
        record(f"fbp_precision_n8192/f32/slice{s}", err)
        assert err <= 1e-4


@pytest.mark.parametrize("dtype", [torch.float16, torch.bfloat16])
@pytest.mark.parametrize("variant", [-1, 8, 5])
def test_precision_n8192_16bit_sampled(n8192, dtype, variant):
    """16-bit rows with the default (packed symmetric) kernel, the unpacked
    symmetric kernel and the generic kernel (FP32 tables from 16-bit rows)."""
    api, sinos, refs = n8192
    g = api.Geometry(4096, 8192, 8192)
    x = to_gpu(sinos)
    f16 = api.fbp(x, g, dtype=dtype, variant=variant)
    f32 = api.fbp(x, g)
    for s, (rows, cols, ref) in enumerate(refs):
        r, c = torch.from_numpy(rows).cuda(), torch.from_numpy(cols).cuda()
        got = to_np(f16[s][r, c])
        dr = ref.max() - ref.min()
        err = np.max(np.abs(got - ref)) / dr
        full32 = f32[s]
        dr32 = (full32.max() - full32.min()).item()
        e32 = ((f16[s] - full32).abs().max().item()) / dr32
        name = str(dtype).replace("torch.", "")
        record(f"fbp_precision_n8192/{name}/variant{variant}/slice{s}/vs_oracle", err)
        record(f"fbp_precision_n8192/{name}/variant{variant}/slice{s}/vs_f32_gpu", e32)
        assert err <= 2e-3, f"{dtype}: {err:.2e} of DR vs the FP64 oracle"
        assert e32 <= 2e-3, f"{dtype}: {e32:.2e} of DR vs the FP32 GPU image"


@pytest.mark.parametrize("dtype", [torch.float16, torch.bfloat16])
def test_precision_n8192_staged_equals_orbit_kernel(n8192, dtype):
    """The bulk-copy-fed kernel (fbp_backproject_staged, default 64 x 64
    shape) on the full-size workload: bit-identical to the packed orbit
    kernel of the same tile over the whole 8192^2 image, and within the
    16-bit bar of the oracle on the sampled pixels."""
    api, sinos, refs = n8192
    g = api.Geometry(4096, 8192, 8192)
    filt, rs = api.filter(to_gpu(sinos), g, dtype=dtype)
    staged = api.backproject_staged(filt, g, rs, chunk=2)
    orbit = api.backproject(filt, g, row_scale=rs, variant=10)
    assert torch.equal(staged, orbit)
    for s, (rows, cols, ref) in enumerate(refs):
        got = to_np(staged[s][torch.from_numpy(rows).cuda(), torch.from_numpy(cols).cuda()])
        err = np.max(np.abs(got - ref)) / (ref.max() - ref.min())
        record(f"fbp_precision_n8192/{str(dtype).replace('torch.', '')}/staged/slice{s}/vs_oracle", err)
        assert err <= 2e-3
    assert api.device_status() == 0


def test_precision_n8192_staged_f32_sampled(n8192):
    """FP32 rows through fbp_backproject_staged at full size: within the FP32
    bar of the oracle on the sampled pixels and of the orbit kernel's image."""
    api, sinos, refs = n8192
    g = api.Geometry(4096, 8192, 8192)
    filt, _ = api.filter(to_gpu(sinos), g)
    staged = api.backproject_staged(filt, g, chunk=2)
    orbit = api.backproject(filt, g, variant=7)       # the block-staged orbit kernel
    for s, (rows, cols, ref) in enumerate(refs):
        got = to_np(staged[s][torch.from_numpy(rows).cuda(), torch.from_numpy(cols).cuda()])
        err = np.max(np.abs(got - ref)) / (ref.max() - ref.min())
        record(f"fbp_precision_n8192/f32/staged/slice{s}/vs_oracle", err)
        assert err <= 1e-4
        dr = (orbit[s].max() - orbit[s].min()).item()
        assert (staged[s] - orbit[s]).abs().max().item() <= 1e-5 * dr
    assert api.device_status() == 0
