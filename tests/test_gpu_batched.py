"""GPU parity: fbp_batched (one filter launch + persistent backprojection
launches over a ragged batch) -- bit-identical per item to the same slice run
alone through fbp_filter + fbp_backproject (or fbp_backproject_staged, for
the items the default runs as staged units) with the same shape, within
tolerance of the oracle, and replayable from a captured CUDA graph."""
import numpy as np
import pytest

import oracle
from gpu_util import assert_within_dr, fbp_api, needs_gpu, to_gpu, to_np, torch
from paper_2505_13955_gb300 import phantoms

pytestmark = [pytest.mark.gpu, needs_gpu]


def ragged(api, dims, seed=0):
    sinos, geoms = [], []
    for i, (K, N) in enumerate(dims):
        ell = phantoms.random_ellipses(phantoms.rng_for(seed + i), count_range=(3, 6))
        sinos.append(to_gpu(phantoms.sinogram(ell, K, N, N)))
        geoms.append(api.Geometry(K, N, N))
    return sinos, geoms


DIMS = [(30, 64), (90, 100), (45, 128), (17, 33), (120, 257), (1, 5), (64, 64), (60, 128)]


def item_shape(api, variant, g, dtype=torch.float32):
    """The single-slice variant a batch item runs: a symmetric variant's own
    shape where the item's geometry has the symmetry, else the generic
    variant with the same threads (12 for 128-thread orbits, 0 for 256)."""
    shape = api.bp_variants()[variant]
    if not shape["symmetric"] or api.variant_supports(variant, g, dtype):
        return variant
    return 12 if shape["threads"] == 128 else 0


@pytest.mark.parametrize("variant", [0, 2, 5, 6, 7, 8, 9, 12])
@pytest.mark.parametrize("kind", ["ramlak", "shepp_logan"])
def test_batched_bit_identical_to_single_slices(variant, kind):
    api = fbp_api()
    sinos, geoms = ragged(api, DIMS)
    outs = api.fbp_batched(sinos, geoms, kind=kind, variant=variant)
    torch.cuda.synchronize()
    orbit_items = 0
    for s, g, o in zip(sinos, geoms, outs):
        v = item_shape(api, variant, g)
        orbit_items += api.bp_variants()[v]["symmetric"]
        single = api.fbp(s, g, kind=kind, variant=v)
        assert torch.equal(o, single), f"K={g.n_angles} N={g.n} ran variant {v}"
    if api.bp_variants()[variant]["symmetric"]:
        assert orbit_items >= 1
    assert api.device_status() == 0


def staged_shape(dtype):
    """The fbp_backproject_staged shape of the default's staged batch units:
    32 x 32 orbits for FP32 rows, 64 x 64 for 16-bit rows."""
    return 0 if dtype == torch.float32 else 1


def single_default(api, s, g, kind="ramlak", dtype=torch.float32):
    """The single-slice run a batch item under the default equals: the staged
    kernel's shape where fbp_batched_item_staged accepts the item,
    else the persistent tile kernel's variant (8 for FP32 rows, packed 10
    for 16-bit rows) or its generic fallback."""
    if api.batched_item_staged(g, dtype):
        filt, rs = api.filter(s, g, kind=kind, dtype=dtype)
        return api.backproject_staged(filt, g, rs, shape=staged_shape(dtype)), "staged"
    v = item_shape(api, 8 if dtype == torch.float32 else 10, g, dtype)
    return api.fbp(s, g, kind=kind, dtype=dtype, variant=v), v


@pytest.mark.parametrize("variant", [8, 10, 11])
@pytest.mark.parametrize("dtype", [torch.float16, torch.bfloat16])
def test_batched_16bit_orbits_bit_identical_to_single_slices(variant, dtype):
    """16-bit rows: packed and unpacked orbit units in the persistent kernel
    equal the single-slice kernels of the same shape."""
    api = fbp_api()
    sinos, geoms = ragged(api, DIMS, seed=50)
    outs = api.fbp_batched(sinos, geoms, dtype=dtype, variant=variant)
    torch.cuda.synchronize()
    for s, g, o in zip(sinos, geoms, outs):
        v = item_shape(api, variant, g, dtype)
        single = api.fbp(s, g, dtype=dtype, variant=v)
        assert torch.equal(o, single), f"K={g.n_angles} N={g.n} ran variant {v}"
    assert api.device_status() == 0


@pytest.mark.parametrize("dtype", [torch.float32, torch.float16, torch.bfloat16])
@pytest.mark.parametrize("kind", ["ramlak", "shepp_logan"])
def test_batched_default_bit_identical_to_single_slices(dtype, kind):
    """The default: items with the orbit symmetry (n a multiple of 64 for
    FP32 rows, 128 for 16-bit rows) run staged units and equal
    fbp_backproject_staged with the same shape; the others run the
    persistent tile kernel (orbit variant 8 / packed 10, or its generic
    fallback)."""
    api = fbp_api()
    sinos, geoms = ragged(api, DIMS, seed=70)
    outs = api.fbp_batched(sinos, geoms, kind=kind, dtype=dtype)
    torch.cuda.synchronize()
    ran = []
    for s, g, o in zip(sinos, geoms, outs):
        single, how = single_default(api, s, g, kind, dtype)
        ran.append(how)
        assert torch.equal(o, single), f"K={g.n_angles} N={g.n} ran {how}"
    n_staged = 3 if dtype == torch.float32 else 1          # n = 64, 64, 128 / n = 128
    assert ran.count("staged") == n_staged and len(ran) == 8
    assert api.device_status() == 0


# pixel / bin ratios below and above 1 and detectors narrower and wider than
# the image: windows of the corner orbits reach far past the detector, into
# the padding of the item's table
PADDING_GEOMS = {
    torch.float32: [dict(n_angles=100, n_det=80, n=128, pixel_size=1.3),
                    dict(n_angles=72, n_det=200, n=128, pixel_size=0.7),
                    dict(n_angles=36, n_det=33, n=64, pixel_size=1.45),
                    dict(n_angles=180, n_det=256, n=192)],
    torch.float16: [dict(n_angles=100, n_det=80, n=256, pixel_size=1.05),
                    dict(n_angles=72, n_det=200, n=128, pixel_size=0.7),
                    dict(n_angles=36, n_det=40, n=128, pixel_size=1.08),
                    dict(n_angles=180, n_det=300, n=256)],
}


@pytest.mark.parametrize("dtype", [torch.float32, torch.float16])
def test_batched_staged_padding_bit_identical(dtype):
    api = fbp_api()
    gen = torch.Generator(device="cuda").manual_seed(31)
    geoms = [api.Geometry(**kw) for kw in PADDING_GEOMS[dtype]]
    assert all(api.batched_item_staged(g, dtype) for g in geoms)
    sinos = [torch.randn((g.n_angles, g.n_det), device="cuda", generator=gen) for g in geoms]
    for order in ("queue", "group_cyclic"):
        scans = [api.Scan(g) for g in geoms]
        outs = api.fbp_batched_scans(sinos, scans, dtype=dtype, order=order)
        torch.cuda.synchronize()
        for s, g, o in zip(sinos, geoms, outs):
            single, how = single_default(api, s, g, dtype=dtype)
            assert how == "staged"
            assert torch.equal(o, single), f"{order}: K={g.n_angles} D={g.n_det} N={g.n} alpha={g.pixel_size}"
    assert api.device_status() == 0


def test_batched_packed_needs_16bit_rows_and_wide_windows_fall_back():
    api = fbp_api()
    sinos, geoms = ragged(api, DIMS, seed=70)
    with pytest.raises(api.FbpError, match="UNSUPPORTED"):
        api.fbp_batched(sinos, geoms, variant=10)         # packed: 16-bit rows only
    # a window wider than the staged batch allows (pixel / bin ratio 1.6):
    # the default runs the item in the persistent tile kernel
    g = api.Geometry(64, 128, 128, pixel_size=1.6)
    assert not api.batched_item_staged(g) and api.batched_item_staged(api.Geometry(64, 128, 128))
    s = torch.randn((64, 128), device="cuda")
    out = api.fbp_batched([s], [g])[0]
    assert torch.equal(out, api.fbp(s, g, variant=item_shape(api, 8, g)))


@pytest.mark.parametrize("dtype", [torch.float32, torch.float16, torch.bfloat16])
def test_batched_matches_oracle(dtype):
    api = fbp_api()
    sinos, geoms = ragged(api, DIMS, seed=100)
    outs = api.fbp_batched(sinos, geoms, dtype=dtype)
    tol = 1e-4 if dtype == torch.float32 else 2e-3
    for s, g, o in zip(sinos, geoms, outs):
        go = oracle.Geometry(g.n_angles, g.n_det, g.n)
        ref = oracle.fbp(to_np(s), go)
        assert_within_dr(to_np(o), ref, tol, f"{g.n_angles}x{g.n}")


def test_batched_graph_capture_replay():
    api = fbp_api()
    sinos, geoms = ragged(api, DIMS, seed=200)
    outs = [torch.empty((g.n, g.n), device="cuda") for g in geoms]
    ws = torch.empty(api.batched_workspace_bytes(sinos, outs, geoms), dtype=torch.uint8, device="cuda")
    eager = [o.clone() for o in api.fbp_batched(sinos, geoms, outs=outs, workspace=ws)]
    for o in outs:
        o.zero_()
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        api.fbp_batched(sinos, geoms, outs=outs, workspace=ws)
    for _ in range(2):
        graph.replay()
    torch.cuda.synchronize()
    for a, b in zip(eager, outs):
        assert torch.equal(a, b)


def test_capture_before_tables_exist_is_refused():
    api = fbp_api()
    # a geometry no other test uses, so its tables do not exist yet
    g = api.Geometry(77, 91, 91, angle_start=0.0123)
    x = torch.zeros((91, 91), device="cuda")
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with pytest.raises(api.FbpError, match="UNSUPPORTED"):
        with torch.cuda.graph(graph, stream=stream):
            api.radon_forward(x, g)
    torch.cuda.synchronize()
    api.prepare(g, kind=None)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        y = api.radon_forward(x, g)
    graph.replay()
    torch.cuda.synchronize()
    assert float(y.abs().max()) == 0.0


def test_ragged_workload_sample_vs_oracle():
    """A sample of the ragged workload (N in {512..4096}, K in {720, 1800,
    3600}): items run in one batch; each is checked against the oracle on
    sampled pixels, and bit-identical to its single-slice run."""
    api = fbp_api()
    w = phantoms.WORKLOADS["fbp_ragged_batch"]
    idx = [0, 1, 2, 3, 4, 5]
    sinos, geoms = [], []
    for i in idx:
        n, k, _, _ = phantoms.slice_spec(w, i)
        sinos.append(to_gpu(phantoms.slice_sinogram(w, i)))
        geoms.append(api.Geometry(k, n, n))
    outs = api.fbp_batched(sinos, geoms)
    rng = np.random.default_rng(1)
    for s, g, o in zip(sinos, geoms, outs):
        # every item of this workload has the symmetry with n a multiple of
        # 128: the default runs it as staged orbit units
        assert api.batched_item_staged(g)
        single, how = single_default(api, s, g)
        assert how == "staged" and torch.equal(o, single)
        go = oracle.Geometry(g.n_angles, g.n_det, g.n)
        q = oracle.filter(to_np(s))
        rows = rng.integers(0, g.n, 300)
        cols = rng.integers(0, g.n, 300)
        ref = oracle.backproject_pixels(q, go, rows, cols)
        got = to_np(o)[rows, cols]
        # DR of the oracle's values (the sampled range: a lower bound of the
        # image's, so the check is the stricter one)
        dr = ref.max() - ref.min()
        assert np.max(np.abs(got - ref)) <= 1e-4 * dr
