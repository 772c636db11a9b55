"""GPU parity for mixed batches of normal and offset scans (Sec. V-A(b)):
fbp_batched_scans in one filter launch and one persistent backprojection
launch, under both work orders.  Each item is bit-identical to the same scan
run alone with the same tile shape (fbp / fbp_offset, variant 0), and within
the FP32 tolerance of the oracle."""
import math

import numpy as np
import pytest

import oracle
from gpu_util import assert_within_dr, fbp_api, needs_gpu, to_gpu, to_np, torch
from paper_2505_13955_gb300 import phantoms

pytestmark = [pytest.mark.gpu, needs_gpu]


def mixed_items(api, specs, seed):
    sinos, scans, raw = [], [], []
    for i, (n, k, offset, fold) in enumerate(specs):
        ell = phantoms.random_ellipses(phantoms.rng_for(seed + i), count_range=(5, 10))
        if offset:
            d, c, ov = 9 * n // 16, n / 16 - 0.5, n / 32
            p = phantoms.sinogram(ell, 2 * k, d, n, angle_step=2 * math.pi / (2 * k), det_center=c)
            g = api.Geometry(2 * k, d, n, angle_step=2 * math.pi / (2 * k), det_center=c)
            scans.append(api.Scan(g, ov, fold))
        else:
            p = phantoms.sinogram(ell, k, n, n)
            scans.append(api.Scan(api.Geometry(k, n, n)))
        raw.append(p)
        sinos.append(to_gpu(p))
    return sinos, scans, raw


SPECS = [(128, 90, True, True), (64, 45, False, False), (96, 60, True, False), (128, 120, False, False),
         (256, 180, True, True), (64, 31, False, False), (160, 100, True, True), (96, 77, False, False)]


@pytest.mark.parametrize("order", ["queue", "group_cyclic"])
def test_mixed_batch_equals_single_scans(order):
    api = fbp_api()
    sinos, scans, raw = mixed_items(api, SPECS, 300)
    outs = api.fbp_batched_scans(sinos, scans, variant=0, order=order)
    assert api.device_status() == 0
    for i, (s, sc) in enumerate(zip(sinos, scans)):
        if sc.overlap:
            ref = api.fbp_offset(s, sc.g, sc.overlap, fold=sc.fold, variant=0)
        else:
            ref = api.fbp(s, sc.g, variant=0)
        assert torch.equal(outs[i], ref), f"item {i} differs from the single-scan path"


@pytest.mark.parametrize("order", ["queue", "group_cyclic"])
@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_mixed_batch_default_equals_single_scans(order, dtype):
    """The default: normal and folded offset items with the orbit symmetry
    (n a multiple of 64 for FP32 rows, 128 for 16-bit rows) run staged units
    and equal fbp_backproject_staged (32 x 32 / 64 x 64 shape) on the item's
    filtered rows; unfolded offset items and the others run the persistent
    kernel's orbit variant 8 / packed 10 or its generic fallback."""
    api = fbp_api()
    sinos, scans, _ = mixed_items(api, SPECS, 350)
    outs = api.fbp_batched_scans(sinos, scans, dtype=dtype, order=order)
    assert api.device_status() == 0
    staged = 0
    for i, (s, sc) in enumerate(zip(sinos, scans)):
        if sc.overlap:
            filt, rs, gv = api.filter_offset(s, sc.g, sc.overlap, sc.fold, dtype=dtype)
        else:
            gv = sc.g
            filt, rs = api.filter(s, gv, dtype=dtype)
        if api.batched_item_staged(gv, dtype):
            staged += 1
            ref = api.backproject_staged(filt, gv, rs, shape=0 if dtype == torch.float32 else 1)
        else:
            v = 8 if dtype == torch.float32 else 10
            if not api.variant_supports(v, gv, dtype):
                v = 0
            ref = api.backproject(filt, gv, row_scale=rs, variant=v)
        assert torch.equal(outs[i], ref), f"item {i}"
    assert staged == 3      # items 0, 3, 4: folded offset scans and a normal scan, n = 128, 128, 256


def test_mixed_batch_matches_oracle():
    api = fbp_api()
    sinos, scans, raw = mixed_items(api, SPECS[:5], 400)
    outs = api.fbp_batched_scans(sinos, scans, order="group_cyclic")
    for i, (p, sc) in enumerate(zip(raw, scans)):
        g = sc.g
        if sc.overlap:
            n_v, c_v, off, w = oracle.offset_virtual(g.n_det, g.det_center, sc.overlap)
            ref = oracle.fbp_weighted(oracle.embed_rows(p, n_v, off),
                                      oracle.Geometry(g.n_angles, n_v, g.n, angle_step=g.angle_step), w)
        else:
            ref = oracle.fbp(p.astype(np.float64), oracle.Geometry(g.n_angles, g.n_det, g.n))
        assert_within_dr(to_np(outs[i]), ref, 1e-4, f"item {i}")


@pytest.mark.parametrize("dtype", [torch.float16, torch.bfloat16])
def test_mixed_batch_16bit_equals_single_scans(dtype):
    api = fbp_api()
    sinos, scans, _ = mixed_items(api, SPECS[:4], 500)
    outs = api.fbp_batched_scans(sinos, scans, dtype=dtype, variant=0)
    for i, (s, sc) in enumerate(zip(sinos, scans)):
        if sc.overlap:
            ref = api.fbp_offset(s, sc.g, sc.overlap, fold=sc.fold, dtype=dtype, variant=0)
        else:
            ref = api.fbp(s, sc.g, dtype=dtype, variant=0)
        assert torch.equal(outs[i], ref), f"item {i}"


def test_group_cyclic_batch_replays_from_a_cuda_graph():
    """The group-cyclic order needs no counter reset: the captured graph holds
    the two launches only, and replays reproduce the eager result."""
    api = fbp_api()
    sinos, scans, _ = mixed_items(api, SPECS, 600)
    for sc in scans:
        gv = api.offset_geometry(sc.g, sc.overlap, sc.fold)[0] if sc.overlap else sc.g
        api.prepare(gv)
    eager = [o.clone() for o in api.fbp_batched_scans(sinos, scans, order="group_cyclic")]
    outs = [torch.zeros_like(o) for o in eager]
    ws = torch.empty(api.batched_scans_workspace_bytes(sinos, outs, scans), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        api.fbp_batched_scans(sinos, scans, order="group_cyclic", outs=outs, workspace=ws)
    for _ in range(2):
        for o in outs:
            o.zero_()
        graph.replay()
        torch.cuda.synchronize()
        for e, o in zip(eager, outs):
            assert torch.equal(e, o)
    assert api.device_status() == 0


def test_mixed_batch_workload_items_sampled():
    """Three items of the mixed benchmark batch (one of each kind at the
    largest size present), through the benchmark's call, against the oracle
    on sampled pixels."""
    api = fbp_api()
    w = phantoms.WORKLOADS["fbp_mixed_batch"]
    specs = [phantoms.scan_spec(w, i) for i in range(w.n_slices)]
    pick = [next(i for i, s in enumerate(specs) if s["offset"] and s["n"] == 4096),
            next(i for i, s in enumerate(specs) if not s["offset"] and s["n"] == 4096),
            next(i for i, s in enumerate(specs) if s["offset"] and s["n"] == 512)]
    sinos, scans, raws = [], [], []
    for i in pick:
        sp = specs[i]
        p = phantoms.scan_sinogram(sp)
        g = api.Geometry(sp["n_angles"], sp["n_det"], sp["n"], angle_step=sp["angle_step"],
                         det_center=sp["det_center"])
        sinos.append(to_gpu(p))
        scans.append(api.Scan(g, sp["overlap"], True))
        raws.append(p)
    outs = api.fbp_batched_scans(sinos, scans, order="group_cyclic")
    rng = np.random.default_rng(8)
    for o, p, sc in zip(outs, raws, scans):
        g = sc.g
        rows = rng.integers(0, g.n, 600)
        cols = rng.integers(0, g.n, 600)
        if sc.overlap:
            n_v, c_v, off, wt = oracle.offset_virtual(g.n_det, g.det_center, sc.overlap)
            q = oracle.filter(oracle.offset_fold(oracle.embed_rows(p, n_v, off), wt))
            go = oracle.Geometry(g.n_angles // 2, n_v, g.n, angle_step=g.angle_step)
        else:
            q = oracle.filter(p.astype(np.float64))
            go = oracle.Geometry(g.n_angles, g.n_det, g.n)
        ref = oracle.backproject_pixels(q, go, rows, cols)
        got = to_np(o)[rows, cols]
        assert_within_dr(got, ref, 1e-4, "mixed workload item")
