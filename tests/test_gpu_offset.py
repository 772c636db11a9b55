"""GPU parity for offset scans (Sec. V-A(b)): fbp_filter_offset (weight,
embed, fold, filter on the virtual detector) against the oracle's weighted
virtual rows filtered in FP64, and the reconstruction through
fbp_backproject on the virtual geometry against the oracle's weighted
full-turn FBP, element by element; the full-size workload on sampled pixels."""
import math

import numpy as np
import pytest

import oracle
from gpu_util import assert_within_dr, fbp_api, needs_gpu, to_gpu, to_np, torch
from paper_2505_13955_gb300 import phantoms

pytestmark = [pytest.mark.gpu, needs_gpu]


def offset_case(N, D, c, K, seed, S=1):
    ell = [phantoms.random_ellipses(phantoms.rng_for(seed + s), count_range=(6, 12)) for s in range(S)]
    p = np.stack([phantoms.sinogram(e, K, D, N, angle_step=2 * math.pi / K, det_center=c) for e in ell])
    return p


def oracle_rows(p, D, c, delta, fold, kind=oracle.RAMLAK):
    """The oracle's weighted (and folded) virtual rows, filtered in FP64."""
    n_v, c_v, off, w = oracle.offset_virtual(D, c, delta)
    pv = oracle.embed_rows(p.astype(np.float64), n_v, off)
    r = oracle.offset_fold(pv, w) if fold else pv * w
    return oracle.filter(r.reshape(-1, n_v), kind).reshape(r.shape[:-1] + (n_v,)), pv, w, n_v


# (N, D, c, delta, K, S): long side above and below the axis, integer and
# half-integer axes, odd row counts, virtual widths that are not powers of two
CASES = [(128, 80, 15.5, 12.0, 242, 3), (128, 80, 64.5, 10.0, 240, 2), (96, 60, 12.0, 11.5, 200, 1),
         (600, 333, 40.0, 30.0, 402, 1), (256, 200, 198.5, 0.5, 120, 1)]


@pytest.mark.parametrize("fold", [1, 0])
@pytest.mark.parametrize("N,D,c,delta,K,S", CASES)
def test_filter_offset_matches_oracle(N, D, c, delta, K, S, fold):
    api = fbp_api()
    p = offset_case(N, D, c, K, 100 + D, S)
    g = api.Geometry(K, D, N, angle_step=2 * math.pi / K, det_center=c)
    q, rs, gv = api.filter_offset(to_gpu(p), g, delta, fold=bool(fold))
    assert rs is None
    ref, _, _, n_v = oracle_rows(p, D, c, delta, fold)
    assert (gv.n_angles, gv.n_det, gv.det_center) == (K // 2 if fold else K, n_v, 0.5 * (n_v - 1))
    assert tuple(q.shape) == (S, gv.n_angles, n_v)
    assert_within_dr(to_np(q), ref, 2e-5, f"offset filter fold={fold}")


@pytest.mark.parametrize("fold", [1, 0])
@pytest.mark.parametrize("kind", ["ramlak", "shepp_logan"])
def test_fbp_offset_matches_the_weighted_full_turn_oracle(fold, kind):
    api = fbp_api()
    N, D, c, delta, K = 128, 80, 15.5, 12.0, 240
    ko = oracle.RAMLAK if kind == "ramlak" else oracle.SHEPP_LOGAN
    p = offset_case(N, D, c, K, 7, 2)
    g = api.Geometry(K, D, N, angle_step=2 * math.pi / K, det_center=c)
    f = to_np(api.fbp_offset(to_gpu(p), g, delta, fold=bool(fold), kind=kind))
    n_v, c_v, off, w = oracle.offset_virtual(D, c, delta)
    gv = oracle.Geometry(K, n_v, N, angle_step=2 * math.pi / K)
    for s in range(2):
        ref = oracle.fbp_weighted(oracle.embed_rows(p[s], n_v, off), gv, w, ko)
        assert_within_dr(f[s], ref, 1e-4, f"offset FBP fold={fold} {kind} slice {s}")


def test_folded_rows_run_the_symmetric_kernels():
    """K/2 even, a centred virtual detector, N a multiple of twice the tile:
    the folded geometry qualifies for the 90-degree orbit kernels, and every
    kernel that accepts it gives the oracle's image."""
    api = fbp_api()
    N, D, c, delta, K = 256, 160, 31.5, 20.0, 360
    p = offset_case(N, D, c, K, 31)
    g = api.Geometry(K, D, N, angle_step=2 * math.pi / K, det_center=c)
    q, _, gv = api.filter_offset(to_gpu(p), g, delta)
    syms = [v["variant"] for v in api.bp_variants() if v["symmetric"] and not v["packed16"]]
    assert any(api.variant_supports(v, gv) for v in syms)
    n_v, c_v, off, w = oracle.offset_virtual(D, c, delta)
    ref = oracle.fbp_weighted(oracle.embed_rows(p[0], n_v, off),
                              oracle.Geometry(K, n_v, N, angle_step=2 * math.pi / K), w)
    for v in api.bp_variants():
        if api.variant_supports(v["variant"], gv) and not v["texture"]:
            f = to_np(api.backproject(q, gv, variant=v["variant"]))
            assert_within_dr(f[0], ref, 1e-4, f"variant {v['variant']}")


@pytest.mark.parametrize("dtype", [torch.float16, torch.bfloat16])
def test_offset_16bit_rows(dtype):
    api = fbp_api()
    N, D, c, delta, K = 256, 160, 31.5, 20.0, 360
    p = offset_case(N, D, c, K, 41)
    g = api.Geometry(K, D, N, angle_step=2 * math.pi / K, det_center=c)
    f = to_np(api.fbp_offset(to_gpu(p), g, delta, dtype=dtype))
    n_v, c_v, off, w = oracle.offset_virtual(D, c, delta)
    ref = oracle.fbp_weighted(oracle.embed_rows(p[0], n_v, off),
                              oracle.Geometry(K, n_v, N, angle_step=2 * math.pi / K), w)
    assert_within_dr(f[0], ref, 2e-3, f"offset FBP {dtype}")


def test_offset_reconstruction_of_the_wide_field():
    """A phantom wider than the detector's own half-width: the offset FBP
    equals the half-turn FBP of a centred detector spanning the whole field
    (the oracle's, from analytic rows of that wider detector)."""
    api = fbp_api()
    N, D, c, delta, K = 256, 160, 31.5, 20.0, 720
    ell = phantoms.random_ellipses(phantoms.rng_for(57))
    p = phantoms.sinogram(ell, K, D, N, angle_step=2 * math.pi / K, det_center=c)
    g = api.Geometry(K, D, N, angle_step=2 * math.pi / K, det_center=c)
    f = to_np(api.fbp_offset(to_gpu(p), g, delta))
    n_v = oracle.offset_virtual(D, c, delta)[0]
    ref = oracle.fbp(phantoms.sinogram(ell, K // 2, n_v, N, dtype=np.float64), oracle.Geometry(K // 2, n_v, N))
    assert_within_dr(f, ref, 1e-4, "offset vs centred wide detector")


@pytest.fixture(scope="module")
def offset_n8192():
    w = phantoms.WORKLOADS["fbp_offset_n8192"]
    D, c, delta = w.offset
    sino = phantoms.slice_sinogram(w, 0)
    n_v, c_v, off, wt = oracle.offset_virtual(D, c, delta)
    r = oracle.offset_fold(oracle.embed_rows(sino.astype(np.float64), n_v, off), wt)
    q = oracle.filter(r)
    go = oracle.Geometry(w.n_angles // 2, n_v, w.n, angle_step=2 * math.pi / w.n_angles)
    rng = np.random.default_rng(71)
    rows = np.concatenate([rng.integers(0, w.n, 1000), [0, w.n - 1, w.n // 2, 0, w.n - 1]])
    cols = np.concatenate([rng.integers(0, w.n, 1000), [0, w.n - 1, w.n // 2, w.n - 1, 0]])
    return w, sino, rows, cols, oracle.backproject_pixels(q, go, rows, cols)


@pytest.mark.parametrize("dtype,tol", [(torch.float32, 1e-4), (torch.float16, 2e-3), (torch.bfloat16, 2e-3)])
def test_offset_n8192_sampled(offset_n8192, dtype, tol):
    """Full size, in the benchmark's launch configuration (fold, default kernel)."""
    api = fbp_api()
    w, sino, rows, cols, ref = offset_n8192
    D, c, delta = w.offset
    g = api.Geometry(w.n_angles, D, w.n, angle_step=2 * math.pi / w.n_angles, det_center=c)
    f = api.fbp_offset(to_gpu(sino[None]), g, delta, dtype=dtype)
    got = to_np(f[0][torch.from_numpy(rows).cuda(), torch.from_numpy(cols).cuda()])
    assert_within_dr(got, ref, tol, f"offset N=8192 {dtype}")
