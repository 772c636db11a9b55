"""GPU parity: fbp_backproject (K2) and full FBP vs the FP64 oracle,
element by element, on seeded inputs spanning several tiles and ragged
edges; every compiled tile variant; 16-bit staged rows; the bounds-checked
build's device status word."""
import numpy as np
import pytest

import oracle
from gpu_util import assert_within_dr, fbp_api, needs_gpu, to_gpu, to_np, torch
from paper_2505_13955_gb300 import phantoms

pytestmark = [pytest.mark.gpu, needs_gpu]

TOL = 1e-4   # max abs error <= 1e-4 x dynamic range (FP32 path)


GEOMS = [
    dict(K=1, D=1, N=1),
    dict(K=3, D=5, N=2),
    dict(K=7, D=9, N=7),
    dict(K=90, D=64, N=64),
    dict(K=45, D=70, N=65),
    dict(K=36, D=100, N=100),
    dict(K=360, D=256, N=256),
    dict(K=33, D=150, N=130, det_center=70.25),
    dict(K=20, D=120, N=96, pixel_size=0.8),
    dict(K=20, D=90, N=96, pixel_size=1.3, angle_start=0.4),
    dict(K=16, D=300, N=130, pixel_size=2.4),
    dict(K=24, D=40, N=150, pixel_size=0.25, det_center=25.0),
    dict(K=50, D=64, N=64, angle_step=0.13),
]


def make(api, G):
    kw = {k: v for k, v in G.items() if k not in ("K", "D", "N")}
    return api.Geometry(G["K"], G["D"], G["N"], **kw), oracle.Geometry(G["K"], G["D"], G["N"], **kw)


@pytest.mark.parametrize("G", GEOMS, ids=lambda G: "x".join(f"{k}{v}" for k, v in G.items()))
def test_backproject_matches_oracle(G):
    api = fbp_api()
    g, go = make(api, G)
    rng = np.random.default_rng(G["K"] * 7 + G["N"])
    q = rng.standard_normal((G["K"], G["D"])).astype(np.float32)
    f = api.backproject(to_gpu(q), g)
    ref = oracle.backproject(q.astype(np.float64), go)
    assert_within_dr(to_np(f), ref, TOL, str(G))


@pytest.mark.parametrize("variant", range(13))
def test_every_table_variant_matches_oracle(variant):
    api = fbp_api()
    shape = api.bp_variants()[variant]
    assert not shape["texture"]
    if shape["packed16"]:
        pytest.skip("16-bit-only variant: covered by the 16-bit test below")
    if shape["symmetric"]:
        # the standard geometry (angle step pi/K, K even, centred detector,
        # N a multiple of 2 tiles), with D != N and a non-unit pixel size
        G = dict(K=70, D=230, N=256, pixel_size=0.9)
    else:
        G = dict(K=70, D=200, N=190, det_center=101.3)
    g, go = make(api, G)
    assert api.variant_supports(variant, g)
    assert not any(api.variant_supports(v["variant"], g) for v in api.bp_variants() if v["packed16"])
    rng = np.random.default_rng(variant)
    q = rng.standard_normal((2, G["K"], G["D"])).astype(np.float32)
    f = api.backproject(to_gpu(q), g, variant=variant)
    for s in range(2):
        ref = oracle.backproject(q[s].astype(np.float64), go)
        assert_within_dr(to_np(f[s]), ref, TOL, f"variant {variant} slice {s}")


def test_symmetric_variants_refuse_other_geometries():
    api = fbp_api()
    sym = [v["variant"] for v in api.bp_variants() if v["symmetric"]]
    assert sym
    q = torch.zeros((71, 64), device="cuda")
    for g in (api.Geometry(71, 64, 64),                       # odd K
              api.Geometry(70, 64, 64, det_center=30.0),      # off-centre detector
              api.Geometry(70, 64, 96),                       # N not a multiple of 2 tiles
              api.Geometry(70, 64, 64, angle_step=0.04)):     # not pi/K
        for v in sym:
            assert not api.variant_supports(v, g)
            with pytest.raises(api.FbpError, match="UNSUPPORTED"):
                api.backproject(q[: g.n_angles], g, variant=v)
        # the default falls back to a generic variant and stays correct
        go = oracle.Geometry(g.n_angles, g.n_det, g.n, angle_step=g.angle_step, det_center=g.det_center)
        qq = torch.randn((g.n_angles, g.n_det), device="cuda")
        assert_within_dr(to_np(api.backproject(qq, g)), oracle.backproject(to_np(qq), go), TOL, "fallback")


def test_scale_and_accumulate():
    api = fbp_api()
    g, go = make(api, dict(K=30, D=80, N=80))
    rng = np.random.default_rng(1)
    q = rng.standard_normal((30, 80)).astype(np.float32)
    base = rng.standard_normal((80, 80)).astype(np.float32)
    out = to_gpu(base)
    api.backproject(to_gpu(q), g, scale=1.0, out=out, accumulate=True)
    ref = base + oracle.backproject(q.astype(np.float64), go, scale=1.0)
    assert_within_dr(to_np(out), ref, TOL, "accumulate")


def test_constant_rows_give_pi_on_disk():
    api = fbp_api()
    N, K = 129, 64
    g = api.Geometry(K, N, N)
    f = to_np(api.backproject(torch.ones((K, N), device="cuda"), g))
    X = np.arange(N) - 0.5 * (N - 1)
    R = np.hypot(*np.meshgrid(X, X))
    np.testing.assert_allclose(f[R <= 0.5 * (N - 1)], np.pi, rtol=2e-6)


@pytest.mark.parametrize("dtype", [torch.float16, torch.bfloat16])
@pytest.mark.parametrize("variant,tol", [(0, TOL), (-1, 2e-3), (7, 2e-3), (10, 2e-3), (11, 2e-3)])
def test_16bit_rows_match_oracle_on_dequantised_rows(dtype, variant, tol):
    """Generic variants stage 16-bit rows as FP32 tables (FP32 tolerance); the
    symmetric default stages 16-bit tables (the 16-bit staging bound)."""
    api = fbp_api()
    g, go = make(api, dict(K=90, D=128, N=128))
    rng = np.random.default_rng(2)
    q = rng.standard_normal((90, 128)).astype(np.float32)
    q16, rs = api.filter(to_gpu(q), g, dtype=dtype)   # any rows will do: use filtered ones
    f = api.backproject(q16, g, row_scale=rs, variant=variant)
    deq = to_np(q16) * to_np(rs)[:, None]
    ref = oracle.backproject(deq, go)
    assert_within_dr(to_np(f), ref, tol, f"16-bit variant {variant}")


def test_fbp_shepp_logan_n256_vs_oracle_and_phantom():
    """Plain FBP, single slice: N = 256, 360 angles, analytic Shepp-Logan
    sinogram in FP32, Ram-Lak."""
    api = fbp_api()
    ell = phantoms.shepp_logan()
    N, K = 256, 360
    p = phantoms.sinogram(ell, K, N, N)
    g, go = make(api, dict(K=K, D=N, N=N))
    f = to_np(api.fbp(to_gpu(p), g, kind="ramlak"))
    ref = oracle.fbp(p.astype(np.float64), go, oracle.RAMLAK)
    assert_within_dr(f, ref, TOL, "shepp-logan fbp")
    truth = phantoms.image(ell, N)
    d = phantoms.edge_distance(ell, N)
    X = np.arange(N) - 0.5 * (N - 1)
    R = np.hypot(*np.meshgrid(X, X))
    m = (d >= 3) & (R <= 0.45 * N)
    assert np.mean(np.abs(f - truth)[m]) <= 0.01 * (ref.max() - ref.min())


def test_checked_build_reports_no_fault_on_valid_geometries():
    from paper_2505_13955_gb300 import build
    build.build_cuda()
    api = fbp_api()
    assert api.device_status("checked") == 0
    extra = [dict(K=70, D=230, N=256, pixel_size=0.9), dict(K=64, D=300, N=256, pixel_size=2.4),
             dict(K=36, D=40, N=128, pixel_size=0.125)]
    for G in GEOMS[3:] + extra:
        g, go = make(api, G)
        q = torch.randn((G["K"], G["D"]), device="cuda")
        ran = 0
        for v in range(len(api.bp_variants())):
            if api.variant_supports(v, g):
                api.backproject(q, g, variant=v, which="checked")
                ran += 1
        assert ran >= 6
        assert api.device_status("checked") == 0, str(G)
