"""GPU parity: radon_forward (K3) vs the oracle's scatter-form projector; the
adjoint identity between K3 and K2; autograd gradients vs the oracle's FP64
gradient and vs finite differences; least-squares refinement vs the oracle's
FP64 run."""
import math

import numpy as np
import pytest

import oracle
from gpu_util import assert_within_dr, fbp_api, needs_gpu, to_gpu, to_np, torch
from paper_2505_13955_gb300 import phantoms

pytestmark = [pytest.mark.gpu, needs_gpu]

TOL = 1e-4

GEOMS = [
    dict(K=1, D=1, N=1),
    dict(K=4, D=6, N=5),
    dict(K=8, D=8, N=8),
    dict(K=12, D=9, N=9, det_center=4.0),
    dict(K=90, D=64, N=64),
    dict(K=37, D=101, N=100),
    dict(K=33, D=150, N=130, det_center=70.25),
    dict(K=20, D=120, N=96, pixel_size=0.8),
    dict(K=20, D=90, N=96, pixel_size=1.3, angle_start=0.4),
    dict(K=16, D=300, N=130, pixel_size=2.4),
    dict(K=24, D=40, N=150, pixel_size=0.25, det_center=25.0),
]


def make(api, G):
    kw = {k: v for k, v in G.items() if k not in ("K", "D", "N")}
    return api.Geometry(G["K"], G["D"], G["N"], **kw), oracle.Geometry(G["K"], G["D"], G["N"], **kw)


@pytest.mark.parametrize("G", GEOMS, ids=lambda G: "x".join(f"{k}{v}" for k, v in G.items()))
def test_forward_matches_oracle(G):
    api = fbp_api()
    g, go = make(api, G)
    rng = np.random.default_rng(G["N"] + G["K"])
    x = rng.standard_normal((G["N"], G["N"])).astype(np.float32)
    p = api.radon_forward(to_gpu(x), g)
    ref = oracle.forward(x.astype(np.float64), go)
    assert_within_dr(to_np(p), ref, TOL, str(G))


def tile_eligible(G):
    a = G.get("pixel_size", 1.0) / G.get("det_spacing", 1.0)
    return 0.9429 <= a <= 1.0


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4, 5])
@pytest.mark.parametrize("G", GEOMS, ids=lambda G: "x".join(f"{k}{v}" for k, v in G.items()))
def test_forward_variants_match_oracle(variant, G):
    """Every forward kernel (0: gather; 1-3: tile-owned with 8/16/32 bins per
    warp; 4: four slices per block; 5: two slices per block) on every
    geometry, with 7 slices so that the multi-slice variants also run their
    two- and one-slice remainders; the tile-owned forms refuse pixel/bin
    ratios outside [0.9429, 1]."""
    api = fbp_api()
    g, go = make(api, G)
    rng = np.random.default_rng(G["N"] + 7 * G["K"])
    x = rng.standard_normal((7, G["N"], G["N"])).astype(np.float32)
    if variant > 0 and not tile_eligible(G):
        with pytest.raises(api.FbpError, match="UNSUPPORTED"):
            api.radon_forward(to_gpu(x), g, variant=variant)
        return
    p = to_np(api.radon_forward(to_gpu(x), g, variant=variant))
    for s in range(7):
        ref = oracle.forward(x[s].astype(np.float64), go)
        assert_within_dr(p[s], ref, TOL, f"variant {variant} {G}")


def test_forward_variant_out_of_range_rejected():
    api = fbp_api()
    g = api.Geometry(8, 8, 8)
    x = torch.zeros((8, 8), device="cuda")
    for v in (-2, api.forward_variant_count()):
        with pytest.raises(api.FbpError, match="INVALID_ARG"):
            api.radon_forward(x, g, variant=v)


def test_forward_tile_full_size_sampled_angles():
    """The tile-owned projector at the refinement workload's size and launch
    (16 slices, N = 1024, 1800 angles), on FBP images of the workload's
    sinograms: sampled angles (including 0, pi/4, pi/2 and their
    neighbours, where the walk axis switches) against the oracle, and every
    bin against the deterministic gather kernel."""
    api = fbp_api()
    w = phantoms.WORKLOADS["gd_refine_n1024"]
    N, K = 1024, 1800
    g = api.Geometry(K, N, N)
    sinos = np.stack([phantoms.slice_sinogram(w, i) for i in range(16)])
    x = api.fbp(to_gpu(sinos), g)
    p = api.radon_forward(x, g)
    p0 = api.radon_forward(x, g, variant=0)
    dr = (p0.max() - p0.min()).item()
    assert (p - p0).abs().max().item() <= 1e-5 * dr
    for v in range(1, api.forward_variant_count()):
        assert (api.radon_forward(x, g, variant=v) - p0).abs().max().item() <= 1e-5 * dr, v
    pn, xn = to_np(p), to_np(x)
    for s in (0, 15):
        for k in (0, 1, 449, 450, 451, 899, 900, 901, 1349, 1350, 1799):
            go = oracle.Geometry(1, N, N, angle_start=k * (math.pi / K))
            ref = oracle.forward(xn[s].astype(np.float64), go)[0]
            assert np.max(np.abs(pn[s, k] - ref)) <= TOL * dr, (s, k)


def test_forward_multi_slice_and_mass():
    api = fbp_api()
    g, go = make(api, dict(K=30, D=64, N=64))
    rng = np.random.default_rng(0)
    X = np.arange(64) - 31.5
    disk = (np.hypot(*np.meshgrid(X, X)) <= 31.0)
    x = (rng.uniform(size=(3, 64, 64)) * disk).astype(np.float32)
    p = to_np(api.radon_forward(to_gpu(x), g))
    for s in range(3):
        np.testing.assert_allclose(p[s].sum(axis=1), x[s].astype(np.float64).sum(), rtol=1e-5)
        assert_within_dr(p[s], oracle.forward(x[s].astype(np.float64), go), TOL, "slice")


@pytest.mark.parametrize("N,K", [(64, 90), (1024, 1800)])
def test_adjoint_dot_product(N, K):
    api = fbp_api()
    g = api.Geometry(K, N, N)
    gen = torch.Generator(device="cuda").manual_seed(N)
    x = torch.randn((N, N), device="cuda", generator=gen)
    y = torch.randn((K, N), device="cuda", generator=gen)
    ax = api.radon_forward(x, g).double()
    aty = api.backproject(y, g, scale=1.0).double()
    lhs = (ax * y.double()).sum().item()
    rhs = (x.double() * aty).sum().item()
    # the dot products cancel heavily; their natural scale is the
    # Cauchy-Schwarz bound |<Ax, y>| <= ||Ax|| ||y||
    scale = min(ax.norm().item() * y.double().norm().item(),
                x.double().norm().item() * aty.norm().item())
    assert abs(lhs - rhs) <= 1e-6 * scale


def test_autograd_gradient_matches_oracle_fp64():
    api = fbp_api()
    N, K = 64, 90
    g, go = make(api, dict(K=K, D=N, N=N))
    rng = np.random.default_rng(3)
    xt = rng.uniform(size=(N, N))
    b = (oracle.forward(xt, go) + rng.standard_normal((K, N))).astype(np.float32)
    x = rng.uniform(size=(N, N)).astype(np.float32)
    xg = to_gpu(x).requires_grad_(True)
    loss = 0.5 * ((api.radon(xg, g) - to_gpu(b)) ** 2).sum()
    loss.backward()
    ref = oracle.gradient(x.astype(np.float64), b.astype(np.float64), go)
    assert_within_dr(to_np(xg.grad), ref, TOL, "gradient")
    # and the transpose op's gradient is the forward projector
    yg = to_gpu(b).requires_grad_(True)
    (api.radon_t(yg, g) * to_gpu(x)).sum().backward()
    assert_within_dr(to_np(yg.grad), oracle.forward(x.astype(np.float64), go), TOL, "A^T grad")


def test_finite_difference_directional_derivative_n1024():
    """Differentiation workload: N = 1024, 1800 angles, Poisson-noised data."""
    api = fbp_api()
    w = phantoms.WORKLOADS["gd_refine_n1024"]
    b = phantoms.slice_sinogram(w, 0)
    g = api.Geometry(1800, 1024, 1024)
    bg = to_gpu(b)
    x = api.fbp(bg, g)
    gen = torch.Generator(device="cuda").manual_seed(7)
    v = torch.randn(x.shape, device="cuda", generator=gen)
    v /= v.pow(2).mean().sqrt()
    xg = x.clone().requires_grad_(True)
    loss = 0.5 * (api.radon(xg, g) - bg).double().pow(2).sum()
    (grad,) = torch.autograd.grad(loss, xg)
    dd = (grad.double() * v.double()).sum().item()
    eps = 1e-2 * x.pow(2).mean().sqrt().item()

    def L(z):
        r = api.radon_forward(z, g).double() - bg.double()
        return 0.5 * (r * r).sum().item()

    fd = (L(x + eps * v) - L(x - eps * v)) / (2 * eps)
    assert abs(fd - dd) <= 1e-3 * abs(dd)


def test_gradient_at_full_size_sampled_vs_oracle():
    api = fbp_api()
    w = phantoms.WORKLOADS["gd_refine_n1024"]
    b = phantoms.slice_sinogram(w, 1)
    N, K = 1024, 1800
    g, go = make(api, dict(K=K, D=N, N=N))
    x = api.fbp(to_gpu(b), g)
    xg = x.clone().requires_grad_(True)
    (0.5 * (api.radon(xg, g) - to_gpu(b)).pow(2).sum()).backward()
    xn = to_np(x)
    r = oracle.forward(xn, go) - b.astype(np.float64)
    rng = np.random.default_rng(0)
    rows = np.concatenate([rng.integers(0, N, 1500), [0, N - 1, 0, N - 1, 511]])
    cols = np.concatenate([rng.integers(0, N, 1500), [0, 0, N - 1, N - 1, 512]])
    ref = oracle.backproject_pixels(r, go, rows, cols, scale=1.0)
    got = to_np(xg.grad)[rows, cols]
    assert np.max(np.abs(got - ref)) <= TOL * (ref.max() - ref.min())


def test_gd_refinement_matches_oracle():
    api = fbp_api()
    N, K = 64, 90
    g, go = make(api, dict(K=K, D=N, N=N))
    ell = phantoms.random_ellipses(phantoms.rng_for(11), count_range=(5, 8))
    p = phantoms.sinogram(ell, K, N, N, dtype=np.float64)
    b = phantoms.poisson_noise(p, N, 1e4, phantoms.rng_for(12))
    lam = oracle.power_lambda_max(go, iters=20)
    eta = 1.0 / lam
    x0 = oracle.fbp(b.astype(np.float64), go)
    x_ref, loss_ref = oracle.gd_refine(x0, b.astype(np.float64), go, eta, 50)
    x, losses = api.lsq_refine(to_gpu(x0), to_gpu(b), g, eta, 50)
    assert all(l1 <= l0 * (1 + 1e-6) for l0, l1 in zip(losses, losses[1:]))
    np.testing.assert_allclose(losses, loss_ref, rtol=1e-4)
    assert_within_dr(to_np(x), x_ref, TOL, "x_50")
