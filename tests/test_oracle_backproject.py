"""Pins for the oracle's backprojection and matched forward projector (CPU).

The paper's backprojection is the O(N_p N_x N_y) sum of Sec. V-A(c) stage 2;
it prints no formula, so the oracle follows the textbook discrete sum
(Kak & Slaney ch. 3) with linear interpolation.  These tests pin it to facts
that do not come from the oracle's own code:

* numpy's ``interp`` (a library routine) reproduces the sum on random rows;
* backprojecting a constant row gives dtheta * K = pi on the inscribed disk;
* the forward projector (scatter form) and the backprojector (gather form)
  are transposes of each other, entry by entry, on brute-force dense matrices
  -- including angles 0, pi/4, pi/2 and detector coordinates near integers;
* projector column sums are 1 and the projector preserves mass;
* rotating the image by 90 degrees shifts the angles by K/2 (and mirrors the
  detector for the wrapped half);
* FBP of a centred unit disk converges to 1 at the centre as the disk grows;
* FBP of the Shepp-Logan phantom approaches the analytic phantom as N grows.
"""
import numpy as np
import pytest

import oracle
from oracle import Geometry
from paper_2505_13955_gb300 import phantoms


def np_backproject(q, g: Geometry, scale):
    """The backprojection sum written with numpy.interp on zero-padded rows."""
    N, K, D = g.n, g.n_angles, g.n_det
    X = np.arange(N) - 0.5 * (N - 1)
    Xg, Yg = np.meshgrid(X, X)  # Xg[r, c] = X(c), Yg[r, c] = Y(r)
    alpha = g.pixel_size / g.det_spacing
    f = np.zeros((N, N))
    xp = np.arange(-1, D + 1)
    for k in range(K):
        th = g.angle_start + k * g.angle_step
        u = alpha * (Xg * np.cos(th) + Yg * np.sin(th)) + g.det_center
        fp = np.concatenate([[0.0], q[k], [0.0]])
        f += np.interp(u, xp, fp, left=0.0, right=0.0)
    return scale * f


@pytest.mark.parametrize("N,D,K,extra", [
    (8, 8, 5, {}),
    (9, 13, 7, {"det_center": 5.3}),
    (16, 12, 6, {"pixel_size": 0.8, "det_spacing": 1.1, "angle_start": 0.3}),
    (12, 12, 4, {"angle_step": 0.7}),
])
def test_backprojection_equals_numpy_interp(N, D, K, extra):
    g = Geometry(K, D, N, **extra)
    rng = np.random.default_rng(N * 100 + K)
    q = rng.standard_normal((K, D))
    np.testing.assert_allclose(oracle.backproject(q, g, 0.37), np_backproject(q, g, 0.37),
                               rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("N,K", [(16, 8), (17, 9), (64, 90)])
def test_backprojection_of_constant_is_pi_on_disk(N, K):
    g = Geometry(K, N, N)
    f = oracle.backproject(np.ones((K, N)), g)
    X = np.arange(N) - 0.5 * (N - 1)
    R = np.hypot(*np.meshgrid(X, X))
    inside = R <= 0.5 * (N - 1)
    np.testing.assert_allclose(f[inside], np.pi, rtol=1e-13)
    # and strictly less where some angle leaves the detector
    assert np.all(f[R > 0.5 * (N - 1) + 1.0] < np.pi)


@pytest.mark.parametrize("pixel_size,det_spacing", [(0.75, 1.5), (1.5, 1.0), (1.0, 1.25)])
def test_backprojection_of_constant_scales_with_pixel_over_bin_size(pixel_size, det_spacing):
    """u = alpha (X cos + Y sin) + c_d with alpha = pixel_size / det_spacing:
    a constant row of D bins covers a pixel at radius R at every angle when
    alpha R <= (D - 1)/2 (value pi), and misses it at the angles where
    |alpha R cos(theta - phi)| > (D + 1)/2, which exist once alpha R > (D + 1)/2
    (value below pi)."""
    N, D, K = 32, 16, 12
    alpha = pixel_size / det_spacing
    g = Geometry(K, D, N, pixel_size=pixel_size, det_spacing=det_spacing)
    f = oracle.backproject(np.ones((K, D)), g)
    X = np.arange(N) - 0.5 * (N - 1)
    R = np.hypot(*np.meshgrid(X, X))
    inside, outside = alpha * R <= 0.5 * (D - 1), alpha * R > 0.5 * (D + 1) + 0.5
    assert inside.sum() > 20 and outside.sum() > 20
    np.testing.assert_allclose(f[inside], np.pi, rtol=1e-13)
    assert np.all(f[outside] < np.pi - 0.1)


def dense_forward(g: Geometry) -> np.ndarray:
    N = g.n
    A = np.empty((g.n_angles * g.n_det, N * N))
    for i in range(N * N):
        e = np.zeros(N * N)
        e[i] = 1.0
        A[:, i] = oracle.forward(e.reshape(N, N), g).ravel()
    return A


def dense_backproject(g: Geometry) -> np.ndarray:
    KD = g.n_angles * g.n_det
    B = np.empty((g.n * g.n, KD))
    for i in range(KD):
        e = np.zeros(KD)
        e[i] = 1.0
        B[:, i] = oracle.backproject(e.reshape(g.n_angles, g.n_det), g, 1.0).ravel()
    return B


@pytest.mark.parametrize("N,D,K,extra", [
    (4, 4, 1, {}),
    (5, 6, 4, {}),                        # includes theta = 0, pi/4, pi/2
    (8, 8, 8, {}),
    (9, 9, 12, {"det_center": 4.0}),      # integer centre: u hits integers exactly
    (16, 12, 6, {"pixel_size": 0.5}),     # half-integer u values
    (10, 14, 7, {"angle_start": 0.1, "det_center": 6.2}),
])
def test_backprojection_is_exact_transpose_of_forward(N, D, K, extra):
    g = Geometry(K, D, N, **extra)
    A = dense_forward(g)
    B = dense_backproject(g)
    np.testing.assert_allclose(B, A.T, rtol=0, atol=1e-13)
    # adjoint identity on random vectors
    rng = np.random.default_rng(K)
    x = rng.standard_normal((N, N))
    y = rng.standard_normal((K, D))
    lhs = np.sum(oracle.forward(x, g) * y)
    rhs = np.sum(x * oracle.backproject(y, g, 1.0))
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_forward_column_sums_and_mass():
    N, K = 24, 10
    g = Geometry(K, N, N)
    X = np.arange(N) - 0.5 * (N - 1)
    Xg, Yg = np.meshgrid(X, X)
    R = np.hypot(Xg, Yg)
    # every pixel whose u stays inside [0, D-1] puts total weight 1 in each row
    for (r, c) in [(0, 0), (12, 3), (5, 17), (11, 11)]:
        e = np.zeros((N, N))
        e[r, c] = 1.0
        p = oracle.forward(e, g)
        if R[r, c] <= 0.5 * (N - 1):
            np.testing.assert_allclose(p.sum(axis=1), 1.0, rtol=1e-13)
    rng = np.random.default_rng(0)
    f = rng.uniform(size=(N, N)) * (R <= 0.5 * (N - 1))
    p = oracle.forward(f, g)
    np.testing.assert_allclose(p.sum(axis=1), f.sum(), rtol=1e-12)


@pytest.mark.parametrize("N,K", [(12, 8), (15, 12)])
def test_rotation_by_90_degrees_shifts_angles(N, K):
    g = Geometry(K, N, N)
    rng = np.random.default_rng(N)
    f = rng.standard_normal((N, N))
    # rotate the image by +90 degrees about its centre: (X, Y) -> (-Y, X)
    # i.e. f_rot[r'][c'] = f[r][c] with c' = N-1-r, r' = c
    f_rot = np.empty_like(f)
    for r in range(N):
        for c in range(N):
            f_rot[c, N - 1 - r] = f[r, c]
    p = oracle.forward(f, g)
    p_rot = oracle.forward(f_rot, g)
    h = K // 2
    # angle k + K/2 of the rotated image sees what angle k saw
    np.testing.assert_allclose(p_rot[h:], p[:K - h], rtol=1e-10, atol=1e-10)
    # angles k < K/2 of the rotated image see angle k + K/2 - pi, i.e. mirrored
    np.testing.assert_allclose(p_rot[:h], p[K - h:, ::-1], rtol=1e-10, atol=1e-10)


@pytest.mark.parametrize("kind", [oracle.RAMLAK, oracle.SHEPP_LOGAN])
def test_disk_fbp_centre_converges_to_density(kind):
    errs = []
    for R in (32, 64, 128):
        D = 2 * R + 41  # odd, so a pixel sits on the axis at c_d
        s = np.arange(D) - 0.5 * (D - 1)
        p = 2.0 * np.sqrt(np.maximum(R * R - s * s, 0.0))
        q = oracle.filter(p[None, :], kind)[0]
        # every angle sees the same row, so f(0, 0) = dtheta * K * q[c_d] = pi q[c_d]
        errs.append(abs(np.pi * q[(D - 1) // 2] - 1.0))
        # and the full backprojection agrees with that 1-D sum at the centre
        if R == 32:
            K = 16
            g = Geometry(K, D, D)
            f = oracle.backproject(np.tile(q, (K, 1)), g)
            assert f[(D - 1) // 2, (D - 1) // 2] == pytest.approx(np.pi * q[(D - 1) // 2], rel=1e-13)
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 5e-3


def interior_mask(ell, N, margin=3.0, radius_frac=0.9):
    d = phantoms.edge_distance(ell, N)
    X = np.arange(N) - 0.5 * (N - 1)
    R = np.hypot(*np.meshgrid(X, X))
    return (d >= margin) & (R <= radius_frac * 0.5 * N)


def test_shepp_logan_fbp_approaches_analytic_phantom():
    ell = phantoms.shepp_logan()
    errs = []
    for N in (128, 256, 512):
        K = int(round(360 * N / 256))
        p = phantoms.sinogram(ell, K, N, N, dtype=np.float64)
        f = oracle.fbp(p, Geometry(K, N, N), oracle.RAMLAK)
        truth = phantoms.image(ell, N)
        m = interior_mask(ell, N)
        dr = f.max() - f.min()
        err = np.mean(np.abs(f - truth)[m]) / dr
        errs.append(err)
    assert errs[0] > errs[1] > errs[2]
    assert errs[-1] <= 0.01


def test_random_ellipses_fbp_close_to_phantom():
    rng = phantoms.rng_for(7)
    ell = phantoms.random_ellipses(rng, count_range=(5, 8), semi_axis_range=(0.1, 0.3))
    N, K = 256, 400
    p = phantoms.sinogram(ell, K, N, N, dtype=np.float64)
    f = oracle.fbp(p, Geometry(K, N, N), oracle.SHEPP_LOGAN)
    truth = phantoms.image(ell, N)
    m = interior_mask(ell, N)
    dr = f.max() - f.min()
    assert np.mean(np.abs(f - truth)[m]) / dr <= 0.01


def test_backproject_pixels_matches_full():
    g = Geometry(30, 40, 33, det_center=18.7)
    rng = np.random.default_rng(5)
    q = rng.standard_normal((30, 40))
    full = oracle.backproject(q, g)
    rows = rng.integers(0, 33, 50)
    cols = rng.integers(0, 33, 50)
    np.testing.assert_array_equal(oracle.backproject_pixels(q, g, rows, cols), full[rows, cols])


def test_gd_decreases_loss_and_matches_gradient_fd():
    N, K = 16, 12
    g = Geometry(K, N, N)
    rng = np.random.default_rng(11)
    x_true = rng.uniform(size=(N, N))
    b = oracle.forward(x_true, g) + 0.01 * rng.standard_normal((K, N))
    lam = oracle.power_lambda_max(g, iters=50)
    # lambda_max bounds the Rayleigh quotient of random vectors
    for _ in range(3):
        v = rng.standard_normal((N, N))
        assert np.sum(oracle.forward(v, g) ** 2) <= lam * np.sum(v * v) * (1 + 1e-6)
    x0 = oracle.fbp(b, g)
    x, losses = oracle.gd_refine(x0, b, g, 1.0 / lam, 20)
    assert all(l1 <= l0 + 1e-12 for l0, l1 in zip(losses, losses[1:]))
    # central finite difference of the loss along a random direction
    v = rng.standard_normal((N, N))
    eps = 1e-4
    fd = (oracle.loss(x + eps * v, b, g) - oracle.loss(x - eps * v, b, g)) / (2 * eps)
    assert np.sum(oracle.gradient(x, b, g) * v) == pytest.approx(fd, rel=1e-7)
