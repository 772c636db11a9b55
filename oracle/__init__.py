"""FP64 CPU oracle for parallel-beam FBP -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  It shares no code with the CUDA library in
``paper_2505_13955_gb300``; the two meet only through the seeded inputs that
``paper_2505_13955_gb300.phantoms`` generates.

The arithmetic lives in ``fbp_oracle.c`` (plain double-precision loops, one
per definition):

* ``taps``                -- band-limited ramp kernels (Kak & Slaney ch. 3),
                             the filter the paper cites for its filtering step
                             (Sec. IV-B; Sec. V-A(c) stage 2);
* ``filter_direct``       -- q_k[j] = tau * sum_m h[j-m] p_k[m];
* ``filter_fft``          -- the same linear convolution through the oracle's
                             own radix-2 FFT (used for D > 2048);
* ``backproject``         -- f = scale * sum_k Q_k(u_k), linear interpolation,
                             zero outside the detector (the O(N_p N_x N_y)
                             backprojection of Sec. V-A(c) stage 2);
* ``forward``             -- the matched forward projector A (scatter form),
                             whose transpose is ``backproject`` with scale 1.

This module adds, in numpy on top of those calls, the least-squares
refinement loop (gradient descent on 0.5 * ||A x - b||^2, step
1/lambda_max(A^T A) from power iteration) and the steps on either side of
the path (Sec. V-A(c) stages 2 and 4): Beer-Lambert conversion of counts,
a Gaussian blur along the detector, and the HU window quantised to uint16.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

RAMLAK = 0
SHEPP_LOGAN = 1

_lib = None


class _Geom(ctypes.Structure):
    _fields_ = [
        ("n_angles", ctypes.c_int),
        ("n_det", ctypes.c_int),
        ("n", ctypes.c_int),
        ("angle_start", ctypes.c_double),
        ("angle_step", ctypes.c_double),
        ("det_center", ctypes.c_double),
        ("det_spacing", ctypes.c_double),
        ("pixel_size", ctypes.c_double),
    ]


@dataclass
class Geometry:
    """Parallel-beam geometry of one slice (the oracle's own copy).

    Angles theta_k = angle_start + k * angle_step, k in [0, n_angles);
    pixel [r][c] sits at X = c - (n-1)/2, Y = r - (n-1)/2 (in pixels);
    its detector coordinate at angle k is
    u = (pixel_size / det_spacing) * (X cos theta_k + Y sin theta_k) + det_center.
    """
    n_angles: int
    n_det: int
    n: int
    angle_start: float = 0.0
    angle_step: float | None = None
    det_center: float | None = None
    det_spacing: float = 1.0
    pixel_size: float = 1.0

    def __post_init__(self):
        if self.angle_step is None:
            self.angle_step = np.pi / self.n_angles if self.n_angles else 0.0
        if self.det_center is None:
            self.det_center = 0.5 * (self.n_det - 1)

    def c_struct(self) -> _Geom:
        return _Geom(self.n_angles, self.n_det, self.n, float(self.angle_start),
                     float(self.angle_step), float(self.det_center),
                     float(self.det_spacing), float(self.pixel_size))


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        gp = ctypes.POINTER(_Geom)
        L.oracle_tap.argtypes = [ctypes.c_int, ctypes.c_long, ctypes.c_double]
        L.oracle_tap.restype = ctypes.c_double
        L.oracle_taps.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, dp]
        for name in ("oracle_filter_direct", "oracle_filter_fft", "oracle_filter"):
            fn = getattr(L, name)
            fn.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                           ctypes.c_double, dp]
            fn.restype = ctypes.c_int
        L.oracle_fft.argtypes = [dp, dp, ctypes.c_int, ctypes.c_int]
        L.oracle_fft.restype = ctypes.c_int
        L.oracle_conv_length.argtypes = [ctypes.c_int]
        L.oracle_conv_length.restype = ctypes.c_int
        L.oracle_backproject.argtypes = [dp, gp, ctypes.c_double, dp]
        L.oracle_backproject.restype = ctypes.c_int
        L.oracle_backproject_pixels.argtypes = [dp, gp, ctypes.c_double, ip, ip,
                                                ctypes.c_long, dp]
        L.oracle_backproject_pixels.restype = ctypes.c_int
        L.oracle_forward.argtypes = [dp, gp, dp]
        L.oracle_forward.restype = ctypes.c_int
        L.oracle_fbp.argtypes = [dp, gp, ctypes.c_int, dp]
        L.oracle_fbp.restype = ctypes.c_int
        L.oracle_num_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def num_threads() -> int:
    return int(lib().oracle_num_threads())


def tap(kind: int, n: int, tau: float = 1.0) -> float:
    return float(lib().oracle_tap(kind, n, tau))


def taps(kind: int, D: int, tau: float = 1.0) -> np.ndarray:
    """h[(D-1)+n] = h(n tau) for |n| <= D-1."""
    h = np.empty(2 * D - 1)
    _check(lib().oracle_taps(kind, D, tau, _dp(h)), "taps")
    return h


def conv_length(D: int) -> int:
    return int(lib().oracle_conv_length(D))


def fft(x: np.ndarray, sign: int = -1) -> np.ndarray:
    """The oracle's own radix-2 FFT (unnormalised both ways)."""
    x = np.asarray(x, dtype=np.complex128)
    re = _f64(x.real.copy())
    im = _f64(x.imag.copy())
    _check(lib().oracle_fft(_dp(re), _dp(im), len(re), sign), "fft")
    return re + 1j * im


def _filter(name: str, p, kind: int, tau: float) -> np.ndarray:
    p = _f64(p)
    shape = p.shape
    D = shape[-1]
    p2 = p.reshape(-1, D)
    q = np.empty_like(p2)
    _check(getattr(lib(), name)(_dp(p2), p2.shape[0], D, kind, tau, _dp(q)), name)
    return q.reshape(shape)


def filter_direct(p, kind: int = RAMLAK, tau: float = 1.0) -> np.ndarray:
    return _filter("oracle_filter_direct", p, kind, tau)


def filter_fft(p, kind: int = RAMLAK, tau: float = 1.0) -> np.ndarray:
    return _filter("oracle_filter_fft", p, kind, tau)


def filter(p, kind: int = RAMLAK, tau: float = 1.0) -> np.ndarray:
    return _filter("oracle_filter", p, kind, tau)


def backproject(q, g: Geometry, scale: float | None = None) -> np.ndarray:
    """f = scale * sum_k Q_k(u_k) for every pixel; scale defaults to dtheta."""
    q = _f64(q).reshape(g.n_angles, g.n_det)
    if scale is None:
        scale = g.angle_step
    f = np.empty((g.n, g.n))
    gs = g.c_struct()
    _check(lib().oracle_backproject(_dp(q), ctypes.byref(gs), scale, _dp(f)), "backproject")
    return f


def backproject_pixels(q, g: Geometry, rows, cols, scale: float | None = None) -> np.ndarray:
    q = _f64(q).reshape(g.n_angles, g.n_det)
    if scale is None:
        scale = g.angle_step
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    cols = np.ascontiguousarray(cols, dtype=np.int32)
    out = np.empty(len(rows))
    gs = g.c_struct()
    _check(lib().oracle_backproject_pixels(_dp(q), ctypes.byref(gs), scale, _ip(rows),
                                           _ip(cols), len(rows), _dp(out)),
           "backproject_pixels")
    return out


def forward(f, g: Geometry) -> np.ndarray:
    f = _f64(f).reshape(g.n, g.n)
    p = np.empty((g.n_angles, g.n_det))
    gs = g.c_struct()
    _check(lib().oracle_forward(_dp(f), ctypes.byref(gs), _dp(p)), "forward")
    return p


def fbp(p, g: Geometry, kind: int = RAMLAK) -> np.ndarray:
    p = _f64(p).reshape(g.n_angles, g.n_det)
    f = np.empty((g.n, g.n))
    gs = g.c_struct()
    _check(lib().oracle_fbp(_dp(p), ctypes.byref(gs), kind, _dp(f)), "fbp")
    return f


# ---------------------------------------------------------------------------
# Least-squares refinement: minimise L(x) = 0.5 ||A x - b||^2 by gradient
# descent x <- x - eta * A^T (A x - b), eta = 1 / lambda_max(A^T A).
# ---------------------------------------------------------------------------
def gradient(x, b, g: Geometry) -> np.ndarray:
    """grad L(x) = A^T (A x - b)."""
    return backproject(forward(x, g) - _f64(b), g, scale=1.0)


def loss(x, b, g: Geometry) -> float:
    r = forward(x, g) - _f64(b)
    return 0.5 * float(np.sum(r * r))


def power_lambda_max(g: Geometry, iters: int = 20, seed: int = 0) -> float:
    """Largest eigenvalue of A^T A by power iteration from a seeded start."""
    rng = np.random.Generator(np.random.PCG64(seed))
    v = rng.standard_normal((g.n, g.n))
    v /= np.linalg.norm(v)
    lam = 0.0
    for _ in range(iters):
        w = backproject(forward(v, g), g, scale=1.0)
        lam = float(np.sum(v * w))
        v = w / np.linalg.norm(w)
    return lam


def gd_refine(x0, b, g: Geometry, eta: float, iters: int):
    """Returns (x_iters, [loss before each step ..., final loss])."""
    x = _f64(x0).copy()
    losses = []
    for _ in range(iters):
        r = forward(x, g) - _f64(b)
        losses.append(0.5 * float(np.sum(r * r)))
        x = x - eta * backproject(r, g, scale=1.0)
    losses.append(loss(x, b, g))
    return x, losses


# ---------------------------------------------------------------------------
# The steps on either side of the path (Sec. V-A(c)): stage 2 converts
# detector counts to line integrals (Beer-Lambert) and blurs them (Gaussian)
# before filtering; stage 4 maps the reconstructed attenuation to CT numbers
# (HU) over a window and quantises to uint16.  The paper fixes neither the
# blur width nor the window: both are parameters here.
# ---------------------------------------------------------------------------
def beer_lambert(I, I0, mu_scale: float = 1.0, floor: float = 1.0) -> np.ndarray:
    """Line integrals from counts by the Beer-Lambert law I = I0 exp(-p):
    p = mu_scale * -ln(max(I, floor) / I0).  I0 is a scalar or one value per
    detector bin (broadcast along the last axis)."""
    I = np.maximum(_f64(I), float(floor))
    return float(mu_scale) * -np.log(I / _f64(I0))


def gaussian_taps(sigma: float) -> np.ndarray:
    """Weights w_k, |k| <= r, r = floor(4 sigma + 1/2): exp(-k^2 / (2 sigma^2))
    normalised to sum 1 (sigma = 0: the single tap w_0 = 1)."""
    if sigma <= 0.0:
        return np.ones(1)
    r = int(4.0 * sigma + 0.5)
    k = np.arange(-r, r + 1, dtype=np.float64)
    w = np.exp(-(k * k) / (2.0 * sigma * sigma))
    return w / w.sum()


def gaussian_blur(p, sigma: float) -> np.ndarray:
    """Blur along the detector (last axis), zero outside [0, D):
    y[j] = sum_k w_k p[j - k]."""
    p = _f64(p)
    w = gaussian_taps(sigma)
    r = (len(w) - 1) // 2
    D = p.shape[-1]
    y = np.zeros_like(p)
    for i, k in enumerate(range(-r, r + 1)):
        lo, hi = max(0, k), min(D, D + k)          # j with 0 <= j - k < D
        if lo < hi:
            y[..., lo:hi] += w[i] * p[..., lo - k:hi - k]
    return y


def preprocess(I, I0, mu_scale: float = 1.0, floor: float = 1.0, sigma: float = 0.0) -> np.ndarray:
    """Stage-2 pre-processing: Beer-Lambert, then the Gaussian blur."""
    return gaussian_blur(beer_lambert(I, I0, mu_scale, floor), sigma)


def hu(mu, mu_water: float, mu_air: float = 0.0) -> np.ndarray:
    """CT number: HU = 1000 (mu - mu_water) / (mu_water - mu_air)."""
    return 1000.0 * (_f64(mu) - mu_water) / (mu_water - mu_air)


def hu_codes(mu, mu_water: float, mu_air: float, hu_min: float, hu_max: float) -> np.ndarray:
    """Stage-4 quantisation in FP64: the HU window [hu_min, hu_max] mapped
    onto [0, 65535], rounded to nearest (ties to even) and clamped."""
    x = (hu(mu, mu_water, mu_air) - hu_min) / (hu_max - hu_min) * 65535.0
    return np.clip(np.rint(x), 0, 65535).astype(np.uint16)


def hu_affine(mu_water: float, mu_air: float, hu_min: float, hu_max: float):
    """(a, b) with code = a * mu + b before rounding, from the definition in
    FP64: a = 1000 * 65535 / ((mu_water - mu_air)(hu_max - hu_min)),
    b = -(1000 mu_water / (mu_water - mu_air) + hu_min) * 65535 / (hu_max - hu_min)."""
    s = 65535.0 / (hu_max - hu_min)
    a = 1000.0 / (mu_water - mu_air) * s
    b = -(1000.0 * mu_water / (mu_water - mu_air) + hu_min) * s
    return a, b


def hu_codes_f32(mu32, a32, b32) -> np.ndarray:
    """The same quantisation taken in FP32 from FP32 values, as a sequence of
    single roundings: t = RN32(a * mu), t = RN32(t + b), code = clamp(RNE(t))."""
    mu32 = np.asarray(mu32, dtype=np.float32)
    t = np.float32(a32) * mu32
    t = (t + np.float32(b32)).astype(np.float32)
    return np.clip(np.rint(t), 0, 65535).astype(np.uint16)


# ---------------------------------------------------------------------------
# Offset scans (Sec. V-A(b): the sample is shifted laterally so that a 360
# degree scan covers a field of view wider than the detector).  A ray (th, s)
# and (th + pi, -s) are the same line, so near the rotation axis every line
# is measured twice and far out on the long side once.  Each row is weighted
# before filtering by a smooth overlap weight (the paper gives none):
#   t = +-s (positive towards the long side), Delta = overlap half-width,
#   w = 0 (t < -Delta), sin^2(pi/4 (1 + t/Delta)) (|t| <= Delta), 1 (t > Delta),
# so that w(t) + w(-t) = 1 and every line counts once.  The ramp filter
# spreads a weighted row beyond the detector's short edge, so rows are
# filtered and backprojected on a virtual detector centred on the axis that
# spans the long side twice (the physical bins embedded, zeros elsewhere);
# the backprojection runs over [0, 2 pi) with scale 2 pi / K.
# ---------------------------------------------------------------------------
def offset_weight(t, overlap: float) -> np.ndarray:
    """w(t) for signed distances t (bins) from the axis, positive towards the long side."""
    t = _f64(t)
    w = np.where(t > overlap, 1.0, 0.0)
    mid = np.abs(t) <= overlap
    w[mid] = np.sin(0.25 * np.pi * (1.0 + t[mid] / overlap)) ** 2
    return w


def offset_virtual(n_det: int, det_center: float, overlap: float):
    """Virtual detector of an offset scan: (n_virtual, centre, offset, weights)
    with physical bin j at virtual bin j + offset and the weights per
    virtual bin.  2 * det_center must be an integer."""
    long_positive = (n_det - 1 - det_center) >= det_center
    half = (n_det - 1 - det_center) if long_positive else det_center
    n_v = int(round(2 * half)) + 1
    c_v = 0.5 * (n_v - 1)
    offset = int(round(c_v - det_center)) if long_positive else 0
    s = np.arange(n_v) - c_v
    w = offset_weight(s if long_positive else -s, overlap)
    return n_v, c_v, offset, w


def embed_rows(p, n_virtual: int, offset: int) -> np.ndarray:
    """Rows of physical bins placed at virtual bins [offset, offset + D)."""
    p = _f64(p)
    out = np.zeros(p.shape[:-1] + (n_virtual,))
    out[..., offset:offset + p.shape[-1]] = p
    return out


def fbp_weighted(p, g: Geometry, weights, kind: int = RAMLAK) -> np.ndarray:
    """FBP of rows weighted per bin before filtering (scale = angle_step)."""
    return fbp(_f64(p) * _f64(weights)[None, :], g, kind)


def offset_fold(pv, weights) -> np.ndarray:
    """Fold the weighted virtual rows of a full turn into half-turn rows.

    With K even and angles th_k = th_0 + 2 pi k / K, th_{k + K/2} = th_k + pi,
    and the line (th + pi, s) is the line (th, -s): on the centred virtual
    detector the row at th_k + pi, read at the mirrored bin n_v - 1 - i,
    measures the line that bin i of the row at th_k measures.  So
        r_k[i] = w[i] p_k[i] + w[n_v - 1 - i] p_{k + K/2}[n_v - 1 - i],  k < K/2,
    and the FBP of r over th_k, k < K/2 (step 2 pi / K = pi / (K/2), a half
    turn) equals the weighted full-turn FBP: the ramp kernel is even, so
    filtering commutes with the mirror, and so does linear interpolation."""
    pv = _f64(pv)
    w = _f64(weights)
    K = pv.shape[-2]
    if K % 2:
        raise ValueError("the fold needs an even number of angles")
    return pv[..., :K // 2, :] * w + (pv[..., K // 2:, :] * w)[..., ::-1]
