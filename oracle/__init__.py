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

This module adds the least-squares refinement loop (gradient descent on
0.5 * ||A x - b||^2, step 1/lambda_max(A^T A) from power iteration) in numpy
on top of those calls.
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
