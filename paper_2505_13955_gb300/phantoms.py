"""Seeded synthetic inputs shaped like the paper's reconstruction workloads.

The paper reconstructs SPring-8 scans of 46 highway specimens (Sec. VI) and
simulated 8192^2 volumes (Sec. V-B(a)); neither is available here.  Seeded
ellipse phantoms stand in for them: the Shepp-Logan head phantom and random
ellipse fields, projected analytically (closed-form line integrals of
ellipses), optionally with Poisson photon noise.  Both the CUDA library's tests
and the FP64 oracle consume the arrays produced here, so neither side's
arithmetic decides what the other is compared on.

This module holds no filtered-backprojection arithmetic.  The heavy loops
(sinogram evaluation, rasterisation) are plain host C in
``csrc/phantom_gen.c``; parameters and noise come from numpy's PCG64 with the
seeds below.

Conventions (pixel units, pixel size 1):
  * ellipse parameters live on the unit disk; radius 1 <-> N/2 pixels;
  * pixel [r][c] is centred at X = c - (N-1)/2, Y = r - (N-1)/2;
  * bin j is centred at s_j = j - det_center; det_center defaults to (D-1)/2;
  * angles theta_k = k * pi / K on [0, pi) (a full turn, 2 pi k / K, for
    offset scans);
  * a sinogram value is the line integral in density x pixels.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csrc", "phantom_gen.c")
_LIB = os.path.join(_HERE, "libphantom.so")
_lib = None

BASE_SEED = 20250519

# Shepp & Logan (1974) head phantom, 10 ellipses, with the original low-contrast
# densities, as tabulated in Kak & Slaney, "Principles of Computerized
# Tomographic Imaging", Table 3.1: centre (x, y), semi-axes (A, B), rotation of
# the A axis from +x in degrees, density.
SHEPP_LOGAN_TABLE = (
    # x0      y0       A      B      deg    rho
    (0.0,     0.0,     0.92,  0.69,  90.0,  2.00),
    (0.0,    -0.0184,  0.874, 0.6624, 90.0, -0.98),
    (0.22,    0.0,     0.31,  0.11,  72.0, -0.02),
    (-0.22,   0.0,     0.41,  0.16, 108.0, -0.02),
    (0.0,     0.35,    0.25,  0.21,  90.0,  0.01),
    (0.0,     0.1,     0.046, 0.046,  0.0,  0.01),
    (0.0,    -0.1,     0.046, 0.046,  0.0,  0.01),
    (-0.08,  -0.605,   0.046, 0.023,  0.0,  0.01),
    (0.0,    -0.606,   0.023, 0.023,  0.0,  0.01),   # the circle sits at y = -0.606 in the table
    (0.06,   -0.605,   0.046, 0.023, 90.0,  0.01),
)


def build(force: bool = False) -> str:
    """Compile the generator's host C into libphantom.so (gcc, OpenMP)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    subprocess.run(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                    "-o", tmp, _SRC, "-lm"], check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        fp = ctypes.POINTER(ctypes.c_float)
        L.phantom_sinogram.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double, dp, fp]
        L.phantom_sinogram.restype = ctypes.c_int
        L.phantom_image.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                    ctypes.c_int, dp]
        L.phantom_image.restype = ctypes.c_int
        L.phantom_edge_distance.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                            ctypes.c_double, dp]
        L.phantom_edge_distance.restype = ctypes.c_int
        _lib = L
    return _lib


def shepp_logan() -> np.ndarray:
    """(10, 6) array: x0, y0, A, B, phi (radians), rho on the unit disk."""
    t = np.array(SHEPP_LOGAN_TABLE, dtype=np.float64)
    t[:, 4] = np.deg2rad(t[:, 4])
    return t


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def random_ellipses(rng: np.random.Generator, count_range=(20, 50),
                    semi_axis_range=(0.02, 0.4), density_range=(0.0, 1.0),
                    fit_radius: float = 0.95) -> np.ndarray:
    """Random ellipse field.

    count ~ U{20..50}; semi-axes ~ U[0.02, 0.4] x field-of-view width
    (= U[0.04, 0.8] on the unit disk); rotation ~ U[0, pi); density ~ U[0, 1];
    centre uniform in the unit disk, redrawn until the ellipse's bounding
    circle lies within ``fit_radius`` of the field of view.  Densities add
    where ellipses overlap.
    """
    n = int(rng.integers(count_range[0], count_range[1] + 1))
    out = np.empty((n, 6))
    for i in range(n):
        A = 2.0 * rng.uniform(*semi_axis_range)
        B = 2.0 * rng.uniform(*semi_axis_range)
        phi = rng.uniform(0.0, np.pi)
        rho = rng.uniform(*density_range)
        bound = max(A, B)
        while True:
            rad = np.sqrt(rng.uniform(0.0, 1.0))
            ang = rng.uniform(0.0, 2.0 * np.pi)
            if rad + bound <= fit_radius:
                break
        out[i] = (rad * np.cos(ang), rad * np.sin(ang), A, B, phi, rho)
    return out


def sinogram(ellipses: np.ndarray, n_angles: int, n_det: int, n: int,
             angle_start: float = 0.0, angle_step: float | None = None,
             det_center: float | None = None, det_spacing: float = 1.0,
             dtype=np.float32) -> np.ndarray:
    """Analytic parallel-beam sinogram [n_angles, n_det] in pixel units."""
    if angle_step is None:
        angle_step = np.pi / n_angles
    if det_center is None:
        det_center = 0.5 * (n_det - 1)
    ell = np.ascontiguousarray(ellipses, dtype=np.float64)
    dp = ctypes.POINTER(ctypes.c_double)
    fp = ctypes.POINTER(ctypes.c_float)
    if dtype == np.float64:
        out = np.empty((n_angles, n_det), dtype=np.float64)
        o64, o32 = out.ctypes.data_as(dp), ctypes.cast(None, fp)
    else:
        out = np.empty((n_angles, n_det), dtype=np.float32)
        o64, o32 = ctypes.cast(None, dp), out.ctypes.data_as(fp)
    rc = _load().phantom_sinogram(ell.ctypes.data_as(dp), len(ell), n_angles, n_det,
                                  angle_start, angle_step, det_center, det_spacing,
                                  0.5 * n, o64, o32)
    if rc != 0:
        raise RuntimeError("phantom_sinogram failed")
    return out


def image(ellipses: np.ndarray, n: int, supersample: int = 1) -> np.ndarray:
    """Rasterised phantom [n, n] (density at pixel centres, or sub-pixel mean)."""
    ell = np.ascontiguousarray(ellipses, dtype=np.float64)
    out = np.empty((n, n))
    dp = ctypes.POINTER(ctypes.c_double)
    rc = _load().phantom_image(ell.ctypes.data_as(dp), len(ell), n, 0.5 * n,
                               supersample, out.ctypes.data_as(dp))
    if rc != 0:
        raise RuntimeError("phantom_image failed")
    return out


def edge_distance(ellipses: np.ndarray, n: int, step: float = 0.25) -> np.ndarray:
    """Distance (pixels) from each pixel centre to the nearest ellipse edge
    (boundary sampled every ``step`` pixels of arc; error <= step / 2)."""
    ell = np.ascontiguousarray(ellipses, dtype=np.float64)
    out = np.empty((n, n))
    dp = ctypes.POINTER(ctypes.c_double)
    rc = _load().phantom_edge_distance(ell.ctypes.data_as(dp), len(ell), n, 0.5 * n,
                                       step, out.ctypes.data_as(dp))
    if rc != 0:
        raise RuntimeError("phantom_edge_distance failed")
    return out


def poisson_noise(p_px: np.ndarray, n: int, photons: float,
                  rng: np.random.Generator) -> np.ndarray:
    """Photon-count noise on line integrals given in pixel units.

    The physical line integral is p_px / n (attenuation per field-of-view
    width); counts ~ Poisson(photons * exp(-p_px / n)); the noisy line
    integral is n * -ln(max(counts, 1) / photons), returned as float32.
    """
    lam = photons * np.exp(-np.asarray(p_px, dtype=np.float64) / n)
    counts = rng.poisson(lam)
    return (n * -np.log(np.maximum(counts, 1) / photons)).astype(np.float32)


def poisson_counts(p_px: np.ndarray, n: int, photons: float,
                   rng: np.random.Generator) -> np.ndarray:
    """Raw detector counts for line integrals in pixel units: the physical
    line integral is p_px / n, counts ~ Poisson(photons * exp(-p_px / n)),
    returned as float32 (the detector's data; converting them back to line
    integrals is the method's Beer-Lambert step, not the generator's)."""
    lam = photons * np.exp(-np.asarray(p_px, dtype=np.float64) / n)
    return rng.poisson(lam).astype(np.float32)


# ---------------------------------------------------------------------------
# The workloads (slice counts, sizes, angle counts, filters, noise).
# ---------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    n_slices: int
    n: int                      # N = D for the uniform workloads
    n_angles: int
    filter: str                 # "ramlak" | "shepp_logan"
    phantom: str                # "shepp_logan" | "random"
    photons: float | None       # Poisson incident photons per ray, None = noise-free
    config_id: int
    ragged: bool = False
    n_choices: tuple = field(default_factory=tuple)
    k_choices: tuple = field(default_factory=tuple)
    counts: bool = False        # inputs are raw detector counts (stage-2 pre-processing on)
    offset: tuple | None = None  # full-turn offset scan: (n_det, det_center, overlap in bins)
    offset_fraction: float = 0.0  # ragged: share of items that are offset scans


# Parameters of the counts-to-codes workload (the paper leaves the blur width
# and the HU window open): blur sigma in bins, water / air attenuation in the
# phantom's density units, the HU window.
PIPELINE = {"blur_sigma": 1.0, "mu_water": 0.5, "mu_air": 0.0, "hu_min": -1000.0, "hu_max": 3000.0}


WORKLOADS = {
    "fbp_single_n256": Workload("fbp_single_n256", 1, 256, 360, "ramlak", "shepp_logan", None, 1),
    "fbp_stack_n2048": Workload("fbp_stack_n2048", 64, 2048, 1800, "shepp_logan", "random", 1e4, 2),
    "fbp_precision_n8192": Workload("fbp_precision_n8192", 16, 8192, 4096, "ramlak", "random", None, 3),
    "fbp_ragged_batch": Workload("fbp_ragged_batch", 200, 0, 0, "ramlak", "random", None, 4,
                                 ragged=True, n_choices=(512, 1024, 2048, 4096),
                                 k_choices=(720, 1800, 3600)),
    "gd_refine_n1024": Workload("gd_refine_n1024", 16, 1024, 1800, "ramlak", "random", 1e4, 5),
    "fbp_pipeline_n8192": Workload("fbp_pipeline_n8192", 16, 8192, 4096, "ramlak", "random", 1e4, 6,
                                   counts=True),
    # offset scan (Sec. V-A(b)): 8192 angles over a full turn, a 4608-bin
    # detector with the axis at bin 511.5, so it covers the 8192-pixel field
    # of view's long side (radius 4095.5) and overlaps the axis by 512 bins
    "fbp_offset_n8192": Workload("fbp_offset_n8192", 16, 8192, 8192, "ramlak", "random", None, 7,
                                 offset=(4608, 511.5, 256.0)),
    # normal and offset scans reconstructed together (Sec. V-A(b)): as the
    # ragged batch, about a third of the items offset scans (scan_spec)
    "fbp_mixed_batch": Workload("fbp_mixed_batch", 200, 0, 0, "ramlak", "random", None, 8,
                                ragged=True, n_choices=(512, 1024, 2048, 4096),
                                k_choices=(720, 1800, 3600), offset_fraction=1.0 / 3.0),
    # adaptive patching of reconstructed 8192^2 slices (sap_slice, SAP)
    "sap_patching_n8192": Workload("sap_patching_n8192", 16, 8192, 0, "", "random", None, 9),
}


def slice_seed(config_id: int, slice_index: int) -> int:
    return BASE_SEED + 1000 * config_id + slice_index


def slice_spec(w: Workload, i: int):
    """(n, n_angles, ellipses, rng) for slice i of workload w (deterministic)."""
    rng = rng_for(slice_seed(w.config_id, i))
    if w.ragged:
        n = int(rng.choice(np.array(w.n_choices)))
        k = int(rng.choice(np.array(w.k_choices)))
    else:
        n, k = w.n, w.n_angles
    ell = shepp_logan() if w.phantom == "shepp_logan" else random_ellipses(rng)
    return n, k, ell, rng


def scan_spec(w: Workload, i: int) -> dict:
    """Item i of a mixed batch: n, the half-turn angle count k, ellipses, and
    whether it is an offset scan.  An offset item has 2k angles over a full
    turn on a detector of 9n/16 bins with the axis at bin n/16 - 1/2 (it
    covers the long side of the n-pixel field of view) and overlap n/32 bins;
    a normal item has k angles over a half turn on n centred bins."""
    n, k, ell, rng = slice_spec(w, i)
    offset = bool(rng.uniform() < w.offset_fraction)
    if offset:
        return {"n": n, "k": k, "ell": ell, "offset": True, "n_angles": 2 * k,
                "n_det": 9 * n // 16, "det_center": n / 16 - 0.5, "overlap": n / 32,
                "angle_step": 2.0 * np.pi / (2 * k)}
    return {"n": n, "k": k, "ell": ell, "offset": False, "n_angles": k, "n_det": n,
            "det_center": 0.5 * (n - 1), "overlap": 0.0, "angle_step": np.pi / k}


def scan_sinogram(spec: dict, dtype=np.float32) -> np.ndarray:
    """Noise-free analytic rows [n_angles, n_det] of a scan_spec item."""
    return sinogram(spec["ell"], spec["n_angles"], spec["n_det"], spec["n"],
                    angle_step=spec["angle_step"], det_center=spec["det_center"], dtype=dtype)


# Adaptive patching of reconstructed slices (Sec. V-B(c)): the stage-4
# output is a slice of uint16 codes.  Synthetic stand-in: a random-ellipse
# phantom rasterised at n pixels, densities mapped linearly to codes
# (SAP_CODES: code = offset + scale * density), plus Gaussian noise of
# sigma codes, rounded and clipped to [0, 65535].
SAP_CODES = {"offset": 8000.0, "scale": 20000.0, "sigma": 150.0}
# Patching parameters of the workload (the paper fixes none): patch side,
# sequence length (1 mod 3), Canny thresholds on M = |gx| + |gy|.
SAP = {"patch": 16, "length": 4096, "canny_lo": 400000, "canny_hi": 1000000}


def sap_slice(n: int, seed: int) -> np.ndarray:
    """uint16 codes [n, n] of a seeded random-ellipse slice (see SAP_CODES)."""
    rng = rng_for(seed)
    ell = random_ellipses(rng)
    dens = image(ell, n)
    c = SAP_CODES
    x = c["offset"] + c["scale"] * dens + rng.normal(0.0, c["sigma"], dens.shape)
    return np.clip(np.rint(x), 0, 65535).astype(np.uint16)


def slice_counts(w: Workload, i: int) -> np.ndarray:
    """Raw detector counts [K, N] (float32) for slice i of a counts workload."""
    n, k, ell, rng = slice_spec(w, i)
    p = sinogram(ell, k, n, n, dtype=np.float64)
    return poisson_counts(p, n, w.photons, rng)


def slice_sinogram(w: Workload, i: int, dtype=np.float32):
    """Sinogram [K, N] for slice i of workload w, with the workload's noise
    (an offset workload: [K, n_det] over a full turn, axis at det_center)."""
    n, k, ell, rng = slice_spec(w, i)
    if w.offset is not None:
        d, c, _ = w.offset
        return sinogram(ell, k, d, n, angle_step=2.0 * np.pi / k, det_center=c, dtype=dtype)
    if w.photons is None:
        return sinogram(ell, k, n, n, dtype=dtype)
    p = sinogram(ell, k, n, n, dtype=np.float64)
    return poisson_noise(p, n, w.photons, rng).astype(dtype)
