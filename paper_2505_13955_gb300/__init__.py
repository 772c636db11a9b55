"""GB300-native parallel-beam filtered backprojection (FBP).

The reconstruction hot path of arXiv 2505.13955 ("ROVAI", Sec. V-A): every
detector row's sinogram is ramp-filtered and backprojected into one slice,
slice by slice.  The compute is hand-written CUDA for sm_103a in libfbp.so
(C ABI: include/fbp.h); this package is its thin Python binding.

``phantoms`` (the seeded input generator) imports without torch or CUDA; the
binding (``api``) is loaded on first attribute access.
"""
from __future__ import annotations

_API_NAMES = {
    "Geometry", "filter", "backproject", "radon_forward", "fbp", "fbp_host", "fbp_batched",
    "bp_variants", "forward_variant_count", "variant_supports", "batched_workspace_bytes", "prepare", "device_status", "release_tables",
    "Preprocess", "HuWindow", "filter_counts", "hu_coefficients", "backproject_u16", "fbp_counts",
    "RadonForward", "RadonBackproject", "radon", "radon_t", "lsq_refine", "FbpError", "lib",
}


def __getattr__(name):
    if name in _API_NAMES:
        from . import api
        return getattr(api, name)
    raise AttributeError(name)
