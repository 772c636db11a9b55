"""ctypes declarations for libfbp.so (the C ABI in include/fbp.h).

Argument marshalling only.  If the library has not been built this module
raises on first use: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_NAMES = {"default": "libfbp.so", "checked": "libfbp_checked.so"}

FBP_OK = 0
FBP_ERR_INVALID_ARG = -1
FBP_ERR_UNSUPPORTED = -2
FBP_ERR_WORKSPACE = -3
FBP_ERR_CUDA = -4
FBP_ERR_DEVICE_STATUS = -5

FBP_FILTER_RAMLAK = 0
FBP_FILTER_SHEPP_LOGAN = 1

FBP_F32 = 0
FBP_F16 = 1
FBP_BF16 = 2

# Every function include/*.h declares, with (restype, argtypes).
_vp = ctypes.c_void_p


class CGeometry(ctypes.Structure):
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


class CBatchItem(ctypes.Structure):
    _fields_ = [("sino", _vp), ("slice", _vp), ("g", CGeometry)]


class CBpShape(ctypes.Structure):
    _fields_ = [("angle_tile", ctypes.c_int), ("tile_x", ctypes.c_int), ("tile_y", ctypes.c_int),
                ("px", ctypes.c_int), ("py", ctypes.c_int), ("threads", ctypes.c_int),
                ("symmetric", ctypes.c_int), ("packed16", ctypes.c_int), ("texture", ctypes.c_int)]


_G = ctypes.POINTER(CGeometry)
class CPreprocess(ctypes.Structure):
    _fields_ = [
        ("flat", ctypes.c_void_p),
        ("flat_value", ctypes.c_float),
        ("count_floor", ctypes.c_float),
        ("mu_scale", ctypes.c_float),
        ("blur_sigma", ctypes.c_float),
    ]


class CHuWindow(ctypes.Structure):
    _fields_ = [
        ("mu_water", ctypes.c_double),
        ("mu_air", ctypes.c_double),
        ("hu_min", ctypes.c_double),
        ("hu_max", ctypes.c_double),
    ]


class CScanItem(ctypes.Structure):
    _fields_ = [("sino", _vp), ("slice", _vp), ("g", CGeometry), ("overlap", ctypes.c_double),
                ("fold", ctypes.c_int)]


class CSapParams(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("patch", ctypes.c_int), ("length", ctypes.c_int),
                ("canny_lo", ctypes.c_int), ("canny_hi", ctypes.c_int)]


FBP_ORDER_QUEUE = 0
FBP_ORDER_GROUP_CYCLIC = 1


class COnchipPeaks(ctypes.Structure):
    _fields_ = [("lds_bytes_per_clk_per_sm", ctypes.c_double), ("fma_per_clk_per_sm", ctypes.c_double),
                ("sm_clock_mhz", ctypes.c_double), ("sm_count", ctypes.c_int)]


class COffsetScan(ctypes.Structure):
    _fields_ = [("overlap", ctypes.c_double), ("fold", ctypes.c_int)]


SIGNATURES = {
    "fbp_version": (ctypes.c_int, []),
    "fbp_geometry_default": (CGeometry, [ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "fbp_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "fbp_last_error_message": (ctypes.c_char_p, []),
    "fbp_filter": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, ctypes.c_int, _G, ctypes.c_int, _vp]),
    "fbp_filter_counts": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, ctypes.c_int, _G, ctypes.c_int,
                                         ctypes.POINTER(CPreprocess), _vp]),
    "fbp_offset_geometry": (ctypes.c_int, [_G, ctypes.POINTER(COffsetScan), _G,
                                           ctypes.POINTER(ctypes.c_int)]),
    "fbp_filter_offset": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, ctypes.c_int, _G, ctypes.c_int,
                                         ctypes.POINTER(COffsetScan), _vp]),
    "fbp_hu_coefficients": (ctypes.c_int, [ctypes.POINTER(CHuWindow), ctypes.POINTER(ctypes.c_float),
                                           ctypes.POINTER(ctypes.c_float)]),
    "fbp_backproject_u16": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _vp, _G, ctypes.c_int, ctypes.c_float,
                                           ctypes.POINTER(CHuWindow), ctypes.c_int, _vp]),
    "fbp_backproject": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _vp, _G, ctypes.c_int, ctypes.c_float,
                                       ctypes.c_int, _vp]),
    "fbp_backproject_variant": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _vp, _G, ctypes.c_int,
                                               ctypes.c_float, ctypes.c_int, ctypes.c_int, _vp]),
    "radon_forward": (ctypes.c_int, [_vp, _vp, _G, ctypes.c_int, _vp]),
    "radon_forward_variant": (ctypes.c_int, [_vp, _vp, _G, ctypes.c_int, ctypes.c_int, _vp]),
    "radon_forward_variant_count": (ctypes.c_int, []),
    "fbp_backproject_noalloc": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _vp, _G, ctypes.c_int,
                                               ctypes.c_float, ctypes.c_int, _vp]),
    "fbp_bp_variant_count": (ctypes.c_int, []),
    "fbp_bp_variant_info": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(CBpShape)]),
    "fbp_bp_variant_supports": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _G]),
    "fbp_batched_item_staged": (ctypes.c_int, [_G, ctypes.c_int]),
    "fbp_batched_workspace_bytes": (ctypes.c_size_t, [ctypes.POINTER(CBatchItem), ctypes.c_int,
                                                      ctypes.c_int]),
    "fbp_batched": (ctypes.c_int, [ctypes.POINTER(CBatchItem), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_int, _vp, ctypes.c_size_t, _vp]),
    "fbp_batched_scans_workspace_bytes": (ctypes.c_size_t, [ctypes.POINTER(CScanItem), ctypes.c_int,
                                                            ctypes.c_int]),
    "fbp_batched_scans": (ctypes.c_int, [ctypes.POINTER(CScanItem), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, ctypes.c_int, _vp, ctypes.c_size_t, _vp]),
    "sap_workspace_bytes": (ctypes.c_size_t, [ctypes.POINTER(CSapParams)]),
    "sap_edges": (ctypes.c_int, [_vp, _vp, ctypes.POINTER(CSapParams), _vp, ctypes.c_size_t, _vp]),
    "sap_patches": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.POINTER(CSapParams), _vp, ctypes.c_size_t, _vp]),
    "sap_depatch_pack": (ctypes.c_int, [_vp, _vp, _vp, ctypes.POINTER(CSapParams), _vp]),
    "fbp_last_device_status": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int)]),
    "fbp_prepare": (ctypes.c_int, [_G, ctypes.c_int, _vp]),
    "fbp_release_tables": (None, []),
    "fbp_measure_onchip_peaks": (ctypes.c_int, [ctypes.POINTER(COnchipPeaks)]),
    "fbp_backproject_staged_workspace_bytes": (ctypes.c_size_t, [_G, ctypes.c_int, ctypes.c_int]),
    "fbp_backproject_staged_shape_count": (ctypes.c_int, [ctypes.c_int]),
    "fbp_backproject_staged": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _vp, _G, ctypes.c_int, ctypes.c_float,
                                              ctypes.c_int, ctypes.c_int, _vp, ctypes.c_size_t, _vp]),
    "fbp_backproject_staged_u16": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _vp, _G, ctypes.c_int, ctypes.c_float,
                                                  ctypes.POINTER(CHuWindow), ctypes.c_int, _vp, ctypes.c_size_t,
                                                  _vp]),
    "fbp_host_workspace_bytes": (ctypes.c_size_t, [_G, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "fbp_host": (ctypes.c_int, [_vp, _vp, _G, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                ctypes.POINTER(CPreprocess), ctypes.POINTER(CHuWindow), ctypes.c_int,
                                ctypes.c_int, _vp, ctypes.c_size_t, _vp]),
}

_libs: dict[str, ctypes.CDLL] = {}


class FbpError(RuntimeError):
    def __init__(self, status: int, message: str):
        self.status = status
        super().__init__(message)


def lib_path(which: str = "default") -> str:
    return os.path.join(HERE, LIB_NAMES[which])


def load(which: str = "default") -> ctypes.CDLL:
    """Load libfbp.so (or the bounds-checked build); raises if it is missing."""
    L = _libs.get(which)
    if L is not None:
        return L
    path = lib_path(which)
    if not os.path.exists(path):
        raise RuntimeError(
            f"{os.path.basename(path)} is not built; build it with "
            "`python -c \"import __graft_entry__ as g; g.build()\"` "
            "(there is no CPU fallback)")
    L = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _libs[which] = L
    return L


def check(status: int, lib: ctypes.CDLL, what: str) -> None:
    if status != FBP_OK:
        name = lib.fbp_status_string(status).decode()
        msg = lib.fbp_last_error_message().decode()
        raise FbpError(status, f"{what}: {name}: {msg}")
