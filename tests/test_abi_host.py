"""The C-ABI library on a CPU-only host: it loads, exports every function that
include/fbp.h declares, and its validation paths reject bad arguments before
any CUDA call.  (No compute call is made here.)"""
import ctypes
import os
import re

import pytest

from batch_layout import align256, staged_table_bytes
from paper_2505_13955_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2505_13955_gb300 import build
    build.build_cuda()
    return _lib.load()


def declared_functions():
    inc = os.path.join(ROOT, "include")
    src = "".join(open(os.path.join(inc, f)).read() for f in sorted(os.listdir(inc)) if f.endswith(".h"))
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w \*]*?\b(\w+)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "sizeof")))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("fbp_filter", "fbp_backproject", "radon_forward", "fbp_batched",
              "fbp_batched_workspace_bytes", "fbp_last_device_status", "fbp_status_string"):
        assert n in names


def test_every_declared_symbol_is_exported_and_bound(L):
    for n in declared_functions():
        assert hasattr(L, n), n
        assert n in _lib.SIGNATURES, f"{n} has no ctypes signature"


def test_status_strings(L):
    for code, name in [(0, "FBP_OK"), (-1, "FBP_ERR_INVALID_ARG"), (-2, "FBP_ERR_UNSUPPORTED"),
                       (-3, "FBP_ERR_WORKSPACE"), (-4, "FBP_ERR_CUDA"), (-5, "FBP_ERR_DEVICE_STATUS")]:
        assert L.fbp_status_string(code).decode() == name
    assert L.fbp_version() >= 100


def test_default_geometry(L):
    g = L.fbp_geometry_default(360, 256, 256)
    assert (g.n_angles, g.n_det, g.n) == (360, 256, 256)
    assert g.angle_step == pytest.approx(3.141592653589793 / 360)
    assert g.det_center == 127.5 and g.det_spacing == 1.0 and g.pixel_size == 1.0


def test_variant_table(L):
    n = L.fbp_bp_variant_count()
    assert n >= 4
    for v in range(n):
        s = _lib.CBpShape()
        assert L.fbp_bp_variant_info(v, ctypes.byref(s)) == 0
        assert s.tile_x == s.px * (s.threads // (s.tile_y // s.py))
        assert s.threads % 32 == 0
    s = _lib.CBpShape()
    assert L.fbp_bp_variant_info(n, ctypes.byref(s)) == _lib.FBP_ERR_INVALID_ARG


def dummy_ptr():
    return ctypes.c_void_p(0x1000)


def test_invalid_arguments_are_rejected_without_cuda(L):
    g = L.fbp_geometry_default(10, 16, 16)
    p = dummy_ptr()
    # NULL geometry
    assert L.fbp_filter(p, p, None, 0, 0, None, 1, None) == _lib.FBP_ERR_INVALID_ARG
    assert "NULL" in L.fbp_last_error_message().decode()
    # bad dtype / kind
    assert L.fbp_filter(p, dummy_ptr(), None, 7, 0, ctypes.byref(g), 1, None) == _lib.FBP_ERR_INVALID_ARG
    assert L.fbp_filter(p, dummy_ptr(), None, 0, 9, ctypes.byref(g), 1, None) == _lib.FBP_ERR_INVALID_ARG
    # 16-bit without row_scale
    assert L.fbp_filter(p, ctypes.c_void_p(0x9000000), None, 1, 0, ctypes.byref(g), 1, None) == _lib.FBP_ERR_INVALID_ARG
    # NULL data
    assert L.fbp_backproject(None, None, 0, p, ctypes.byref(g), 1, 1.0, 0, None) == _lib.FBP_ERR_INVALID_ARG
    assert L.radon_forward(p, None, ctypes.byref(g), 1, None) == _lib.FBP_ERR_INVALID_ARG
    # aliasing
    assert L.fbp_filter(p, p, None, 0, 0, ctypes.byref(g), 1, None) == _lib.FBP_ERR_INVALID_ARG
    # negative slice count; zero slices is a no-op
    assert L.fbp_backproject(p, None, 0, p, ctypes.byref(g), -1, 1.0, 0, None) == _lib.FBP_ERR_INVALID_ARG
    assert L.radon_forward(p, dummy_ptr(), ctypes.byref(g), 0, None) == 0
    # geometry limits
    bad = L.fbp_geometry_default(10, 16, 16)
    bad.det_spacing = 0.0
    assert L.fbp_backproject(p, None, 0, ctypes.c_void_p(0x9000000), ctypes.byref(bad), 1, 1.0, 0, None) == _lib.FBP_ERR_INVALID_ARG
    wide = L.fbp_geometry_default(10, 9000, 16)
    assert L.fbp_filter(p, ctypes.c_void_p(0x90000000), None, 0, 0, ctypes.byref(wide), 1, None) == _lib.FBP_ERR_UNSUPPORTED
    fine = L.fbp_geometry_default(10, 16, 16)
    fine.pixel_size = 3.0
    assert L.radon_forward(p, ctypes.c_void_p(0x9000000), ctypes.byref(fine), 1, None) == _lib.FBP_ERR_UNSUPPORTED
    nan = L.fbp_geometry_default(10, 16, 16)
    nan.det_center = float("nan")
    assert L.radon_forward(p, ctypes.c_void_p(0x9000000), ctypes.byref(nan), 1, None) == _lib.FBP_ERR_INVALID_ARG
    # bad variant
    assert L.fbp_backproject_variant(p, None, 0, ctypes.c_void_p(0x9000000), ctypes.byref(g), 1, 1.0, 0, 99, None) == _lib.FBP_ERR_INVALID_ARG
    # forward-projector variants: range, and the tile-owned form's pixel/bin ratio
    nf = L.radon_forward_variant_count()
    assert nf == 6
    for v in (-2, nf):
        assert L.radon_forward_variant(p, dummy_ptr(), ctypes.byref(g), 0, v, None) == _lib.FBP_ERR_INVALID_ARG
    half = L.fbp_geometry_default(10, 16, 16)
    half.pixel_size = 0.5
    for v in range(1, nf):
        assert L.radon_forward_variant(p, dummy_ptr(), ctypes.byref(half), 0, v, None) == _lib.FBP_ERR_UNSUPPORTED
    assert L.radon_forward_variant(p, dummy_ptr(), ctypes.byref(half), 0, 0, None) == 0
    assert L.radon_forward_variant(p, dummy_ptr(), ctypes.byref(half), 0, -1, None) == 0


def test_pipeline_entry_points_validate_on_the_host(L):
    """fbp_filter_counts / fbp_hu_coefficients / fbp_backproject_u16 reject
    bad arguments before any CUDA call."""
    g = L.fbp_geometry_default(10, 16, 16)
    p = dummy_ptr()
    ok = _lib.CPreprocess(None, 1e4, 1.0, 16.0, 1.0)
    assert L.fbp_filter_counts(p, dummy_ptr(), None, 0, 0, ctypes.byref(g), 1, None, None) == _lib.FBP_ERR_INVALID_ARG
    for bad in (_lib.CPreprocess(None, 0.0, 1.0, 16.0, 0.0), _lib.CPreprocess(None, 1e4, 0.0, 16.0, 0.0),
                _lib.CPreprocess(None, 1e4, 1.0, -1.0, 0.0), _lib.CPreprocess(None, 1e4, 1.0, 16.0, 3.9),
                _lib.CPreprocess(None, 1e4, 1.0, float("nan"), 0.0)):
        assert L.fbp_filter_counts(p, dummy_ptr(), None, 0, 0, ctypes.byref(g), 1, ctypes.byref(bad), None) == _lib.FBP_ERR_INVALID_ARG
    assert L.fbp_filter_counts(p, dummy_ptr(), None, 0, 0, ctypes.byref(g), 0, ctypes.byref(ok), None) == 0
    a, b = ctypes.c_float(), ctypes.c_float()
    w = _lib.CHuWindow(0.5, 0.0, -1000.0, 3000.0)
    assert L.fbp_hu_coefficients(ctypes.byref(w), ctypes.byref(a), ctypes.byref(b)) == 0
    assert a.value == pytest.approx(1000.0 / 0.5 * 65535.0 / 4000.0, rel=1e-7) and b.value == 0.0
    for bad in (_lib.CHuWindow(0.5, 0.5, -1000.0, 3000.0), _lib.CHuWindow(0.5, 0.0, 5.0, 5.0),
                _lib.CHuWindow(float("inf"), 0.0, -1000.0, 3000.0)):
        assert L.fbp_hu_coefficients(ctypes.byref(bad), ctypes.byref(a), ctypes.byref(b)) == _lib.FBP_ERR_INVALID_ARG
        assert L.fbp_backproject_u16(p, None, 0, dummy_ptr(), ctypes.byref(g), 1, 1.0, ctypes.byref(bad), -1, None) == _lib.FBP_ERR_INVALID_ARG
    assert L.fbp_hu_coefficients(None, ctypes.byref(a), ctypes.byref(b)) == _lib.FBP_ERR_INVALID_ARG
    assert L.fbp_backproject_u16(p, None, 0, None, ctypes.byref(g), 1, 1.0, ctypes.byref(w), -1, None) == _lib.FBP_ERR_INVALID_ARG
    assert L.fbp_backproject_u16(p, None, 0, dummy_ptr(), ctypes.byref(g), 0, 1.0, ctypes.byref(w), -1, None) == 0


def test_libraries_resolve_every_symbol_at_load(L):
    """Both shared libraries load with immediate binding: no function the
    translation units call on one another is left undefined (a lazy load
    would only fail at the first call of the missing function, on a GPU)."""
    from paper_2505_13955_gb300 import build
    for name in ("libfbp.so", "libfbp_checked.so"):
        ctypes.CDLL(os.path.join(build.HERE, name), mode=os.RTLD_NOW)


def test_batched_workspace_query_and_validation(L):
    items = (_lib.CBatchItem * 3)()
    dims = [(720, 512, 512), (1800, 1024, 1024), (3600, 2048, 2048)]
    for i, (K, D, N) in enumerate(dims):
        items[i].sino = 0x1000 * (i + 1)
        items[i].slice = 0x100000 * (i + 1)
        items[i].g = L.fbp_geometry_default(K, D, N)
    n32 = L.fbp_batched_workspace_bytes(items, 3, 0)
    n16 = L.fbp_batched_workspace_bytes(items, 3, 1)
    # counters, then per item its rows, (16-bit) row scales and padded table,
    # then (16-bit) one S per item
    for i in range(3):
        assert L.fbp_batched_item_staged(ctypes.byref(items[i].g), 0) == 1
    t32 = [staged_table_bytes(K, D, N, f32=True) for K, D, N in dims]
    t16 = [staged_table_bytes(K, D, N, f32=False) for K, D, N in dims]
    assert n32 == 256 + sum(align256(K * D * 4) + t for (K, D, _), t in zip(dims, t32))
    assert n16 == 256 + sum(align256(K * D * 2) + align256(K * 4) + t for (K, D, _), t in zip(dims, t16)) + 256
    # the tables: between the unpadded K/2 x (D + 1) entries and the rows' 6x
    for (K, D, N), t in zip(dims, t32):
        assert K // 2 * (D + 1) * 32 <= t <= 6 * K * D * 4
    # items without staged units keep the rows-only layout
    for i, (K, D, N) in enumerate(dims):
        items[i].g = L.fbp_geometry_default(K + 1, D, N)          # odd K: no orbit symmetry
        assert L.fbp_batched_item_staged(ctypes.byref(items[i].g), 0) == 0
    raw32 = sum(align256((K + 1) * D * 4) for K, D, _ in dims)
    assert L.fbp_batched_workspace_bytes(items, 3, 0) == 256 + raw32
    for i, (K, D, N) in enumerate(dims):
        items[i].g = L.fbp_geometry_default(K, D, N)
    # a window wider than 72 entries (pixel / bin ratio 1.6), and no geometry
    wide = L.fbp_geometry_default(720, 512, 512)
    wide.pixel_size = 1.6
    assert L.fbp_batched_item_staged(ctypes.byref(wide), 0) == 0
    wide.pixel_size = 1.45                                     # FP32 rows: 32 x 32 tiles, window 69
    assert L.fbp_batched_item_staged(ctypes.byref(wide), 0) == 1
    assert L.fbp_batched_item_staged(ctypes.byref(wide), 1) == 0   # 16-bit: 64 x 64 tiles, window 133
    wide.pixel_size = 1.05
    assert L.fbp_batched_item_staged(ctypes.byref(wide), 1) == 1   # window 99
    odd = L.fbp_geometry_default(720, 512, 576)                # n = 9 x 64: FP32 only
    assert L.fbp_batched_item_staged(ctypes.byref(odd), 0) == 1
    assert L.fbp_batched_item_staged(ctypes.byref(odd), 2) == 0
    assert L.fbp_batched_item_staged(None, 0) == 0
    # count limits and NULL pointers
    assert L.fbp_batched_workspace_bytes(items, 0, 0) == 0
    assert L.fbp_batched_workspace_bytes(items, 257, 0) == 0
    items[1].sino = None
    assert L.fbp_batched_workspace_bytes(items, 3, 0) == 0
    items[1].sino = 0x2000
    # workspace checks happen before any launch
    assert L.fbp_batched(items, 3, 0, 0, -1, None, 0, None) == _lib.FBP_ERR_WORKSPACE
    assert L.fbp_batched(items, 3, 0, 0, -1, ctypes.c_void_p(0x10010), n32, None) == _lib.FBP_ERR_WORKSPACE
    assert L.fbp_batched(items, 3, 0, 0, -1, ctypes.c_void_p(0x10000), n32 - 256, None) == _lib.FBP_ERR_WORKSPACE
    assert L.fbp_batched(items, 3, 5, 0, -1, ctypes.c_void_p(0x10000), n32, None) == _lib.FBP_ERR_INVALID_ARG


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(_lib, "HERE", str(tmp_path))
    monkeypatch.setattr(_lib, "_libs", {})
    with pytest.raises(RuntimeError, match="not built"):
        _lib.load()


def test_binding_exposes_its_public_calls():
    """The Python binding keeps one function per C entry point it wraps."""
    from paper_2505_13955_gb300 import api
    for name in ("filter", "filter_counts", "filter_offset", "backproject", "backproject_u16", "backproject_staged",
                 "backproject_staged_u16",
                 "backproject_staged_workspace_bytes", "radon_forward", "fbp", "fbp_offset", "fbp_counts", "fbp_host",
                 "host_workspace_bytes", "fbp_batched", "fbp_batched_scans", "sap_edges", "sap_patches",
                 "sap_depatch_pack", "sap_host", "prepare", "device_status", "release_tables",
                 "measure_onchip_peaks", "lsq_refine", "radon", "radon_t"):
        assert callable(getattr(api, name, None)), name
