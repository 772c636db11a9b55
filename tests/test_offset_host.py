"""Offset-scan host logic of the C ABI on a CPU-only host: the virtual
detector fbp_offset_geometry derives (Sec. V-A(b), offset scans) equals the
oracle's, and bad arguments are rejected before any CUDA call."""
import ctypes
import math

import pytest

import oracle
from batch_layout import align256, staged_table_bytes
from paper_2505_13955_gb300 import _lib


@pytest.fixture(scope="module")
def L():
    from paper_2505_13955_gb300 import build
    build.build_cuda()
    return _lib.load()


def scan(L, K, D, n, c, full=True):
    g = L.fbp_geometry_default(K, D, n)
    g.angle_step = (2 * math.pi if full else math.pi) / K
    g.det_center = c
    return g


@pytest.mark.parametrize("D,c,delta,fold", [(64, 10.0, 6.0, 1), (65, 50.5, 8.0, 0), (101, 50.0, 20.0, 1),
                                             (300, 31.5, 31.5, 1), (4608, 511.5, 256.0, 1),
                                             (80, 15.5, 12.0, 0)])
def test_virtual_geometry_matches_the_oracle(L, D, c, delta, fold):
    K, n = 360, 128
    g = scan(L, K, D, n, c)
    gv = _lib.CGeometry()
    off = ctypes.c_int(-1)
    o = _lib.COffsetScan(delta, fold)
    assert L.fbp_offset_geometry(ctypes.byref(g), ctypes.byref(o), ctypes.byref(gv), ctypes.byref(off)) == 0
    n_v, c_v, off_o, _ = oracle.offset_virtual(D, c, delta)
    assert (gv.n_det, gv.det_center, off.value) == (n_v, c_v, off_o)
    assert gv.n_angles == (K // 2 if fold else K) and gv.n == n
    assert gv.angle_step == g.angle_step and gv.angle_start == g.angle_start
    assert gv.det_spacing == g.det_spacing and gv.pixel_size == g.pixel_size
    # the offset pointer is optional
    assert L.fbp_offset_geometry(ctypes.byref(g), ctypes.byref(o), ctypes.byref(gv), None) == 0


def test_offset_geometry_rejects_bad_scans(L):
    gv = _lib.CGeometry()
    ok = _lib.COffsetScan(6.0, 1)

    def st(g, o=ok):
        return L.fbp_offset_geometry(ctypes.byref(g), ctypes.byref(o), ctypes.byref(gv), None)

    assert L.fbp_offset_geometry(None, ctypes.byref(ok), ctypes.byref(gv), None) == _lib.FBP_ERR_INVALID_ARG
    assert st(scan(L, 360, 64, 64, 10.0, full=False)) == _lib.FBP_ERR_INVALID_ARG   # half turn
    assert "full turn" in L.fbp_last_error_message().decode()
    assert st(scan(L, 361, 64, 64, 10.0)) == _lib.FBP_ERR_INVALID_ARG               # odd K with fold
    assert st(scan(L, 361, 64, 64, 10.0), _lib.COffsetScan(6.0, 0)) == 0            # ... fine unfolded
    assert st(scan(L, 360, 64, 64, 10.25)) == _lib.FBP_ERR_INVALID_ARG              # not a half bin
    assert st(scan(L, 360, 64, 64, -1.0)) == _lib.FBP_ERR_INVALID_ARG               # axis off the detector
    assert st(scan(L, 360, 64, 64, 10.0), _lib.COffsetScan(10.5, 1)) == _lib.FBP_ERR_INVALID_ARG  # > short side
    assert st(scan(L, 360, 64, 64, 10.0), _lib.COffsetScan(0.0, 1)) == _lib.FBP_ERR_INVALID_ARG
    assert st(scan(L, 360, 64, 64, 10.0), _lib.COffsetScan(float("nan"), 1)) == _lib.FBP_ERR_INVALID_ARG
    assert st(scan(L, 360, 64, 64, 10.0), _lib.COffsetScan(6.0, 2)) == _lib.FBP_ERR_INVALID_ARG
    assert st(scan(L, 360, 6000, 64, 100.0)) == _lib.FBP_ERR_UNSUPPORTED            # n_v > 8192


def test_filter_offset_validates_before_any_cuda_call(L):
    p = ctypes.c_void_p(0x1000)
    g = scan(L, 360, 64, 64, 10.0)
    o = _lib.COffsetScan(6.0, 1)
    assert L.fbp_filter_offset(p, p, None, 0, 0, ctypes.byref(g), 1, None, None) == _lib.FBP_ERR_INVALID_ARG
    assert L.fbp_filter_offset(None, p, None, 0, 0, ctypes.byref(g), 1, ctypes.byref(o), None) == \
        _lib.FBP_ERR_INVALID_ARG
    assert L.fbp_filter_offset(p, ctypes.c_void_p(0x2000), None, 1, 0, ctypes.byref(g), 1, ctypes.byref(o),
                               None) == _lib.FBP_ERR_INVALID_ARG          # 16-bit without row_scale
    assert L.fbp_filter_offset(p, ctypes.c_void_p(0x2000), None, 0, 5, ctypes.byref(g), 1, ctypes.byref(o),
                               None) == _lib.FBP_ERR_INVALID_ARG          # bad kind
    assert L.fbp_filter_offset(p, ctypes.c_void_p(0x1004), None, 0, 0, ctypes.byref(g), 1, ctypes.byref(o),
                               None) == _lib.FBP_ERR_INVALID_ARG          # filt overlaps sino
    assert "overlaps" in L.fbp_last_error_message().decode()
    assert L.fbp_filter_offset(p, p, None, 0, 0, ctypes.byref(g), 0, ctypes.byref(o), None) == 0  # nothing to do


def test_batched_scans_validate_before_any_cuda_call(L):
    g = scan(L, 360, 64, 64, 10.0)
    items = (_lib.CScanItem * 2)()
    for it in items:
        it.sino, it.slice, it.g, it.overlap, it.fold = 0x1000, 0x2000, g, 6.0, 1
    items[1].g = L.fbp_geometry_default(90, 64, 64)
    items[1].overlap = 0.0
    n = L.fbp_batched_scans_workspace_bytes(items, 2, 0)
    # counter block, then 180 folded rows of the virtual detector and their
    # padded table (a centred half turn: staged units), then 90 x 64 rows
    # and theirs
    n_v, c_v = oracle.offset_virtual(64, 10.0, 6.0)[:2]
    assert n_v == 107
    gv = _lib.CGeometry()
    off = ctypes.c_int(0)
    o = _lib.COffsetScan(6.0, 1)
    assert L.fbp_offset_geometry(ctypes.byref(items[0].g), ctypes.byref(o), ctypes.byref(gv), ctypes.byref(off)) == 0
    assert L.fbp_batched_item_staged(ctypes.byref(gv), 0) == 1
    t0 = staged_table_bytes(180, n_v, 64, det_center=c_v, angle_step=2 * math.pi / 360)
    t1 = staged_table_bytes(90, 64, 64)
    assert t0 > 0 and t1 > 0
    assert n == 256 + align256(180 * n_v * 4) + t0 + 90 * 64 * 4 + t1
    ws = ctypes.c_void_p(0x100000)
    assert L.fbp_batched_scans(items, 2, 0, 0, -1, 7, ws, n, None) == _lib.FBP_ERR_INVALID_ARG   # order
    assert L.fbp_batched_scans(items, 2, 0, 0, -1, 1, ws, n - 1, None) == _lib.FBP_ERR_WORKSPACE
    items[0].overlap = 20.0                                                   # > short side
    assert L.fbp_batched_scans(items, 2, 0, 0, -1, 1, ws, n, None) == _lib.FBP_ERR_INVALID_ARG
    assert "item 0" in L.fbp_last_error_message().decode()
    assert L.fbp_batched_scans_workspace_bytes(items, 2, 0) == 0
    items[0].overlap = 6.0
    items[1].sino = None
    assert L.fbp_batched_scans(items, 2, 0, 0, -1, 0, ws, n, None) == _lib.FBP_ERR_INVALID_ARG
    assert L.fbp_batched_scans(None, 2, 0, 0, -1, 0, ws, n, None) == _lib.FBP_ERR_INVALID_ARG
