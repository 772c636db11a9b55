"""SAP entry points (include/sap.h) on a CPU-only host: parameter and
workspace validation before any CUDA call, and the workspace size."""
import ctypes

import pytest

from paper_2505_13955_gb300 import _lib


@pytest.fixture(scope="module")
def L():
    from paper_2505_13955_gb300 import build
    build.build_cuda()
    return _lib.load()


def params(n=256, patch=16, length=22, lo=10, hi=20):
    return _lib.CSapParams(n, patch, length, lo, hi)


@pytest.mark.parametrize("bad", [dict(n=100), dict(n=8), dict(n=32768), dict(patch=12), dict(patch=2),
                                 dict(n=16, patch=32, length=1), dict(length=23), dict(length=0),
                                 dict(length=257), dict(lo=-1), dict(lo=30, hi=20)])
def test_bad_parameters_are_rejected(L, bad):
    p = params(**bad)
    assert L.sap_workspace_bytes(ctypes.byref(p)) == 0
    q = ctypes.c_void_p(0x1000)
    ws = ctypes.c_void_p(0x100000)
    assert L.sap_edges(q, q, ctypes.byref(p), ws, 1 << 30, None) == _lib.FBP_ERR_INVALID_ARG
    assert L.sap_patches(q, q, q, q, ctypes.byref(p), ws, 1 << 30, None) == _lib.FBP_ERR_INVALID_ARG
    assert L.sap_depatch_pack(q, q, q, ctypes.byref(p), None) == _lib.FBP_ERR_INVALID_ARG


def test_workspace_size_and_checks(L):
    p = params(n=256, patch=16, length=256)          # 16 x 16 patches, every node split
    need = L.sap_workspace_bytes(ctypes.byref(p))
    n2 = 256 * 256
    assert need >= n2 * 5                            # labels + classes for the edges
    nodes = (4 ** 5 - 1) // 3                        # levels 0..4 (side 256 .. 16)
    assert need >= nodes * 28
    q = ctypes.c_void_p(0x1000)
    ws = ctypes.c_void_p(0x100000)
    assert L.sap_edges(q, q, ctypes.byref(p), None, need, None) == _lib.FBP_ERR_WORKSPACE
    assert L.sap_edges(q, q, ctypes.byref(p), ctypes.c_void_p(0x100010), need, None) == _lib.FBP_ERR_WORKSPACE
    assert L.sap_edges(q, q, ctypes.byref(p), ws, need - 1, None) == _lib.FBP_ERR_WORKSPACE
    assert L.sap_patches(q, q, None, q, ctypes.byref(p), ws, need, None) == _lib.FBP_ERR_INVALID_ARG
    assert L.sap_edges(None, q, ctypes.byref(p), ws, need, None) == _lib.FBP_ERR_INVALID_ARG
    assert L.sap_edges(q, q, None, ws, need, None) == _lib.FBP_ERR_INVALID_ARG


def test_host_stack_call_checks_its_arguments():
    """sap_host validates the host stack before touching a device."""
    import torch
    from paper_2505_13955_gb300 import api
    p = api.SapParams(64, 8, 10, 1, 2)
    with pytest.raises(ValueError):
        api.sap_host(torch.zeros((2, 64, 64), dtype=torch.int32), p)
    with pytest.raises(ValueError):
        api.sap_host(torch.zeros((2, 64, 32), dtype=torch.int16), p)
    with pytest.raises(ValueError):
        api.sap_host(torch.zeros((64, 64), dtype=torch.int16), p)
    with pytest.raises(ValueError):
        api.sap_host(torch.zeros((2, 64, 128), dtype=torch.int16)[:, :, ::2], p)
