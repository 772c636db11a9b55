"""Shared helpers for the GPU parity tests."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

needs_gpu = pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")


def fbp_api():
    from paper_2505_13955_gb300 import api
    return api


def to_gpu(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def to_np(t):
    return t.detach().float().cpu().numpy().astype(np.float64)


def dyn_range(a):
    return float(np.max(a) - np.min(a))


def assert_within_dr(gpu, ref, frac, what=""):
    """max |gpu - ref| <= frac * (max(ref) - min(ref)); when the reference is
    constant (a single pixel, say) its magnitude stands in for the range."""
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    dr = dyn_range(ref) if ref.size else 0.0
    if dr == 0.0 and ref.size:
        dr = float(np.max(np.abs(ref)))
    err = float(np.max(np.abs(gpu - ref))) if ref.size else 0.0
    assert err <= frac * dr + 1e-30, f"{what}: max abs err {err:.3e} > {frac:g} x DR {dr:.3e}"
    return err / dr if dr else 0.0


def geometries(api, oracle_mod, K, D, N, **kw):
    return api.Geometry(K, D, N, **kw), oracle_mod.Geometry(K, D, N, **kw)
