"""Python binding of libfbp.so: same names as the C ABI, torch tensors in/out.

PyTorch provides device memory and streams; every step of the computation
runs in the library's CUDA kernels.  Tensors must be contiguous CUDA tensors
of the stated dtypes; results are enqueued on the current torch stream.

  filter(sino, g)            -> fbp_filter       (K1, FFT ramp filter)
  backproject(filt, g)       -> fbp_backproject  (K2, pixel-driven, linear interp.)
  radon_forward(img, g)      -> radon_forward    (K3, matched forward projector)
  fbp(sino, g)               -> fbp_filter + fbp_backproject
  fbp_batched(sinos, gs)     -> fbp_batched      (ragged batch, persistent launch)
  filter_offset(sino, g, ..) -> fbp_filter_offset (full-turn offset scans)
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass

import torch

from . import _lib

_DTYPES = {torch.float32: _lib.FBP_F32, torch.float16: _lib.FBP_F16, torch.bfloat16: _lib.FBP_BF16}
_KINDS = {"ramlak": _lib.FBP_FILTER_RAMLAK, "ram-lak": _lib.FBP_FILTER_RAMLAK,
          "shepp_logan": _lib.FBP_FILTER_SHEPP_LOGAN, "shepp-logan": _lib.FBP_FILTER_SHEPP_LOGAN}

FbpError = _lib.FbpError


@dataclass
class Geometry:
    """Parallel-beam geometry of a slice (mirrors ``fbp_geometry``).

    Angles th_k = angle_start + k * angle_step (default k*pi/K on [0, pi)),
    detector centre det_center (default (D-1)/2), bin width det_spacing,
    pixel width pixel_size.  Pixel [r][c] sits at X = c-(n-1)/2, Y = r-(n-1)/2.
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
            self.angle_step = math.pi / self.n_angles if self.n_angles > 0 else 0.0
        if self.det_center is None:
            self.det_center = 0.5 * (self.n_det - 1)

    def c(self) -> _lib.CGeometry:
        return _lib.CGeometry(int(self.n_angles), int(self.n_det), int(self.n),
                              float(self.angle_start), float(self.angle_step),
                              float(self.det_center), float(self.det_spacing),
                              float(self.pixel_size))


def lib(which: str = "default"):
    return _lib.load(which)


def _stream(device) -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _ptr(t: torch.Tensor | None) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr() if t is not None else None)


def _need(t: torch.Tensor, name: str, dtype=None):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor (there is no CPU path)")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must have dtype {dtype}, got {t.dtype}")


def _slices(t: torch.Tensor, tail: tuple[int, ...], name: str) -> int:
    if t.dim() == len(tail):
        if tuple(t.shape) != tail:
            raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tail}")
        return 1
    if t.dim() == len(tail) + 1 and tuple(t.shape[1:]) == tail:
        return int(t.shape[0])
    raise ValueError(f"{name} has shape {tuple(t.shape)}, expected [S, {', '.join(map(str, tail))}]")


def kind_id(kind) -> int:
    if isinstance(kind, int):
        return kind
    return _KINDS[kind.lower()]


def filter(sino: torch.Tensor, g: Geometry, kind="ramlak", dtype=torch.float32,
           out: torch.Tensor | None = None, row_scale: torch.Tensor | None = None,
           which: str = "default"):
    """fbp_filter: ramp-filter every row.  Returns (filt, row_scale or None)."""
    _need(sino, "sino", torch.float32)
    S = _slices(sino, (g.n_angles, g.n_det), "sino")
    if out is None:
        out = torch.empty(sino.shape, dtype=dtype, device=sino.device)
    _need(out, "out", dtype)
    if dtype != torch.float32 and row_scale is None:
        row_scale = torch.empty(sino.shape[:-1], dtype=torch.float32, device=sino.device)
    L = lib(which)
    gc = g.c()
    st = L.fbp_filter(_ptr(sino), _ptr(out), _ptr(row_scale), _DTYPES[dtype], kind_id(kind),
                      ctypes.byref(gc), S, _stream(sino.device))
    _lib.check(st, L, "fbp_filter")
    return out, (row_scale if dtype != torch.float32 else None)


@dataclass
class Preprocess:
    """Stage-2 pre-processing for fbp_filter_counts: p = mu_scale * -ln(max(I,
    count_floor) / I0) (I0 = `flat` per bin, or `flat_value`), then a Gaussian
    blur of width blur_sigma bins along the detector."""
    flat_value: float = 1.0
    flat: torch.Tensor | None = None
    count_floor: float = 1.0
    mu_scale: float = 1.0
    blur_sigma: float = 0.0

    def c(self):
        if self.flat is not None:
            _need(self.flat, "flat", torch.float32)
        return _lib.CPreprocess(_ptr(self.flat) if self.flat is not None else None,
                                float(self.flat_value), float(self.count_floor),
                                float(self.mu_scale), float(self.blur_sigma))


@dataclass
class HuWindow:
    """Stage-4 mapping: HU = 1000 (mu - mu_water) / (mu_water - mu_air), the
    window [hu_min, hu_max] onto uint16 codes [0, 65535]."""
    mu_water: float
    mu_air: float = 0.0
    hu_min: float = -1000.0
    hu_max: float = 3000.0

    def c(self):
        return _lib.CHuWindow(float(self.mu_water), float(self.mu_air), float(self.hu_min),
                              float(self.hu_max))


def filter_counts(counts: torch.Tensor, g: Geometry, pre: Preprocess, kind="ramlak",
                  dtype=torch.float32, out: torch.Tensor | None = None,
                  row_scale: torch.Tensor | None = None, which: str = "default"):
    """fbp_filter_counts: Beer-Lambert + blur + ramp filter from detector
    counts in one pass.  Returns (filt, row_scale or None)."""
    _need(counts, "counts", torch.float32)
    S = _slices(counts, (g.n_angles, g.n_det), "counts")
    if out is None:
        out = torch.empty(counts.shape, dtype=dtype, device=counts.device)
    _need(out, "out", dtype)
    if dtype != torch.float32 and row_scale is None:
        row_scale = torch.empty(counts.shape[:-1], dtype=torch.float32, device=counts.device)
    L = lib(which)
    gc, pc = g.c(), pre.c()
    st = L.fbp_filter_counts(_ptr(counts), _ptr(out), _ptr(row_scale), _DTYPES[dtype], kind_id(kind),
                             ctypes.byref(gc), S, ctypes.byref(pc), _stream(counts.device))
    _lib.check(st, L, "fbp_filter_counts")
    return out, (row_scale if dtype != torch.float32 else None)


def hu_coefficients(w: HuWindow, which: str = "default"):
    """The FP32 (a, b) of code = clamp(rint(RN(RN(a mu) + b)), 0, 65535)."""
    L = lib(which)
    wc = w.c()
    a, b = ctypes.c_float(), ctypes.c_float()
    _lib.check(L.fbp_hu_coefficients(ctypes.byref(wc), ctypes.byref(a), ctypes.byref(b)), L,
               "fbp_hu_coefficients")
    return a.value, b.value


def backproject_u16(filt: torch.Tensor, g: Geometry, window: HuWindow,
                    row_scale: torch.Tensor | None = None, scale: float | None = None,
                    out: torch.Tensor | None = None, variant: int = -1, which: str = "default"):
    """fbp_backproject_u16: backprojection with the HU window quantised to
    uint16 in the epilogue.  Returns an int16-typed tensor holding the uint16
    codes' bit patterns (``.view(torch.uint16)`` / ``.numpy().view('u2')``)."""
    _need(filt, "filt")
    if filt.dtype not in _DTYPES:
        raise ValueError(f"unsupported filt dtype {filt.dtype}")
    S = _slices(filt, (g.n_angles, g.n_det), "filt")
    shape = (g.n, g.n) if filt.dim() == 2 else (S, g.n, g.n)
    if out is None:
        out = torch.empty(shape, dtype=torch.int16, device=filt.device)
    _need(out, "out", torch.int16)
    if tuple(out.shape) != shape:
        raise ValueError(f"out has shape {tuple(out.shape)}, expected {shape}")
    if row_scale is not None:
        _need(row_scale, "row_scale", torch.float32)
    if scale is None:
        scale = g.angle_step
    L = lib(which)
    gc, wc = g.c(), window.c()
    st = L.fbp_backproject_u16(_ptr(filt), _ptr(row_scale), _DTYPES[filt.dtype], _ptr(out),
                               ctypes.byref(gc), S, float(scale), ctypes.byref(wc), int(variant),
                               _stream(filt.device))
    _lib.check(st, L, "fbp_backproject_u16")
    return out


def fbp_counts(counts: torch.Tensor, g: Geometry, pre: Preprocess, window: HuWindow | None = None,
               kind="ramlak", dtype=torch.float32, variant: int = -1):
    """The fused reconstruction of Sec. V-A(c) stages 2 and 4: detector counts
    in, FP32 attenuation (window None) or uint16 HU codes out."""
    filt, rs = filter_counts(counts, g, pre, kind=kind, dtype=dtype)
    staged = variant < 0 and staged_preferred(g)
    S = 1 if counts.dim() == 2 else counts.shape[0]
    if window is None:
        if staged:
            return backproject_staged(filt, g, rs, chunk=staged_chunk(g, dtype, S))
        return backproject(filt, g, row_scale=rs, variant=variant)
    if staged:
        return backproject_staged_u16(filt, g, window, row_scale=rs, chunk=staged_chunk(g, dtype, S))
    return backproject_u16(filt, g, window, row_scale=rs, variant=variant)


def offset_geometry(g: Geometry, overlap: float, fold: bool = True, which: str = "default"):
    """fbp_offset_geometry: (virtual geometry of the filtered rows, virtual
    index of physical bin 0) for a full-turn offset scan with geometry g."""
    L = lib(which)
    gc, oc, gv = g.c(), _lib.COffsetScan(float(overlap), int(bool(fold))), _lib.CGeometry()
    off = ctypes.c_int(0)
    _lib.check(L.fbp_offset_geometry(ctypes.byref(gc), ctypes.byref(oc), ctypes.byref(gv),
                                     ctypes.byref(off)), L, "fbp_offset_geometry")
    return Geometry(gv.n_angles, gv.n_det, gv.n, gv.angle_start, gv.angle_step, gv.det_center,
                    gv.det_spacing, gv.pixel_size), int(off.value)


def filter_offset(sino: torch.Tensor, g: Geometry, overlap: float, fold: bool = True, kind="ramlak",
                  dtype=torch.float32, out: torch.Tensor | None = None,
                  row_scale: torch.Tensor | None = None, which: str = "default"):
    """fbp_filter_offset: weight, embed (and fold) the rows of a full-turn
    offset scan and filter them on the virtual detector.  Returns
    (filt, row_scale or None, virtual geometry)."""
    _need(sino, "sino", torch.float32)
    S = _slices(sino, (g.n_angles, g.n_det), "sino")
    gv, _ = offset_geometry(g, overlap, fold, which)
    shape = (gv.n_angles, gv.n_det) if sino.dim() == 2 else (S, gv.n_angles, gv.n_det)
    if out is None:
        out = torch.empty(shape, dtype=dtype, device=sino.device)
    _need(out, "out", dtype)
    if tuple(out.shape) != shape:
        raise ValueError(f"out has shape {tuple(out.shape)}, expected {shape}")
    if dtype != torch.float32 and row_scale is None:
        row_scale = torch.empty(shape[:-1], dtype=torch.float32, device=sino.device)
    L = lib(which)
    gc, oc = g.c(), _lib.COffsetScan(float(overlap), int(bool(fold)))
    st = L.fbp_filter_offset(_ptr(sino), _ptr(out), _ptr(row_scale), _DTYPES[dtype], kind_id(kind),
                             ctypes.byref(gc), S, ctypes.byref(oc), _stream(sino.device))
    _lib.check(st, L, "fbp_filter_offset")
    return out, (row_scale if dtype != torch.float32 else None), gv


def fbp_offset(sino: torch.Tensor, g: Geometry, overlap: float, fold: bool = True, kind="ramlak",
               dtype=torch.float32, out: torch.Tensor | None = None, variant: int = -1):
    """FBP of a full-turn offset scan: fbp_filter_offset, then fbp_backproject
    on the virtual geometry with scale = angle_step."""
    filt, rs, gv = filter_offset(sino, g, overlap, fold, kind=kind, dtype=dtype)
    if variant < 0 and staged_preferred(gv):
        # folded rows: a centred half turn, so the staged orbit path applies
        S = 1 if sino.dim() == 2 else sino.shape[0]
        return backproject_staged(filt, gv, rs, out=out, chunk=staged_chunk(gv, dtype, S))
    return backproject(filt, gv, row_scale=rs, out=out, variant=variant)


def backproject(filt: torch.Tensor, g: Geometry, row_scale: torch.Tensor | None = None,
                scale: float | None = None, out: torch.Tensor | None = None,
                accumulate: bool = False, variant: int = -1, which: str = "default"):
    """fbp_backproject: f = scale * sum_k Q_k(u_k) (scale defaults to angle_step).
    With the default variant, a geometry for which staged_preferred(g) holds
    takes fbp_backproject_staged (with tables for as many slices as
    staged_chunk allows, allocated per call), as fbp does."""
    _need(filt, "filt")
    if filt.dtype not in _DTYPES:
        raise ValueError(f"unsupported filt dtype {filt.dtype}")
    S = _slices(filt, (g.n_angles, g.n_det), "filt")
    shape = (g.n, g.n) if filt.dim() == 2 else (S, g.n, g.n)
    if out is None:
        out = (torch.zeros if accumulate else torch.empty)(shape, dtype=torch.float32,
                                                           device=filt.device)
    if variant < 0 and which == "default" and staged_preferred(g):
        return backproject_staged(filt, g, row_scale, scale=scale, out=out, accumulate=accumulate,
                                  chunk=staged_chunk(g, filt.dtype, S))
    _need(out, "out", torch.float32)
    if tuple(out.shape) != shape:
        raise ValueError(f"out has shape {tuple(out.shape)}, expected {shape}")
    if row_scale is not None:
        _need(row_scale, "row_scale", torch.float32)
    if scale is None:
        scale = g.angle_step
    L = lib(which)
    gc = g.c()
    st = L.fbp_backproject_variant(_ptr(filt), _ptr(row_scale), _DTYPES[filt.dtype], _ptr(out),
                                   ctypes.byref(gc), S, float(scale), int(bool(accumulate)),
                                   int(variant), _stream(filt.device))
    _lib.check(st, L, "fbp_backproject")
    return out


def backproject_staged_workspace_bytes(g: Geometry, dtype=torch.float16, chunk: int = 1) -> int:
    """fbp_backproject_staged_workspace_bytes: workspace for `chunk` slices at a time."""
    gc = g.c()
    n = lib().fbp_backproject_staged_workspace_bytes(ctypes.byref(gc), _DTYPES[dtype], int(chunk))
    if n == 0:
        raise FbpError(_lib.FBP_ERR_INVALID_ARG, "fbp_backproject_staged_workspace_bytes: invalid arguments")
    return int(n)


def staged_shape_count(dtype=torch.float16) -> int:
    return int(lib().fbp_backproject_staged_shape_count(_DTYPES[dtype]))


def backproject_staged(filt: torch.Tensor, g: Geometry, row_scale: torch.Tensor | None = None,
                       scale: float | None = None, out: torch.Tensor | None = None, accumulate: bool = False,
                       shape: int = -1, workspace: torch.Tensor | None = None, chunk: int = 1):
    """fbp_backproject_staged: backprojection from tables written once per
    slice (a workspace of `chunk` slices is allocated if none is given).
    16-bit rows (with their row_scale) are bit-identical to backproject with
    the packed orbit variant of the same tile."""
    _need(filt, "filt")
    if filt.dtype not in _DTYPES:
        raise ValueError(f"unsupported filt dtype {filt.dtype}")
    S = _slices(filt, (g.n_angles, g.n_det), "filt")
    if filt.dtype != torch.float32:
        if row_scale is None:
            raise ValueError("16-bit rows need their row_scale")
        _need(row_scale, "row_scale", torch.float32)
    shape_out = (g.n, g.n) if filt.dim() == 2 else (S, g.n, g.n)
    if out is None:
        out = torch.empty(shape_out, dtype=torch.float32, device=filt.device)
    _need(out, "out", torch.float32)
    if workspace is None:
        workspace = torch.empty(backproject_staged_workspace_bytes(g, filt.dtype, min(chunk, S)),
                                dtype=torch.uint8, device=filt.device)
    L = lib()
    gc = g.c()
    sc = g.angle_step if scale is None else scale
    st = L.fbp_backproject_staged(_ptr(filt), _ptr(row_scale if filt.dtype != torch.float32 else None),
                                  _DTYPES[filt.dtype], _ptr(out), ctypes.byref(gc), S, float(sc), int(accumulate),
                                  int(shape), _ptr(workspace), workspace.numel(), _stream(filt.device))
    _lib.check(st, L, "fbp_backproject_staged")
    return out


def backproject_staged_u16(filt: torch.Tensor, g: Geometry, window: HuWindow,
                           row_scale: torch.Tensor | None = None, scale: float | None = None,
                           out: torch.Tensor | None = None, shape: int = -1,
                           workspace: torch.Tensor | None = None, chunk: int = 1):
    """fbp_backproject_staged_u16: the staged backprojection with the HU window
    quantised to uint16 in the epilogue (int16-typed tensor of the codes)."""
    _need(filt, "filt")
    if filt.dtype not in _DTYPES:
        raise ValueError(f"unsupported filt dtype {filt.dtype}")
    S = _slices(filt, (g.n_angles, g.n_det), "filt")
    if filt.dtype != torch.float32:
        if row_scale is None:
            raise ValueError("16-bit rows need their row_scale")
        _need(row_scale, "row_scale", torch.float32)
    shape_out = (g.n, g.n) if filt.dim() == 2 else (S, g.n, g.n)
    if out is None:
        out = torch.empty(shape_out, dtype=torch.int16, device=filt.device)
    _need(out, "out", torch.int16)
    if workspace is None:
        workspace = torch.empty(backproject_staged_workspace_bytes(g, filt.dtype, min(chunk, S)),
                                dtype=torch.uint8, device=filt.device)
    L = lib()
    gc, wc = g.c(), window.c()
    sc = g.angle_step if scale is None else scale
    st = L.fbp_backproject_staged_u16(_ptr(filt), _ptr(row_scale if filt.dtype != torch.float32 else None),
                                      _DTYPES[filt.dtype], _ptr(out), ctypes.byref(gc), S, float(sc),
                                      ctypes.byref(wc), int(shape), _ptr(workspace), workspace.numel(),
                                      _stream(filt.device))
    _lib.check(st, L, "fbp_backproject_staged_u16")
    return out


def radon_forward(img: torch.Tensor, g: Geometry, out: torch.Tensor | None = None,
                  which: str = "default", variant: int = -1):
    """radon_forward: the matched projector A (transpose of backproject, scale 1).
    variant -1 = library default, 0 = deterministic gather, 1..5 = tile-owned
    (floating-point atomics across tiles; 4 and 5 take four / two slices per
    block)."""
    _need(img, "slice", torch.float32)
    S = _slices(img, (g.n, g.n), "slice")
    shape = (g.n_angles, g.n_det) if img.dim() == 2 else (S, g.n_angles, g.n_det)
    if out is None:
        out = torch.empty(shape, dtype=torch.float32, device=img.device)
    _need(out, "out", torch.float32)
    L = lib(which)
    gc = g.c()
    st = L.radon_forward_variant(_ptr(img), _ptr(out), ctypes.byref(gc), S, int(variant),
                                 _stream(img.device))
    _lib.check(st, L, "radon_forward")
    return out


def staged_supported(g: Geometry) -> bool:
    """Whether fbp_backproject_staged takes geometry g (the 90-degree orbit
    geometry: angle step pi/K with K even, centred detector, n a multiple of 64)."""
    return (g.n_angles % 2 == 0 and g.n % 64 == 0 and abs(g.angle_step * g.n_angles - math.pi) <= 1e-9 * math.pi
            and abs(g.det_center - 0.5 * (g.n_det - 1)) <= 1e-9 * (1 + g.n_det))


def staged_preferred(g: Geometry) -> bool:
    """Whether the default path takes fbp_backproject_staged: the orbit
    geometry and n >= 1024 (a small slice is launch-bound, and the extra table
    pass and its few orbits cost more than they save: 120 vs 176 Gupdates/s
    for one 256^2 slice, K = 360)."""
    return staged_supported(g) and g.n >= 1024


STAGED_TABLE_BUDGET = 2 << 30     # bytes of staged tables the default paths allocate at most


def staged_chunk(g: Geometry, dtype, S: int) -> int:
    """Slices per pass of the default paths' staged backprojection: every
    slice at once (one launch, no tail of a partly filled last wave) while
    their tables fit in STAGED_TABLE_BUDGET bytes, else as many as fit."""
    per = backproject_staged_workspace_bytes(g, dtype, 2) - backproject_staged_workspace_bytes(g, dtype, 1)
    return max(1, min(S, STAGED_TABLE_BUDGET // max(per, 1)))


def fbp(sino: torch.Tensor, g: Geometry, kind="ramlak", dtype=torch.float32,
        out: torch.Tensor | None = None, variant: int = -1):
    """Filtered backprojection: fbp_filter then fbp_backproject (scale =
    angle_step).  With the default variant, rows take fbp_backproject_staged
    where staged_preferred(g) (with tables for as many slices as staged_chunk
    allows, allocated per call)."""
    filt, rs = filter(sino, g, kind=kind, dtype=dtype)
    if variant < 0 and staged_preferred(g):
        S = 1 if sino.dim() == 2 else sino.shape[0]
        return backproject_staged(filt, g, rs, out=out, chunk=staged_chunk(g, dtype, S))
    return backproject(filt, g, row_scale=rs, out=out, variant=variant)


def host_workspace_bytes(g: Geometry, dtype=torch.float32, chunk: int = 2, n_streams: int = 3,
                         codes: bool = False) -> int:
    """fbp_host_workspace_bytes: device bytes fbp_host needs."""
    L = lib()
    gc = g.c()
    n = L.fbp_host_workspace_bytes(ctypes.byref(gc), _DTYPES[dtype], int(chunk), int(n_streams), int(codes))
    if n == 0:
        raise FbpError(_lib.FBP_ERR_INVALID_ARG, "fbp_host_workspace_bytes: invalid arguments")
    return int(n)


def fbp_host(sino: torch.Tensor, g: Geometry, kind="ramlak", dtype=torch.float32,
             out: torch.Tensor | None = None, variant: int = -1, chunk: int = 2,
             n_streams: int = 3, device=None, pre: "Preprocess | None" = None,
             window: "HuWindow | None" = None, workspace: torch.Tensor | None = None) -> torch.Tensor:
    """fbp_host: FBP of a stack held in host memory; returns (or fills) a host tensor.

    With `pre` the input is detector counts (fbp_filter_counts); with
    `window` the output is the uint16 HU codes (fbp_backproject_u16), held in
    an int16 tensor.  The C call cuts the stack into chunks of `chunk` slices
    on `n_streams` streams (copy in, filter, backproject, copy out), so the
    copies of one chunk overlap another's kernels; use pinned host tensors
    (``tensor.pin_memory()``) for that.  Blocks until the result is in `out`.
    """
    if sino.is_cuda:
        raise ValueError("fbp_host takes a host (CPU) tensor; use fbp for device tensors")
    if sino.dtype != torch.float32 or not sino.is_contiguous():
        raise ValueError("sino must be a contiguous float32 tensor")
    S = _slices(sino, (g.n_angles, g.n_det), "sino")
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    odt = torch.int16 if window is not None else torch.float32
    squeeze = sino.dim() == 2
    if out is None:
        out = torch.empty((S, g.n, g.n), dtype=odt, pin_memory=True)
    if out.is_cuda or out.dtype != odt or not out.is_contiguous() or out.numel() != S * g.n * g.n:
        raise ValueError(f"out must be a contiguous host {odt} tensor of {S} x {g.n} x {g.n}")
    chunk = max(1, min(chunk, S))
    n_streams = max(1, min(n_streams, -(-S // chunk)))
    if workspace is None:
        workspace = torch.empty(host_workspace_bytes(g, dtype, chunk, n_streams, window is not None),
                                dtype=torch.uint8, device=dev)
    L = lib()
    gc = g.c()
    pc = pre.c() if pre is not None else None
    wc = window.c() if window is not None else None
    with torch.cuda.device(dev):
        st = L.fbp_host(_ptr(sino), _ptr(out), ctypes.byref(gc), S, kind_id(kind), _DTYPES[dtype], int(variant),
                        ctypes.byref(pc) if pc is not None else None,
                        ctypes.byref(wc) if wc is not None else None, chunk, n_streams, _ptr(workspace),
                        workspace.numel(), _stream(dev))
    _lib.check(st, L, "fbp_host")
    return out[0] if squeeze and out.dim() == 3 else out


def forward_variant_count(which: str = "default") -> int:
    """Number of radon_forward kernels (0 = gather, 1..5 = tile-owned)."""
    return int(lib(which).radon_forward_variant_count())


def bp_variants() -> list[dict]:
    L = lib()
    out = []
    for v in range(L.fbp_bp_variant_count()):
        s = _lib.CBpShape()
        _lib.check(L.fbp_bp_variant_info(v, ctypes.byref(s)), L, "fbp_bp_variant_info")
        out.append({"variant": v, "angle_tile": s.angle_tile, "tile_x": s.tile_x,
                    "tile_y": s.tile_y, "px": s.px, "py": s.py, "threads": s.threads,
                    "symmetric": bool(s.symmetric), "packed16": bool(s.packed16),
                    "texture": bool(s.texture)})
    return out


def variant_supports(variant: int, g: Geometry, dtype=torch.float32) -> bool:
    """Whether fbp_backproject_variant accepts `variant` for rows of `dtype`
    and geometry g."""
    gc = g.c()
    return bool(lib().fbp_bp_variant_supports(int(variant), _DTYPES[dtype], ctypes.byref(gc)))


def batched_item_staged(g: Geometry, dtype=torch.float32) -> bool:
    """fbp_batched_item_staged: whether a batch item with rows of geometry g
    (an offset item's virtual geometry) runs staged units by default."""
    gc = g.c()
    return bool(lib().fbp_batched_item_staged(ctypes.byref(gc), _DTYPES[dtype]))


def _items(sinos, outs, geoms):
    arr = (_lib.CBatchItem * len(sinos))()
    for i, (s, o, g) in enumerate(zip(sinos, outs, geoms)):
        arr[i].sino = s.data_ptr()
        arr[i].slice = o.data_ptr()
        arr[i].g = g.c()
    return arr


def batched_workspace_bytes(sinos, outs, geoms, dtype=torch.float32) -> int:
    L = lib()
    n = L.fbp_batched_workspace_bytes(_items(sinos, outs, geoms), len(sinos), _DTYPES[dtype])
    if n == 0:
        raise FbpError(_lib.FBP_ERR_INVALID_ARG,
                       "fbp_batched_workspace_bytes: " + L.fbp_last_error_message().decode())
    return int(n)


def fbp_batched(sinos: list, geoms: list, kind="ramlak", dtype=torch.float32, variant: int = -1,
                outs: list | None = None, workspace: torch.Tensor | None = None):
    """fbp_batched: ragged batch of slices in one filter launch and one
    persistent backprojection launch.  Returns the list of output slices."""
    if len(sinos) != len(geoms):
        raise ValueError("sinos and geoms differ in length")
    for i, (s, g) in enumerate(zip(sinos, geoms)):
        _need(s, f"sinos[{i}]", torch.float32)
        _slices(s, (g.n_angles, g.n_det), f"sinos[{i}]")
    dev = sinos[0].device
    if outs is None:
        outs = [torch.empty((g.n, g.n), dtype=torch.float32, device=dev) for g in geoms]
    items = _items(sinos, outs, geoms)
    L = lib()
    need = L.fbp_batched_workspace_bytes(items, len(sinos), _DTYPES[dtype])
    if need == 0:
        raise FbpError(_lib.FBP_ERR_INVALID_ARG, "fbp_batched: " + L.fbp_last_error_message().decode())
    if workspace is None:
        workspace = torch.empty(need, dtype=torch.uint8, device=dev)
    st = L.fbp_batched(items, len(sinos), kind_id(kind), _DTYPES[dtype], int(variant),
                       _ptr(workspace), workspace.numel(), _stream(dev))
    _lib.check(st, L, "fbp_batched")
    return outs


_ORDERS = {"queue": _lib.FBP_ORDER_QUEUE, "group_cyclic": _lib.FBP_ORDER_GROUP_CYCLIC}


@dataclass
class Scan:
    """One item of a mixed batch: a normal scan (overlap 0) or a full-turn
    offset scan (overlap > 0, folded when `fold`)."""
    g: Geometry
    overlap: float = 0.0
    fold: bool = True


def _scan_items(sinos, outs, scans):
    arr = (_lib.CScanItem * len(sinos))()
    for i, (s, o, sc) in enumerate(zip(sinos, outs, scans)):
        arr[i].sino = s.data_ptr()
        arr[i].slice = o.data_ptr()
        arr[i].g = sc.g.c()
        arr[i].overlap = float(sc.overlap)
        arr[i].fold = int(bool(sc.fold))
    return arr


def fbp_batched_scans(sinos: list, scans: list, kind="ramlak", dtype=torch.float32, variant: int = -1,
                      order: str = "queue", outs: list | None = None,
                      workspace: torch.Tensor | None = None):
    """fbp_batched_scans: a ragged batch of normal and offset scans in one
    filter launch and one persistent backprojection launch, with the work
    order "queue" (atomic work queue, largest items first) or "group_cyclic"
    (static cyclic assignment of cost-sorted tiles).  Returns the slices."""
    if len(sinos) != len(scans):
        raise ValueError("sinos and scans differ in length")
    for i, (s, sc) in enumerate(zip(sinos, scans)):
        _need(s, f"sinos[{i}]", torch.float32)
        _slices(s, (sc.g.n_angles, sc.g.n_det), f"sinos[{i}]")
    dev = sinos[0].device
    if outs is None:
        outs = [torch.empty((sc.g.n, sc.g.n), dtype=torch.float32, device=dev) for sc in scans]
    items = _scan_items(sinos, outs, scans)
    L = lib()
    need = L.fbp_batched_scans_workspace_bytes(items, len(sinos), _DTYPES[dtype])
    if need == 0:
        raise FbpError(_lib.FBP_ERR_INVALID_ARG,
                       "fbp_batched_scans: " + L.fbp_last_error_message().decode())
    if workspace is None:
        workspace = torch.empty(need, dtype=torch.uint8, device=dev)
    st = L.fbp_batched_scans(items, len(sinos), kind_id(kind), _DTYPES[dtype], int(variant),
                             _ORDERS[order], _ptr(workspace), workspace.numel(), _stream(dev))
    _lib.check(st, L, "fbp_batched_scans")
    return outs


def batched_scans_workspace_bytes(sinos, outs, scans, dtype=torch.float32) -> int:
    L = lib()
    n = L.fbp_batched_scans_workspace_bytes(_scan_items(sinos, outs, scans), len(sinos), _DTYPES[dtype])
    if n == 0:
        raise FbpError(_lib.FBP_ERR_INVALID_ARG,
                       "fbp_batched_scans_workspace_bytes: " + L.fbp_last_error_message().decode())
    return int(n)


# ---------------------------------------------------------------------------
# Adaptive patching of reconstructed slices and 2-bit masks (include/sap.h).
# uint16 slices travel in int16 tensors (the same bits), as in backproject_u16.
# ---------------------------------------------------------------------------
@dataclass
class SapParams:
    """Patching parameters: slice side n, patch side P, sequence length
    (1 mod 3), Canny thresholds on M = |gx| + |gy|."""
    n: int
    patch: int = 16
    length: int = 4096
    canny_lo: int = 400000
    canny_hi: int = 1000000

    def c(self):
        return _lib.CSapParams(int(self.n), int(self.patch), int(self.length), int(self.canny_lo),
                               int(self.canny_hi))


def sap_workspace_bytes(p: SapParams, which: str = "default") -> int:
    pc = p.c()
    n = lib(which).sap_workspace_bytes(ctypes.byref(pc))
    if n == 0:
        L = lib(which)
        raise FbpError(_lib.FBP_ERR_INVALID_ARG, "sap_workspace_bytes: " + L.fbp_last_error_message().decode())
    return int(n)


def _sap_ws(p: SapParams, workspace, device):
    need = sap_workspace_bytes(p)
    if workspace is None:
        workspace = torch.empty(need, dtype=torch.uint8, device=device)
    return workspace


def sap_edges(slice16: torch.Tensor, p: SapParams, out: torch.Tensor | None = None,
              workspace: torch.Tensor | None = None, which: str = "default"):
    """sap_edges: Canny edge map (uint8, 1 on edges) of one uint16 slice."""
    _need(slice16, "slice", torch.int16)
    if tuple(slice16.shape) != (p.n, p.n):
        raise ValueError(f"slice has shape {tuple(slice16.shape)}, expected {(p.n, p.n)}")
    if out is None:
        out = torch.empty((p.n, p.n), dtype=torch.uint8, device=slice16.device)
    _need(out, "edges", torch.uint8)
    workspace = _sap_ws(p, workspace, slice16.device)
    L = lib(which)
    pc = p.c()
    st = L.sap_edges(_ptr(slice16), _ptr(out), ctypes.byref(pc), _ptr(workspace), workspace.numel(),
                     _stream(slice16.device))
    _lib.check(st, L, "sap_edges")
    return out


def sap_patches(slice16: torch.Tensor, edges: torch.Tensor, p: SapParams,
                patches: torch.Tensor | None = None, leaves: torch.Tensor | None = None,
                workspace: torch.Tensor | None = None, which: str = "default"):
    """sap_patches: the adaptive quadtree and its Z-order patch sequence.
    Returns (patches [length, P, P] float32, leaves [length, 3] int32)."""
    _need(slice16, "slice", torch.int16)
    _need(edges, "edges", torch.uint8)
    dev = slice16.device
    if patches is None:
        patches = torch.empty((p.length, p.patch, p.patch), dtype=torch.float32, device=dev)
    if leaves is None:
        leaves = torch.empty((p.length, 3), dtype=torch.int32, device=dev)
    _need(patches, "patches", torch.float32)
    _need(leaves, "leaves", torch.int32)
    workspace = _sap_ws(p, workspace, dev)
    L = lib(which)
    pc = p.c()
    st = L.sap_patches(_ptr(slice16), _ptr(edges), _ptr(patches), _ptr(leaves), ctypes.byref(pc),
                       _ptr(workspace), workspace.numel(), _stream(dev))
    _lib.check(st, L, "sap_patches")
    return patches, leaves


def sap_depatch_pack(mask_patches: torch.Tensor, leaves: torch.Tensor, p: SapParams,
                     out: torch.Tensor | None = None, which: str = "default"):
    """sap_depatch_pack: mask patches [length, P, P] (uint8 classes 0..3) back
    onto the slice through the quadtree, packed 2 bits per pixel [n, n/4]."""
    _need(mask_patches, "mask_patches", torch.uint8)
    _need(leaves, "leaves", torch.int32)
    if out is None:
        out = torch.empty((p.n, p.n // 4), dtype=torch.uint8, device=mask_patches.device)
    _need(out, "packed", torch.uint8)
    L = lib(which)
    pc = p.c()
    st = L.sap_depatch_pack(_ptr(mask_patches), _ptr(leaves), _ptr(out), ctypes.byref(pc),
                            _stream(mask_patches.device))
    _lib.check(st, L, "sap_depatch_pack")
    return out


def sap_host(slices: torch.Tensor, p: SapParams, patches: torch.Tensor | None = None,
             leaves: torch.Tensor | None = None, n_streams: int = 8, device=None):
    """Adaptive patching of a stack of uint16 slices held in host memory
    (int16 tensor [S, n, n], pinned for asynchronous copies): each slice is
    copied in, patched (sap_edges + sap_patches) and its patches and leaves
    copied out, on `n_streams` streams so that one slice's copies overlap
    another's kernels, and one slice's serial tail (the one-block selection,
    the tree's small top levels) overlaps another's edge detection.  The
    slices are copied in one at a time on a stream of their own.  Returns host (patches [S, length, P, P],
    leaves [S, length, 3]); blocks until they are filled."""
    if slices.is_cuda:
        raise ValueError("sap_host takes a host tensor; use sap_edges / sap_patches on device tensors")
    if slices.dtype != torch.int16 or not slices.is_contiguous() or slices.dim() != 3:
        raise ValueError("slices must be a contiguous int16 tensor [S, n, n]")
    S = int(slices.shape[0])
    if tuple(slices.shape[1:]) != (p.n, p.n):
        raise ValueError(f"slices have shape {tuple(slices.shape)}, expected [S, {p.n}, {p.n}]")
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    if patches is None:
        patches = torch.empty((S, p.length, p.patch, p.patch), dtype=torch.float32, pin_memory=True)
    if leaves is None:
        leaves = torch.empty((S, p.length, 3), dtype=torch.int32, pin_memory=True)
    n_streams = max(1, min(n_streams, S))
    caller = torch.cuda.current_stream(dev)
    streams = [torch.cuda.Stream(dev) for _ in range(n_streams)]
    # the slices come in one after another on a copy stream, each at the full
    # host-link bandwidth, so that slice 0's kernels start after one slice's
    # copy instead of after all of them; twice as many input buffers as
    # streams let the copies run ahead of the kernels, and a buffer is
    # refilled once the kernels that read it are done
    copier = torch.cuda.Stream(dev)
    need = sap_workspace_bytes(p)
    n_in = min(S, 2 * n_streams)
    ins = [torch.empty((p.n, p.n), dtype=torch.int16, device=dev) for _ in range(n_in)]
    bufs = [(torch.empty((p.n, p.n), dtype=torch.uint8, device=dev),
             torch.empty(need, dtype=torch.uint8, device=dev),
             torch.empty((p.length, p.patch, p.patch), dtype=torch.float32, device=dev),
             torch.empty((p.length, 3), dtype=torch.int32, device=dev)) for _ in range(n_streams)]
    copier.wait_stream(caller)
    for st in streams:
        st.wait_stream(caller)
    read_done = [None] * n_in
    for i in range(S):
        st = streams[i % n_streams]
        b = i % n_in
        d_in = ins[b]
        d_e, d_ws, d_p, d_l = bufs[i % n_streams]
        if read_done[b] is not None:
            copier.wait_event(read_done[b])
        with torch.cuda.stream(copier):
            d_in.copy_(slices[i], non_blocking=True)
            arrived = torch.cuda.Event()
            arrived.record(copier)
        st.wait_event(arrived)
        with torch.cuda.stream(st):
            sap_edges(d_in, p, out=d_e, workspace=d_ws)
            sap_patches(d_in, d_e, p, patches=d_p, leaves=d_l, workspace=d_ws)
            read_done[b] = torch.cuda.Event()
            read_done[b].record(st)
            patches[i].copy_(d_p, non_blocking=True)
            leaves[i].copy_(d_l, non_blocking=True)
    for st in streams:
        st.synchronize()
    copier.synchronize()
    return patches, leaves


def prepare(g: Geometry, kind="ramlak", device=None):
    """Build the geometry's constant tables now (before CUDA graph capture)."""
    L = lib()
    gc = g.c()
    k = -1 if kind is None else kind_id(kind)
    dev = torch.device("cuda") if device is None else torch.device(device)
    _lib.check(L.fbp_prepare(ctypes.byref(gc), k, _stream(dev)), L, "fbp_prepare")


def device_status(which: str = "default", device=None) -> int:
    """Synchronise, read and clear the device status word (0 = no fault)."""
    L = lib(which)
    code = ctypes.c_int(0)
    dev = torch.device("cuda") if device is None else torch.device(device)
    st = L.fbp_last_device_status(_stream(dev), ctypes.byref(code))
    if st not in (_lib.FBP_OK, _lib.FBP_ERR_DEVICE_STATUS):
        _lib.check(st, L, "fbp_last_device_status")
    return int(code.value)


def release_tables():
    lib().fbp_release_tables()


def measure_onchip_peaks(device=None) -> dict:
    """Measured per-SM ceilings of the device (fbp_measure_onchip_peaks):
    shared-load bytes and FP32 FMA lane operations per SM clock, the SM
    clock seen during the probe, and the SM count."""
    L = lib()
    dev = torch.device("cuda") if device is None else torch.device(device)
    out = _lib.COnchipPeaks()
    with torch.cuda.device(dev):
        _lib.check(L.fbp_measure_onchip_peaks(ctypes.byref(out)), L, "fbp_measure_onchip_peaks")
    return {"lds_bytes_per_clk_per_sm": out.lds_bytes_per_clk_per_sm,
            "fma_per_clk_per_sm": out.fma_per_clk_per_sm,
            "sm_clock_mhz": out.sm_clock_mhz, "sm_count": out.sm_count}


# ---------------------------------------------------------------------------
# Differentiation: A and A^T as a torch.autograd.Function pair.
# ---------------------------------------------------------------------------
class RadonForward(torch.autograd.Function):
    """y = A x (radon_forward); the gradient is A^T (fbp_backproject, scale 1)."""

    @staticmethod
    def forward(ctx, x: torch.Tensor, g: Geometry):
        ctx.g = g
        return radon_forward(x.contiguous(), g)

    @staticmethod
    def backward(ctx, gy: torch.Tensor):
        return backproject(gy.contiguous(), ctx.g, scale=1.0), None


class RadonBackproject(torch.autograd.Function):
    """x = A^T y (fbp_backproject, scale 1); the gradient is A (radon_forward)."""

    @staticmethod
    def forward(ctx, y: torch.Tensor, g: Geometry):
        ctx.g = g
        return backproject(y.contiguous(), g, scale=1.0)

    @staticmethod
    def backward(ctx, gx: torch.Tensor):
        return radon_forward(gx.contiguous(), ctx.g), None


def radon(x: torch.Tensor, g: Geometry) -> torch.Tensor:
    """Differentiable A x."""
    return RadonForward.apply(x, g)


def radon_t(y: torch.Tensor, g: Geometry) -> torch.Tensor:
    """Differentiable A^T y."""
    return RadonBackproject.apply(y, g)


def lsq_refine(x0: torch.Tensor, b: torch.Tensor, g: Geometry, eta: float, iters: int,
               return_losses: bool = True):
    """Gradient-descent least-squares refinement min 0.5 ||A x - b||^2 on the
    device: x <- x - eta * grad, the gradient taken by autograd through
    RadonForward (so it is A^T (A x - b), computed by the library's kernels).
    Returns (x, losses); the loss before each step is kept on the device and
    copied once at the end."""
    x = x0.detach().clone().requires_grad_(True)
    losses = []
    for _ in range(iters):
        r = radon(x, g) - b
        loss = 0.5 * (r.double() * r.double()).sum()
        (gx,) = torch.autograd.grad(loss, x)
        losses.append(loss.detach())
        with torch.no_grad():
            x -= eta * gx.float()
    with torch.no_grad():
        r = radon_forward(x.detach(), g) - b
        losses.append(0.5 * (r.double() * r.double()).sum())
    out = [float(v) for v in torch.stack(losses).cpu()] if return_losses else None
    return x.detach(), out
