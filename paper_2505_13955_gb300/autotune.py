"""Autotuner for the backprojection tile shape.

Picks, by timing on the device, the fastest compiled backprojection variant
(angle stage, pixels per thread, tile, symmetric or not) for a workload, and
caches the choice in a JSON file keyed by the workload's (N, K) mix, the row
dtype, the device name and its SM count.  Two cases:

* ``tune_single(g, dtype)`` -- fbp_backproject on one geometry: every variant
  that ``variant_supports`` accepts is timed on one slice of random rows;
* ``tune_batched(sinos, geoms, dtype)`` -- fbp_batched on a ragged batch: the
  variants its persistent kernel supports (symmetric ones included: orbit
  units where an item has the symmetry) are timed on the batch itself.

Timing: CUDA events on the current stream, one warm-up launch, best of
``reps``.  Cache: $FBP_AUTOTUNE_CACHE, else ~/.cache/fbp_gb300/autotune.json.
"""
from __future__ import annotations

import json
import os
import threading

import torch

from . import api

_lock = threading.Lock()


def cache_path() -> str:
    p = os.environ.get("FBP_AUTOTUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "fbp_gb300", "autotune.json")


def _device_key(device=None) -> str:
    dev = torch.device("cuda") if device is None else torch.device(device)
    props = torch.cuda.get_device_properties(dev)
    return f"{props.name}|sm{props.multi_processor_count}"


def _load() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(key: str, value: dict) -> None:
    with _lock:
        data = _load()
        data[key] = value
        path = cache_path()
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        os.replace(tmp, path)


def _time(fn, reps: int) -> float:
    stream = torch.cuda.current_stream()
    fn()
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        best = min(best, a.elapsed_time(b))
    return best


def _dtype_name(dtype) -> str:
    return {torch.float32: "f32", torch.float16: "f16", torch.bfloat16: "bf16"}[dtype]


def single_key(g: api.Geometry, dtype, device=None) -> str:
    return (f"single|{_device_key(device)}|{_dtype_name(dtype)}|K{g.n_angles}|D{g.n_det}|N{g.n}|"
            f"a{g.pixel_size / g.det_spacing:.6g}|c{g.det_center - 0.5 * (g.n_det - 1):.6g}|"
            f"s{g.angle_step * g.n_angles:.9g}")


def batched_key(geoms, dtype, device=None) -> str:
    # v3: the default (-1, staged batch units) is a candidate beside every
    # persistent-kernel shape
    mix = sorted({(g.n_angles, g.n) for g in geoms})
    return f"batched-v3|{_device_key(device)}|{_dtype_name(dtype)}|" + ",".join(f"{k}x{n}" for k, n in mix)


def tune_single(g: api.Geometry, dtype=torch.float32, reps: int = 3, force: bool = False,
                variants=None) -> dict:
    """Fastest fbp_backproject variant for geometry g and rows of `dtype`."""
    key = single_key(g, dtype)
    if not force:
        hit = _load().get(key)
        if hit is not None:
            return hit
    gen = torch.Generator(device="cuda").manual_seed(0)
    rows = torch.randn((g.n_angles, g.n_det), device="cuda", generator=gen)
    filt, rs = api.filter(rows, g, dtype=dtype)
    out = torch.empty((g.n, g.n), device="cuda")
    # the texture-unit variant synchronises on every call and is never the
    # default: it is timed only when asked for explicitly
    cands = variants if variants is not None else [s["variant"] for s in api.bp_variants() if not s["texture"]]
    times = {}
    for v in cands:
        if not api.variant_supports(v, g, dtype):
            continue
        times[v] = _time(lambda: api.backproject(filt, g, row_scale=rs, out=out, variant=v), reps)
    best = min(times, key=times.get)
    upd = g.n * g.n * g.n_angles
    result = {"variant": int(best), "ms": times[best],
              "gupdates_per_s": upd / times[best] / 1e6,
              "times_ms": {str(k): t for k, t in times.items()}}
    _store(key, result)
    return result


def tune_batched(sinos, geoms, dtype=torch.float32, reps: int = 2, force: bool = False,
                 kind="ramlak", variants=None) -> dict:
    """Fastest backprojection of fbp_batched on this batch: -1 (the default:
    staged batch units for the items whose geometry allows them, the
    persistent tile kernel for the rest) or a persistent-kernel variant."""
    key = batched_key(geoms, dtype)
    if not force:
        hit = _load().get(key)
        if hit is not None:
            return hit
    outs = [torch.empty((g.n, g.n), device="cuda") for g in geoms]
    ws = torch.empty(api.batched_workspace_bytes(sinos, outs, geoms, dtype), dtype=torch.uint8,
                     device="cuda")
    shapes = api.bp_variants()
    # symmetric shapes run orbit units for the items with the symmetry and
    # generic tiles of the same threads for the others; packed shapes only
    # for 16-bit rows
    cands = variants if variants is not None else [-1] + [
        s["variant"] for s in shapes
        if not s["texture"] and not (s["packed16"] and dtype == torch.float32)]
    times = {}
    for v in cands:
        try:
            times[v] = _time(lambda: api.fbp_batched(sinos, geoms, kind=kind, dtype=dtype, variant=v,
                                                     outs=outs, workspace=ws), reps)
        except api.FbpError:
            continue
    best = min(times, key=times.get)
    upd = sum(g.n * g.n * g.n_angles for g in geoms)
    result = {"variant": int(best), "ms": times[best],
              "gupdates_per_s": upd / times[best] / 1e6,
              "times_ms": {str(k): t for k, t in times.items()}}
    _store(key, result)
    return result
