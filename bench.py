"""Benchmark: backprojection throughput (Gupdates/s, slices/s) at N = 8192.

One step = one pass of the whole hot path -- ramp filter (fbp_filter) then
pixel-driven backprojection (fbp_backproject) -- over one batch of the
precision workload: 16 slices, N = D = 8192, 4096 angles on [0, pi),
seeded random-ellipse sinograms (noise-free), FP32 unless --dtype says
otherwise.  One update = one (pixel, angle) accumulation; a slice has
N^2 * K of them.

Timing: W untimed warm-up steps, then exactly K steps bracketed by a barrier
and torch.cuda.synchronize(), timed with CUDA events on the launching
stream; the per-step input (2.15 GB of sinograms) is larger than L2, so no
flush is needed.  The dominant kernel (backprojection) is bracketed by its
own events inside the timed region for the roofline figure.  SM clocks and
throttle reasons are sampled with nvidia-smi during the timed region.

Multi-GPU (torchrun, one rank per GPU): slices are independent (one slice
per detector row), so each rank reconstructs its own 16 slices with no
collective; the step time is the max over ranks and the value counts every
rank's updates (weak scaling).

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (one slice's full filtering plus the
backprojection of a square block of its pixels), extrapolated to whole
slices.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "backprojection Gupdates/s & slices/s at N=8192; % of roofline vs plain FP32 FBP"
UNIT = "Gupdates/s"
WORKLOAD = "fbp_precision_n8192"
SMS = 152
FP32_LANES = 128
ALU_OPS_PER_UPDATE = 4          # coordinate step, fraction, interpolate, accumulate
SHARED_BYTES_PER_CLK = 128      # shared-memory load bandwidth per SM
SAMPLES_PER_UPDATE = 2          # linear interpolation reads two detector samples
BP_KERNEL_REGEX = "bp_kernel"


def roofline_peak(sm_mhz: float, dtype: str) -> dict:
    """Backprojection ceilings in updates/s: the FP32 ALU ceiling
    (lanes x SMs x clock / 4 ops) and the on-chip load ceiling
    (128 B/clk/SM / (2 samples x sample bytes)); the roofline is the lower."""
    sample_bytes = 4 if dtype == "f32" else 2
    c_alu = SMS * FP32_LANES * sm_mhz * 1e6 / ALU_OPS_PER_UPDATE
    c_lds = SMS * SHARED_BYTES_PER_CLK * sm_mhz * 1e6 / (SAMPLES_PER_UPDATE * sample_bytes)
    return {"c_alu": c_alu / 1e9, "c_lds": c_lds / 1e9, "peak": min(c_alu, c_lds) / 1e9,
            "basis": f"min(C_alu = {SMS} SMs x {FP32_LANES} FP32 lanes x {sm_mhz:.0f} MHz / "
                     f"{ALU_OPS_PER_UPDATE} ops, C_lds = {SMS} x {SHARED_BYTES_PER_CLK} B/clk x "
                     f"{sm_mhz:.0f} MHz / ({SAMPLES_PER_UPDATE} x {sample_bytes} B)) per update"}


# ---------------------------------------------------------------------------
# Distributed plumbing (pure host logic; tested with gloo on CPU)
# ---------------------------------------------------------------------------
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def shard_slices(n_slices_per_rank: int, rank: int) -> list[int]:
    """Slice indices of the workload that a rank reconstructs (weak scaling:
    every rank gets its own n_slices_per_rank slices)."""
    return list(range(rank * n_slices_per_rank, (rank + 1) * n_slices_per_rank))


def aggregate(elapsed_ms_per_rank: list[float], units_per_rank: list[int]) -> tuple[float, float]:
    """(whole-job units per second, max-over-ranks step time in ms)."""
    t = max(elapsed_ms_per_rank)
    return sum(units_per_rank) / (t / 1e3), t


def allgather_floats(values: list[float], group=None) -> list[list[float]]:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return [values]
    ws = dist.get_world_size()
    t = torch.tensor(values, dtype=torch.float64)
    if dist.get_backend() == "nccl":
        t = t.cuda()
    out = [torch.zeros_like(t) for _ in range(ws)]
    dist.all_gather(out, t, group=group)
    return [o.cpu().tolist() for o in out]


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


# ---------------------------------------------------------------------------
# Clock sampling during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=2)

    def summary(self) -> dict:
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for name, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# Inputs
# ---------------------------------------------------------------------------
def make_inputs(w, slices: list[int]) -> np.ndarray:
    from paper_2505_13955_gb300 import phantoms
    out = np.empty((len(slices), w.n_angles, w.n), dtype=np.float32)
    for i, s in enumerate(slices):
        out[i] = phantoms.slice_sinogram(w, s)
    return out


def bp_source_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in ("bp_tile.cuh", "backproject.cu"):
        with open(os.path.join(ROOT, "paper_2505_13955_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def captured_traffic(variant: int, dtype: str, n_slices: int):
    """DRAM bytes per backprojection launch from the committed ncu capture,
    scaled by slices; None when the kernel sources changed since the capture
    or the launch differs (variant, dtype)."""
    try:
        with open(os.path.join(ROOT, "profiles", "bp_traffic.json")) as f:
            t = json.load(f)
    except (OSError, ValueError):
        return None
    if t.get("source_hash") != bp_source_hash() or t.get("dtype") != dtype:
        return None
    if variant not in (-1, t.get("variant")):
        return None
    return float(t["dram_bytes_per_slice"]) * n_slices


def peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


# ---------------------------------------------------------------------------
# CPU baseline (the FP64 oracle, as it stands)
# ---------------------------------------------------------------------------
def cpu_sample(w, block: int) -> dict:
    """Oracle on one slice: full filtering of its K rows plus backprojection of
    a block x block pixel square (all K angles); whole-slice time is
    extrapolated as t_filter + t_block * N^2 / block^2."""
    import oracle
    from paper_2505_13955_gb300 import phantoms
    N, K = w.n, w.n_angles
    p = phantoms.slice_sinogram(w, 0).astype(np.float64)
    g = oracle.Geometry(K, N, N)
    t0 = time.perf_counter()
    q = oracle.filter(p, oracle.RAMLAK if w.filter == "ramlak" else oracle.SHEPP_LOGAN)
    t1 = time.perf_counter()
    c0 = N // 2 - block // 2
    rr, cc = np.meshgrid(np.arange(c0, c0 + block), np.arange(c0, c0 + block), indexing="ij")
    oracle.backproject_pixels(q, g, rr.ravel(), cc.ravel())
    t2 = time.perf_counter()
    t_slice = (t1 - t0) + (t2 - t1) * (N * N) / (block * block)
    return {"value": N * N * K / t_slice / 1e9, "unit": UNIT, "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": f"1 slice N={N} K={K}: filter all {K} rows ({t1 - t0:.2f} s) + "
                      f"backproject a {block}x{block} pixel block over all angles "
                      f"({t2 - t1:.2f} s), extrapolated to the full slice",
            "seconds": t2 - t0}


def run_reference(args) -> None:
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from paper_2505_13955_gb300 import phantoms
    w = phantoms.WORKLOADS[args.workload]
    block = 1024 if args.steps + args.warmup <= 20 else 512
    for _ in range(args.warmup):
        cpu_sample(w, block // 2)
    vals, secs = [], []
    sample = None
    for _ in range(args.steps):
        r = cpu_sample(w, block)
        vals.append(r["value"])
        secs.append(r["seconds"])
        sample = r
    value = float(np.median(vals))
    slice_s = w.n * w.n * w.n_angles / (value * 1e9)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * slice_s * w.n_slices, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{w.name}: S={w.n_slices} N=D={w.n} K={w.n_angles} "
                   f"random ellipses, Ram-Lak", "sample": "see cpu_baseline"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": sample["cores"], "kind": "oracle",
                         "sample": sample["sample"]},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "slices_per_s": 1.0 / slice_s,
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_ours(args) -> None:
    import torch
    import torch.distributed as dist

    ws, rank, local = dist_env()
    if ws > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    from paper_2505_13955_gb300 import api, phantoms
    w = phantoms.WORKLOADS[args.workload]
    N, K, S = w.n, w.n_angles, (args.slices or w.n_slices)
    dtype = {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}[args.dtype]
    kind = w.filter
    g = api.Geometry(K, N, N)

    host = make_inputs(w, shard_slices(S, rank))
    sino = torch.from_numpy(host).to(dev)
    filt = torch.empty(sino.shape, dtype=dtype, device=dev)
    rs = torch.empty((S, K), dtype=torch.float32, device=dev) if dtype != torch.float32 else None
    out = torch.empty((S, N, N), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    api.prepare(g, kind=kind, device=dev)

    n_steps = args.steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(n_steps)]

    def step(evs=None):
        if evs:
            evs[0].record(stream)
        api.filter(sino, g, kind=kind, dtype=dtype, out=filt, row_scale=rs)
        if evs:
            evs[1].record(stream)
        api.backproject(filt, g, row_scale=rs, out=out, variant=args.variant)
        if evs:
            evs[2].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    assert api.device_status() == 0

    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev.index) as clocks:
        barrier()
        torch.cuda.synchronize()
        t_start.record(stream)
        for i in range(n_steps):
            step(ev[i])
        t_end.record(stream)
        torch.cuda.synchronize()
        barrier()
    elapsed = t_start.elapsed_time(t_end)
    bp_ms = [e[1].elapsed_time(e[2]) for e in ev]
    filt_ms = [e[0].elapsed_time(e[1]) for e in ev]
    updates_per_step = S * N * N * K
    per_rank = allgather_floats([elapsed / n_steps, float(updates_per_step)])
    job_rate, ms_step = aggregate([r[0] for r in per_rank], [int(r[1]) for r in per_rank])
    value = job_rate / 1e9
    slices_per_s = S * len(per_rank) / (ms_step / 1e3)

    # end to end through the public API with host buffers: pinned H2D of the
    # step's sinograms, filter + backprojection, D2H of the slices
    e2e = None
    if args.e2e_steps > 0:
        pin_in = torch.from_numpy(host).pin_memory()
        pin_out = torch.empty((S, N, N), dtype=torch.float32).pin_memory()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

        def e2e_step():
            x = pin_in.to(dev, non_blocking=True)
            f = api.fbp(x, g, kind=kind, dtype=dtype, variant=args.variant)
            pin_out.copy_(f, non_blocking=True)

        e2e_step()
        torch.cuda.synchronize()
        barrier()
        e0.record(stream)
        for _ in range(args.e2e_steps):
            e2e_step()
        e1.record(stream)
        torch.cuda.synchronize()
        t_e2e = e0.elapsed_time(e1) / args.e2e_steps
        per_rank_e2e = allgather_floats([t_e2e, float(updates_per_step)])
        e2e_rate, _ = aggregate([r[0] for r in per_rank_e2e], [int(r[1]) for r in per_rank_e2e])
        e2e = {"value": e2e_rate / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": int(pin_in.numel() * 4),
               "d2h_bytes_per_step": int(pin_out.numel() * 4),
               "ms_per_step": t_e2e}
        del pin_in, pin_out

    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return

    pk = peaks()
    csum = clocks.summary()
    sm_max = pk.get("sm_max_mhz") or 2070.0
    rp = roofline_peak(sm_max, args.dtype)
    peak_gups = rp["peak"]
    bp_avg = float(np.mean(bp_ms))
    achieved = updates_per_step / (bp_avg / 1e3) / 1e9
    traffic = args.traffic_bytes
    if traffic is None:
        traffic = captured_traffic(args.variant, args.dtype, S)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": n_steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"f32": "f32", "f16": "f16 rows, f32 accumulate", "bf16": "bf16 rows, f32 accumulate"}[args.dtype],
        "data": "synthetic",
        "config": {"workload": f"{w.name}: S={S} slices per GPU, N=D={N}, K={K} angles on [0,pi), "
                               f"seeded random ellipses (20-50), noise-free, Ram-Lak",
                   "l2": "inputs larger than L2 (2.15 GB sinograms per step), no flush",
                   "parallelism": f"slices sharded over {ws} GPU(s), no collective",
                   "bp_variant": args.variant},
        "slices_per_s": slices_per_s,
        "bp_ms_per_step": bp_avg, "filter_ms_per_step": float(np.mean(filt_ms)),
        "bp_gupdates_per_s": achieved,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_gups, "unit": UNIT,
                     "frac": achieved / peak_gups, "traffic": traffic,
                     "kernel": BP_KERNEL_REGEX, "c_alu": rp["c_alu"], "c_lds": rp["c_lds"],
                     "peak_basis": rp["basis"] + " (sm_max_mhz from MEASURED_PEAKS.json)",
                     "traffic_basis": "ncu dram bytes per slice x slices, kernel unchanged since capture"},
        "clocks": csum,
        "gpu_launches": 2 * n_steps,
    }
    if e2e is not None:
        line["e2e"] = e2e
    if not args.no_cpu_baseline and ws == 1:
        line["cpu_baseline"] = {k: v for k, v in cpu_sample(w, args.cpu_block).items() if k != "seconds"}
    print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--dtype", choices=["f32", "f16", "bf16"], default="f32")
    ap.add_argument("--variant", type=int, default=-1)
    ap.add_argument("--slices", type=int, default=None,
                    help="slices per GPU (default: the workload's 16); small cases for profiling")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--cpu-block", type=int, default=1024)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--traffic-bytes", type=float, default=None,
                    help="DRAM bytes per backprojection launch from an ncu capture")
    args = ap.parse_args(argv)
    args.warmup = max(3, args.warmup)   # at least 3 untimed warm-up steps
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
