"""Benchmark: backprojection throughput (Gupdates/s, slices/s) at N = 8192.

Default workload (the headline): 16 slices per GPU, N = D = 8192, 4096
angles on [0, pi), seeded random-ellipse sinograms (noise-free), Ram-Lak.
One step = one pass of the whole hot path over the batch: fbp_filter then
fbp_backproject.  One update = one (pixel, angle) accumulation; a slice has
N^2 K of them.  `value` is for plain FP32 rows; the same line reports the
FP16- and BF16-staged forms measured in the same run, as ratios to FP32.

Other workloads (--workload): fbp_single_n256 (1 slice, N = 256, K = 360),
fbp_stack_n2048 (64 slices, N = 2048, K = 1800, Poisson noise, Shepp-Logan
filter), fbp_ragged_batch (200 slices of mixed N and K in one persistent
launch replayed from a CUDA graph, against per-slice launches), and
gd_refine_n1024 (gradient-descent least squares, 16 slices, N = 1024,
K = 1800; a step is one iteration, A and A^T), fbp_pipeline_n8192 (detector
counts to uint16 CT-number codes) and fbp_offset_n8192 (full-turn offset
scans, 16 slices, 8192 angles, a 4608-bin detector off the axis) and
fbp_mixed_batch (200 normal and offset scans in one persistent launch, work
queue against the paper's group-and-cyclic order) and sap_patching_n8192
(adaptive patching of 16 reconstructed 8192^2 uint16 slices, slices/s).

Timing: W >= 3 untimed warm-up steps, then exactly K steps bracketed by a
barrier and torch.cuda.synchronize(), timed with CUDA events on the
launching stream; the dominant kernel is bracketed by its own events inside
the timed region for the roofline.  Inputs of the headline workload (2.15 GB
of sinograms per step) exceed L2, so no flush is needed.  SM clocks and
throttle reasons are sampled with nvidia-smi during the timed region.

Multi-GPU (torchrun, one rank per GPU): slices are independent (one slice
per detector row), so each rank reconstructs its own slices with no
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
SAP_METRIC = "SAP patching slices/s at N=8192 (Canny + adaptive quadtree + Z-order patches)"
WORKLOAD = "fbp_precision_n8192"
FP32_LANES = 128                # nominal FP32 lanes per SM
ALU_OPS_PER_UPDATE = 4          # coordinate step, fraction, interpolate, accumulate
SHARED_BYTES_PER_CLK = 128      # nominal shared-memory load bandwidth per SM
SAMPLES_PER_UPDATE = 2          # linear interpolation reads two detector samples
BP_KERNEL_REGEX = "bp_kernel|bp_orbit_kernel"
BP_STAGED_REGEX = "bp_staged_kernel"
GRAPH_BELOW_UPDATES = 1e9     # uniform steps smaller than this are replayed from a CUDA graph


def roofline_peak(sm_mhz: float, dtype: str, sms: int, onchip: dict | None = None) -> dict:
    """Backprojection ceilings in Gupdates/s at `sm_mhz`: the FP32 ALU ceiling
    (FMA lane operations per SM clock x SMs x clock / 4 ops) and the
    shared-load ceiling (bytes per SM clock x SMs x clock / (2 samples x
    sample bytes)), each from the nominal per-SM rates (128 lanes, 128 B) and,
    when `onchip` is given, from the rates measured on this GPU
    (fbp_measure_onchip_peaks).  The roofline is the lower of the two, taken
    from the measured rates when there are any."""
    sample_bytes = 4 if dtype == "f32" else 2
    clk = sm_mhz * 1e6

    def ceil(lanes, lds_b):
        c_alu = sms * lanes * clk / ALU_OPS_PER_UPDATE / 1e9
        c_lds = sms * lds_b * clk / (SAMPLES_PER_UPDATE * sample_bytes) / 1e9
        return c_alu, c_lds

    c_alu, c_lds = ceil(FP32_LANES, SHARED_BYTES_PER_CLK)
    out = {"c_alu_nominal": c_alu, "c_lds_nominal": c_lds, "peak_nominal": min(c_alu, c_lds),
           "sms": sms, "sm_mhz": sm_mhz}
    basis = (f"min(C_alu = {sms} SMs x {{lanes}} FP32 FMA/clk x {sm_mhz:.0f} MHz / {ALU_OPS_PER_UPDATE} ops, "
             f"C_lds = {sms} SMs x {{lds}} B/clk x {sm_mhz:.0f} MHz / ({SAMPLES_PER_UPDATE} x {sample_bytes} B)) "
             "per update")
    if onchip:
        m_alu, m_lds = ceil(onchip["fma_per_clk_per_sm"], onchip["lds_bytes_per_clk_per_sm"])
        out.update({"c_alu": m_alu, "c_lds": m_lds, "peak": min(m_alu, m_lds),
                    "bound": "lds" if m_lds <= m_alu else "alu", "measured": True,
                    "basis": basis.format(lanes=f"{onchip['fma_per_clk_per_sm']:.1f} (measured)",
                                          lds=f"{onchip['lds_bytes_per_clk_per_sm']:.1f} (measured)")})
    else:
        out.update({"c_alu": c_alu, "c_lds": c_lds, "peak": min(c_alu, c_lds),
                    "bound": "lds" if c_lds <= c_alu else "alu", "measured": False,
                    "basis": basis.format(lanes=FP32_LANES, lds=SHARED_BYTES_PER_CLK) + " (nominal)"})
    return out


def roofline_entry(achieved: float, rp: dict, kernel: str, traffic=None, **extra) -> dict:
    """The line's roofline object for an updates-per-second kernel."""
    r = {"bound": rp["bound"], "achieved": achieved, "peak": rp["peak"], "unit": UNIT,
         "frac": achieved / rp["peak"], "traffic": traffic, "kernel": kernel,
         "c_alu": rp["c_alu"], "c_lds": rp["c_lds"],
         "peak_nominal": rp["peak_nominal"], "frac_nominal": achieved / rp["peak_nominal"],
         "peak_basis": rp["basis"] + f", sm_max_mhz {rp['sm_mhz']:.0f} from MEASURED_PEAKS.json"}
    r.update(extra)
    return r


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
# Inputs, peaks, captured traffic
# ---------------------------------------------------------------------------
def make_inputs(w, slices: list[int]) -> np.ndarray:
    from paper_2505_13955_gb300 import phantoms
    out = np.empty((len(slices), w.n_angles, w.n), dtype=np.float32)
    for i, s in enumerate(slices):
        out[i] = phantoms.slice_sinogram(w, s)
    return out


def peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


BP_SOURCES = ("bp_tile.cuh", "bp_orbit.cuh", "backproject.cu", "bp_staged.cuh", "bp_staged.cu")
# the files that hold the staged kernel's device code (the pair arithmetic,
# the pipeline, the kernel): its captured traffic stays valid across edits
# of the other kernels' launch code
STAGED_SOURCES = ("bp_orbit.cuh", "bp_staged.cuh", "bp_staged.cu")


def bp_source_hash(files=BP_SOURCES) -> str:
    """Hash of the backprojection kernels' code: the sources with comments
    and blank lines removed, so that an edit of the comments keeps a
    captured traffic figure valid."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2505_13955_gb300", "csrc", f)) as fh:
            for line in fh:
                code = re.sub(r"//.*", "", line).rstrip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def captured_traffic(variant: int, dtype: str, n_slices: int, n: int, k: int):
    """DRAM bytes per backprojection launch from the committed ncu capture,
    scaled by slices; None when the kernel sources changed since the capture
    or the launch differs (variant, dtype, image size, angle count)."""
    try:
        with open(os.path.join(ROOT, "profiles", "bp_traffic.json")) as f:
            entries = json.load(f)
    except (OSError, ValueError):
        return None
    for t in entries if isinstance(entries, list) else [entries]:
        if t.get("source_hash") != bp_source_hash(tuple(t.get("sources", BP_SOURCES))) or t.get("dtype") != dtype:
            continue
        if variant != t.get("variant") or t.get("n") != n or t.get("k") != k:
            continue
        return float(t["dram_bytes_per_slice"]) * n_slices
    return None


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
    block = min(block, N)
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


def cpu_sample_pipeline(w, block: int) -> dict:
    """Oracle on one counts slice: Beer-Lambert + Gaussian blur and filtering
    of all K rows, backprojection of a block x block pixel square over all
    angles and its uint16 codes; whole-slice time extrapolated by pixel
    count (as cpu_sample)."""
    import oracle
    from paper_2505_13955_gb300 import phantoms
    P = phantoms.PIPELINE
    N, K = w.n, w.n_angles
    I = phantoms.slice_counts(w, 0).astype(np.float64)
    g = oracle.Geometry(K, N, N)
    t0 = time.perf_counter()
    p = oracle.preprocess(I, w.photons, mu_scale=float(N), floor=1.0, sigma=P["blur_sigma"])
    q = oracle.filter(p, oracle.RAMLAK)
    t1 = time.perf_counter()
    block = min(block, N)
    c0 = N // 2 - block // 2
    rr, cc = np.meshgrid(np.arange(c0, c0 + block), np.arange(c0, c0 + block), indexing="ij")
    mu = oracle.backproject_pixels(q, g, rr.ravel(), cc.ravel())
    oracle.hu_codes(mu, P["mu_water"], P["mu_air"], P["hu_min"], P["hu_max"])
    t2 = time.perf_counter()
    t_slice = (t1 - t0) + (t2 - t1) * (N * N) / (block * block)
    return {"value": N * N * K / t_slice / 1e9, "unit": UNIT, "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": f"1 counts slice N={N} K={K}: Beer-Lambert + blur + filter of all {K} rows "
                      f"({t1 - t0:.2f} s) + backprojection and uint16 codes of a {block}x{block} pixel "
                      f"block over all angles ({t2 - t1:.2f} s), extrapolated to the full slice"}


def cpu_sample_offset(w, block: int) -> dict:
    """Oracle on one offset-scan slice: weight, embed and fold its rows,
    filter all folded rows, backproject a block x block pixel square over
    all folded angles; whole-slice time extrapolated by pixel count."""
    import oracle
    from paper_2505_13955_gb300 import phantoms
    D, c, delta = w.offset
    N, K = w.n, w.n_angles
    p = phantoms.slice_sinogram(w, 0).astype(np.float64)
    t0 = time.perf_counter()
    n_v, c_v, off, wt = oracle.offset_virtual(D, c, delta)
    q = oracle.filter(oracle.offset_fold(oracle.embed_rows(p, n_v, off), wt))
    t1 = time.perf_counter()
    block = min(block, N)
    c0 = N // 2 - block // 2
    rr, cc = np.meshgrid(np.arange(c0, c0 + block), np.arange(c0, c0 + block), indexing="ij")
    oracle.backproject_pixels(q, oracle.Geometry(K // 2, n_v, N, angle_step=2 * np.pi / K), rr.ravel(), cc.ravel())
    t2 = time.perf_counter()
    t_slice = (t1 - t0) + (t2 - t1) * (N * N) / (block * block)
    return {"value": N * N * (K // 2) / t_slice / 1e9, "unit": UNIT, "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": f"1 offset slice: weight + fold + filter all {K // 2} folded rows ({t1 - t0:.2f} s) + "
                      f"backproject a {block}x{block} block ({t2 - t1:.2f} s), extrapolated to the full slice"}


def cpu_sample_gd(w) -> dict:
    """Oracle FP64 gradient A^T (A x - b) of one slice (one GD iteration's work)."""
    import oracle
    from paper_2505_13955_gb300 import phantoms
    N, K = w.n, w.n_angles
    b = phantoms.slice_sinogram(w, 0).astype(np.float64)
    g = oracle.Geometry(K, N, N)
    x = np.zeros((N, N))
    t0 = time.perf_counter()
    oracle.gradient(x, b, g)
    t1 = time.perf_counter()
    return {"value": 2 * N * N * K / (t1 - t0) / 1e9, "unit": UNIT, "cores": oracle.num_threads(),
            "kind": "oracle", "sample": f"one FP64 gradient A^T (A x - b) of 1 slice N={N} K={K} ({t1 - t0:.2f} s)"}


def cpu_sample_sap(n_sample: int, n: int) -> dict:
    """Oracle patching (Canny, greedy quadtree, patch means) of one
    n_sample^2 slice, scaled to n^2 slices by pixel count."""
    from oracle import sap
    from paper_2505_13955_gb300 import phantoms
    c = phantoms.SAP
    img = phantoms.sap_slice(n_sample, 12345)
    length = min(c["length"], 1 + 3 * (((n_sample // c["patch"]) ** 2 - 1) // 3))
    t0 = time.perf_counter()
    e = sap.canny(img, c["canny_lo"], c["canny_hi"])
    leaves, _ = sap.quadtree(img, e, c["patch"], length)
    sap.extract_patches(img, leaves, c["patch"])
    t1 = time.perf_counter()
    per_slice = (t1 - t0) * (n * n) / (n_sample * n_sample)
    from oracle import num_threads
    return {"value": 1.0 / per_slice, "unit": "slices/s", "cores": num_threads(), "kind": "oracle",
            "sample": f"Canny + quadtree ({length} patches) + patch means of one {n_sample}^2 slice "
                      f"({t1 - t0:.2f} s), scaled to {n}^2 by pixel count"}


def run_reference(args) -> None:
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from paper_2505_13955_gb300 import phantoms
    w = phantoms.WORKLOADS[args.workload]
    block = 1024 if args.steps + args.warmup <= 20 else 512
    metric, unit = METRIC, UNIT
    # each workload's oracle sample, in its own metric: (sample function, seconds per slice from a value)
    if w.name == "sap_patching_n8192":
        metric, unit = SAP_METRIC, "slices/s"
        fn, slice_seconds = (lambda _b: cpu_sample_sap(2048, w.n)), (lambda v: 1.0 / v)
        what = f"{w.name}: S={w.n_slices} uint16 slices, n={w.n}"
    elif w.name == "gd_refine_n1024":
        fn, slice_seconds = (lambda _b: cpu_sample_gd(w)), (lambda v: 2 * w.n * w.n * w.n_angles / (v * 1e9))
        what = f"{w.name}: S={w.n_slices} N=D={w.n} K={w.n_angles}, one gradient step per slice"
    elif w.offset is not None and not w.ragged:
        fn = lambda b: cpu_sample_offset(w, b)
        slice_seconds = lambda v: w.n * w.n * (w.n_angles // 2) / (v * 1e9)
        what = f"{w.name}: S={w.n_slices} N={w.n} K={w.n_angles} over a full turn, folded"
    else:
        if w.ragged or not w.filter:
            w = phantoms.WORKLOADS[WORKLOAD]      # ragged batches: per-update cost of the uniform stack
        fn, slice_seconds = (lambda b: cpu_sample(w, b)), (lambda v: w.n * w.n * w.n_angles / (v * 1e9))
        what = f"{w.name}: S={w.n_slices} N=D={w.n} K={w.n_angles} random ellipses, {w.filter}"
    for _ in range(args.warmup):
        fn(block // 2)
    vals = []
    sample = None
    for _ in range(args.steps):
        r = fn(block)
        vals.append(r["value"])
        sample = r
    value = float(np.median(vals))
    slice_s = slice_seconds(value)
    line = {
        "impl": "reference", "metric": metric, "value": value, "unit": unit, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * slice_s * w.n_slices, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": what, "sample": "see cpu_baseline"},
        "cpu_baseline": {"value": value, "unit": unit, "cores": sample["cores"], "kind": "oracle",
                         "sample": sample["sample"]},
        "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "slices_per_s": 1.0 / slice_s,
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
class Timed:
    """W warm-up steps, then K steps between a barrier and synchronisation,
    timed with CUDA events on `stream`; `step(evs)` may record its own
    events for the dominant kernel."""

    def __init__(self, stream, steps: int, warmup: int, n_events: int = 0):
        import torch
        self.torch = torch
        self.stream = stream
        self.steps = steps
        self.warmup = warmup
        self.clocks = None
        self.ev = [[torch.cuda.Event(enable_timing=True) for _ in range(n_events)]
                   for _ in range(steps)]

    def run(self, step, clocks_index: int | None):
        torch = self.torch
        for _ in range(self.warmup):
            step(None)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        sampler = ClockSampler(clocks_index) if clocks_index is not None else None
        if sampler:
            sampler.__enter__()
        try:
            barrier()
            torch.cuda.synchronize()
            a.record(self.stream)
            for i in range(self.steps):
                step(self.ev[i] if self.ev[i] else None)
            b.record(self.stream)
            torch.cuda.synchronize()
            barrier()
        finally:
            if sampler:
                sampler.__exit__(None, None, None)
        self.clocks = sampler.summary() if sampler else None
        return a.elapsed_time(b) / self.steps

    def between(self, i: int, j: int) -> float:
        return float(np.mean([e[i].elapsed_time(e[j]) for e in self.ev]))

    def spread(self, i: int, j: int) -> dict:
        """Median, min and max over the timed steps of the time from event i
        to event j of each step."""
        t = [e[i].elapsed_time(e[j]) for e in self.ev]
        return {"median": float(np.median(t)), "min": float(np.min(t)), "max": float(np.max(t)),
                "n": len(t)}


def init_device():
    import torch
    import torch.distributed as dist
    ws, rank, local = dist_env()
    if ws > 1:
        torch.cuda.set_device(local)
        if not dist.is_initialized():
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    return ws, rank, torch.device("cuda", torch.cuda.current_device())


_ONCHIP: dict = {}


def device_ceilings(dev) -> tuple[float, int, dict | None]:
    """(sm_max_mhz from MEASURED_PEAKS.json, the device's SM count, the on-chip
    rates measured on it by fbp_measure_onchip_peaks, once per process)."""
    import torch
    from paper_2505_13955_gb300 import api
    if dev.index not in _ONCHIP:
        try:
            _ONCHIP[dev.index] = api.measure_onchip_peaks(dev)
        except Exception as e:           # the nominal ceilings stand in, and the line says so
            print(f"on-chip probe failed: {e}", file=sys.stderr)
            _ONCHIP[dev.index] = None
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    return peaks().get("sm_max_mhz") or 2070.0, sms, _ONCHIP[dev.index]


def base_line(args, ws, value, ms_step, dtype_label, config) -> dict:
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": dtype_label, "data": "synthetic",
            "config": config}


DT = {"f32": "float32", "f16": "float16", "bf16": "bfloat16"}
DT_LABEL = {"f32": "f32", "f16": "f16 rows, f32 accumulate", "bf16": "bf16 rows, f32 accumulate"}


def resolved_variant(api, g, dtype: str, variant: int) -> int:
    """The tile variant fbp_backproject runs for `variant` (-1 = default)."""
    if variant >= 0:
        return variant
    import torch
    tdt = getattr(torch, DT[dtype])
    # the library's default choice (backproject.cu: bp_default_variant)
    for v in ((10, 8, 11, 6) if dtype != "f32" else (7, 5)):
        if api.variant_supports(v, g, tdt):
            return v
    return 0


def run_uniform(args) -> None:
    """Uniform stacks (headline N = 8192, N = 2048 stack, N = 256 single):
    one step = fbp_filter + fbp_backproject over the whole stack."""
    import torch
    from paper_2505_13955_gb300 import api, phantoms

    ws, rank, dev = init_device()
    w = phantoms.WORKLOADS[args.workload]
    N, K, S = w.n, w.n_angles, (args.slices or w.n_slices)
    g = api.Geometry(K, N, N)
    host = make_inputs(w, shard_slices(S, rank))
    sino = torch.from_numpy(host).to(dev)
    out = torch.empty((S, N, N), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    api.prepare(g, kind=w.filter, device=dev)
    updates = S * N * N * K
    use_graph = args.graph == "on" or (args.graph == "auto" and updates < GRAPH_BELOW_UPDATES)
    dtypes = [args.dtype] + ([d for d in ("f16", "bf16") if d != args.dtype] if args.all_dtypes else [])
    results = {}
    for dt in dtypes:
        tdt = getattr(torch, DT[dt])
        filt = torch.empty(sino.shape, dtype=tdt, device=dev)
        rs = torch.empty((S, K), dtype=torch.float32, device=dev) if dt != "f32" else None
        # the bulk-copy-fed kernel from per-slice tables (its workspace holds
        # the whole stack's tables, allocated before timing)
        staged = args.variant < 0 and api.staged_preferred(g)
        wsp = torch.empty(api.backproject_staged_workspace_bytes(g, tdt, S), dtype=torch.uint8, device=dev) \
            if staged else None
        T = Timed(stream, args.steps, args.warmup, n_events=3)

        def filter_only():
            api.filter(sino, g, kind=w.filter, dtype=tdt, out=filt, row_scale=rs)

        def bp_only():
            if staged:
                api.backproject_staged(filt, g, rs, out=out, workspace=wsp)
            else:
                api.backproject(filt, g, row_scale=rs, out=out, variant=args.variant)

        def step(evs):
            if evs:
                evs[0].record(stream)
            filter_only()
            if evs:
                evs[1].record(stream)
            bp_only()
            if evs:
                evs[2].record(stream)

        clocks_at = dev.index if dt == args.dtype else None
        ms = T.run(step, None if use_graph else clocks_at)
        assert api.device_status() == 0
        res = {"bp_ms": T.between(1, 2), "filter_ms": T.between(0, 1), "step_spread": T.spread(0, 2),
               "clocks": T.clocks}
        if use_graph:
            # a step this short is bound by the host's launch path: the step,
            # the filter alone and the backprojection alone are each captured
            # once in a CUDA graph and replayed (all work stays in every step)
            eager = {"ms_per_step": ms, "bp_ms_per_step": res["bp_ms"], "filter_ms_per_step": res["filter_ms"]}
            gs = torch.cuda.Stream(dev)
            graphs = []
            for fn in (lambda: step(None), filter_only, bp_only):
                gr = torch.cuda.CUDAGraph()
                with torch.cuda.graph(gr, stream=gs):
                    fn()
                graphs.append(gr)
            with torch.cuda.stream(gs):
                # the rate: replays back to back, events only around the run
                # (an event per replay is host work on the launch path that
                # bounds a step this short); the per-step spread from a second
                # run with an event pair around each replay
                Tg = Timed(gs, args.steps, args.warmup)
                ms = Tg.run(lambda _: graphs[0].replay(), clocks_at)
                clocks_g = Tg.clocks
                Ts = Timed(gs, min(args.steps, 2000), 1, n_events=2)

                def replay(evs):
                    evs[0].record(gs)
                    graphs[0].replay()
                    evs[1].record(gs)

                Ts.run(lambda evs: replay(evs) if evs else graphs[0].replay(), None)
                f_ms = Timed(gs, args.steps, 1).run(lambda _: graphs[1].replay(), None)
                b_ms = Timed(gs, args.steps, 1).run(lambda _: graphs[2].replay(), None)
            torch.cuda.synchronize()
            assert api.device_status() == 0
            res = {"bp_ms": b_ms, "filter_ms": f_ms, "step_spread": Ts.spread(0, 1), "clocks": clocks_g,
                   "eager": eager}
            del graphs
        per_rank = allgather_floats([ms, float(updates)])
        rate, ms_step = aggregate([r[0] for r in per_rank], [int(r[1]) for r in per_rank])
        results[dt] = dict(res, value=rate / 1e9, ms_per_step=ms_step,
                           slices_per_s=S * len(per_rank) / (ms_step / 1e3), staged=staged)
        if staged:
            # the block-staged orbit kernel on the same rows, for comparison
            # (named explicitly: api.backproject's default takes the staged kernel)
            vo = resolved_variant(api, g, dt, -1)
            To = Timed(stream, 3, 3)
            ms_o = To.run(lambda _: api.backproject(filt, g, row_scale=rs, out=out, variant=vo), None)
            results[dt]["orbit_kernel"] = {"bp_ms_per_step": ms_o,
                                           "bp_gupdates_per_s": updates / (ms_o / 1e3) / 1e9,
                                           "bp_variant": vo}
        del filt, rs, wsp

    # the texture-unit backprojection (the measured alternative to staged
    # tables): backprojection only, on the same FP32 rows
    tex = None
    tvs = [v["variant"] for v in api.bp_variants() if v["texture"]]
    if args.texture and tvs and api.variant_supports(tvs[0], g):
        filt, _ = api.filter(sino, g, kind=w.filter)
        Tt = Timed(stream, 2, args.warmup)
        ms_tex = Tt.run(lambda _: api.backproject(filt, g, out=out, variant=tvs[0]), None)
        assert api.device_status() == 0
        tex = {"variant": tvs[0], "bp_ms_per_step": ms_tex,
               "bp_gupdates_per_s": updates / (ms_tex / 1e3) / 1e9}
        del filt

    e2e = None
    if args.e2e_steps > 0:
        tdt = getattr(torch, DT[args.dtype])
        pin_in = torch.from_numpy(host).pin_memory()
        pin_out = torch.empty((S, N, N), dtype=torch.float32).pin_memory()

        def e2e_step(_):
            # the public host-buffer call: chunked copies overlapped with kernels
            api.fbp_host(pin_in, g, kind=w.filter, dtype=tdt, out=pin_out, variant=args.variant)

        T = Timed(stream, args.e2e_steps, 1)
        t_e2e = T.run(e2e_step, None)
        per_rank_e2e = allgather_floats([t_e2e, float(updates)])
        e2e_rate, _ = aggregate([r[0] for r in per_rank_e2e], [int(r[1]) for r in per_rank_e2e])
        e2e = {"value": e2e_rate / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": int(pin_in.numel() * 4),
               "d2h_bytes_per_step": int(pin_out.numel() * 4), "ms_per_step": t_e2e}
        del pin_in, pin_out

    if rank != 0:
        return None
    main = results[args.dtype]
    sm_max, sms, onchip = device_ceilings(dev)
    rp = roofline_peak(sm_max, args.dtype, sms, onchip)
    achieved = updates / (main["bp_ms"] / 1e3) / 1e9
    variant = "fbp_backproject_staged (default shape)" if main["staged"] else \
        resolved_variant(api, g, args.dtype, args.variant)
    traffic = args.traffic_bytes
    if traffic is None:
        traffic = captured_traffic(variant, args.dtype, S, N, K)
    phantom = "Shepp-Logan" if w.phantom == "shepp_logan" else "random ellipses (20-50)"
    noise = f"Poisson {w.photons:g} photons" if w.photons else "noise-free"
    line = base_line(args, ws, main["value"], main["ms_per_step"], DT_LABEL[args.dtype], {
        "workload": f"{w.name}: S={S} slices per GPU, N=D={N}, K={K} angles on [0,pi), "
                    f"seeded {phantom}, {noise}, {w.filter}",
        "l2": "inputs larger than L2 (sinograms per step exceed 129 MB), no flush"
              if S * K * N * 4 > 129e6 else "inputs smaller than L2 (launch-bound case)",
        "parallelism": f"slices sharded over {ws} GPU(s), no collective",
        "bp_variant": variant,
        "launch": "CUDA-graph replay of the step (filter + backprojection), eager timings in 'eager'"
                  if use_graph else "eager launches"})
    hbm = peaks().get("hbm_gbs") or 6800.0

    def filter_hbm(filter_ms, dt):
        # K1's algorithmic bytes: every FP32 input sample read once and every
        # filtered sample written once (plus one row scale per 16-bit row)
        out_b = 4 if dt == "f32" else 2
        nbytes = S * K * N * (4 + out_b) + (0 if dt == "f32" else S * K * 4)
        gbs = nbytes / (filter_ms / 1e3) / 1e9 if filter_ms else None
        return {"gb_per_s": gbs, "hbm_frac": gbs / hbm if gbs else None,
                "bytes_per_step": nbytes, "peak_gb_per_s": hbm}

    line.update({
        "slices_per_s": main["slices_per_s"],
        "bp_ms_per_step": main["bp_ms"], "filter_ms_per_step": main["filter_ms"],
        "filter_hbm": filter_hbm(main["filter_ms"], args.dtype),
        # filter + backprojection time of each timed step (CUDA events)
        "step_ms_spread": main["step_spread"],
        "bp_gupdates_per_s": achieved,
        "roofline": roofline_entry(achieved, rp, BP_STAGED_REGEX if main["staged"] else BP_KERNEL_REGEX, traffic,
                                   traffic_basis="ncu dram bytes per slice x slices, kernel unchanged "
                                                 "since capture (null otherwise)"),
        "onchip_measured": onchip,
        "clocks": main["clocks"],
        # filter, backprojection (+ the table pass of the staged path)
        "gpu_launches": (3 if main["staged"] else 2) * args.steps,
    })
    if "eager" in main:
        line["eager"] = main["eager"]
    for dt in dtypes[1:]:
        r = results[dt]
        rpd = roofline_peak(sm_max, dt, sms, onchip)
        ach = updates / (r["bp_ms"] / 1e3) / 1e9
        vdt = "fbp_backproject_staged (default shape)" if r["staged"] else resolved_variant(api, g, dt, args.variant)
        line[f"staged_{dt}"] = {
            "value": r["value"], "unit": UNIT, "ratio_to_f32": r["value"] / main["value"],
            "bp_gupdates_per_s": ach, "bp_ratio_to_f32": ach / achieved,
            "roofline_frac": ach / rpd["peak"], "roofline_peak": rpd["peak"],
            "roofline_frac_nominal": ach / rpd["peak_nominal"], "roofline_bound": rpd["bound"],
            "traffic": captured_traffic(vdt, dt, S, N, K),
            "slices_per_s": r["slices_per_s"], "ms_per_step": r["ms_per_step"],
            "bp_ms_per_step": r["bp_ms"], "filter_ms_per_step": r["filter_ms"],
            "filter_hbm": filter_hbm(r["filter_ms"], dt),
            "bp_variant": vdt}
        if "orbit_kernel" in r:
            line[f"staged_{dt}"]["orbit_kernel"] = r["orbit_kernel"]
    if "orbit_kernel" in main:
        line["orbit_kernel"] = main["orbit_kernel"]
    if tex is not None:
        tex["ratio_to_table"] = tex["bp_gupdates_per_s"] / achieved
        line["texture_alternative"] = tex
    if e2e is not None:
        line["e2e"] = e2e
    if not args.no_cpu_baseline and ws == 1:
        line["cpu_baseline"] = {k: v for k, v in cpu_sample(w, args.cpu_block).items() if k != "seconds"}
    return line


def run_pipeline(args) -> None:
    """Counts to codes (Sec. V-A(c) stages 2-4 on one GPU): one step =
    fbp_filter_counts (Beer-Lambert + Gaussian blur + ramp filter) and
    fbp_backproject_u16 (HU window to uint16) over the stack; the plain FP32
    FBP of the same stack's line integrals is timed in the same run."""
    import torch
    from paper_2505_13955_gb300 import api, phantoms

    ws, rank, dev = init_device()
    w = phantoms.WORKLOADS["fbp_pipeline_n8192"]
    N, K, S = w.n, w.n_angles, (args.slices or w.n_slices)
    g = api.Geometry(K, N, N)
    host = np.empty((S, K, N), dtype=np.float32)
    for i, s in enumerate(shard_slices(S, rank)):
        host[i] = phantoms.slice_counts(w, s)
    counts = torch.from_numpy(host).to(dev)
    P = phantoms.PIPELINE
    pre = api.Preprocess(flat_value=w.photons, count_floor=1.0, mu_scale=float(N),
                         blur_sigma=P["blur_sigma"])
    win = api.HuWindow(P["mu_water"], P["mu_air"], P["hu_min"], P["hu_max"])
    filt = torch.empty(counts.shape, dtype=torch.float32, device=dev)
    codes = torch.empty((S, N, N), dtype=torch.int16, device=dev)
    stream = torch.cuda.current_stream(dev)
    api.prepare(g, kind=w.filter, device=dev)
    updates = S * N * N * K
    staged = args.variant < 0 and api.staged_preferred(g)
    wsp = torch.empty(api.backproject_staged_workspace_bytes(g, torch.float32, S), dtype=torch.uint8,
                      device=dev) if staged else None
    T = Timed(stream, args.steps, args.warmup, n_events=3)

    def step(evs):
        if evs:
            evs[0].record(stream)
        api.filter_counts(counts, g, pre, kind=w.filter, out=filt)
        if evs:
            evs[1].record(stream)
        if staged:
            api.backproject_staged_u16(filt, g, win, out=codes, workspace=wsp)
        else:
            api.backproject_u16(filt, g, win, out=codes, variant=args.variant)
        if evs:
            evs[2].record(stream)

    ms = T.run(step, dev.index)
    assert api.device_status() == 0
    per_rank = allgather_floats([ms, float(updates)])
    rate, ms_step = aggregate([r[0] for r in per_rank], [int(r[1]) for r in per_rank])
    f_ms, bp_ms, clocks = T.between(0, 1), T.between(1, 2), T.clocks

    # the plain path on line integrals of the same stack, for the ratio
    out = torch.empty((S, N, N), dtype=torch.float32, device=dev)
    T2 = Timed(stream, args.steps, args.warmup)
    lines = -torch.log(counts.clamp_min(1.0) / w.photons) * N     # input preparation, not timed

    def plain(_):
        api.filter(lines, g, kind=w.filter, out=filt)
        if staged:
            api.backproject_staged(filt, g, out=out, workspace=wsp)
        else:
            api.backproject(filt, g, out=out, variant=args.variant)

    plain_ms = T2.run(plain, None)
    del lines, out

    e2e = None
    if args.e2e_steps > 0:
        pin_in = torch.from_numpy(host).pin_memory()
        pin_out = torch.empty((S, N, N), dtype=torch.int16).pin_memory()

        def e2e_step(_):
            api.fbp_host(pin_in, g, kind=w.filter, out=pin_out, variant=args.variant, pre=pre, window=win)

        T3 = Timed(stream, args.e2e_steps, 1)
        t_e2e = T3.run(e2e_step, None)
        per_rank_e2e = allgather_floats([t_e2e, float(updates)])
        e2e_rate, _ = aggregate([r[0] for r in per_rank_e2e], [int(r[1]) for r in per_rank_e2e])
        e2e = {"value": e2e_rate / 1e9, "unit": UNIT, "h2d_bytes_per_step": int(pin_in.numel() * 4),
               "d2h_bytes_per_step": int(pin_out.numel() * 2), "ms_per_step": t_e2e}
        del pin_in, pin_out

    if rank != 0:
        return None
    pk = peaks()
    sm_max, sms, onchip = device_ceilings(dev)
    rp = roofline_peak(sm_max, "f32", sms, onchip)
    achieved = updates / (bp_ms / 1e3) / 1e9
    hbm = pk.get("hbm_gbs")
    fbytes = S * K * N * 8.0                 # counts read + filtered rows written
    line = base_line(args, ws, rate / 1e9, ms_step, "f32", {
        "workload": f"{w.name}: S={S} slices per GPU, N=D={N}, K={K}, raw Poisson counts "
                    f"({w.photons:g} photons), Beer-Lambert + Gaussian blur sigma={P['blur_sigma']} + "
                    f"Ram-Lak + backprojection + HU window [{P['hu_min']}, {P['hu_max']}] to uint16",
        "l2": "inputs larger than L2, no flush",
        "parallelism": f"slices sharded over {ws} GPU(s), no collective",
        "bp_variant": "fbp_backproject_staged_u16 (default shape)" if staged else
                      resolved_variant(api, g, "f32", args.variant)})
    line.update({
        "slices_per_s": S * len(per_rank) / (ms_step / 1e3),
        "filter_counts_ms_per_step": f_ms, "bp_u16_ms_per_step": bp_ms,
        "filter_counts_gb_per_s": fbytes / (f_ms / 1e3) / 1e9,
        "filter_counts_hbm_frac": (fbytes / (f_ms / 1e3) / 1e9 / hbm) if hbm else None,
        "plain_fbp_ms_per_step": plain_ms, "ratio_to_plain_fbp": plain_ms / ms_step,
        "roofline": roofline_entry(achieved, rp, BP_KERNEL_REGEX),
        "clocks": clocks, "gpu_launches": (3 if staged else 2) * args.steps,
    })
    if e2e is not None:
        line["e2e"] = e2e
    if not args.no_cpu_baseline and ws == 1:
        line["cpu_baseline"] = cpu_sample_pipeline(w, args.cpu_block)
    return line


def run_offset(args) -> None:
    """Full-turn offset scans (Sec. V-A(b)): one step = fbp_filter_offset
    (overlap weight, virtual detector, fold of the rows half a turn apart)
    and fbp_backproject on the folded half-turn geometry.  The unfolded path
    (K weighted full-turn rows, backprojected over the full turn) is timed in
    the same run.  Updates are counted once per line: N^2 K/2 per slice."""
    import torch
    from paper_2505_13955_gb300 import api, phantoms

    ws, rank, dev = init_device()
    w = phantoms.WORKLOADS["fbp_offset_n8192"]
    D, c, delta = w.offset
    N, K, S = w.n, w.n_angles, (args.slices or w.n_slices)
    g = api.Geometry(K, D, N, angle_step=2 * np.pi / K, det_center=c)
    host = np.empty((S, K, D), dtype=np.float32)
    for i, s in enumerate(shard_slices(S, rank)):
        host[i] = phantoms.slice_sinogram(w, s)
    sino = torch.from_numpy(host).to(dev)
    del host
    out = torch.empty((S, N, N), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    updates = S * N * N * (K // 2)
    results = {}
    for fold in (True, False):
        gv, _ = api.offset_geometry(g, delta, fold)
        api.prepare(gv, kind=w.filter, device=dev)
        filt = torch.empty((S, gv.n_angles, gv.n_det), dtype=torch.float32, device=dev)
        # folded rows are a centred half turn: the staged path applies
        staged = args.variant < 0 and api.staged_preferred(gv)
        wsp = torch.empty(api.backproject_staged_workspace_bytes(gv, torch.float32, S), dtype=torch.uint8,
                          device=dev) if staged else None
        T = Timed(stream, args.steps if fold else max(1, args.steps // 2), args.warmup, n_events=3)

        def step(evs):
            if evs:
                evs[0].record(stream)
            api.filter_offset(sino, g, delta, fold, kind=w.filter, out=filt)
            if evs:
                evs[1].record(stream)
            if staged:
                api.backproject_staged(filt, gv, out=out, workspace=wsp)
            else:
                api.backproject(filt, gv, out=out, variant=args.variant)
            if evs:
                evs[2].record(stream)

        ms = T.run(step, dev.index if fold else None)
        assert api.device_status() == 0
        per_rank = allgather_floats([ms, float(updates)])
        rate, ms_step = aggregate([r[0] for r in per_rank], [int(r[1]) for r in per_rank])
        results[fold] = {"value": rate / 1e9, "ms_per_step": ms_step, "filter_ms": T.between(0, 1),
                         "bp_ms": T.between(1, 2), "clocks": T.clocks, "gv": gv,
                         "staged": staged,
                         "variant": "fbp_backproject_staged (default shape)" if staged else
                                    resolved_variant(api, gv, "f32", args.variant),
                         "slices_per_s": S * len(per_rank) / (ms_step / 1e3)}
        del filt
    if rank != 0:
        return None
    main, unf = results[True], results[False]
    sm_max, sms, onchip = device_ceilings(dev)
    rp = roofline_peak(sm_max, "f32", sms, onchip)
    achieved = updates / (main["bp_ms"] / 1e3) / 1e9
    gv = main["gv"]
    line = base_line(args, ws, main["value"], main["ms_per_step"], "f32", {
        "workload": f"{w.name}: S={S} slices per GPU, N={N}, K={K} angles on [0,2pi), offset detector "
                    f"D={D} with the axis at bin {c} (virtual detector {gv.n_det} bins), overlap "
                    f"half-width {delta} bins, seeded random ellipses (20-50), noise-free, {w.filter}; "
                    f"updates counted once per line (N^2 K/2 per slice)",
        "l2": "inputs larger than L2, no flush",
        "parallelism": f"slices sharded over {ws} GPU(s), no collective",
        "bp_variant": main["variant"]})
    line.update({
        "slices_per_s": main["slices_per_s"],
        "filter_offset_ms_per_step": main["filter_ms"], "bp_ms_per_step": main["bp_ms"],
        "bp_gupdates_per_s": achieved,
        "roofline": roofline_entry(achieved, rp, BP_KERNEL_REGEX),
        "unfolded": {"value": unf["value"], "unit": UNIT, "ms_per_step": unf["ms_per_step"],
                     "filter_offset_ms_per_step": unf["filter_ms"], "bp_ms_per_step": unf["bp_ms"],
                     "bp_variant": unf["variant"], "slices_per_s": unf["slices_per_s"]},
        "speedup_fold_vs_unfolded": unf["ms_per_step"] / main["ms_per_step"],
        "clocks": main["clocks"], "gpu_launches": (3 if main["staged"] else 2) * args.steps,
    })
    if not args.no_cpu_baseline and ws == 1:
        line["cpu_baseline"] = cpu_sample_offset(w, args.cpu_block)
    return line


def batch_launches(api, rows_geoms, tdt, variant) -> int:
    """Kernels one fbp_batched / fbp_batched_scans call launches: the batched
    filter; under the default (-1), for the items that run staged units, the
    table pass (and, for 16-bit rows, the per-item scale pass) and the staged
    persistent kernel; the persistent tile kernel for the other items."""
    import torch
    staged = sum(api.batched_item_staged(g, tdt) for g in rows_geoms) if variant < 0 else 0
    n = 1
    if staged:
        n += 2 + (tdt != torch.float32)
    if staged < len(rows_geoms):
        n += 1
    return n


def batch_roofline(api, dev, args, per_gpu_rate: float, variant: int) -> dict:
    """Roofline of a batch line: the whole graph-replayed step (batched
    filter, table pass and backprojection) against the backprojection
    ceiling of the rows' dtype -- a lower bound of the backprojection
    kernel's own fraction, which the step cannot time apart inside the
    graph."""
    smhz, sms, onchip = device_ceilings(dev)
    rp = roofline_peak(smhz, args.dtype, sms, onchip)
    kernel = ("bp_staged_batch_kernel (staged units) and bp_persistent_kernel" if variant < 0
              else f"bp_persistent_kernel (variant {variant})")
    return roofline_entry(per_gpu_rate, rp, kernel,
                          achieved_basis="updates of the batch / graph-replayed step time (filter and table "
                                         "pass included)")


def default_backproject(api, f, g, r, o, staged_ws):
    """One slice's backprojection as the library's single-slice default path
    (api.fbp) runs it: the staged kernel where api.staged_preferred(g), else
    fbp_backproject's default variant."""
    if api.staged_preferred(g):
        api.backproject_staged(f, g, r, out=o, workspace=staged_ws)
    else:
        api.backproject(f, g, row_scale=r, out=o, variant=-1)


def staged_workspace(api, geoms, tdt, dev):
    import torch
    need = max([api.backproject_staged_workspace_bytes(g, tdt, 1) for g in geoms if api.staged_preferred(g)],
               default=256)
    return torch.empty(need, dtype=torch.uint8, device=dev)


def run_ragged(args) -> None:
    """Ragged batch: all items in one fbp_batched call (one filter launch + one
    persistent backprojection launch), captured once in a CUDA graph and
    replayed; compared in the same run with per-slice fbp_filter +
    fbp_backproject launches.  The tile variant comes from the autotuner."""
    import torch
    from paper_2505_13955_gb300 import api, autotune, phantoms

    ws, rank, dev = init_device()
    w = phantoms.WORKLOADS["fbp_ragged_batch"]
    S = args.slices or w.n_slices
    idx = shard_slices(S, rank)
    sinos, geoms = [], []
    for i in idx:
        n, k, _, _ = phantoms.slice_spec(w, i)
        sinos.append(torch.from_numpy(phantoms.slice_sinogram(w, i)).to(dev))
        geoms.append(api.Geometry(k, n, n))
    updates = sum(g.n * g.n * g.n_angles for g in geoms)
    for g in geoms:
        api.prepare(g, kind=w.filter, device=dev)
    tdt = getattr(torch, DT[args.dtype])
    outs = [torch.empty((g.n, g.n), device=dev) for g in geoms]
    if args.variant >= 0:
        tuned = {"variant": args.variant}
    elif args.autotune:
        tuned = autotune.tune_batched(sinos, geoms, tdt, kind=w.filter)
    else:
        tuned = {"variant": -1}                     # the library's batch default, untuned
    variant = tuned["variant"]
    n_staged = sum(api.batched_item_staged(g, tdt) for g in geoms) if variant < 0 else 0
    wsp = torch.empty(api.batched_workspace_bytes(sinos, outs, geoms, tdt), dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(dev)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        api.fbp_batched(sinos, geoms, kind=w.filter, dtype=tdt, variant=variant, outs=outs, workspace=wsp)
    with torch.cuda.stream(stream):
        T = Timed(stream, args.steps, args.warmup)
        ms = T.run(lambda _: graph.replay(), dev.index)
        clocks = T.clocks
        # per-slice launches on the same stream: with the library's default
        # path for each slice (the baseline), and with the shape each item
        # ran in the batch
        filts = [torch.empty_like(s, dtype=tdt) for s in sinos]
        rss = [torch.empty((g.n_angles,), device=dev) if args.dtype != "f32" else None for g in geoms]
        sws = staged_workspace(api, geoms, tdt, dev)

        def per_slice_with(v):
            def run(_):
                for s, g, f, r, o in zip(sinos, geoms, filts, rss, outs):
                    api.filter(s, g, kind=w.filter, dtype=tdt, out=f, row_scale=r)
                    if v == "default":
                        default_backproject(api, f, g, r, o, sws)
                    elif v < 0 and api.batched_item_staged(g, tdt):
                        api.backproject_staged(f, g, r, out=o, workspace=sws_batch,
                                               shape=0 if tdt == torch.float32 else 5)
                    else:
                        vv = v if v >= 0 else (8 if tdt == torch.float32 else 10)
                        if not api.variant_supports(vv, g, tdt):
                            vv = 12 if api.bp_variants()[vv]["threads"] == 128 else 0
                        api.backproject(f, g, row_scale=r, out=o, variant=vv)
            return run

        sws_batch = torch.empty(max([api.backproject_staged_workspace_bytes(g, tdt, 1) for g in geoms
                                     if api.batched_item_staged(g, tdt)], default=256),
                                dtype=torch.uint8, device=dev)
        ms_single = Timed(stream, max(1, args.steps // 2), args.warmup).run(per_slice_with("default"), None)
        ms_same = Timed(stream, max(1, args.steps // 2), args.warmup).run(per_slice_with(variant), None)
    assert api.device_status() == 0
    per_rank = allgather_floats([ms, float(updates)])
    rate, ms_step = aggregate([r[0] for r in per_rank], [int(r[1]) for r in per_rank])
    if rank != 0:
        return None
    line = base_line(args, ws, rate / 1e9, ms_step, DT_LABEL[args.dtype], {
        "workload": f"{w.name}: {len(idx)} slices per GPU, N in {w.n_choices}, K in {w.k_choices}, "
                    "random ellipses, Ram-Lak; one persistent launch per step, CUDA-graph replay",
        "parallelism": f"slices sharded over {ws} GPU(s), no collective",
        "bp_variant": variant if variant >= 0 else
        f"library batch default: staged 32 x 32 orbit units for {n_staged} of {len(idx)} items, "
        f"persistent orbit variant {8 if args.dtype == 'f32' else 10} for the rest", "autotune": tuned})
    line.update({"slices_per_s": len(idx) * len(per_rank) / (ms_step / 1e3),
                 "per_slice_launches": {"value": updates / (ms_single / 1e3) / 1e9, "unit": UNIT,
                                        "ms_per_step": ms_single,
                                        "bp_variant": "library default per slice (fbp: staged kernel where "
                                                      "n >= 1024 and the orbit geometry, else variant 7)"},
                 "speedup_vs_per_slice": ms_single / ms,
                 "per_slice_launches_same_variant": {"value": updates / (ms_same / 1e3) / 1e9, "unit": UNIT,
                                                     "ms_per_step": ms_same,
                                                     "bp_variant": "each item's batch shape, one slice per launch"},
                 "clocks": clocks, "gpu_launches": batch_launches(api, geoms, tdt, variant) * args.steps})
    line["roofline"] = batch_roofline(api, dev, args, rate / 1e9 / ws, variant)
    return line


def run_mixed(args) -> None:
    """Normal and offset scans reconstructed together (Sec. V-A(b)): all
    items in one fbp_batched_scans call (one filter launch + one persistent
    backprojection launch), captured in a CUDA graph and replayed, once with
    the atomic work queue and once with the paper's group-and-cyclic order;
    per-scan launches of the same items are timed in the same run.  Updates
    are counted once per line (N^2 K for a normal item, N^2 K/2 for an
    offset item of K full-turn angles)."""
    import torch
    from paper_2505_13955_gb300 import api, phantoms

    ws, rank, dev = init_device()
    w = phantoms.WORKLOADS["fbp_mixed_batch"]
    S = args.slices or w.n_slices
    idx = shard_slices(S, rank)
    sinos, scans = [], []
    for i in idx:
        sp = phantoms.scan_spec(w, i)
        g = api.Geometry(sp["n_angles"], sp["n_det"], sp["n"], angle_step=sp["angle_step"],
                         det_center=sp["det_center"])
        sinos.append(torch.from_numpy(phantoms.scan_sinogram(sp)).to(dev))
        scans.append(api.Scan(g, sp["overlap"], True))
    rows_geoms = [api.offset_geometry(sc.g, sc.overlap, sc.fold)[0] if sc.overlap else sc.g for sc in scans]
    for gv in rows_geoms:
        api.prepare(gv, kind=w.filter, device=dev)
    updates = sum(g.n * g.n * g.n_angles for g in rows_geoms)
    n_off = sum(1 for sc in scans if sc.overlap)
    tdt = getattr(torch, DT[args.dtype])
    variant = args.variant              # -1: the library's batch default (staged units where they apply)
    n_staged = sum(api.batched_item_staged(g, tdt) for g in rows_geoms) if variant < 0 else 0
    outs = [torch.empty((g.n, g.n), device=dev) for g in rows_geoms]
    wsp = torch.empty(api.batched_scans_workspace_bytes(sinos, outs, scans, tdt), dtype=torch.uint8,
                      device=dev)
    stream = torch.cuda.Stream(dev)
    res = {}
    for order in ("queue", "group_cyclic"):
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            api.fbp_batched_scans(sinos, scans, kind=w.filter, dtype=tdt, variant=variant, order=order,
                                  outs=outs, workspace=wsp)
        with torch.cuda.stream(stream):
            T = Timed(stream, args.steps, args.warmup)
            res[order] = (T.run(lambda _: graph.replay(), dev.index if order == "queue" else None), T.clocks)
        del graph
    with torch.cuda.stream(stream):
        filts = [torch.empty((g.n_angles, g.n_det), dtype=tdt, device=dev) for g in rows_geoms]
        rss = [torch.empty((g.n_angles,), device=dev) if args.dtype != "f32" else None for g in rows_geoms]

        sws = staged_workspace(api, rows_geoms, tdt, dev)

        def per_scan(_):
            # each scan alone through the library's default single-scan path
            for s, sc, gv, f, r, o in zip(sinos, scans, rows_geoms, filts, rss, outs):
                if sc.overlap:
                    api.filter_offset(s, sc.g, sc.overlap, sc.fold, kind=w.filter, dtype=tdt, out=f,
                                      row_scale=r)
                else:
                    api.filter(s, sc.g, kind=w.filter, dtype=tdt, out=f, row_scale=r)
                default_backproject(api, f, gv, r, o, sws)

        T2 = Timed(stream, max(1, args.steps // 2), args.warmup)
        ms_single = T2.run(per_scan, None)
    assert api.device_status() == 0
    ms, clocks = res["queue"]
    per_rank = allgather_floats([ms, float(updates)])
    rate, ms_step = aggregate([r[0] for r in per_rank], [int(r[1]) for r in per_rank])
    per_rank_c = allgather_floats([res["group_cyclic"][0], float(updates)])
    rate_c, ms_c = aggregate([r[0] for r in per_rank_c], [int(r[1]) for r in per_rank_c])
    if rank != 0:
        return None
    line = base_line(args, ws, rate / 1e9, ms_step, DT_LABEL[args.dtype], {
        "workload": f"{w.name}: {len(idx)} scans per GPU ({n_off} offset: full turn, detector 9N/16 bins "
                    f"off the axis, folded), N in {w.n_choices}, half-turn K in {w.k_choices}, random "
                    "ellipses, Ram-Lak; one persistent launch per step, CUDA-graph replay, atomic work queue",
        "parallelism": f"scans sharded over {ws} GPU(s), no collective",
        "bp_variant": variant if variant >= 0 else
        f"library batch default: staged 32 x 32 orbit units for {n_staged} of {len(idx)} items, persistent "
        f"orbit variant {8 if args.dtype == 'f32' else 10} (generic 64 x 64 tiles without the symmetry) "
        "for the rest"})
    line.update({"slices_per_s": len(idx) * len(per_rank) / (ms_step / 1e3),
                 "group_cyclic": {"value": rate_c / 1e9, "unit": UNIT, "ms_per_step": ms_c,
                                  "ratio_to_queue": ms_step / ms_c},
                 "per_scan_launches": {"value": updates / (ms_single / 1e3) / 1e9, "unit": UNIT,
                                       "ms_per_step": ms_single,
                                       "bp_variant": "library default per scan (staged kernel where n >= 1024 "
                                                     "and the orbit geometry, else variant 7 / 5)"},
                 "speedup_vs_per_scan": ms_single / ms,
                 "clocks": clocks, "gpu_launches": batch_launches(api, rows_geoms, tdt, variant) * args.steps})
    line["roofline"] = batch_roofline(api, dev, args, rate / 1e9 / ws, variant)
    return line


SAP_STREAMS = 8          # slices of the patching workload in flight
SAP_BYTES_PER_PIXEL = 8   # codes read by Canny (2) + edge map written (1) + codes and edges read by
                          # the tree sums (3) + codes read by the patch means (2)


def run_sap(args) -> None:
    """Adaptive patching of reconstructed slices (Sec. V-B(c)): one step =
    sap_edges + sap_patches for each of the stack's 16 uint16 slices
    (n = 8192, 16 x 16 patches, 4096 per slice); the 2-bit mask path
    (sap_depatch_pack of random four-class patches) is timed after it.
    Throughput in slices/s; the roofline is HBM bandwidth at the step's
    algorithmic bytes (8 per pixel)."""
    import torch
    from paper_2505_13955_gb300 import api, phantoms

    ws, rank, dev = init_device()
    w = phantoms.WORKLOADS["sap_patching_n8192"]
    c = phantoms.SAP
    n, S = w.n, (args.slices or w.n_slices)
    host = np.empty((S, n, n), dtype=np.uint16)
    for i, s_ in enumerate(shard_slices(S, rank)):
        host[i] = phantoms.sap_slice(n, phantoms.slice_seed(w.config_id, s_))
    slices = torch.from_numpy(host.view(np.int16)).to(dev)
    p = api.SapParams(n, c["patch"], c["length"], c["canny_lo"], c["canny_hi"])
    # SAP_STREAMS slices in flight, each stream with its own workspace and
    # edge map: one slice's serial tail (the one-block selection, the small
    # top levels of the tree) overlaps another slice's Canny
    n_str = min(SAP_STREAMS, S)
    wsps = [torch.empty(api.sap_workspace_bytes(p), dtype=torch.uint8, device=dev) for _ in range(n_str)]
    edgess = [torch.empty((n, n), dtype=torch.uint8, device=dev) for _ in range(n_str)]
    patches = torch.empty((S, p.length, p.patch, p.patch), dtype=torch.float32, device=dev)
    leaves = torch.empty((S, p.length, 3), dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    side = [torch.cuda.Stream(dev) for _ in range(n_str)]
    T = Timed(stream, args.steps, args.warmup, n_events=3)

    def step(evs):
        start = torch.cuda.Event()
        start.record(stream)
        for k in range(n_str):
            side[k].wait_event(start)
        for i in range(S):
            k = i % n_str
            with torch.cuda.stream(side[k]):
                if evs and i == 0:
                    evs[0].record(side[k])
                api.sap_edges(slices[i], p, out=edgess[k], workspace=wsps[k])
                if evs and i == 0:
                    evs[1].record(side[k])
                api.sap_patches(slices[i], edgess[k], p, patches=patches[i], leaves=leaves[i], workspace=wsps[k])
                if evs and i == 0:
                    evs[2].record(side[k])
        for k in range(n_str):
            done = torch.cuda.Event()
            done.record(side[k])
            stream.wait_event(done)

    ms = T.run(step, dev.index)
    assert api.device_status() == 0
    edges_ms, patches_ms, clocks = T.between(0, 1), T.between(1, 2), T.clocks
    rng = np.random.default_rng(0)
    masks = torch.from_numpy(rng.integers(0, 4, (S, p.length, p.patch, p.patch)).astype(np.uint8)).to(dev)
    packed = torch.empty((S, n, n // 4), dtype=torch.uint8, device=dev)
    T2 = Timed(stream, args.steps, args.warmup)

    def unpatch(_):
        for i in range(S):
            api.sap_depatch_pack(masks[i], leaves[i], p, out=packed[i])

    ms_pack = T2.run(unpatch, None)
    assert api.device_status() == 0

    e2e = None
    if args.e2e_steps > 0:
        pin_in = torch.from_numpy(host.view(np.int16)).pin_memory()
        pin_p = torch.empty(patches.shape, dtype=torch.float32).pin_memory()
        pin_l = torch.empty(leaves.shape, dtype=torch.int32).pin_memory()

        def e2e_step(_):
            # the public host-buffer call: copies of one slice overlap another's kernels
            api.sap_host(pin_in, p, patches=pin_p, leaves=pin_l)

        T3 = Timed(stream, args.e2e_steps, 1)
        t_e2e = T3.run(e2e_step, None)
        e2e = {"value": S / (t_e2e / 1e3), "unit": "slices/s", "h2d_bytes_per_step": int(pin_in.numel() * 2),
               "d2h_bytes_per_step": int(pin_p.numel() * 4 + pin_l.numel() * 4), "ms_per_step": t_e2e}
    per_rank = allgather_floats([ms, float(S)])
    rate, ms_step = aggregate([r[0] for r in per_rank], [int(r[1]) for r in per_rank])
    if rank != 0:
        return None
    hbm = peaks().get("hbm_gbs") or 6800.0
    gbs = SAP_BYTES_PER_PIXEL * n * n * S / (ms / 1e3) / 1e9
    line = base_line(args, ws, rate, ms_step, "u16 codes, exact integer / f64", {
        "workload": f"{w.name}: S={S} uint16 slices per GPU, n={n}, seeded random-ellipse phantoms "
                    f"(codes {phantoms.SAP_CODES}), patch {p.patch}, {p.length} patches per slice, Canny "
                    f"thresholds {p.canny_lo}/{p.canny_hi}",
        "l2": "inputs larger than L2 (2.1 GB of slices per step), no flush",
        "streams": f"{n_str} slices in flight, each stream with its own workspace",
        "parallelism": f"slices sharded over {ws} GPU(s), no collective"})
    line["metric"] = SAP_METRIC
    line["unit"] = "slices/s"
    line.update({
        "sap_edges_ms_per_slice": edges_ms, "sap_patches_ms_per_slice": patches_ms,
        "depatch_pack": {"ms_per_step": ms_pack, "slices_per_s": S / (ms_pack / 1e3),
                         "gb_per_s": (p.length * p.patch ** 2 + n * n // 4) * S / (ms_pack / 1e3) / 1e9},
        "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                     "traffic": None, "kernel": "whole SAP step",
                     "basis": f"{SAP_BYTES_PER_PIXEL} algorithmic bytes per pixel per step / step time; "
                              "peak = measured HBM copy (MEASURED_PEAKS.json)"},
        "clocks": clocks, "gpu_launches": S * (5 + 3 * int(np.log2(n // p.patch)) + 5) * args.steps})
    if e2e is not None:
        line["e2e"] = e2e
    if not args.no_cpu_baseline and ws == 1:
        line["cpu_baseline"] = cpu_sample_sap(max(256, min(2048, args.cpu_block)), n)
    return line


def run_gd(args) -> None:
    """Least-squares refinement: one step = one gradient-descent iteration
    x <- x - eta A^T (A x - b) over the stack (radon_forward, then
    fbp_backproject with scale 1); A and A^T are timed separately.  Then the
    refinement as specified -- 50 iterations from the FBP start -- is timed
    once, with the loss 0.5 ||A x - b||^2 before and after."""
    import torch
    from paper_2505_13955_gb300 import api, phantoms

    ws, rank, dev = init_device()
    w = phantoms.WORKLOADS["gd_refine_n1024"]
    N, K, S = w.n, w.n_angles, (args.slices or w.n_slices)
    g = api.Geometry(K, N, N)
    b = torch.from_numpy(make_inputs(w, shard_slices(S, rank))).to(dev)
    api.prepare(g, kind=w.filter, device=dev)
    x = api.fbp(b, g, kind=w.filter)
    # step size 1 / lambda_max(A^T A) from power iterations on the device (not timed)
    v = torch.randn((N, N), device=dev)
    lam = 1.0
    for _ in range(10):
        v = api.backproject(api.radon_forward(v, g), g, scale=1.0)
        lam = v.norm().item()
        v /= lam
    eta = 1.0 / (1.05 * lam)
    r = torch.empty_like(b)
    grad = torch.empty_like(x)
    stream = torch.cuda.current_stream(dev)
    T = Timed(stream, args.steps, args.warmup, n_events=3)

    def step(evs):
        if evs:
            evs[0].record(stream)
        api.radon_forward(x, g, out=r, variant=args.fwd_variant)
        if evs:
            evs[1].record(stream)
        r.sub_(b)
        api.backproject(r, g, scale=1.0, out=grad)
        if evs:
            evs[2].record(stream)
        x.sub_(eta * grad)

    ms = T.run(step, dev.index)
    assert api.device_status() == 0

    # the refinement itself: 50 iterations from the FBP start, the loss
    # 0.5 ||A x - b||^2 evaluated on the device before and after
    x.copy_(api.fbp(b, g, kind=w.filter))

    def loss():
        api.radon_forward(x, g, out=r, variant=args.fwd_variant)
        r.sub_(b)
        return 0.5 * (r.double() ** 2).sum()

    l0 = loss()
    a50, b50 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a50.record(stream)
    for _ in range(50):
        step(None)
    b50.record(stream)
    torch.cuda.synchronize()
    refine = {"iterations": 50, "ms": a50.elapsed_time(b50), "loss_start": float(l0),
              "loss_end": float(loss())}
    assert api.device_status() == 0
    updates = 2 * S * N * N * K
    per_rank = allgather_floats([ms, float(updates)])
    rate, ms_step = aggregate([r_[0] for r_ in per_rank], [int(r_[1]) for r_ in per_rank])
    if rank != 0:
        return None
    a_ms, at_ms = T.between(0, 1), T.between(1, 2)
    fwd_variant = args.fwd_variant if args.fwd_variant >= 0 else 4
    sm_max, sms, onchip = device_ceilings(dev)
    rp = roofline_peak(sm_max, "f32", sms, onchip)
    a_rate = S * N * N * K / a_ms / 1e6
    line = base_line(args, ws, rate / 1e9, ms_step, "f32", {
        "workload": f"{w.name}: S={S} slices per GPU, N=D={N}, K={K}, Poisson 1e4 photons, "
                    "one gradient-descent iteration (A and A^T) per step",
        "parallelism": f"slices sharded over {ws} GPU(s), no collective"})
    line["config"]["forward_variant"] = fwd_variant
    line.update({"forward_A": {"ms": a_ms, "gupdates_per_s": a_rate},
                 "adjoint_AT": {"ms": at_ms, "gupdates_per_s": S * N * N * K / at_ms / 1e6},
                 # the forward projector dominates the step; it has the
                 # backprojection's per-update accounting (one pixel-angle pair)
                 "roofline": roofline_entry(a_rate, rp, "fwd_tile_kernel" if fwd_variant else "fwd_strip_kernel"),
                 "refine_50": refine,
                 "eta": eta, "clocks": T.clocks,
                 # the forward projector, then A^T: the staged table pass and kernel
                 # (one pass over the stack) where staged_preferred, else one kernel
                 "gpu_launches": (3 if api.staged_preferred(g) and api.staged_chunk(g, torch.float32, S) >= S
                                  else 2) * args.steps,
                 "adjoint_kernel": "fbp_backproject_staged" if api.staged_preferred(g) else
                                   f"fbp_backproject variant {resolved_variant(api, g, 'f32', -1)}"})
    if not args.no_cpu_baseline and ws == 1:
        line["cpu_baseline"] = cpu_sample_gd(w)
    return line


RUNNERS = {
    "fbp_ragged_batch": run_ragged,
    "gd_refine_n1024": run_gd,
    "fbp_pipeline_n8192": run_pipeline,
    "fbp_offset_n8192": run_offset,
    "fbp_mixed_batch": run_mixed,
    "sap_patching_n8192": run_sap,
}

# Compact runs of the other workloads after the headline (one GPU): the key,
# the workload, and what differs from the headline's arguments.  Slice counts
# below a workload's own are stated in its config ("slices_per_gpu").
SUB_RECORDS = (
    # (steps sized so that every timed region lasts at least ~0.5 s: the clock
    # sampler reads nvidia-smi every 200 ms)
    ("config1_fbp_single_n256", "fbp_single_n256",
     dict(steps=40000, e2e_steps=20, all_dtypes=False, texture=False, cpu_block=256)),
    ("config2_fbp_stack_n2048", "fbp_stack_n2048",
     dict(steps=5, e2e_steps=1, all_dtypes=True, texture=False, cpu_block=256)),
    ("config4_fbp_ragged_batch", "fbp_ragged_batch", dict(steps=5)),
    ("config5_gd_refine_n1024", "gd_refine_n1024", dict(steps=30)),
    ("f1_pipeline_n8192", "fbp_pipeline_n8192", dict(steps=3, slices=4, e2e_steps=1, cpu_block=256)),
    ("f2_offset_n8192", "fbp_offset_n8192", dict(steps=4, slices=4, cpu_block=256)),
    ("f3_mixed_batch", "fbp_mixed_batch", dict(steps=5)),
    ("f4_sap_patching_n8192", "sap_patching_n8192", dict(steps=50, slices=16, e2e_steps=2, cpu_block=1024)),
)
SUB_DROP = ("n_gpus", "higher_is_better", "scaling", "vs_baseline", "data")


def run_sub_records(args, head: dict) -> dict:
    """Every other workload in a compact form (fewer steps, fewer slices for
    the 8192^2 counts, offset and patching stacks), each with its own value,
    step time, roofline where one applies, CPU baseline and clocks."""
    import copy
    import torch
    out = {}
    for key, workload, over in SUB_RECORDS:
        a = copy.copy(args)
        a.workload, a.warmup, a.variant, a.fwd_variant = workload, 3, -1, -1
        a.dtype, a.traffic_bytes, a.slices, a.sub_records = "f32", None, None, False
        for name, v in over.items():
            setattr(a, name, v)
        t0 = time.perf_counter()
        try:
            sub = RUNNERS.get(workload, run_uniform)(a)
        except Exception as e:           # one workload's failure must not hide the others
            sub = {"error": f"{type(e).__name__}: {e}"}
        torch.cuda.empty_cache()
        if sub is None:
            continue
        for name in SUB_DROP:
            sub.pop(name, None)
        if a.slices is not None and "config" in sub:
            sub["config"]["slices_per_gpu"] = a.slices
        if "cpu_baseline" not in sub and "error" not in sub and "cpu_baseline" in head \
                and workload in ("fbp_ragged_batch", "fbp_mixed_batch"):
            cb = dict(head["cpu_baseline"])
            cb["sample"] = "the headline stack's oracle sample (per-update cost): " + cb["sample"]
            sub["cpu_baseline"] = cb
        sub["wall_s"] = time.perf_counter() - t0
        out[key] = sub
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--dtype", choices=["f32", "f16", "bf16"], default="f32")
    ap.add_argument("--all-dtypes", action=argparse.BooleanOptionalAction, default=True,
                    help="also time FP16- and BF16-staged rows in the same run")
    ap.add_argument("--variant", type=int, default=-1)
    ap.add_argument("--graph", choices=["auto", "on", "off"], default="auto",
                    help="uniform stacks: replay each step from a CUDA graph (auto: steps under "
                         f"{GRAPH_BELOW_UPDATES:.0e} updates, which the host's launch path would bound)")
    ap.add_argument("--autotune", action=argparse.BooleanOptionalAction, default=True,
                    help="ragged batch with --variant -1: pick the backprojection by the autotuner "
                         "(--no-autotune: the library's batch default)")
    ap.add_argument("--fwd-variant", type=int, default=-1,
                    help="radon_forward kernel for the refinement workload (-1 = default)")
    ap.add_argument("--slices", type=int, default=None,
                    help="slices per GPU (default: the workload's); small cases for profiling")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--texture", action=argparse.BooleanOptionalAction, default=True,
                    help="also time the texture-unit backprojection (FP32 rows) in the same run")
    ap.add_argument("--cpu-block", type=int, default=1024)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--traffic-bytes", type=float, default=None,
                    help="DRAM bytes per backprojection launch from an ncu capture")
    ap.add_argument("--sub-records", action=argparse.BooleanOptionalAction, default=True,
                    help="after the headline workload (one GPU), also run every other workload "
                         "in a compact form and attach its line under sub_records")
    args = ap.parse_args(argv)
    args.warmup = max(3, args.warmup)   # at least 3 untimed warm-up steps
    if args.impl == "reference":
        run_reference(args)
        return
    ws, rank, _ = init_device()
    line = RUNNERS.get(args.workload, run_uniform)(args)
    if args.sub_records and args.workload == WORKLOAD and ws == 1 and line is not None:
        line["sub_records"] = run_sub_records(args, line)
    if rank == 0 and line is not None:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
