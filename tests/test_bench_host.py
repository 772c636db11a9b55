"""Host logic of bench.py's multi-GPU path, run as two gloo ranks on CPU:
slices shard with no overlap, per-rank times gather to every rank, and the
job rate is total units over the slowest rank's time."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        env = bench.dist_env()
        mine = bench.shard_slices(16, rank)
        elapsed = 100.0 + 50.0 * rank          # rank 1 is the slow one
        units = 16 * 8192 * 8192 * 4096
        gathered = bench.allgather_floats([elapsed, float(units)])
        bench.barrier()
        rate, t = bench.aggregate([g[0] for g in gathered], [int(g[1]) for g in gathered])
        q.put((rank, env, mine, gathered, rate, t))
    finally:
        dist.destroy_process_group()


def test_two_rank_sharding_and_aggregation():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, env0, s0, g0, rate0, t0), (r1, env1, s1, g1, rate1, t1) = res
    assert env0 == (2, 0, 0) and env1 == (2, 1, 1)
    assert set(s0).isdisjoint(s1) and len(s0) == len(s1) == 16
    assert g0 == g1 == [[100.0, float(16 * 8192 * 8192 * 4096)], [150.0, float(16 * 8192 * 8192 * 4096)]]
    assert t0 == t1 == 150.0
    assert rate0 == pytest.approx(2 * 16 * 8192 * 8192 * 4096 / 0.150)


def test_aggregate_single_rank():
    rate, t = bench.aggregate([80.0], [1000])
    assert t == 80.0 and rate == pytest.approx(1000 / 0.08)


class _FakeEvent:
    """Stands in for torch.cuda.Event on a CPU host: each record() advances
    a shared clock by 1 ms before taking the time."""
    clock = 0.0

    def __init__(self, enable_timing=False):
        self.t = None

    def record(self, stream=None):
        _FakeEvent.clock += 1.0
        self.t = _FakeEvent.clock

    def elapsed_time(self, other):
        return other.t - self.t


def test_timed_reports_each_steps_time_and_their_spread(monkeypatch):
    import torch
    monkeypatch.setattr(torch.cuda, "Event", _FakeEvent)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    T = bench.Timed(None, steps=5, warmup=3, n_events=2)
    work = iter([1.0, 3.0, 2.0, 5.0, 4.0])
    calls = []

    def step(evs):
        calls.append(evs is not None)
        if evs:
            evs[0].record()
            _FakeEvent.clock += next(work)
            evs[1].record()

    ms = T.run(step, None)
    assert calls == [False] * 3 + [True] * 5                 # warm-up steps record nothing
    # each step spans its work + 1 ms of the second record; 5 steps + the bracketing events
    assert T.spread(0, 1) == {"median": 4.0, "min": 2.0, "max": 6.0, "n": 5}
    assert T.between(0, 1) == 4.0
    assert ms == (15.0 + 10.0 + 1.0) / 5


@pytest.mark.slow
def test_reference_arm_prints_one_contract_line():
    """`bench.py --impl reference` times the FP64 oracle on the host cores
    (no GPU involved) and prints one JSON line with the contract's keys."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"],
                       cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "Gupdates/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] >= 3
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_roofline_ceilings_nominal_and_measured():
    """The FP32-row ceiling is the shared-load path (8 B per update through
    128 B/clk/SM = 16 updates/clk/SM) and the 16-bit one ties it with the
    ALU (32 updates/clk/SM); measured per-SM rates replace the nominal ones
    and the binding unit follows them; the SM count is a parameter."""
    rp = bench.roofline_peak(2000.0, "f32", 100)
    assert rp["measured"] is False and rp["bound"] == "lds"
    assert rp["c_lds"] == pytest.approx(100 * 16 * 2000e6 / 1e9)
    assert rp["c_alu"] == pytest.approx(100 * 32 * 2000e6 / 1e9)
    assert rp["peak"] == rp["peak_nominal"] == rp["c_lds"]
    r16 = bench.roofline_peak(2000.0, "f16", 100)
    assert r16["c_lds"] == pytest.approx(r16["c_alu"])
    onchip = {"lds_bytes_per_clk_per_sm": 120.0, "fma_per_clk_per_sm": 100.0}
    m = bench.roofline_peak(2000.0, "f16", 100, onchip)
    assert m["measured"] is True
    assert m["c_lds"] == pytest.approx(100 * 120 / 4 * 2000e6 / 1e9)      # 30 updates/clk/SM
    assert m["c_alu"] == pytest.approx(100 * 100 / 4 * 2000e6 / 1e9)      # 25 updates/clk/SM
    assert m["bound"] == "alu" and m["peak"] == m["c_alu"]
    assert m["peak_nominal"] == pytest.approx(r16["peak"])
    e = bench.roofline_entry(0.5 * m["peak"], m, "k")
    assert e["frac"] == pytest.approx(0.5) and e["bound"] == "alu"
    assert e["frac_nominal"] == pytest.approx(0.5 * m["peak"] / m["peak_nominal"])


def test_sub_records_cover_every_workload_and_survive_a_failure(monkeypatch):
    """The default run attaches one compact line per other workload (BASELINE
    configs 1, 2, 4, 5 and the next rows f1-f4); a runner that raises is
    recorded as an error without losing the others; overrides reach the
    runner and the ragged batches borrow the headline's CPU baseline."""
    import argparse
    keys = [k for k, _, _ in bench.SUB_RECORDS]
    for want in ("config1", "config2", "config4", "config5", "f1_", "f2_", "f3_", "f4_"):
        assert sum(k.startswith(want) for k in keys) == 1, want
    seen = {}

    def fake(a):
        seen[a.workload] = a
        if a.workload == "gd_refine_n1024":
            raise RuntimeError("boom")
        return {"metric": "m", "value": 1.0, "n_gpus": 1, "config": {"workload": a.workload}}

    monkeypatch.setattr(bench, "RUNNERS", {w: fake for _, w, _ in bench.SUB_RECORDS})
    monkeypatch.setattr(bench, "run_uniform", fake)
    args = argparse.Namespace(steps=20, warmup=5, variant=3, fwd_variant=2, dtype="bf16", traffic_bytes=1.0,
                              slices=None, sub_records=True, e2e_steps=2, all_dtypes=True, texture=True,
                              cpu_block=1024, no_cpu_baseline=False)
    head = {"cpu_baseline": {"value": 3.0, "sample": "s"}}
    out = bench.run_sub_records(args, head)
    assert list(out) == keys
    assert out["config5_gd_refine_n1024"]["error"] == "RuntimeError: boom"
    assert "n_gpus" not in out["config1_fbp_single_n256"]
    assert out["f4_sap_patching_n8192"]["config"]["slices_per_gpu"] == 16
    assert out["config4_fbp_ragged_batch"]["cpu_baseline"]["value"] == 3.0
    assert "cpu_baseline" not in out["config2_fbp_stack_n2048"]
    a = seen["fbp_single_n256"]
    assert (a.steps, a.warmup, a.variant, a.dtype, a.texture) == (40000, 3, -1, "f32", False)
    assert args.steps == 20 and args.variant == 3          # the headline's arguments are untouched
