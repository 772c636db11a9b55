"""GPU: the tile-shape autotuner picks a variant that exists and runs, caches
it by workload key, and the cached choice is returned without re-timing."""
import json

import pytest

from gpu_util import fbp_api, needs_gpu, torch

pytestmark = [pytest.mark.gpu, needs_gpu]


def test_autotune_single_and_batched(tmp_path, monkeypatch):
    monkeypatch.setenv("FBP_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    from paper_2505_13955_gb300 import autotune
    api = fbp_api()
    g = api.Geometry(64, 128, 128)
    r = autotune.tune_single(g, torch.float16, reps=1)
    assert api.variant_supports(r["variant"], g, torch.float16)
    assert r["gupdates_per_s"] > 0 and str(r["variant"]) in r["times_ms"]
    # every supported variant was timed
    supported = [v["variant"] for v in api.bp_variants() if api.variant_supports(v["variant"], g, torch.float16)]
    assert sorted(int(k) for k in r["times_ms"]) == supported
    again = autotune.tune_single(g, torch.float16, reps=1)
    assert again == r
    sinos = [torch.randn((30, 64), device="cuda"), torch.randn((50, 96), device="cuda")]
    geoms = [api.Geometry(30, 64, 64), api.Geometry(50, 96, 96)]
    rb = autotune.tune_batched(sinos, geoms, reps=1)
    # the default (-1: staged units where an item allows them) and every
    # persistent shape but the texture and packed ones were timed
    cands = [-1] + [v["variant"] for v in api.bp_variants() if not v["texture"] and not v["packed16"]]
    assert sorted(int(k) for k in rb["times_ms"]) == sorted(cands)
    assert rb["variant"] in cands
    outs = api.fbp_batched(sinos, geoms, variant=rb["variant"])
    assert all(torch.isfinite(o).all() for o in outs)
    data = json.load(open(tmp_path / "tune.json"))
    assert len(data) == 2
