"""The parameter autotuner: cache keys and files on the CPU; on the GPU a
tuning run picks a converging candidate, caches it and is reused."""

import json

import numpy as np
import pytest

from paper_2401_06747_b300 import autotune


def test_keys_and_candidates():
    assert autotune.size_class(2160, 3840) == "2^23"
    assert autotune.density_bucket(0.04) == "4%"
    assert autotune.density_bucket(0.05) == "4%" and autotune.density_bucket(0.07) == "8%"
    k = autotune.cache_key("B300", 2160, 3840, 3, 0.04, "tonal")
    assert k == "B300|2^23|c3|4%|tonal"
    c = autotune.candidates({"b": (1, 2), "a": (3,)})
    assert c == [{"a": 3, "b": 1}, {"a": 3, "b": 2}]
    assert len(autotune.candidates(autotune.INPAINT_GRID)) == 12
    # tiling stage: subdomain layout and its size threshold, row staging, strip rows, RAS block side
    assert len(autotune.candidates(autotune.INPAINT_SHAPES)) == 36
    assert len(autotune.candidates(autotune.TONAL_SHAPES)) == 32
    assert {c["tonal_block"] for c in autotune.candidates(autotune.TONAL_SHAPES)} == {32, 64}


def test_cache_round_trip(tmp_path):
    p = str(tmp_path / "tune.json")
    assert autotune.load_cache(p) == {}
    autotune.save_cache(p, {"k": {"params": {"oras_theta": 0.2}}})
    assert json.load(open(p)) == {"k": {"params": {"oras_theta": 0.2}}}
    assert autotune.load_cache(p)["k"]["params"]["oras_theta"] == 0.2


@pytest.mark.gpu
def test_tune_on_gpu(tmp_path):
    from gpu_util import need_gpu, dev, torch
    from synthdata import synth_rgb, random_mask
    import paper_2401_06747_b300 as hdi
    need_gpu()
    f = dev(synth_rgb(192, 256, seeds=(1, 2, 3), dtype=np.float32))
    c = dev(random_mask(192, 256, 0.04, 5))
    p = str(tmp_path / "tune.json")
    grid = {"oras_theta": (0.2, 0.3), "oras_eta": (1e-2, 1e-3)}
    shapes = {"oras_warp": (0, 1), "strip_rows": (0, 8)}
    best = autotune.tune(0, f, c, "inpaint", tol=1e-6, cache_path=p, grid=grid, shapes=shapes)
    assert best["oras_theta"] in (0.2, 0.3) and best["oras_eta"] in (1e-2, 1e-3)
    assert best["oras_warp"] in (0, 1) and best["strip_rows"] in (0, 8)
    cache = json.load(open(p))
    (entry,) = cache.values()
    assert entry["params"] == best and len(entry["table"]) == 8
    assert {r["stage"] for r in entry["table"]} == {"tiling", "parameters"}
    assert autotune.tune(0, f, c, "inpaint", cache_path=p, grid=grid) == best   # from the cache
    out = torch.empty_like(f)
    st = hdi.Context(0, **best).inpaint(f, c, out, tol=1e-6)
    assert st["rel_res"] <= 1e-6
