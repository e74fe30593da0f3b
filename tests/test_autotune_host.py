"""The autotuner's host logic without a GPU: the cache key, the choice of the
fastest candidate, and that a cached result skips the timing (a fake timer
stands in for the CUDA-event timing; the grid build needs the device, so the
tune() round trip is in the GPU tests)."""
import json

import pytest

from paper_2304_11165_b300 import autotune


def test_cache_key_rounds_the_fill_and_names_every_field():
    k = autotune.cache_key("NVIDIA B300", "f32r", 1, 0.6749)
    assert k == "NVIDIA B300|f32r|1|fill0.7"
    assert autotune.cache_key("NVIDIA B300", "f32r", 2, 0.6749) != k
    assert autotune.cache_key("NVIDIA B300", "f32", 1, 0.6749) != k
    assert autotune.cache_key("NVIDIA B300", "f32r", 1, 0.61) == "NVIDIA B300|f32r|1|fill0.6"


def test_pick_best_takes_the_least_time_per_update():
    table = [dict(block=4, variant="async", ctas_per_sm=0, ns_per_voxel_update=0.030),
             dict(block=8, variant="async", ctas_per_sm=0, ns_per_voxel_update=0.025),
             dict(block=4, variant="pipelined", ctas_per_sm=4, ns_per_voxel_update=0.025)]
    assert autotune.pick_best(table) is table[1]


def test_cache_round_trip(tmp_path, monkeypatch):
    path = tmp_path / "tune.json"
    monkeypatch.setenv("SBG_AUTOTUNE_CACHE", str(path))
    assert autotune.cache_path() == str(path)
    autotune._save_cache({"k": {"block": 4}})
    assert json.load(open(path)) == {"k": {"block": 4}}
    assert autotune._load_cache() == {"k": {"block": 4}}
    path.write_text("not json")
    assert autotune._load_cache() == {}
