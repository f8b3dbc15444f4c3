"""Host logic of the tile autotuner (paper_1402_4089_gb300/tune.py): candidate
enumeration, choice of the fastest measured tile, the per-device cache and the
fallback when no explicit tile runs.  The timing itself is replaced by a fake
(the measurement runs on the GPU in the bench)."""
import json

import numpy as np
import pytest

from paper_1402_4089_gb300 import tune


@pytest.fixture
def fake(monkeypatch, tmp_path):
    import torch
    monkeypatch.setenv("HMC_TUNE_CACHE", str(tmp_path / "tune.json"))
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda *a: "FakeGPU")
    calls = []

    def timer(times):
        def time_tile(X, y, K, prior, scale, xs, st, chains, engine, tile, stream=None, reps=5, layout="free"):
            calls.append((engine, tile, layout))
            us = times.get((engine, tile[0], tile[3]))
            if us is None:
                return None, None
            return us, {"problems": [{"nclusters": 3, "group_chains": chains, "smem": 1000}]}
        monkeypatch.setattr(tune, "time_tile", time_tile)
    return calls, timer, tmp_path / "tune.json"


def _xy():
    return np.zeros((100, 30), np.float32), np.zeros(100, np.int32)


def test_picks_the_fastest_and_caches_it(fake):
    calls, timer, cache = fake
    timer({(1, 4, 3): 50.0, (1, 2, 2): 40.0, (1, 16, 4): 90.0})
    X, y = _xy()
    eng, tile, table = tune.autotune(X, y, 3, chains=2)
    assert (eng, tile) == (1, (2, 0, 0, 2))
    # every CUDA-core candidate was tried: cluster sizes x ring depths, and the two-pass CUDA-core engine
    assert len(calls) == len(tune.SIMT_S) * len(tune.RING) + 1
    assert [c for c in calls if c[0] == 4] == [(4, (0, 0, 0, 0), "free")]
    assert sorted(r["us"] for r in table) == [40.0, 50.0, 90.0]
    d = json.load(open(cache))
    (key, entry), = d.items()
    assert "FakeGPU" in key and "chains=2" in key and entry["tile"] == [2, 0, 0, 2]
    n = len(calls)
    assert tune.autotune(X, y, 3, chains=2)[:2] == (1, (2, 0, 0, 2))    # from the cache, no new timing
    assert len(calls) == n


def test_reduced_precision_tries_both_engines(fake):
    calls, timer, _ = fake
    timer({(2, 8, 3): 30.0, (1, 4, 4): 31.0})
    X, y = _xy()
    eng, tile, _ = tune.autotune(X, y, 3, x_storage="bf16", chains=1)
    assert (eng, tile) == (2, (8, 0, 0, 3))
    assert {c[0] for c in calls} == {1, 2, 3}
    assert len(calls) == (len(tune.SIMT_S) + len(tune.TC_S)) * len(tune.RING) + 1     # one two-pass candidate


def test_two_pass_engine_can_win(fake):
    calls, timer, _ = fake
    timer({(2, 8, 3): 30.0, (3, 0, 0): 20.0})
    X, y = _xy()
    assert tune.autotune(X, y, 3, x_storage="bf16", chains=4)[:2] == (3, (0, 0, 0, 0))
    assert [c for c in calls if c[0] == 3] == [(3, (0, 0, 0, 0), "free")]


def test_two_pass_cuda_core_engine_can_win(fake):
    calls, timer, _ = fake
    timer({(1, 4, 3): 50.0, (4, 0, 0): 35.0})
    X, y = _xy()
    assert tune.autotune(X, y, 3, chains=1)[:2] == (4, (0, 0, 0, 0))


def test_no_tile_runs_leaves_the_choice_to_the_library(fake):
    calls, timer, cache = fake
    timer({})
    X, y = _xy()
    assert tune.autotune(X, y, 3) == (0, None, [])
    assert not cache.exists()


def test_layout_is_part_of_the_key_and_passed_through(fake):
    calls, timer, cache = fake
    timer({(1, 1, 2): 10.0})
    X, y = _xy()
    tune.autotune(X, y, 3, layout="unconstrained")
    assert all(c[2] == "unconstrained" for c in calls)
    (key,) = json.load(open(cache)).keys()
    assert key.endswith("layout=unconstrained")
