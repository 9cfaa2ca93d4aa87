"""Autotuner: selection and caching logic on CPU (fake timings), a real tune
on the GPU."""
import json

import pytest
import torch


def test_picks_fastest_and_caches(tmp_path, monkeypatch):
    from paper_2103_04856_gb300 import autotune
    fake = {(16, 0): 0.20, (13, 0): 0.21, (8, 0): 0.25, (16, 64): 0.15, (16, 32): 0.30, (8, 64): 0.40}
    calls = []

    def timer(shapes, cand, steps=30, **kw):
        calls.append((cand["tile_y"], cand["max_run"]))
        return fake[(cand["tile_y"], cand["max_run"])]

    monkeypatch.setattr(autotune, "time_candidate", timer)
    cache = str(tmp_path / "cache.json")
    best = autotune.tune([(64, 64, 64), (32, 32, 32)], cache=cache)
    assert (best["tile_y"], best["max_run"]) == (16, 64)
    assert len(calls) == 3 * len(autotune.CANDIDATES)           # three interleaved rounds
    assert calls[:len(autotune.CANDIDATES)] == calls[len(autotune.CANDIDATES):2 * len(autotune.CANDIDATES)]
    stored = json.load(open(cache))
    assert list(stored.values())[0]["tile_y"] == 16
    # second call: from the cache, no timing; the key ignores shape order
    calls.clear()
    again = autotune.tune([(32, 32, 32), (64, 64, 64)], cache=cache)
    assert calls == [] and again["max_run"] == 64
    # force re-times
    autotune.tune([(32, 32, 32), (64, 64, 64)], cache=cache, force=True)
    assert len(calls) == 3 * len(autotune.CANDIDATES)


def test_symmetric_problems_are_tuned_and_cached_apart(tmp_path, monkeypatch):
    """Polynomials symmetric in kappa1, kappa2 run another instantiation of
    the sweep: they are timed with a symmetric polynomial and cached under
    their own key."""
    from paper_2103_04856_gb300 import autotune
    seen = []

    def timer(shapes, cand, steps=30, symmetric=False, **kw):
        seen.append(symmetric)
        return {True: {16: 0.10, 13: 0.11}, False: {16: 0.17, 13: 0.16}}[symmetric].get(cand["tile_y"], 1.0) + \
            0.01 * cand["max_run"]

    monkeypatch.setattr(autotune, "time_candidate", timer)
    cache = str(tmp_path / "cache.json")
    sym = autotune.tune([(64, 64, 64)], cache=cache, symmetric=True)
    gen = autotune.tune([(64, 64, 64)], cache=cache)
    assert (sym["tile_y"], gen["tile_y"]) == (16, 13)
    assert sym["symmetric"] and not gen["symmetric"]
    assert set(seen) == {True, False} and len(json.load(open(cache))) == 2


def test_rejects_fp64():
    from paper_2103_04856_gb300 import autotune
    with pytest.raises(ValueError):
        autotune.tune([(8, 8, 8)], prec="fp64", cache=None)


@pytest.mark.gpu
def test_real_tune_small(tmp_path):
    from paper_2103_04856_gb300 import autotune
    shapes = [(32, 32, 64), (24, 40, 32)]
    best = autotune.tune(shapes, cache=str(tmp_path / "c.json"), steps=3)
    assert {"tile_y", "max_run", "sweep_ms"} <= set(best)
    assert best["sweep_ms"] > 0 and len(best["tried"]) == len(autotune.CANDIDATES)
    assert min(r["sweep_ms"] for r in best["tried"]) == best["sweep_ms"]


def test_bench_counts_algorithmic_flops_per_polynomial():
    """The roofline's algorithmic flops: 211 per voxel-step in general, 185
    for polynomials symmetric in kappa1, kappa2 (a20 = a02, a10 = a01), whose
    sqrt(D+) terms have weight zero and are not evaluated; a workload counts
    each problem by its own polynomial."""
    import numpy as np
    import bench
    from paper_2103_04856_gb300 import inputs as I
    assert bench.flops_per_voxel_step((1.0, 0.0, 1.0, 0.0, 0.0, 0.0)) == 185
    assert bench.flops_per_voxel_step((0.0, 1.0, 0.0, 0.0, 0.0, 0.0)) == 185
    assert bench.flops_per_voxel_step((1.0, 0.3, 0.2, 0.0, 0.0, 0.0)) == 211
    assert bench.flops_per_voxel_step((1.0, 0.0, 1.0, 0.1, -0.1, 0.0)) == 211
    val = I.validation_set_128()
    assert bench.workload_flops(val) == 185.0 * sum(int(np.prod(i.shape)) for i in val)
