"""Launch-shape autotuner for the fused sweep.

The sweep's tile height (32 x 8 or 32 x 16 columns per CTA) and the cap on
planes a CTA processes per problem (0 = one CTA per SM with equal shares)
trade halo recomputation, registers and balance against each other, and the
best choice depends on the grid sizes.  `tune` times every candidate with
CUDA events on synthetic noise fields of the requested shapes (L2 flushed
between steps, medians of repeated steps) through the library's own batched
step, and caches the winner in a JSON file keyed by GPU name, precision, the
multiset of shapes and whether the polynomials are symmetric in kappa1,
kappa2 (those problems run another instantiation of the sweep, without the
sqrt(D+) terms, whose best tile can differ).

    from paper_2103_04856_gb300 import autotune
    best = autotune.tune([(128, 128, 128)] * 4)        # {'tile_y': 16, 'max_run': 0, ...}
    prob = pfc.Problem(..., tile_y=best["tile_y"], tile_z=best["max_run"])
"""
from __future__ import annotations

import json
import os
import time

import numpy as np
import torch

from . import inputs
from . import pfc

CANDIDATES = [
    {"tile_y": 16, "max_run": 0},
    {"tile_y": 13, "max_run": 0},
    {"tile_y": 8, "max_run": 0},
    {"tile_y": 16, "max_run": 64},
    {"tile_y": 16, "max_run": 32},
    {"tile_y": 8, "max_run": 64},
]
DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "autotune_cache.json")


def cache_key(shapes, prec: str = "fp32", symmetric: bool = False) -> str:
    dev = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    shp = ",".join("x".join(str(int(d)) for d in s) for s in sorted(tuple(s) for s in shapes))
    return f"{dev}|{prec}|{shp}" + ("|sym" if symmetric else "")


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(path, data):
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


# polynomials (paper order) the candidates are timed with: a general one, and
# one symmetric in kappa1, kappa2 (a20 = a02, a10 = a01)
A_GENERAL = (1.0, 0.3, 0.6, 0.1, -0.1, 0.0)
A_SYMMETRIC = (1.0, 0.3, 1.0, 0.1, 0.1, 0.0)


def time_candidate(shapes, cand, steps: int = 30, warmup: int = 5, flush_mb: int = 256, eps: float = 1.5,
                   symmetric: bool = False):
    """Median device time (ms) of one batched fused sweep over noise fields."""
    a = A_SYMMETRIC if symmetric else A_GENERAL
    probs = [pfc.Problem.from_shape(s, eps=eps, a=a, prec="fp32",
                                    tile_y=cand["tile_y"], tile_z=cand["max_run"]) for s in shapes]
    A = [torch.tensor(inputs.noise(s, 0.3, 0.1, 1000 + k).astype(np.float32), device="cuda")
         for k, s in enumerate(shapes)]
    B = [torch.empty_like(a) for a in A]
    flush = torch.empty(flush_mb << 20, dtype=torch.uint8, device="cuda")
    batch = pfc.Batch(probs)
    batch.timing(True)
    sweeps = []
    for k in range(warmup + steps):
        flush.zero_()
        batch.step(A, B, [1e-4] * len(A))
        _, sw = batch.last_timing()
        if k >= warmup:
            sweeps.append(sw)
        A, B = B, A
    batch.close()
    return float(np.median(sweeps))


def tune(shapes, prec: str = "fp32", cache: str | None = DEFAULT_CACHE, force: bool = False,
         candidates=None, steps: int = 30, symmetric: bool = False, rounds: int = 3):
    """Best launch shape for these problem shapes (each (nz, ny, nx)); cached.
    ``symmetric``: the problems' polynomials are all symmetric in kappa1,
    kappa2.  Candidates are timed in ``rounds`` interleaved rounds (so that
    a drift of the clock or of a neighbour's load does not favour the ones
    timed first); each one's time is the median over all its steps."""
    if prec != "fp32":
        raise ValueError("the batched sweep is FP32; FP64 uses the library defaults")
    key = cache_key(shapes, prec, symmetric)
    data = _load(cache) if cache else {}
    if not force and key in data:
        return data[key]
    cands = list(candidates or CANDIDATES)
    times = [[] for _ in cands]
    per_round = max(1, steps // max(rounds, 1))
    for _ in range(max(rounds, 1)):
        for j, cand in enumerate(cands):
            times[j].append(time_candidate(shapes, cand, steps=per_round, symmetric=symmetric))
    results = [{**cand, "sweep_ms": float(np.median(t))} for cand, t in zip(cands, times)]
    best = min(results, key=lambda r: r["sweep_ms"])
    entry = {"tile_y": best["tile_y"], "max_run": best["max_run"], "sweep_ms": best["sweep_ms"],
             "symmetric": bool(symmetric),
             "voxels": int(sum(int(np.prod(s)) for s in shapes)), "tried": results,
             "when": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime())}
    if cache:
        data[key] = entry
        _store(cache, data)
    return entry
