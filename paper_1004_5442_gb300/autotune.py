"""Autotuner of the batched step: tries each kernel variant (tile 2, 4, 5)
and work-item height on a batch built from the given workloads, keeps the
fastest, and caches the choice in a JSON file keyed by the batch's shape
signature (instance sizes and boundary kinds).  Tuning runs on a batch of
its own, so a caller's simulation state is never advanced by it.
"""
from __future__ import annotations

import hashlib
import json
import os
import time

from . import binding as Bd

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_CACHE = os.path.join(HERE, "_build", "autotune_cache.json")
CANDIDATES = [(t, r) for t in (2, 4, 5) for r in (8, 16, 32, 64)]


def signature(workloads) -> str:
    shapes = sorted((w.nx, w.ny, w.bc_x, w.bc_y) for w in workloads)
    return hashlib.sha256(json.dumps(shapes).encode()).hexdigest()[:20]


def _load(path):
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def tune_workloads(workloads, steps: int = 6, candidates=CANDIDATES, cache_path: str = DEFAULT_CACHE,
                   use_cache: bool = True) -> dict:
    """Best (tile, rows_per_item) for these workloads, with all timings."""
    key = signature(workloads)
    cache = _load(cache_path) if use_cache else {}
    if key in cache:
        return dict(cache[key], cached=True)
    timings = []
    with Bd.Batch(workloads) as b:
        for tile, rows in candidates:
            b.tune(tile, rows)
            b.step(2)
            b.sync()
            t0 = time.perf_counter()
            b.step(steps)
            b.sync()
            timings.append({"tile": tile, "rows_per_item": rows, "ms_per_step": 1e3 * (time.perf_counter() - t0) / steps})
    best = min(timings, key=lambda d: d["ms_per_step"])
    result = {"tile": best["tile"], "rows_per_item": best["rows_per_item"], "timings": timings}
    if use_cache:
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
        cache = _load(cache_path)
        cache[key] = result
        with open(cache_path, "w") as fh:
            json.dump(cache, fh, indent=1)
    return dict(result, cached=False)
