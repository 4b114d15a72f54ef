"""Autotuners: the ragged launch knobs, and the constants mode of a plan.

Every combination of the ragged launch knobs (schedule of the persistent
small-length launch, order of its work items, its CTAs per SM, and the
cluster grid multiplier of the 2^14..2^16 launches) is timed on the caller's
own batch with CUDA events (median of `reps` runs after a warm-up run); the
fastest is applied to the plan and cached in a JSON file keyed by device,
variant, longest length and the batch's length histogram, so later plans for
the same kind of batch skip the search.
"""
from __future__ import annotations

import itertools
import json
import os
import statistics
import threading

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")
GRID = {"schedule": (0, 1), "order": (0, 1), "small_ctas_per_sm": (1, 2), "cluster_mult": (1, 2)}

_lock = threading.Lock()


def _load_cache(path: str) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save_cache(path: str, cache: dict) -> None:
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def batch_signature(log2n) -> str:
    """Length histogram of a batch (counts per log2 N), as a cache key part."""
    import torch

    counts = torch.bincount(log2n.to(torch.int64), minlength=32).cpu().tolist()
    return ",".join(str(c) for c in counts)


def tune_ragged(plan, x, log2n, offsets, out=None, reps: int = 5, use_cache: bool = True,
                cache_path: str = CACHE) -> dict:
    """Pick the fastest knob setting of `plan` for this batch; returns it.
    The search runs the batch 1 + reps times per setting (16 settings)."""
    import torch

    key = f"{torch.cuda.get_device_name()}|v{plan.variant}|L{plan.max_log2n}|{batch_signature(log2n)}"
    with _lock:
        cache = _load_cache(cache_path) if use_cache else {}
        hit = cache.get(key)
    if hit:
        plan.tune(**hit["knobs"])
        return dict(hit["knobs"])
    if out is None:
        out = torch.empty_like(x)
    stream = torch.cuda.current_stream()
    results = []
    for combo in itertools.product(*GRID.values()):
        knobs = dict(zip(GRID, combo))
        plan.tune(**knobs)
        plan.exec(x, log2n, offsets, out)
        times = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            plan.exec(x, log2n, offsets, out)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        results.append((statistics.median(times), knobs))
    best_ms, best = min(results, key=lambda r: r[0])
    plan.tune(**best)
    if use_cache:
        with _lock:
            cache = _load_cache(cache_path)
            cache[key] = {"knobs": best, "ms": best_ms,
                          "all": [{"knobs": k, "ms": t} for t, k in results]}
            _save_cache(cache_path, cache)
    return dict(best)


def tune_constants(plan, x, reps: int = 5, use_cache: bool = True, cache_path: str = CACHE) -> dict:
    """Time `plan`'s forward transform of x with the band constants read from
    the table and evaluated on the fly (Sect. 7.1; CUDA events, median of
    `reps` runs after a warm-up run), apply the faster mode and return
    {"mode": ..., "table_ms": ..., "fly_ms": ...}.  Cached per device, length,
    variant, batch and storage type."""
    import torch

    key = f"{torch.cuda.get_device_name()}|const|v{plan.variant}|n{plan.log2n}|b{plan.batch}|d{plan.dtype}"
    with _lock:
        cache = _load_cache(cache_path) if use_cache else {}
        hit = cache.get(key)
    if hit:
        plan.constants = hit["mode"]
        return dict(hit)
    stream = torch.cuda.current_stream()
    out = torch.empty_like(x)
    res = {}
    for mode in ("table", "fly"):
        plan.constants = mode
        plan.fwd(x, out)
        times = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            plan.fwd(x, out)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        res[mode + "_ms"] = statistics.median(times)
    res["mode"] = "fly" if res["fly_ms"] < res["table_ms"] else "table"
    plan.constants = res["mode"]
    if use_cache:
        with _lock:
            cache = _load_cache(cache_path)
            cache[key] = res
            _save_cache(cache_path, cache)
    return dict(res)
