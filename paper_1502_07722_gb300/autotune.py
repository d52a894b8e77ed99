"""Autotuner for the tile edge and the sort interval of a batch (or a single simulation).

For each candidate (tile, sort_every) it builds the batch, advances a few warm-up steps and times
enough graph-replayed steps to include at least one cell sort, with CUDA events on the batch's
stream. The fastest candidate is cached per GPU model and workload signature in a JSON file next
to this module, so later runs reuse it without measuring.
"""
from __future__ import annotations

import hashlib
import json
import os

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), ".autotune_cache.json")
TILES = (12, 16, 20)
SORTS = (40, 80, 160)


def _signature(phys_list) -> str:
    keys = ("nx", "nz", "slab_k", "ppc_ion", "ppc_electron", "mode", "laser_profile")
    sig = json.dumps([[p.get(k) for k in keys] for p in phys_list])
    return hashlib.sha256(sig.encode()).hexdigest()[:16]


def _load():
    if os.path.exists(CACHE):
        try:
            with open(CACHE) as f:
                return json.load(f)
        except (OSError, ValueError):
            return {}
    return {}


def tune_batch(phys_list, tiles=TILES, sorts=SORTS, warmup=3, use_cache=True, verbose=False):
    """Return {"tile": T, "sort_every": k, "ms_per_step": t, "trials": [...]} for this batch."""
    import torch

    import paper_1502_07722_gb300 as gb

    gpu = torch.cuda.get_device_name()
    key = f"{gpu}|{_signature(phys_list)}"
    cache = _load()
    if use_cache and key in cache:
        return cache[key]
    trials = []
    steps = 2 * max(sorts)
    for T in tiles:
        for se in sorts:
            b = gb.Batch(phys_list, tile=T, sort_every=se)
            b.step(warmup)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(b.stream)
            b.step(steps)
            e1.record(b.stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / steps
            trials.append({"tile": T, "sort_every": se, "ms_per_step": ms})
            if verbose:
                print(f"tile {T:3d} sort_every {se:3d}: {ms:.4f} ms/step")
            b.close()
            del b
            torch.cuda.empty_cache()
    best = min(trials, key=lambda t: t["ms_per_step"])
    result = dict(best, trials=trials, gpu=gpu)
    cache[key] = result
    tmp = CACHE + f".{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1)
    os.replace(tmp, CACHE)
    return result
