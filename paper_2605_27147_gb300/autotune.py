"""Autotuner for batched sorts.

For a batch shape (instance count, total elements, largest instance) it
captures the batched sort into a CUDA graph for every candidate pair of

* tile_log2          -- on-chip tile capacity 2^10 .. 2^12 (how much of the
                        merge tree is merged in shared memory before the HBM merges)
* merge_lanes        -- chunks each CTA of the HBM merge kernel prepares ahead
                        (its search lanes: 4, 8 or 16); few lanes spread a
                        round's chunks over more CTAs, many hide more latency

times each graph's replays with CUDA events, and keeps the fastest.  Results
are cached in memory and in a JSON file (``$PS_AUTOTUNE_CACHE``, default
``~/.cache/paper_2605_27147_gb300/autotune.json``) keyed by the GPU name and a
bucketed shape, so a shape is tuned once per machine.  Timing uses the
caller's inputs; they are restored from a pristine copy before every replay.
"""
from __future__ import annotations

import json
import math
import os
import threading

TILE_LOG2 = (10, 11, 12)
MERGE_LANES = (4, 8, 16)
_lock = threading.Lock()
_mem: dict = {}


def _cache_path() -> str:
    return os.environ.get("PS_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "paper_2605_27147_gb300", "autotune.json"))


CACHE_VERSION = 4   # entries of other versions (other tuning knobs) are not reused


def shape_key(gpu: str, count: int, total: int, max_n: int) -> str:
    b = lambda x: int(round(math.log2(max(1, x)) * 2))   # half-octave buckets
    return f"v{CACHE_VERSION}|{gpu}|c{b(count)}|t{b(total)}|m{b(max_n)}"


def _load_file() -> dict:
    try:
        with open(_cache_path()) as f:
            return json.load(f)
    except Exception:
        return {}


def _store_file(d: dict) -> None:
    try:
        path = _cache_path()
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".{os.getpid()}.tmp"
        with open(tmp, "w") as f:
            json.dump(d, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass


def tune(keys, offsets, perm, max_n: int, *, reps: int = 3, stream=None, use_cache: bool = True,
         candidates=None) -> dict:
    """Best (tile_log2, merge_lanes) for sorting this batch, with timings.

    keys / perm: CUDA int32 tensors (keys are restored after tuning);
    offsets: CUDA int64 tensor of count + 1 entries."""
    import torch

    from . import binding

    count = offsets.numel() - 1
    total = keys.numel()
    gpu = torch.cuda.get_device_name(keys.device)
    key = shape_key(gpu, count, total, max_n)
    if use_cache:
        with _lock:
            if key in _mem:
                return dict(_mem[key], cached=True)
            disk = _load_file()
            if key in disk:
                _mem[key] = disk[key]
                return dict(disk[key], cached=True)
    stream = stream or torch.cuda.Stream(keys.device)
    pristine = keys.clone()
    cands = candidates or [(t, l) for t in TILE_LOG2 for l in MERGE_LANES]
    results = []
    for tile_log2, merge_lanes in cands:
        with binding.Context(max_n, want_perm=perm is not None, max_total=total, max_count=count,
                             tile_log2=tile_log2, merge_lanes=merge_lanes, stream=stream) as ctx:
            g = ctx.graph_batched(keys, offsets, perm)
            times = []
            with torch.cuda.stream(stream):
                for i in range(reps + 1):
                    keys.copy_(pristine)
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    g.launch()
                    e1.record(stream)
                    ctx.sync()
                    if i:
                        times.append(e0.elapsed_time(e1))
            g.close()
        results.append({"tile_log2": tile_log2, "merge_lanes": merge_lanes, "ms": min(times)})
    keys.copy_(pristine)
    torch.cuda.synchronize(keys.device)
    best = min(results, key=lambda r: r["ms"])
    out = {"tile_log2": best["tile_log2"], "merge_lanes": best["merge_lanes"], "ms": best["ms"],
           "trials": results, "shape": key}
    with _lock:
        _mem[key] = out
        if use_cache:
            disk = _load_file()
            disk[key] = out
            _store_file(disk)
    return dict(out, cached=False)
