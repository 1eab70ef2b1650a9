"""Autotuner for the library's launch knobs.

Results never depend on the tuning (every domain is a counter space of its
own), only speed does, so a workload can be timed under each candidate
tuning -- ring length (the refill granularity: a top-up fills a whole ring),
warps per block, lanes per chain, Dirichlet lookahead, producer warps -- and
the fastest kept.  Timing is on the device with CUDA events on the launching
stream, after warm-up, median of a few launches.  Choices are cached per
(device name, workload key) in memory and, when a path is given, in a JSON
file.
"""
from __future__ import annotations

import itertools
import json
import os
import statistics

from . import brng as B

_MEM: dict = {}

# candidate spaces per workload kind (the library's defaults are among them)
SPACES = {
    "normal_gamma": {"buf_len": [16, 32], "warps_per_block": [1, 2, 4, 8, 16],
                     "producer_warps": [B.PRODUCERS_NONE, 4]},
    "triangle": {"buf_len": [64, 256], "lanes_per_chain": [4, 8, 16]},
    "lda": {"buf_len": [16, 32], "lookahead": [4, 8, 16], "warps_per_block": [2, 4]},
    "mixed": {"buf_len": [8, 16], "warps_per_block": [2, 4]},
}


def candidates(space: dict):
    """Every combination of a space's values, as tuning dicts."""
    keys = sorted(space)
    return [dict(zip(keys, vals)) for vals in itertools.product(*(space[k] for k in keys))]


def _device_name():
    import torch
    return torch.cuda.get_device_name(torch.cuda.current_device())


def autotune(handle, launch, space: dict, stream, key: str, reps: int = 3, warm: int = 1,
             cache_path: str | None = None):
    """Time `launch()` (which enqueues the workload on `stream` through the
    library) under each tuning of `space` applied to `handle`; return
    (best tuning, its median ms, {tuning-json: ms}) and leave `handle` tuned
    to the best.  `key` names the workload (sizes included) for the cache."""
    import torch

    ck = "%s|%s" % (_device_name(), key)
    if ck not in _MEM and cache_path and os.path.exists(cache_path):
        try:
            _MEM.update(json.load(open(cache_path)))
        except (OSError, ValueError):
            pass
    if ck in _MEM:
        best = _MEM[ck]
        handle.tune(**best["tuning"])
        return best["tuning"], best["ms"], best["table"]
    table = {}
    for tune in candidates(space):
        try:
            handle.tune(**tune)
        except B.BrngError:
            continue  # e.g. the rings do not fit in shared memory
        for _ in range(warm):
            launch()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for a, b in ev:
            a.record(stream)
            launch()
            b.record(stream)
        torch.cuda.synchronize()
        table[json.dumps(tune, sort_keys=True)] = statistics.median(a.elapsed_time(b) for a, b in ev)
    if not table:
        raise RuntimeError("autotune: no candidate tuning could run")
    best_key = min(table, key=table.get)
    best = {"tuning": json.loads(best_key), "ms": table[best_key], "table": table}
    _MEM[ck] = best
    if cache_path:
        try:
            with open(cache_path, "w") as f:
                json.dump(_MEM, f, indent=1, sort_keys=True)
        except OSError:
            pass
    handle.tune(**best["tuning"])
    return best["tuning"], best["ms"], table
