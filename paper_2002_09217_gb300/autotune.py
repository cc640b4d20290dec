"""Autotuner of the step kernel's launch shape.

For a grid (nx, ny, boundaries) and precision it times a few steps of every valid
(lanes_per_node, tile_x) pair on the current GPU with CUDA events and returns the fastest;
results are cached per device name in ``autotune_cache.json`` next to this file (created
on first use, not part of the sources).  Results do not depend on the choice (the step is
the same arithmetic for every shape), only the speed does.
"""
from __future__ import annotations

import json
import os
import threading

from . import pond

_HERE = os.path.dirname(os.path.abspath(__file__))
CACHE = os.path.join(_HERE, "autotune_cache.json")
_lock = threading.Lock()

LANES = (8, 16)
TILES = (1, 2, 4, 8, 16)


def _key(w, precision: str, device: str) -> str:
    return "%s|%dx%d|bc%d%d|%s" % (device, w.nx, w.ny, w.bc_x, w.bc_y, precision)


def _load() -> dict:
    try:
        with open(CACHE) as fh:
            return json.load(fh)
    except Exception:
        return {}


def _save(d: dict):
    tmp = CACHE + ".%d.tmp" % os.getpid()
    with open(tmp, "w") as fh:
        json.dump(d, fh, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


def tune(w, precision: str = "mixed", steps: int = 6, warmup: int = 2, use_cache: bool = True,
         stream=None) -> dict:
    """Best {'lanes_per_node', 'tile_x', 'ms_per_step'} for workload w (an inputs.Workload)."""
    import torch
    dev = torch.cuda.get_device_name()
    key = _key(w, precision, dev)
    with _lock:
        cache = _load() if use_cache else {}
        if key in cache:
            return cache[key]
    stream = stream if stream is not None else torch.cuda.Stream()
    trials = {}
    for lanes in LANES:
        for tx in TILES:
            if tx > max(1, w.nx) * 2 and tx > 1:
                continue
            with pond.from_workload(w, precision=precision, lanes_per_node=lanes, tile_x=tx,
                                    stream=stream) as sim:
                sim.init_fields(*w.fields())
                sim.step(warmup)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                sim.step(steps)
                b.record(stream)
                b.synchronize()
                trials[(lanes, tx)] = a.elapsed_time(b) / steps
    (lanes, tx), ms = min(trials.items(), key=lambda kv: kv[1])
    best = {"lanes_per_node": lanes, "tile_x": tx, "ms_per_step": ms,
            "trials": {"%d/%d" % k: v for k, v in trials.items()}}
    with _lock:
        cache = _load()
        cache[key] = best
        _save(cache)
    return best
