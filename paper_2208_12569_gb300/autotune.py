"""Autotuner for the tracer's scheduling knobs.

The knobs of fqsl_params that change how work is scheduled but never what is
computed (refill_lanes, sync_dirs, chunk_tiles, blocks_per_sm) are timed on the
caller's own workload with CUDA events, and the fastest setting is cached per
GPU name and workload key in a JSON file. Results are identical for every
setting (the tests check bitwise equality), so tuning is safe to apply.
"""
from __future__ import annotations

import itertools
import json
import os
import threading

import torch

from . import fqsl

KNOBS = ("refill_lanes", "sync_dirs", "chunk_tiles", "blocks_per_sm")
DEFAULT_SPACE = {
    "refill_lanes": (1, 16, 32),
    "sync_dirs": (0, 1),
    "chunk_tiles": (1, 4),
    "blocks_per_sm": (0, 2, 3),
}
_lock = threading.Lock()


def cache_path() -> str:
    root = os.environ.get("XDG_CACHE_HOME") or os.path.join(os.path.expanduser("~"), ".cache")
    return os.path.join(root, "fqsl", "autotune.json")


def _load(path):
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _time(run, reps):
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for e0, e1 in ev:
        e0.record()
        run()
        e1.record()
    torch.cuda.synchronize()
    ts = sorted(e0.elapsed_time(e1) for e0, e1 in ev)
    return ts[len(ts) // 2]


def tune(run_with, base: fqsl.Params, key: str, space=None, reps: int = 5, warmup: int = 1,
         path: str | None = None, force: bool = False):
    """Return (best params, table of timings).

    run_with(params) must launch the workload on the current stream. The search
    is exhaustive over ``space`` (default DEFAULT_SPACE). The result is cached
    under (GPU name, key) unless ``path`` is '' (no cache)."""
    space = dict(DEFAULT_SPACE if space is None else space)
    gpu = torch.cuda.get_device_name()
    full_key = "%s|%s" % (gpu, key)
    path = cache_path() if path is None else path
    if path and not force:
        hit = _load(path).get(full_key)
        if hit:
            p = fqsl.Params.from_buffer_copy(base)
            for k in KNOBS:
                if k in hit["best"]:
                    setattr(p, k, int(hit["best"][k]))
            return p, hit["table"]
    names = [k for k in KNOBS if k in space]
    table = []
    best, best_ms = None, float("inf")
    for combo in itertools.product(*(space[k] for k in names)):
        p = fqsl.Params.from_buffer_copy(base)
        for k, v in zip(names, combo):
            setattr(p, k, int(v))
        for _ in range(warmup):
            run_with(p)
        ms = _time(lambda: run_with(p), reps)
        table.append(dict(zip(names, combo), ms=ms))
        if ms < best_ms:
            best, best_ms = p, ms
    if path:
        with _lock:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            data = _load(path)
            data[full_key] = {"best": {k: getattr(best, k) for k in names}, "ms": best_ms, "table": table}
            tmp = path + ".tmp%d" % os.getpid()
            with open(tmp, "w") as fh:
                json.dump(data, fh, indent=1)
            os.replace(tmp, path)
    return best, table
