"""Autotuner for the launch shape of the counting kernels.

The knobs (niorca_set_tuning) are the CTAs per SM of each persistent
warp-tier kernel and the thresholds that send a vertex to a warp or to a
whole CTA: the GPU counterpart of the paper's OpenMP schedule and chunk-size
study (Sec. 8, Figs. 10-11). Every setting gives identical counts. The tuner
times whole calls with CUDA events and walks the knobs one at a time
(coordinate descent), keeping a candidate only if it is faster. Results are
cached as JSON, keyed by GPU name and a bucket of the graph's shape
(log2 of vertices, mean degree and skew), in $NIORCA_TUNING_CACHE or
~/.cache/niorca/tuning.json.
"""
from __future__ import annotations

import json
import math
import os
import threading

import torch

from . import _lib

SEARCH = {
    "grid_c4": (4, 8, 16),
    "grid_tri": (2, 4, 8, 16),
    "grid_relabel": (4, 8, 16),
    "grid_agg": (4, 8, 16),
    "grid_solve": (4, 8, 16),
    "warp_maxd": (32, 64),
    "c4_warp_maxw": (768, 1152, 1536),
    "long_row_class": (24, 28, 32, 36),   # rows of degree >= 128, 256, 512, 1024 get a CTA
}

_lock = threading.Lock()


def cache_path() -> str:
    p = os.environ.get("NIORCA_TUNING_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "niorca", "tuning.json")


def shape_bucket(n: int, m: int, dmax: int) -> str:
    """Coarse shape class: log2 n, log2 mean degree, log2 (d_max / mean degree)."""
    mean = max(m / max(n, 1), 1.0)
    return f"n{round(math.log2(max(n, 1)))}_d{round(math.log2(mean))}_s{round(math.log2(max(dmax, 1) / mean))}"


def _key(bucket: str) -> str:
    return f"{torch.cuda.get_device_name()}|{bucket}"


def load(bucket: str):
    try:
        with open(cache_path()) as fh:
            return json.load(fh).get(_key(bucket))
    except (OSError, ValueError):
        return None


def store(bucket: str, params: dict) -> None:
    path = cache_path()
    with _lock:
        try:
            with open(path) as fh:
                db = json.load(fh)
        except (OSError, ValueError):
            db = {}
        db[_key(bucket)] = params
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".tmp{os.getpid()}"
        with open(tmp, "w") as fh:
            json.dump(db, fh, indent=1, sort_keys=True)
        os.replace(tmp, path)


def _time(run, reps: int) -> float:
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    run()
    torch.cuda.synchronize()
    s.record()
    for _ in range(reps):
        run()
    e.record()
    torch.cuda.synchronize()
    return s.elapsed_time(e) / reps


def tune(run, reps: int = 3, search: dict | None = None) -> dict:
    """Coordinate descent over the knobs; `run()` enqueues one call. Leaves
    the best setting active and returns it with its time."""
    search = search or SEARCH
    best = _lib.get_tuning()
    best_ms = _time(run, reps)
    for knob, values in search.items():
        for v in values:
            if v == best[knob]:
                continue
            _lib.set_tuning(**{**best, knob: v})
            ms = _time(run, reps)
            if ms < best_ms:
                best_ms = ms
                best = {**best, knob: v}
        _lib.set_tuning(**best)
    _lib.check()
    return {"params": best, "ms": best_ms}


def tune_graph(rowptr: torch.Tensor, colidx: torch.Tensor, use_cache: bool = True, reps: int = 3) -> dict:
    """Tune (or load from the cache) the knobs for one graph's shape and apply them."""
    n = rowptr.numel() - 1
    m = colidx.numel()
    dmax = int((rowptr[1:] - rowptr[:-1]).max().item()) if n > 0 else 0
    bucket = shape_bucket(n, m, dmax)
    if use_cache:
        hit = load(bucket)
        if hit:
            _lib.set_tuning(**hit["params"])
            return {**hit, "bucket": bucket, "cached": True}
    out = torch.empty((n, 15), dtype=torch.int64, device=rowptr.device)
    res = tune(lambda: _lib.count(rowptr, colidx, out), reps)
    store(bucket, res)
    return {**res, "bucket": bucket, "cached": False}


def tune_batch(rowptr, colidx, vtx_offset, edge_offset, use_cache: bool = True, reps: int = 3) -> dict:
    """Same for a packed batch (bucket of the union graph, tagged 'batch')."""
    n = rowptr.numel() - 1
    m = colidx.numel()
    dmax = int((rowptr[1:] - rowptr[:-1]).max().item()) if n > 0 else 0
    bucket = "batch_" + shape_bucket(n, m, dmax)
    if use_cache:
        hit = load(bucket)
        if hit:
            _lib.set_tuning(**hit["params"])
            return {**hit, "bucket": bucket, "cached": True}
    out = torch.empty((n, 15), dtype=torch.int64, device=rowptr.device)
    res = tune(lambda: _lib.count_batch(rowptr, colidx, vtx_offset, edge_offset, out), reps)
    store(bucket, res)
    return {**res, "bucket": bucket, "cached": False}
