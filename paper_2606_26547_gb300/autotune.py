"""Launch-shape autotuner for the batched sweep kernel.

Times every candidate (threads per block, words per shared-memory chunk) of
hdc_sweep_eval on the caller's own data with CUDA events, keeps the fastest
and caches the choice per (device, shape) in a JSON file.  Results of the
kernel do not depend on the launch shape, so tuning never changes output.
"""
from __future__ import annotations

import json
import os

import torch

from . import hdc

CANDIDATES = ((64, 16), (64, 32), (64, 64), (128, 16), (128, 32), (128, 64), (256, 8), (256, 16), (256, 32))


def cache_path() -> str:
    return os.environ.get("HDC_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "hdc_gb300", "autotune.json"))


def _load() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(cache: dict) -> None:
    p = cache_path()
    try:
        os.makedirs(os.path.dirname(p), exist_ok=True)
        tmp = p + ".tmp%d" % os.getpid()
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, p)
    except OSError:
        pass  # a read-only home only loses the cache


def sweep_key(N, D, C, strides, bits) -> str:
    name = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    return "sweep|%s|N%d|D%d|C%d|s%s|b%s" % (name, N, D, C, ",".join(map(str, strides)), ",".join(map(str, bits)))


def pick_fastest(timings: dict):
    """The candidate with the smallest time (ties: the first listed)."""
    best = None
    for cand in CANDIDATES:
        t = timings.get(cand)
        if t is not None and (best is None or t < timings[best]):
            best = cand
    return best


def tune_sweep(H, y, acc, D, C, strides, bits, reps: int = 3, use_cache: bool = True):
    """(block_threads, words_per_chunk) for hdc_sweep_eval on this shape."""
    key = sweep_key(H.shape[0], D, C, strides, bits)
    cache = _load() if use_cache else {}
    if key in cache:
        return tuple(cache[key])
    timings = {}
    for bt, wc in CANDIDATES:
        try:
            sw = hdc.Sweep(D, C, strides, bits, H.shape[0], H.device, bt, wc)
            sw(H, y, acc)
            torch.cuda.synchronize()
        except hdc.HdcError:
            continue  # shared memory does not fit this shape
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            sw(H, y, acc)
        b.record()
        b.synchronize()
        timings[(bt, wc)] = a.elapsed_time(b) / reps
    best = pick_fastest(timings) or (0, 0)
    if use_cache:
        cache[key] = list(best)
        _store(cache)
    return best
