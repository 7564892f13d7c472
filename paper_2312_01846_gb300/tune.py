"""Autotuner for the batched scan's launch shapes.

It times a short scan (from the aufbau determinants, after a few warm-up
steps) for every combination of
  - emit_warps: warps per CTA of the element generator (the CTA's shape),
  - bucket_elems: intermediate elements per merge bucket (the work one merge
    CTA takes at a time, hence its shared-memory table size),
  - workers: host threads feeding the per-instance streams,
and keeps the fastest.  Results are cached per GPU name and workload in
_build/tune_cache.json next to the library.
"""
from __future__ import annotations

import hashlib
import itertools
import json
import os
import time

import numpy as np
import torch

from . import Scan, _HERE

CACHE = os.path.join(_HERE, "_build", "tune_cache.json")
DEFAULT_SPACE = {"emit_warps": [4, 8], "bucket_elems": [768, 1024, 1536], "workers": [4, 8, 16]}


def _key(systems, caps, n_lanczos, space):
    sig = ";".join(f"{s.n}/{s.na}/{s.nb}/{c}" for s, c in zip(systems, caps))
    sig += "|" + json.dumps(space, sort_keys=True) + f"|NL{n_lanczos}"
    return torch.cuda.get_device_name() + "|" + hashlib.sha1(sig.encode()).hexdigest()[:16]


def _load():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def time_scan(systems, caps, n_lanczos=10, steps=2, warmup=3, **shape):
    """Elements per second of `steps` scan steps after `warmup` steps."""
    inst = [(s, np.array([0], dtype=np.uint64), np.array([1.0]), c) for s, c in zip(systems, caps)]
    sc = Scan(inst, n_lanczos=n_lanczos, **shape)
    try:
        for _ in range(warmup):
            sc.step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        infos = [sc.step() for _ in range(steps)]
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
    finally:
        sc.close()
    return sum(x["n_elements"] for st in infos for x in st) / dt


def tune_scan(systems, caps, n_lanczos=10, steps=2, warmup=3, space=None, use_cache=True):
    """Best {emit_warps, bucket_elems, workers} for these instances, with the
    timing of every combination tried."""
    space = space or DEFAULT_SPACE
    key = _key(systems, caps, n_lanczos, space)
    cache = _load()
    if use_cache and key in cache:
        return cache[key]
    names = sorted(space)
    results = []
    for combo in itertools.product(*(space[n] for n in names)):
        shape = dict(zip(names, combo))
        results.append(dict(shape, elements_per_s=time_scan(systems, caps, n_lanczos, steps, warmup,
                                                             **shape)))
    best = max(results, key=lambda r: r["elements_per_s"])
    entry = {"best": {n: best[n] for n in names}, "best_elements_per_s": best["elements_per_s"],
             "results": results, "steps": steps, "warmup": warmup}
    cache[key] = entry
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + f".{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1)
    os.replace(tmp, CACHE)
    return entry
