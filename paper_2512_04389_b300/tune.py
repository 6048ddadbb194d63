"""Autotuner for the per-block sparse/dense switch.

The paper runs each block with a sparse kernel or a dense routine chosen by
the block's density (Section 1); the density threshold that pays off
depends on the precision and the GPU.  ``tune`` factors and solves the given
system once per candidate threshold and keeps the fastest, timing with CUDA
events on the current stream.  Results are cached in a JSON file (path from
the ``SLU_TUNE_CACHE`` environment variable, default
``~/.cache/slu_b300_tune.json``) under a key made of the pattern's hash, the
precision and the blocking options, so a pattern is tuned once.
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np

from . import slu as S

CANDIDATES = (0.0, 0.05, 0.3, 0.6)


def _key(n, colptr, rowidx, opts):
    h = hashlib.sha1()
    h.update(np.int64(n).tobytes())
    h.update(np.ascontiguousarray(colptr, dtype=np.int64).tobytes())
    h.update(np.ascontiguousarray(rowidx, dtype=np.int32).tobytes())
    h.update(json.dumps(sorted(opts.items()), default=str).encode())
    return h.hexdigest()


def _cache_path():
    return os.environ.get("SLU_TUNE_CACHE",
                          os.path.expanduser("~/.cache/slu_b300_tune.json"))


def _load():
    try:
        with open(_cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save(cache):
    p = _cache_path()
    os.makedirs(os.path.dirname(p) or ".", exist_ok=True)
    tmp = p + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1)
    os.replace(tmp, p)


def tune(n, colptr, rowidx, values, rhs, candidates=CANDIDATES, reps=2,
         use_cache=True, **opts):
    """Return ``(best_threshold, timings)``; ``values`` and ``rhs`` are CUDA
    float64 tensors, ``opts`` the other plan options (precision, blocking,
    ...).  Timings map each candidate to its factor + solve milliseconds."""
    import torch
    key = _key(n, colptr, rowidx, opts)
    cache = _load() if use_cache else {}
    if key in cache:
        e = cache[key]
        return e["threshold"], e["timings"]
    timings = {}
    for thr in candidates:
        P = S.Plan(n, colptr, rowidx, dense_threshold=thr, **opts)
        F = S.Factor(P, values)
        F.solve(rhs)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            F.refactor(values)
            F.solve(rhs)
        e1.record()
        torch.cuda.synchronize()
        timings[str(thr)] = e0.elapsed_time(e1) / reps
        del F, P
    best = float(min(timings, key=timings.get))
    if use_cache:
        cache[key] = {"threshold": best, "timings": timings}
        _save(cache)
    return best, timings
