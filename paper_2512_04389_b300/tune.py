"""Autotuner for the block shapes and the per-block sparse/dense switch.

The paper runs each block with a sparse kernel or a dense routine chosen by
the block's density (Section 1), and Algorithm 3 sizes the irregular blocks
from sampling parameters: the number of samples S (``sample_points``,
capped at n / ``b_min``) sets the finest block n / S, and ``max_num``
bounds how many sample steps one block may merge.  Which density threshold
and which block sizes pay off depends on the precision, the pattern and the
GPU, so
``tune`` factors and solves the given system once per candidate and keeps
the fastest, timing with CUDA events on the current stream.  Results are
cached in a JSON file (path from the ``SLU_TUNE_CACHE`` environment
variable, default ``~/.cache/slu_b300_tune.json``) under a key made of the
library sources' digest, the pattern's hash, the precision and the other
plan options, so a pattern is tuned once per build of the library.
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np

from . import slu as S

THRESHOLDS = (0.0, 0.3)
MAX_NUM = (3, 2, 1)
SAMPLE_POINTS = (1000, 2000)
B_MIN = (32, 8, 64, 128)
REGULAR_BLOCKS = (32, 64, 128, 256)


def candidates(blocking="irregular", n=None):
    """Plan options tried by default.  Regular blocking: the thresholds
    (block size fixed by the caller); "regular_sizes": block size and
    threshold.  Irregular blocking: threshold 0 with every (sample_points, b_min,
    max_num), plus threshold 0.3 with the paper's defaults; candidates whose
    effective sample count S = min(sample_points, n / b_min) coincides are
    tried once (their plans are identical)."""
    if blocking == "regular":
        return [{"dense_threshold": t} for t in THRESHOLDS]
    if blocking == "regular_sizes":
        # the regular blocking's own search, over as many candidates as the
        # irregular one: block size and threshold
        return [{"blocking": "regular", "regular_block": b, "dense_threshold": t}
                for b in REGULAR_BLOCKS for t in THRESHOLDS
                if n is None or b <= max(n, 1)]
    out, seen = [], set()
    for sp in SAMPLE_POINTS:
        for bm in B_MIN:
            for m in MAX_NUM:
                eff = min(sp, n // bm) if n else (sp, bm)
                if (eff, m) in seen:
                    continue
                seen.add((eff, m))
                out.append({"dense_threshold": 0.0, "sample_points": sp,
                            "b_min": bm, "max_num": m})
    out.append({"dense_threshold": 0.3, "sample_points": 1000, "b_min": 32,
                "max_num": 3})
    return out


TC_MODES = (3, 1, 0)


def default_candidates(n, opts):
    """The blocking candidates ``tune`` tries when none are given:
    ``candidates`` for the blocking in ``opts``.  A batch (``n`` a list) is
    not merged by sample count, since members of different orders merge
    differently.  For FP32, ``tune`` then tries the tile modes ``TC_MODES``
    (``tc_passes``: 3xTF32, one TF32 pass, the FP32 pipe with zero sub-tiles
    skipped) on the best blocking; refinement makes up the accuracy of one
    TF32 pass and the timing includes its iterations."""
    return candidates(opts.get("blocking", "irregular"),
                      None if isinstance(n, (list, tuple)) else n)


_SOURCES = None


def _source_digest():
    """Digest of the library's sources: a timing measured with other kernels
    does not carry over, so a rebuilt library tunes afresh."""
    global _SOURCES
    if _SOURCES is None:
        h = hashlib.sha1()
        d = os.path.join(os.path.dirname(os.path.abspath(__file__)), "csrc")
        for f in sorted(os.listdir(d)):
            if f.endswith((".cu", ".cuh", ".cpp", ".hpp")):
                with open(os.path.join(d, f), "rb") as fh:
                    h.update(f.encode())
                    h.update(fh.read())
        _SOURCES = h.hexdigest()
    return _SOURCES


def _key(n, colptr, rowidx, opts):
    """Cache key; a batch (lists of the members' n, colptr, rowidx) hashes
    every member in order."""
    h = hashlib.sha1()
    h.update(_source_digest().encode())
    members = zip(n, colptr, rowidx) if isinstance(n, (list, tuple)) else [(n, colptr, rowidx)]
    for m, cp, ri in members:
        h.update(np.int64(m).tobytes())
        h.update(np.ascontiguousarray(cp, dtype=np.int64).tobytes())
        h.update(np.ascontiguousarray(ri, dtype=np.int32).tobytes())
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


def tune(n, colptr, rowidx, values, rhs, cands=None, reps=2, use_cache=True,
         **opts):
    """Return ``(best, timings)``: ``best`` is the dict of tuned plan options
    (``dense_threshold`` and, for irregular blocking, ``max_num``) to pass to
    ``Plan`` together with ``opts``; ``timings`` maps each candidate (as
    JSON) to its factor + solve milliseconds.  ``values`` and ``rhs`` are
    CUDA float64 tensors, ``opts`` the fixed plan options (precision,
    blocking, ...).  ``n``, ``colptr``, ``rowidx`` may be lists (a batch:
    the candidates are tried on the batch plan, all of them, since members
    of different orders merge different candidates)."""
    import torch
    staged = cands is None and opts.get("precision") == "fp32"
    if cands is None:
        cands = default_candidates(n, opts)
    key = _key(n, colptr, rowidx, dict(opts, cands=cands, tc_modes=staged))
    cache = _load() if use_cache else {}
    if key in cache:
        e = cache[key]
        return e["best"], e["timings"]
    timings = {}

    def run(cs):
        best, best_ms = None, float("inf")
        for c in cs:
            k = json.dumps(c, sort_keys=True)
            if k in timings:
                ms = timings[k]
            else:
                # the device analysis gives the host analysis's plan, faster
                P = S.Plan(n, colptr, rowidx, device=True, **opts, **c)
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
                ms = e0.elapsed_time(e1) / reps
                timings[k] = ms
                del F, P
            if ms < best_ms:
                best, best_ms = dict(c), ms
        return best

    best = run(cands)
    if staged:              # the FP32 tile modes on the best blocking
        base = {k: v for k, v in best.items() if k != "tc_passes"}
        best = run([base] + [dict(base, tc_passes=t) for t in TC_MODES if t != 3])
    if use_cache:
        cache[key] = {"best": best, "timings": timings}
        _save(cache)
    return best, timings
