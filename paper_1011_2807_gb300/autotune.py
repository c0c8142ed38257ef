"""Autotuner for the join's tile sizes.

The S block size (fixed when an index is built), the threads per CTA and the number of
S blocks per launch (or per batched work item) are picked per class of join, by timing
candidate configurations on a small sample of the join itself; the Section 4.4 level
margin is then timed on the winning configuration.  A class is keyed by
dtype and the rounded base-2 logarithms of |S|, |R|, the mean query length and k, so
every join of similar shape reuses one measurement.  Results are cached in a JSON file
(``$KNN_TUNE_CACHE``, else ``~/.cache/knnjoin_gb300/tune.json``).

All timing runs go through the library's own entry points; the tuner holds no join
arithmetic of its own.
"""
from __future__ import annotations

import json
import math
import os
import threading

import numpy as np

_lock = threading.Lock()

# blocks_per_launch 0: the library's default (as many S blocks as keep a launch's
# postings within ~48 MB of L2, at most 16)
DEFAULT = {"block_size": 16384, "threads": 512, "blocks_per_launch": 0, "level_margin": 0.3}
MARGINS = (0.25, 0.35, 0.45)


def cache_path() -> str:
    p = os.environ.get("KNN_TUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "knnjoin_gb300", "tune.json")


def _load() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except Exception:
        return {}


def _store(d: dict) -> None:
    p = cache_path()
    try:
        os.makedirs(os.path.dirname(p), exist_ok=True)
        tmp = p + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(d, f, indent=1, sort_keys=True)
        os.replace(tmp, p)
    except OSError:
        pass   # a read-only home only costs re-tuning


def class_key(n_s: int, n_r: int, mean_nnz: float, k: int, dtype: str) -> str:
    lg = lambda x: int(round(math.log2(max(1.0, float(x)))))
    return f"{dtype}:s{lg(n_s)}:r{lg(n_r)}:q{lg(mean_nnz)}:k{lg(k)}"


def heuristic(n_s: int) -> dict:
    """Untuned default: the largest block that does not exceed |S| (2048..16384)."""
    bs = 2048
    while bs < 16384 and bs < n_s:
        bs *= 2
    return dict(DEFAULT, block_size=bs)


def lookup(n_s: int, n_r: int, mean_nnz: float, k: int, dtype: str = "u8") -> dict:
    with _lock:
        d = _load()
    got = dict(d.get(class_key(n_s, n_r, mean_nnz, k, dtype), heuristic(n_s)))
    got.setdefault("level_margin", DEFAULT["level_margin"])
    return got


def candidates(n_s: int, threads: int | None = None):
    """Configurations to try: blocks 2048..32768 not far beyond |S|; threads that keep
    4 * threads <= block <= 64 * threads; 4, 8 or 16 blocks per launch."""
    out = []
    for bs in (2048, 4096, 8192, 16384, 32768):
        if bs > 2 * max(2048, n_s):
            continue
        for t in ((threads,) if threads else (256, 512, 1024)):
            if not (4 * t <= bs <= 64 * t):
                continue
            for bpl in (4, 8, 16):
                out.append({"block_size": bs, "threads": t, "blocks_per_launch": bpl})
    return out


def tune(S, R_sample, k: int, *, threads: int | None = None, reps: int = 2, store: bool = True,
         max_trials: int = 24, tune_margin: bool = True) -> dict:
    """Times the candidates on (S, R_sample) and returns (and caches) the fastest."""
    import torch
    from . import binding

    dtype = "u8" if np.asarray(S.values).dtype == np.uint8 else "f32"
    mean_nnz = R_sample.nnz / max(1, R_sample.n_rows)
    key = class_key(S.n_rows, R_sample.n_rows, mean_nnz, k, dtype)
    Rd = binding.DeviceCSR.from_host(R_sample)
    best, best_ms = None, float("inf")
    trials = []
    cands = candidates(S.n_rows, threads)[:max_trials]
    by_block = {}
    for c in cands:
        by_block.setdefault(c["block_size"], []).append(c)
    for bs, cs in by_block.items():
        idx = binding.knn_join_build_index(S, block_size=bs)
        try:
            for c in cs:
                kw = dict(threads=c["threads"], blocks_per_launch=c["blocks_per_launch"],
                          level_margin=DEFAULT["level_margin"], skip_validation=True)
                binding.knn_join(idx, Rd, k, **kw)   # warm-up (and validation of R on first use)
                torch.cuda.synchronize()
                ms = float("inf")
                for _ in range(reps):
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record()
                    binding.knn_join(idx, Rd, k, **kw)
                    e1.record()
                    torch.cuda.synchronize()
                    ms = min(ms, e0.elapsed_time(e1))
                trials.append(dict(c, ms=ms))
                if ms < best_ms:
                    best, best_ms = dict(c), ms
        finally:
            idx.close()
    if best is not None and tune_margin:
        idx = binding.knn_join_build_index(S, block_size=best["block_size"])
        try:
            for mg in MARGINS:
                kw = dict(threads=best["threads"], blocks_per_launch=best["blocks_per_launch"], level_margin=mg,
                          skip_validation=True)
                binding.knn_join(idx, Rd, k, **kw)
                torch.cuda.synchronize()
                ms = float("inf")
                for _ in range(reps):
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record()
                    binding.knn_join(idx, Rd, k, **kw)
                    e1.record()
                    torch.cuda.synchronize()
                    ms = min(ms, e0.elapsed_time(e1))
                trials.append(dict(best, level_margin=mg, ms=ms))
                if ms < best_ms:
                    best_ms = ms
                    best["level_margin"] = mg
        finally:
            idx.close()
    if best is None:
        best = heuristic(S.n_rows)
    best.setdefault("level_margin", DEFAULT["level_margin"])
    best["ms"] = best_ms
    best["trials"] = len(trials)
    if store:
        with _lock:
            d = _load()
            d[key] = best
            _store(d)
    return best
