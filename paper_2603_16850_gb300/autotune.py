"""Scan chunk-length autotuner.

The chunked scans reduce every chunk of L consecutive rows of a sequence to one aggregate
and walk the aggregates of a sequence in order, so L trades the per-chunk serial work
(proportional to L) against the length of the per-sequence carry chain (T / L) and the
number of independent chunks (parallelism). The best L depends on the GPU, the dynamics,
d, the Jacobian mode, the precision and T, so it is measured: ``tune_chunk`` times a
few candidates on the caller's own problem with CUDA events and caches the fastest in a
JSON file, keyed by (GPU name, kind, d, jac, prec, T rounded up to a power of two).
The solver's default path (``chunk=0`` in the Python binding) then uses the cached choice
for the same configuration, and falls back to the library's own default without one.

The diagonal look-back scan fixes its own tile length (it is tied to d), so tuning applies
to the dense (full-Jacobian) paths.
"""
from __future__ import annotations

import json
import math
import os
from typing import Callable, Dict, Iterable, Optional

DEFAULT_CANDIDATES = (16, 32, 64, 128, 256)


def cache_path() -> str:
    return os.environ.get("DEER_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "deer_gb300",
                                       "autotune.json"))


def make_key(gpu: str, kind: str, d: int, jac: str, prec: str, T: int) -> str:
    tb = 1 << max(0, math.ceil(math.log2(max(int(T), 1))))
    return f"{gpu}|{kind}|d{d}|{jac}|{prec}|T{tb}"


def load_cache(path: Optional[str] = None) -> Dict[str, dict]:
    p = path or cache_path()
    try:
        with open(p) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def store(key: str, entry: dict, path: Optional[str] = None) -> None:
    p = path or cache_path()
    os.makedirs(os.path.dirname(p), exist_ok=True)
    cache = load_cache(p)
    cache[key] = entry
    tmp = p + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, p)


def pick_best(candidates: Iterable[int], time_fn: Callable[[int], float]) -> dict:
    """Time every candidate with ``time_fn(L) -> milliseconds`` (inf = failed) and return
    the fastest with all timings."""
    timings = {}
    for L in candidates:
        try:
            timings[int(L)] = float(time_fn(int(L)))
        except Exception:  # a candidate the solver rejects is skipped
            timings[int(L)] = float("inf")
    best = min(timings, key=lambda k: timings[k])
    if not math.isfinite(timings[best]):
        raise RuntimeError("no chunk length candidate ran")
    return {"chunk": best, "ms": timings[best], "timings": {str(k): v for k, v in timings.items()}}


def tune_chunk(dyn, s0, T: int, x=None, candidates=DEFAULT_CANDIDATES, repeats: int = 2,
               path: Optional[str] = None, **opts) -> int:
    """Time deer_solve for each candidate chunk length on this problem (after one warm-up
    each) and cache the fastest. Returns it."""
    import torch

    from . import deer_solve

    def time_fn(L: int) -> float:
        deer_solve(dyn, s0, T, x, chunk=L, **opts)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(repeats):
            deer_solve(dyn, s0, T, x, chunk=L, **opts)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / repeats

    res = pick_best(candidates, time_fn)
    key = make_key(torch.cuda.get_device_name(), dyn.kind, dyn.d, opts.get("jac", "full"),
                   opts.get("prec", "fp64"), T)
    store(key, res, path)
    return res["chunk"]


def cached_chunk(dyn, T: int, jac: str = "full", prec: str = "fp64",
                 path: Optional[str] = None, gpu: Optional[str] = None) -> int:
    """The tuned chunk length for this configuration, or 0 (the library default)."""
    if gpu is None:
        import torch
        gpu = torch.cuda.get_device_name()
    key = make_key(gpu, dyn.kind, dyn.d, jac, prec, T)
    return int(_cache_cached(path or cache_path()).get(key, {}).get("chunk", 0))


_MEMO: Dict[str, tuple] = {}


def _cache_cached(path: str) -> Dict[str, dict]:
    """The cache file's contents, re-read only when the file changed (the solver's default
    path consults it on every call)."""
    try:
        mtime = os.path.getmtime(path)
    except OSError:
        return {}
    hit = _MEMO.get(path)
    if hit is None or hit[0] != mtime:
        hit = (mtime, load_cache(path))
        _MEMO[path] = hit
    return hit[1]
