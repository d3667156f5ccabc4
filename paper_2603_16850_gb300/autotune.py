"""Autotuner of the solver's launch configuration.

The chunked scans reduce every chunk of L consecutive rows of a sequence to one aggregate
and walk the aggregates of a sequence in order, so L trades the per-chunk serial work
(proportional to L) against the length of the per-sequence carry chain (T / L) and the
number of independent chunks (parallelism). Beside L, the form of the loop matters: the
Newton iterations driven from the host or as one CUDA graph on the device
(``device_loop``), and, for short sequences, the whole solve in one cluster-per-sequence
launch (``block_solve``) against the multi-kernel loop. The best choice depends on the GPU,
the dynamics, d, the Jacobian mode, the precision and T, so it is measured: ``tune`` times
candidates on the caller's own problem with CUDA events (chunk lengths first, then the
loop forms with the best length) and caches the fastest configuration in a JSON file,
keyed by (GPU name, kind, d, jac, prec, T rounded up to a power of two); ``tune_chunk``
tunes L alone. The solver's default path then uses the cached configuration for the same
key: the chunk length where the caller passes ``chunk=0``, the loop forms where the caller
does not set them, and the library's own defaults without an entry.

The diagonal look-back scan fixes its own tile length (it is tied to d), so the chunk
length matters to the dense (full-Jacobian) paths.
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


def cached_options(dyn, T: int, jac: str = "full", prec: str = "fp64",
                   path: Optional[str] = None, gpu: Optional[str] = None) -> dict:
    """The tuned launch options for this configuration (keys among ``chunk``,
    ``device_loop``, ``block_solve``), or {} without an entry."""
    if gpu is None:
        import torch
        gpu = torch.cuda.get_device_name()
    key = make_key(gpu, dyn.kind, dyn.d, jac, prec, T)
    entry = _cache_cached(path or cache_path()).get(key, {})
    out = {}
    if int(entry.get("chunk", 0)) > 0:
        out["chunk"] = int(entry["chunk"])
    for k in ("device_loop", "block_solve"):
        if k in entry:
            out[k] = bool(entry[k])
    return out


def cached_chunk(dyn, T: int, jac: str = "full", prec: str = "fp64",
                 path: Optional[str] = None, gpu: Optional[str] = None) -> int:
    """The tuned chunk length for this configuration, or 0 (the library default)."""
    return cached_options(dyn, T, jac, prec, path, gpu).get("chunk", 0)


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


def pick_best_config(candidates: Iterable[dict], time_fn: Callable[[dict], float]) -> dict:
    """Time every option dict with ``time_fn(opts) -> milliseconds`` (inf = failed) and
    return the fastest, its time and all timings (in candidate order)."""
    rows = []
    for c in candidates:
        try:
            ms = float(time_fn(dict(c)))
        except Exception:  # a configuration the solver rejects is skipped
            ms = float("inf")
        rows.append((dict(c), ms))
    best, best_ms = min(rows, key=lambda r: r[1])
    if not math.isfinite(best_ms):
        raise RuntimeError("no configuration candidate ran")
    return {**best, "ms": best_ms, "timings": [{**c, "ms": ms} for c, ms in rows]}


def tune(dyn, s0, T: int, x=None, candidates=DEFAULT_CANDIDATES, repeats: int = 2,
         path: Optional[str] = None, **opts) -> dict:
    """Tune the chunk length with the multi-kernel host loop, then the loop forms with it:
    the device-resident loop, and the whole solve in one launch (which the library takes
    only for short sequences and otherwise ignores). Caches and returns the fastest
    configuration (``chunk``, ``device_loop``, ``block_solve``, ``ms``, ``timings``)."""
    import torch

    from . import deer_solve

    def time_fn(c: dict) -> float:
        o = dict(opts, **c)
        deer_solve(dyn, s0, T, x, **o)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(repeats):
            deer_solve(dyn, s0, T, x, **o)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / repeats

    loop = dict(device_loop=False, block_solve=False)
    first = pick_best_config([dict(loop, chunk=int(L)) for L in candidates], time_fn)
    L = first["chunk"]
    second = pick_best_config([dict(loop, chunk=L), dict(loop, chunk=L, device_loop=True),
                               dict(chunk=L, device_loop=False, block_solve=True)], time_fn)
    res = {k: second[k] for k in ("chunk", "device_loop", "block_solve", "ms")}
    res["timings"] = first["timings"] + second["timings"][1:]
    key = make_key(torch.cuda.get_device_name(), dyn.kind, dyn.d, opts.get("jac", "full"),
                   opts.get("prec", "fp64"), T)
    store(key, res, path)
    return res
