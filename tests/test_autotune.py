"""Launch-configuration autotuner: host logic on the CPU (key, cache round trip, selection
with failing candidates, which cached options the default path takes), and GPU tuning runs
whose choices are then read back from the cache and served to the default path."""
import math

import numpy as np
import pytest

from paper_2603_16850_gb300 import autotune as at


def test_key_rounds_T_up_to_power_of_two():
    assert at.make_key("G", "massaction", 8, "full", "fp32", 16384).endswith("|T16384")
    assert at.make_key("G", "massaction", 8, "full", "fp32", 16385).endswith("|T32768")
    assert at.make_key("G", "gru", 64, "diag", "fp32", 1) == "G|gru|d64|diag|fp32|T1"


def test_pick_best_skips_failures_and_takes_fastest():
    times = {16: 3.0, 32: 1.5, 64: float("inf"), 128: 2.0}

    def fn(L):
        if L == 256:
            raise ValueError("rejected")
        return times[L]

    res = at.pick_best([16, 32, 64, 128, 256], fn)
    assert res["chunk"] == 32 and res["ms"] == 1.5
    assert math.isinf(res["timings"]["256"]) and math.isinf(res["timings"]["64"])


def test_pick_best_raises_when_nothing_ran():
    with pytest.raises(RuntimeError):
        at.pick_best([16, 32], lambda L: float("inf"))


def test_cache_round_trip(tmp_path):
    p = str(tmp_path / "sub" / "tune.json")
    assert at.load_cache(p) == {}
    at.store("k1", {"chunk": 64, "ms": 1.0}, p)
    at.store("k2", {"chunk": 32, "ms": 2.0}, p)
    c = at.load_cache(p)
    assert c["k1"]["chunk"] == 64 and c["k2"]["chunk"] == 32


@pytest.mark.gpu
def test_tune_chunk_on_gpu(tmp_path):
    import torch

    import paper_2603_16850_gb300 as deer
    import synth
    p = synth.massaction(64, 8, 12, 2048, seed=4)
    dyn = deer.Dynamics.massaction(torch.tensor(p["topology"], dtype=torch.int32, device="cuda"),
                                   torch.tensor(p["params"], dtype=torch.float32, device="cuda"),
                                   8, p["dt"])
    s0 = torch.tensor(p["s0"], dtype=torch.float32, device="cuda")
    path = str(tmp_path / "tune.json")
    best = at.tune_chunk(dyn, s0, 2048, candidates=(32, 64, 128), path=path, jac="full",
                         prec="fp32", tol=5e-7, confirm=2, init="s0", reset=True)
    assert best in (32, 64, 128)
    assert at.cached_chunk(dyn, 2048, "full", "fp32", path=path) == best
    s, info = deer.deer_solve(dyn, s0, 2048, chunk=best, jac="full", prec="fp32", tol=5e-7,
                              confirm=2, init="s0", reset=True)
    assert bool(info.converged.all())
    assert np.isfinite(s.cpu().numpy()).all()


def test_cached_choice_serves_the_default_path(tmp_path, monkeypatch):
    """A tuned entry for (GPU, kind, d, Jacobian mode, precision, T bucket) is what the
    solver's default chunk (0) resolves to; other configurations keep the library default;
    a rewritten cache file is picked up."""
    path = str(tmp_path / "tune.json")
    monkeypatch.setenv("DEER_AUTOTUNE_CACHE", path)

    class Dyn:
        kind, d = "massaction_rk4", 8

    at.store(at.make_key("GB300", "massaction_rk4", 8, "full", "fp32", 16384),
             {"chunk": 128, "ms": 1.0}, path)
    assert at.cached_chunk(Dyn, 10000, "full", "fp32", gpu="GB300") == 128
    assert at.cached_chunk(Dyn, 20000, "full", "fp32", gpu="GB300") == 0
    assert at.cached_chunk(Dyn, 10000, "diag", "fp32", gpu="GB300") == 0
    assert at.cached_chunk(Dyn, 10000, "full", "fp32", gpu="other") == 0
    import os
    import time
    time.sleep(0.01)
    at.store(at.make_key("GB300", "massaction_rk4", 8, "full", "fp32", 16384),
             {"chunk": 64, "ms": 0.5}, path)
    os.utime(path, (time.time() + 5, time.time() + 5))
    assert at.cached_chunk(Dyn, 10000, "full", "fp32", gpu="GB300") == 64


def test_pick_best_config_and_cached_options(tmp_path):
    """Option dicts are timed in order, failures skipped; a cached configuration yields its
    chunk length and loop forms, an entry with chunk only yields the chunk."""
    times = [3.0, 1.0, float("inf")]
    cands = [dict(chunk=32), dict(chunk=32, device_loop=True), dict(chunk=64)]
    res = at.pick_best_config(cands, lambda c: times[cands.index(c)])
    assert res["chunk"] == 32 and res["device_loop"] is True and res["ms"] == 1.0
    assert [t["ms"] for t in res["timings"]][:2] == [3.0, 1.0]
    with pytest.raises(RuntimeError):
        at.pick_best_config(cands[:1], lambda c: float("inf"))
    path = str(tmp_path / "t.json")

    class Dyn:
        kind, d = "brusselator_euler", 2

    at.store(at.make_key("G", Dyn.kind, 2, "full", "fp64", 1024),
             {"chunk": 16, "device_loop": True, "block_solve": False, "ms": 1.0}, path)
    at.store(at.make_key("G", Dyn.kind, 2, "full", "fp64", 64), {"chunk": 8, "ms": 1.0}, path)
    assert at.cached_options(Dyn, 1000, "full", "fp64", path=path, gpu="G") == \
        {"chunk": 16, "device_loop": True, "block_solve": False}
    assert at.cached_options(Dyn, 50, "full", "fp64", path=path, gpu="G") == {"chunk": 8}
    assert at.cached_options(Dyn, 5000, "full", "fp64", path=path, gpu="G") == {}


@pytest.mark.gpu
def test_tune_configuration_serves_the_default_path(tmp_path, monkeypatch):
    """tune() on the Brusselator (T = 1024, FP64) caches a configuration; the default path
    then solves with it (the explicit choice of the caller still wins), and the result is
    the rollout either way."""
    import torch

    import paper_2603_16850_gb300 as deer
    import synth
    from oracle import dynamics as odyn
    from oracle import newton as onewton
    path = str(tmp_path / "tune.json")
    monkeypatch.setenv("DEER_AUTOTUNE_CACHE", path)
    p = synth.brusselator(T=1024)
    dyn = deer.Dynamics.brusselator(torch.tensor(p["params"], device="cuda"), p["dt"])
    s0 = torch.tensor(p["s0"], device="cuda")
    opts = dict(jac="full", prec="fp64", tol=1e-12, reset=True)
    res = at.tune(dyn, s0, 1024, candidates=(16, 64), **opts)
    assert res["chunk"] in (16, 64) and len(res["timings"]) == 4
    assert at.cached_options(dyn, 1024, "full", "fp64") == \
        {k: res[k] for k in ("chunk", "device_loop", "block_solve")}
    ref = onewton.rollout(odyn.Brusselator(p["params"], p["dt"]), p["s0"], 1024)[0]
    for extra in ({}, {"block_solve": False, "device_loop": True}):
        s, info = deer.deer_solve(dyn, s0, 1024, **opts, **extra)
        assert bool(info.converged.all())
        err = np.max(np.abs(s.cpu().numpy() - ref)) / np.max(np.abs(ref))
        assert err <= 1e-10
