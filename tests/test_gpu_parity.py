"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (normwise, per sequence: max |s_gpu - s_ref| / max |s_ref|): 1e-10 in FP64
mode and 1e-5 in FP32 mode for converged trajectories; per-iteration iterates in FP64
agree to 1e-11 (they differ only by the association order of the scan).
"""
import numpy as np
import pytest
import torch

import synth
from oracle import dynamics as odyn
from oracle import elk as oelk
from oracle import newton as onewton

pytestmark = pytest.mark.gpu

DEV = "cuda"
# float32 solves: scaled residual 5e-7 (a few units of float32 roundoff, so the test can
# always be met) on two consecutive iterates. The second pass puts one more Newton step
# on top of the first, which removes the smooth part of the remaining error; a single
# pass leaves residuals with a common sign that add up along the conserved directions
# of the kinetics.
FP32_TOL = 5e-7
FP32 = dict(tol=FP32_TOL, confirm=2, prec="fp32")


def _deer():
    import paper_2603_16850_gb300 as deer
    return deer


def _t(a, dt=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dt, device=DEV)


def _relerr(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return np.max(np.abs(got - ref)) / max(np.max(np.abs(ref)), 1e-300)


def _ma_problem(B, d, R, T, seed, dt=1e-3, integ="rk4"):
    return synth.massaction(B, d, R, T, seed, dt=dt, integrator=integ)


def _ma_dyn(p, dtype):
    deer = _deer()
    return deer.Dynamics.massaction(_t(p["topology"], torch.int32), _t(p["params"], dtype),
                                    p["d"], p["dt"], p["kind"].split("_")[1])


def _ma_oracle(p):
    return odyn.MassAction(p["topology"], p["params"], p["dt"], p["kind"].split("_")[1], d=p["d"])


# ---------------------------------------------------------------------------
def test_brusselator_full_size_fp64():
    """Brusselator d=2, Euler dt=0.01, a=1, b=3, s0=(1,1), T=1024, full Newton, FP64,
    tol 1e-12: the converged trajectory equals the sequential rollout. Undamped Newton from
    the constant guess overflows on this limit cycle (the oracle's iterates do too), so the
    reset heuristic is on, as the paper uses it for unstable iterates."""
    deer = _deer()
    p = synth.brusselator(T=1024)
    dyn = deer.Dynamics.brusselator(_t(p["params"]), p["dt"])
    s, info = deer.deer_solve(dyn, _t(p["s0"]), 1024, jac="full", tol=1e-12, prec="fp64",
                              init="s0", reset=True)
    ref = onewton.rollout(odyn.Brusselator(p["params"], p["dt"]), p["s0"], 1024)[0]
    assert bool(info.converged[0])
    assert _relerr(s.cpu().numpy(), ref) <= 1e-10
    o = onewton.solve(odyn.Brusselator(p["params"], p["dt"]), p["s0"], 1024, "full", tol=1e-12,
                      init="s0", reset=True)
    assert o["converged"][0]
    assert abs(int(info.iters[0]) - int(o["iters"][0])) <= max(2, int(o["iters"][0]) // 10)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_brusselator_iterates_match_oracle(k):
    """After k iterations (cap k) the GPU iterate equals k oracle forward-substitution
    steps (T=300: four 64-row chunks and a ragged tail)."""
    deer = _deer()
    T = 300
    p = synth.brusselator(T=T)
    od = odyn.Brusselator(p["params"], p["dt"])
    dyn = deer.Dynamics.brusselator(_t(p["params"]), p["dt"])
    s, info = deer.deer_solve(dyn, _t(p["s0"]), T, jac="full", tol=0.0, max_iters=k, init="s0")
    assert info.status == 1 and int(info.iters[0]) == k
    ref = onewton.initial_guess(od, p["s0"], T, "s0")
    for _ in range(k):
        ref = onewton.quasi_newton_step(od, p["s0"], ref, "full")
    assert _relerr(s.cpu().numpy(), ref[0]) <= 1e-11


@pytest.mark.parametrize("jac,damp,dp", [("full", "none", 0.0), ("diag", "none", 0.0),
                                         ("identity", "none", 0.0), ("zero", "none", 0.0),
                                         ("full", "scale", 0.3), ("diag", "clip", 0.9)])
def test_massaction_modes_fp64(jac, damp, dp):
    deer = _deer()
    B, d, R, T = 3, 4, 6, 200
    p = _ma_problem(B, d, R, T, seed=4, dt=0.02)
    od = _ma_oracle(p)
    dyn = _ma_dyn(p, torch.float64)
    # two iterations from the same start, then the fixed point
    s2, _ = deer.deer_solve(dyn, _t(p["s0"]), T, jac=jac, damp=damp, damp_param=dp, tol=0.0,
                            max_iters=2, init="s0")
    ref = onewton.initial_guess(od, p["s0"], T, "s0")
    for _ in range(2):
        ref = onewton.quasi_newton_step(od, p["s0"], ref, jac, damp, dp)
    assert _relerr(s2.cpu().numpy(), ref.reshape(-1, d)) <= 1e-11
    s, info = deer.deer_solve(dyn, _t(p["s0"]), T, jac=jac, damp=damp, damp_param=dp, tol=1e-12,
                              init="s0", reset=True)
    assert bool(info.converged.all())
    roll = onewton.rollout(od, p["s0"], T)
    for b in range(B):
        assert _relerr(s.cpu().numpy()[b * T:(b + 1) * T], roll[b]) <= 1e-10


@pytest.mark.parametrize("d,R,jac", [(16, 24, "full"), (32, 48, "full"), (16, 24, "diag")])
def test_massaction_wide_fp64_iterates(d, R, jac):
    """d = 16 / 32 (lane-per-species Jacobians, lane-per-column scans): two iterations and
    the fixed point against the oracle in FP64 (T = 150: several chunks and a tail)."""
    deer = _deer()
    B, T = 2, 150
    p = _ma_problem(B, d, R, T, seed=d + 1, dt=0.01)
    od = _ma_oracle(p)
    dyn = _ma_dyn(p, torch.float64)
    s2, _ = deer.deer_solve(dyn, _t(p["s0"]), T, jac=jac, tol=0.0, max_iters=2, init="s0")
    ref = onewton.initial_guess(od, p["s0"], T, "s0")
    for _ in range(2):
        ref = onewton.quasi_newton_step(od, p["s0"], ref, jac)
    assert _relerr(s2.cpu().numpy(), ref.reshape(-1, d)) <= 1e-11
    s, info = deer.deer_solve(dyn, _t(p["s0"]), T, jac=jac, tol=1e-12, init="s0", reset=True,
                              max_iters=400)
    assert bool(info.converged.all())
    roll = onewton.rollout(od, p["s0"], T)
    assert _relerr(s.cpu().numpy(), roll.reshape(-1, d)) <= 1e-10


@pytest.mark.parametrize("d,R", [(2, 3), (8, 12), (16, 24), (32, 48)])
def test_massaction_rk4_fp32_full(d, R):
    deer = _deer()
    B, T = 4, 700
    p = _ma_problem(B, d, R, T, seed=d)
    dyn = _ma_dyn(p, torch.float32)
    s, info = deer.deer_solve(dyn, _t(p["s0"], torch.float32), T, jac="full", init="s0",
                              reset=True, **FP32)
    assert bool(info.converged.all()), info
    roll = onewton.rollout(_ma_oracle(p), p["s0"], T)
    for b in range(B):
        assert _relerr(s.cpu().numpy()[b * T:(b + 1) * T], roll[b]) <= 1e-5


@pytest.mark.parametrize("d,prec", [(8, "fp64"), (64, "fp32")])
def test_gru_quasi_deer(d, prec):
    deer = _deer()
    B, T = 2, 400
    dt = torch.float32 if prec == "fp32" else torch.float64
    g = synth.gru(B, T, d, d, seed=1)
    dyn = deer.Dynamics.gru(_t(g["W"], dt), _t(g["U"], dt))
    x = _t(g["x"].reshape(-1, d), dt)
    extra = dict(tol=1e-12, prec="fp64") if prec == "fp64" else FP32
    s, info = deer.deer_solve(dyn, _t(g["s0"], dt), T, x, jac="diag", init="zeros", **extra)
    assert bool(info.converged.all())
    roll = onewton.rollout(odyn.GRU(g["W"], g["U"], g["x"]), g["s0"], T)
    lim = 1e-10 if prec == "fp64" else 1e-5
    for b in range(B):
        assert _relerr(s.cpu().numpy()[b * T:(b + 1) * T], roll[b]) <= lim


@pytest.mark.parametrize("jac", ["diag", "zero"])
def test_gru_tensor_core_linearisation_matches_simt(jac):
    """GRU d = 64 float32: the tcgen05 linearisation (three products per step as tf32 MMAs
    split to float32 accuracy) and the SIMT one give the same iterates up to float32
    rounding, and both converge to the float64 rollout within 1e-5."""
    deer = _deer()
    B, T, d = 3, 1000, 64  # 3000 rows: 23 tiles of 128 and a ragged last tile
    g = synth.gru(B, T, d, d, seed=5)
    dyn = deer.Dynamics.gru(_t(g["W"], torch.float32), _t(g["U"], torch.float32))
    x = _t(g["x"].reshape(-1, d), torch.float32)
    s0 = _t(g["s0"], torch.float32)
    out = {}
    try:
        for tc in (True, False):
            deer.set_tensor_cores(tc)
            s2, _ = deer.deer_solve(dyn, s0, T, x, jac=jac, tol=0.0, max_iters=2,
                                    init="zeros", prec="fp32")
            s, info = deer.deer_solve(dyn, s0, T, x, jac=jac, init="zeros", max_iters=T,
                                      **FP32)
            assert bool(info.converged.all()), (tc, info.iters.max())
            out[tc] = (s2.cpu().numpy(), s.cpu().numpy())
    finally:
        deer.set_tensor_cores(True)
    assert _relerr(out[True][0], out[False][0]) <= 2e-6
    roll = onewton.rollout(odyn.GRU(g["W"], g["U"], g["x"]), g["s0"], T)
    for tc in (True, False):
        for b in range(B):
            assert _relerr(out[tc][1][b * T:(b + 1) * T], roll[b]) <= 1e-5


@pytest.mark.parametrize("lam", [0.5, 10.0])
def test_gru_quasi_elk_iterates(lam):
    """Kalman-filter damped quasi-DEER (quasi-ELK): each iterate equals the oracle's
    filtered means; the fixed point equals the rollout."""
    deer = _deer()
    B, T, d = 2, 260, 8
    g = synth.gru(B, T, d, d, seed=3)
    od = odyn.GRU(g["W"], g["U"], g["x"])
    dyn = deer.Dynamics.gru(_t(g["W"]), _t(g["U"]))
    x = _t(g["x"].reshape(-1, d))
    s2, _ = deer.deer_solve(dyn, _t(g["s0"]), T, x, jac="diag", damp="elk", damp_param=lam,
                            tol=0.0, max_iters=2, init="zeros")
    ref = onewton.initial_guess(od, g["s0"], T, "zeros")
    for _ in range(2):
        ref = oelk.elk_filter_step(od, g["s0"], ref, "diag", lam)
    assert _relerr(s2.cpu().numpy(), ref.reshape(-1, d)) <= 1e-11
    s, info = deer.deer_solve(dyn, _t(g["s0"]), T, x, jac="diag", damp="elk", damp_param=lam,
                              tol=1e-12, init="zeros", max_iters=20 * T)
    assert bool(info.converged.all())
    roll = onewton.rollout(od, g["s0"], T)
    assert _relerr(s.cpu().numpy(), roll.reshape(-1, d)) <= 1e-10


def test_linear_converges_in_one_iteration():
    deer = _deer()
    lds = synth.linear_lds(B=3, T=500, d=8, seed=5)
    dyn = deer.Dynamics.linear(_t(lds["A"]))
    s, info = deer.deer_solve(dyn, _t(lds["s0"]), 500, _t(lds["x"].reshape(-1, 8)), jac="full",
                              tol=1e-9, init="zeros")
    assert info.iters.tolist() == [1, 1, 1]
    roll = onewton.rollout(odyn.Linear(lds["A"], lds["x"]), lds["s0"], 500)
    assert _relerr(s.cpu().numpy(), roll.reshape(-1, 8)) <= 1e-10


def test_ragged_batch_matches_per_sequence_rollouts():
    deer = _deer()
    lengths = [0, 1, 2, 300, 77, 129, 64]
    off = synth.offsets_from_lengths(lengths)
    B, d, R = len(lengths), 4, 6
    p = _ma_problem(B, d, R, 1, seed=9, dt=0.02)
    dyn = _ma_dyn(p, torch.float64)
    s, info = deer.deer_solve_batched(dyn, _t(p["s0"]), off, jac="full", tol=1e-12, init="s0")
    assert bool(info.converged.all())
    assert int(info.iters[0]) == 0 and int(info.iters[1]) == 1
    od = _ma_oracle(p)
    sn = s.cpu().numpy()
    for b, L in enumerate(lengths):
        if L == 0:
            continue
        sub = odyn.MassAction(p["topology"][b:b + 1], p["params"][b:b + 1], p["dt"], "rk4", d=d)
        roll = onewton.rollout(sub, p["s0"][b:b + 1], L)[0]
        assert _relerr(sn[off[b]:off[b + 1]], roll) <= 1e-10


@pytest.mark.parametrize("d,R,jac,prec", [(8, 12, "diag", "fp32"), (16, 24, "diag", "fp32"),
                                          (32, 48, "diag", "fp32"), (8, 12, "identity", "fp32"),
                                          (4, 6, "diag", "fp64"), (32, 48, "diag", "fp64")])
def test_diag_lookback_ragged(d, R, jac, prec):
    """Single-pass look-back diagonal scans (tiles of 8192 / d rows, 1024 for d = 4; Picard
    reads no a) on a ragged batch whose lengths are below, at and above the tile length:
    every sequence equals its float64 rollout within 1e-5 (float32) or 1e-10 (float64).
    float32 uses d >= 8: the standard-form diagonal update has a float32 residual floor
    near 5e-7 on the longer d = 4 sequences, where the float32 test cannot be met."""
    deer = _deer()
    L = 8192 // d if d >= 8 else 1024
    lengths = [L - 1, 1, L + 3, L, 37]
    off = synth.offsets_from_lengths(lengths)
    B = len(lengths)
    p = _ma_problem(B, d, R, 1, seed=21)
    dt = torch.float32 if prec == "fp32" else torch.float64
    dyn = _ma_dyn(p, dt)
    extra = FP32 if prec == "fp32" else dict(tol=1e-12, prec="fp64")
    s, info = deer.deer_solve_batched(dyn, _t(p["s0"], dt), off, jac=jac, init="s0",
                                      reset=True, max_iters=4000, **extra)
    assert bool(info.converged.all()), (info.iters.max(), info.max_resid.max())
    sn = s.cpu().numpy()
    lim = 1e-5 if prec == "fp32" else 1e-10
    for b, n in enumerate(lengths):
        sub = odyn.MassAction(p["topology"][b:b + 1], p["params"][b:b + 1], p["dt"], "rk4", d=d)
        roll = onewton.rollout(sub, p["s0"][b:b + 1], n)[0]
        assert _relerr(sn[off[b]:off[b + 1]], roll) <= lim


@pytest.mark.parametrize("case", ["full_fp64_d4", "full_fp32_d8", "full_fp32_d16",
                                  "diag_fp64_d8", "diag_fp64_d2", "elk_fp64_gru8",
                                  "mixed_d16", "gru64_fp32_tc"])
def test_sliding_window_matches_rollout(case):
    """Sliding window (Sec. 3.2): the converged prefix of every sequence is frozen and later
    iterations solve only from its first failing chunk on. The fixed point is unchanged: on
    ragged batches every path (fused d <= 8, wide dense, three-pass and look-back diagonal,
    quasi-ELK, mixed precision, tensor-core GRU) returns the sequential rollout, and no more
    rows are linearised than without the window (up to a margin: frozen rows sit anywhere
    within the tolerance, which can cost the rows after them an extra iteration)."""
    deer = _deer()
    from paper_2603_16850_gb300 import _native as N
    lib = N.load()
    kind, prec, d = case.split("_")[0], case.split("_")[1], case.split("_")[-1]
    lengths = [900, 1, 257, 2000, 64]
    off = synth.offsets_from_lengths(lengths)
    B = len(lengths)
    x = None
    if kind in ("full", "diag", "mixed"):
        dd = int(d[1:])
        R = {2: 3, 4: 6, 8: 12, 16: 24}[dd]
        p = _ma_problem(B, dd, R, 1, seed=31)
        tdt = torch.float32 if prec == "fp32" else torch.float64
        dyn = _ma_dyn(p, tdt)
        s0 = _t(p["s0"], tdt)
        opts = dict(jac="full" if kind != "diag" else "diag", init="zeros", reset=True,
                    max_iters=3000)
        if prec == "fp32":
            opts.update(FP32)
        elif kind == "mixed":
            opts.update(tol=1e-12, prec="mixed_bf16")
        else:
            opts.update(tol=1e-12, prec="fp64")
        rolls = [onewton.rollout(odyn.MassAction(p["topology"][b:b + 1], p["params"][b:b + 1],
                                                 p["dt"], "rk4", d=dd), p["s0"][b:b + 1], n)[0]
                 for b, n in enumerate(lengths)]
    else:
        dd = 8 if case.endswith("gru8") else 64
        g = synth.gru(1, sum(lengths), dd, dd, seed=32)
        tdt = torch.float32 if prec == "fp32" else torch.float64
        dyn = deer.Dynamics.gru(_t(g["W"], tdt), _t(g["U"], tdt))
        x = _t(g["x"].reshape(-1, dd), tdt)
        s0 = _t(np.zeros((B, dd)), tdt)
        opts = dict(jac="diag", init="zeros", max_iters=3000)
        if kind == "elk":
            opts.update(damp="elk", damp_param=2.0)
        opts.update(FP32 if prec == "fp32" else dict(tol=1e-12, prec="fp64"))
        xs = g["x"][0]
        rolls = []
        for b, n in enumerate(lengths):
            sub = odyn.GRU(g["W"], g["U"], xs[off[b]:off[b + 1]][None])
            rolls.append(onewton.rollout(sub, np.zeros((1, dd)), n)[0])
    rows = {}
    for win in (False, True):
        lib.deer_profile_reset()
        lib.deer_profile_enable(1)
        s, info = deer.deer_solve_batched(dyn, s0, off, x, window=win, **opts)
        torch.cuda.synchronize()
        lib.deer_profile_enable(0)
        prof = N.deer_profile()
        lib.deer_profile_read(prof)
        rows[win] = int(prof.rows[1])
        assert bool(info.converged.all()), (case, win, info.iters.max())
        sn = s.cpu().numpy()
        # float64 rows are frozen once their scaled residual is below tol, so along the
        # conserved directions of the kinetics the frozen prefix carries up to ~T tol of
        # drift (the unwindowed iteration keeps refining it while later rows converge)
        lim = 1e-5 if prec == "fp32" else (1e-9 if (kind == "mixed" or win) else 1e-10)
        for b in range(B):
            assert _relerr(sn[off[b]:off[b + 1]], rolls[b]) <= lim, (case, win, b)
    assert rows[True] <= 1.25 * rows[False], rows


@pytest.mark.parametrize("kind", ["massaction_rk4", "gru", "brusselator"])
def test_sequential_rollout_parity(kind):
    deer = _deer()
    if kind == "massaction_rk4":
        p = _ma_problem(5, 8, 12, 400, seed=2)
        dyn, s0, T, x = _ma_dyn(p, torch.float64), p["s0"], 400, None
        ref = onewton.rollout(_ma_oracle(p), p["s0"], 400)
    elif kind == "gru":
        g = synth.gru(3, 200, 16, 16, seed=2)
        dyn, s0, T = deer.Dynamics.gru(_t(g["W"]), _t(g["U"])), g["s0"], 200
        x = _t(g["x"].reshape(-1, 16))
        ref = onewton.rollout(odyn.GRU(g["W"], g["U"], g["x"]), g["s0"], 200)
    else:
        p = synth.brusselator(T=1024)
        dyn, s0, T, x = deer.Dynamics.brusselator(_t(p["params"]), p["dt"]), p["s0"], 1024, None
        ref = onewton.rollout(odyn.Brusselator(p["params"], p["dt"]), p["s0"], 1024)
    s = deer.deer_rollout(dyn, _t(s0), T, x)
    assert _relerr(s.cpu().numpy(), ref.reshape(s.shape)) <= 1e-12


def test_nonfinite_input_is_reported():
    deer = _deer()
    p = synth.brusselator(T=100)
    dyn = deer.Dynamics.brusselator(_t(p["params"]), p["dt"])
    s0 = _t([[float("nan"), 1.0]])
    with pytest.raises(RuntimeError, match="non-finite"):
        deer.deer_solve(dyn, s0, 100, jac="full", tol=1e-12)


@pytest.mark.parametrize("window", [False, True])
def test_full_size_batched_massaction_fp32_sampled(window):
    """B=4096 systems, d=8, 12 reactions, RK4 dt=1e-3, T=16384, full Newton, FP32 (with and
    without the sliding window, the benchmark runs with it): sampled trajectories equal the
    FP64 oracle rollout within 1e-5."""
    deer = _deer()
    B, d, R, T = 4096, 8, 12, 16384
    p = _ma_problem(B, d, R, T, seed=0)
    dyn = _ma_dyn(p, torch.float32)
    s, info = deer.deer_solve(dyn, _t(p["s0"], torch.float32), T, jac="full", init="zeros",
                              reset=True, window=window, **FP32)
    assert bool(info.converged.all()), (info.max_resid.max(), info.iters.max())
    assert float(info.max_resid.max()) <= FP32_TOL
    rng = np.random.default_rng(0)
    # two random systems and the one that needed the most iterations
    pick = np.concatenate([rng.choice(B, size=2, replace=False), [int(info.iters.argmax())]])
    sub = odyn.MassAction(p["topology"][pick], p["params"][pick], p["dt"], "rk4", d=d)
    roll = onewton.rollout(sub, p["s0"][pick], T)
    sv = s.view(B, T, d)
    for i, b in enumerate(pick):
        assert _relerr(sv[b].cpu().numpy(), roll[i]) <= 1e-5


@pytest.mark.parametrize("window", [False, True])
def test_full_size_gru_quasi_deer_fp32_sampled(window):
    """GRU d=64, inputs 64, T=65536, B=64, weights N(0,1/d), inputs N(0,1), quasi-DEER,
    FP32, tol 1e-5 (scaled residual), with and without the sliding window: sampled
    trajectories equal the FP64 oracle rollout within 1e-5."""
    deer = _deer()
    B, T, d = 64, 65536, 64
    g = synth.gru(B, T, d, d, seed=0, dtype=np.float32)
    dyn = deer.Dynamics.gru(_t(g["W"], torch.float32), _t(g["U"], torch.float32))
    x = torch.tensor(g["x"].reshape(-1, d), device=DEV)
    s, info = deer.deer_solve(dyn, _t(g["s0"], torch.float32), T, x, jac="diag", tol=1e-5,
                              confirm=2, prec="fp32", init="zeros", window=window)
    assert bool(info.converged.all()), (info.max_resid.max(), info.iters.max())
    pick = [0, int(info.iters.argmax())]
    sub = odyn.GRU(g["W"], g["U"], g["x"][pick].astype(np.float64))
    roll = onewton.rollout(sub, g["s0"][pick], T)
    sv = s.view(B, T, d)
    for i, b in enumerate(pick):
        assert _relerr(sv[b].cpu().numpy(), roll[i]) <= 1e-5


@pytest.mark.parametrize("lam", [1.0])
def test_gru_d64_quasi_elk_fp32(lam):
    deer = _deer()
    B, T, d = 3, 3000, 64
    g = synth.gru(B, T, d, d, seed=4)
    dyn = deer.Dynamics.gru(_t(g["W"], torch.float32), _t(g["U"], torch.float32))
    x = _t(g["x"].reshape(-1, d), torch.float32)
    s, info = deer.deer_solve(dyn, _t(g["s0"], torch.float32), T, x, jac="diag", damp="elk",
                              damp_param=lam, init="zeros", **FP32)
    assert bool(info.converged.all())
    roll = onewton.rollout(odyn.GRU(g["W"], g["U"], g["x"]), g["s0"], T)
    for b in range(B):
        assert _relerr(s.cpu().numpy()[b * T:(b + 1) * T], roll[b]) <= 1e-5


@pytest.mark.parametrize("d,R", [(16, 24), (32, 48)])
def test_mixed_bf16_ragged_matches_fp64_rollout(d, R):
    """Mixed precision (bf16 Jacobians E = A - I, float32 scan accumulation, float64
    state and residual) on a ragged batch: the fixed point is refined against the float64
    residual, so it equals the float64 rollout to float64 accuracy."""
    deer = _deer()
    lengths = [300, 1000, 77, 2000, 1]
    off = synth.offsets_from_lengths(lengths)
    B = len(lengths)
    p = _ma_problem(B, d, R, 1, seed=12)
    dyn = _ma_dyn(p, torch.float64)
    s, info = deer.deer_solve_batched(dyn, _t(p["s0"]), off, jac="full", tol=1e-12,
                                      prec="mixed_bf16", init="s0", reset=True, max_iters=500)
    assert bool(info.converged.all()), info
    od = _ma_oracle(p)
    sn = s.cpu().numpy()
    for b, L in enumerate(lengths):
        sub = odyn.MassAction(p["topology"][b:b + 1], p["params"][b:b + 1], p["dt"], "rk4", d=d)
        roll = onewton.rollout(sub, p["s0"][b:b + 1], L)[0]
        assert _relerr(sn[off[b]:off[b + 1]], roll) <= 1e-9


@pytest.mark.parametrize("d,lam", [(2, 0.7), (4, 3.0), (8, 1.0)])
def test_dense_elk_iterates_and_fixed_point(d, lam):
    """Dense ELK (full-Jacobian Kalman-filter step, Sec. 4.2-4.3): two iterations equal the
    oracle's filtered means (elk_filter_step with the full Jacobian) and the iteration
    converges to the sequential rollout."""
    deer = _deer()
    B, T = 3, 300
    R = {2: 3, 4: 6, 8: 12}[d]
    p = _ma_problem(B, d, R, T, seed=50 + d, dt=0.01)
    od = _ma_oracle(p)
    dyn = _ma_dyn(p, torch.float64)
    s2, _ = deer.deer_solve(dyn, _t(p["s0"]), T, jac="full", damp="elk", damp_param=lam,
                            tol=0.0, max_iters=2, init="s0")
    ref = onewton.initial_guess(od, p["s0"], T, "s0")
    for _ in range(2):
        ref = oelk.elk_filter_step(od, p["s0"], ref, "full", lam)
    assert _relerr(s2.cpu().numpy(), ref.reshape(-1, d)) <= 1e-11
    s, info = deer.deer_solve(dyn, _t(p["s0"]), T, jac="full", damp="elk", damp_param=lam,
                              tol=1e-12, init="s0", max_iters=2000)
    assert bool(info.converged.all()), info.iters.max()
    roll = onewton.rollout(od, p["s0"], T)
    for b in range(B):
        assert _relerr(s.cpu().numpy()[b * T:(b + 1) * T], roll[b]) <= 1e-10


@pytest.mark.parametrize("d,lam,lengths", [(4, 2.0, [6000]), (8, 0.5, [4000, 2500]),
                                            (16, 1.0, [3000])])
def test_dense_elk_covariance_in_parallel_over_time(d, lam, lengths):
    """Dense ELK on few long sequences, where the covariance recursion runs in parallel
    over time (chunk aggregates of the filter's associative elements, a carry across
    chunks, the per-row recursion restarted from the carried covariance): two iterations
    equal the oracle's sequential Kalman filter (elk_filter_step), and the rollout is a
    fixed point of the step (a warm start there is accepted at once and left in place).
    From s0 the damped iteration needs thousands of iterations at these horizons: with
    dt = 0.01 every A_t is close to I, so the residual Jacobian has singular values of
    order 1/T, and error along them shrinks only by lambda / (lambda + sigma^2) per step.
    d = 16 also covers the smaller thread blocks of that size."""
    deer = _deer()
    off = synth.offsets_from_lengths(lengths)
    R = {4: 6, 8: 12, 16: 24}[d]
    p = _ma_problem(len(lengths), d, R, 1, seed=70 + d, dt=0.01)
    dyn = _ma_dyn(p, torch.float64)
    s2, _ = deer.deer_solve_batched(dyn, _t(p["s0"]), off, jac="full", damp="elk",
                                    damp_param=lam, tol=0.0, max_iters=2, init="s0",
                                    chunk=128)
    s2 = s2.cpu().numpy()
    for b, n in enumerate(lengths):
        sub = odyn.MassAction(p["topology"][b:b + 1], p["params"][b:b + 1], p["dt"], "rk4", d=d)
        s0b = p["s0"][b:b + 1]
        ref = onewton.initial_guess(sub, s0b, n, "s0")
        for _ in range(2):
            ref = oelk.elk_filter_step(sub, s0b, ref, "full", lam)
        assert _relerr(s2[off[b]:off[b + 1]], ref[0]) <= 1e-11, b
    rolls = []
    for b, n in enumerate(lengths):
        sub = odyn.MassAction(p["topology"][b:b + 1], p["params"][b:b + 1], p["dt"], "rk4", d=d)
        rolls.append(onewton.rollout(sub, p["s0"][b:b + 1], n)[0])
    s, info = deer.deer_solve_batched(dyn, _t(p["s0"]), off, jac="full", damp="elk",
                                      damp_param=lam, tol=1e-11, init="user", chunk=128,
                                      s_init=_t(np.concatenate(rolls)), max_iters=3)
    assert bool(info.converged.all()) and int(info.iters.max()) <= 2, info
    sn = s.cpu().numpy()
    for b in range(len(lengths)):
        assert _relerr(sn[off[b]:off[b + 1]], rolls[b]) <= 1e-9, b


@pytest.mark.parametrize("window", [False, True])
def test_dense_elk_fp32_ragged_converges(window):
    """Dense ELK in float32 on a ragged batch, within 1e-5 of the float64 rollout. The
    sliding window does not apply to damped steps (they converge linearly, so rows would
    be frozen with too little margin for float32): the option is accepted and ignored."""
    deer = _deer()
    lengths = [700, 33, 1500]
    off = synth.offsets_from_lengths(lengths)
    p = _ma_problem(3, 8, 12, 1, seed=55)
    dyn = _ma_dyn(p, torch.float32)
    s, info = deer.deer_solve_batched(dyn, _t(p["s0"], torch.float32), off, jac="full",
                                      damp="elk", damp_param=0.5, init="zeros", reset=True,
                                      window=window, max_iters=3000, **FP32)
    assert bool(info.converged.all()), info.iters.max()
    sn = s.cpu().numpy()
    for b, n in enumerate(lengths):
        sub = odyn.MassAction(p["topology"][b:b + 1], p["params"][b:b + 1], p["dt"], "rk4", d=8)
        roll = onewton.rollout(sub, p["s0"][b:b + 1], n)[0]
        assert _relerr(sn[off[b]:off[b + 1]], roll) <= 1e-5


def test_host_inputs_round_trip_into_preallocated_output():
    """The end-to-end form of the API: host (pinned) inputs are copied to the GPU, the
    trajectory comes back into the caller's pinned buffer, and equals the device-resident
    solve bit for bit; a mismatched output buffer is rejected before any work."""
    deer = _deer()
    p = _ma_problem(4, 8, 12, 300, seed=21)
    dyn_d = _ma_dyn(p, torch.float32)
    s0_d = _t(p["s0"], torch.float32)
    opts = dict(jac="full", init="zeros", reset=True, window=True, **FP32)
    s_dev, info_d = deer.deer_solve(dyn_d, s0_d, 300, **opts)
    dyn_h = deer.Dynamics.massaction(dyn_d.topology.cpu().pin_memory(),
                                     dyn_d.params.cpu().pin_memory(), 8, p["dt"])
    out = torch.empty((4 * 300, 8), dtype=torch.float32, pin_memory=True)
    s_h, info_h = deer.deer_solve(dyn_h, s0_d.cpu().pin_memory(), 300, out=out, **opts)
    assert s_h.data_ptr() == out.data_ptr() and not s_h.is_cuda
    assert torch.equal(s_h, s_dev.cpu()) and info_h.iters.tolist() == info_d.iters.tolist()
    with pytest.raises(ValueError):
        deer.deer_solve(dyn_h, s0_d.cpu(), 300, out=torch.empty((10, 8)), **opts)


def test_bounded_wait_times_out_and_context_stays_usable():
    """The failure path of the device waits, made on the GPU without a fault: the look-back
    scan's wait for a predecessor flag that nothing sets runs out at its spin limit, the
    kernel records DEER_ERR_TIMEOUT and finishes, and the next solve runs normally."""
    import time
    deer = _deer()
    t0 = time.perf_counter()
    st = deer.selftest_wait_timeout()
    torch.cuda.synchronize()
    assert st == -5 and time.perf_counter() - t0 < 30.0
    p = synth.brusselator(T=200)
    dyn = deer.Dynamics.brusselator(_t(p["params"]), p["dt"])
    s, info = deer.deer_solve(dyn, _t(p["s0"]), 200, jac="full", tol=1e-12, init="s0")
    ref = onewton.rollout(odyn.Brusselator(p["params"], p["dt"]), p["s0"], 200)[0]
    assert bool(info.converged[0]) and _relerr(s.cpu().numpy(), ref) <= 1e-10


@pytest.mark.parametrize("kind", ["massaction_d32", "rnn_d32"])
def test_dense_tensor_core_compose_matches_simt(kind):
    """The d = 32 float32 chunk products on the tensor cores (warp-level tf32 MMAs with the
    three-term split) give the iterates of the SIMT chunk pass to float32 accuracy, and
    both converge to the FP64 oracle's rollout (a ragged tail of chunks, several chunks per
    sequence)."""
    deer = _deer()
    B, T, d = 3, 700, 32
    if kind == "massaction_d32":
        p = _ma_problem(B, d, 48, T, seed=17)
        dyn = _ma_dyn(p, torch.float32)
        s0, x = _t(p["s0"], torch.float32), None
        roll = onewton.rollout(_ma_oracle(p), p["s0"], T)
    else:
        p = synth.mean_field_rnn(B, T, d, 0.5, seed=2)
        dyn = deer.Dynamics.rnn_tanh(_t(p["W"], torch.float32))
        s0, x = _t(p["s0"], torch.float32), _t(p["x"].reshape(-1, d), torch.float32)
        roll = onewton.rollout(odyn.MeanFieldRNN(p["W"], p["x"]), p["s0"], T)
    out = {}
    try:
        for tc in (True, False):
            deer.set_tensor_cores(tc)
            it2, _ = deer.deer_solve(dyn, s0, T, x, jac="full", tol=0.0, max_iters=2,
                                     prec="fp32", init="zeros", chunk=64)
            full, info = deer.deer_solve(dyn, s0, T, x, jac="full", init="zeros", chunk=64,
                                         reset=True, **dict(FP32, tol=5e-8))
            assert bool(info.converged.all())
            out[tc] = (it2.cpu().numpy(), full.cpu().numpy(), info.iters.tolist())
    finally:
        deer.set_tensor_cores(True)
    # two float32 roundings of the chunk products, amplified by two Newton steps far from
    # the fixed point
    assert _relerr(out[True][0], out[False][0]) <= 1e-4
    for tc in (True, False):
        for b in range(B):
            assert _relerr(out[tc][1][b * T:(b + 1) * T], roll[b]) <= 1e-5
