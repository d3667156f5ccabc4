"""The whole-solve kernel for short sequences (one thread-block cluster per sequence runs
every Newton iteration: linearisation, convergence test, cluster-wide scan). Each case is solved
with it and with the multi-kernel loop (block_solve=False): both reach the FP64 oracle's
sequential rollout within the tolerance of their precision, two iterations from the same
start equal the oracle's Newton iterates (the scan's association order is the only
difference, within 1e-11 in FP64), and the whole solve is one kernel launch beside the
set-up kernels.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import dynamics as odyn
from oracle import newton as onewton

pytestmark = pytest.mark.gpu

DEV = "cuda"


def _deer():
    import paper_2603_16850_gb300 as deer
    return deer


def _t(a, dt=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dt, device=DEV)


def _relerr(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return np.max(np.abs(got - ref)) / max(np.max(np.abs(ref)), 1e-300)


def _problem(name, dt=torch.float64):
    """(lengths, s0 host, oracle dynamics per sequence b, GPU dynamics, GPU inputs)."""
    deer = _deer()
    if name == "brusselator":
        p = synth.brusselator(T=1024)
        return ([1024], p["s0"], lambda b: odyn.Brusselator(p["params"], p["dt"]),
                deer.Dynamics.brusselator(_t(p["params"], dt), p["dt"]), None)
    if name in ("ma4_rk4", "ma2_euler"):
        d, R, integ = (4, 6, "rk4") if name == "ma4_rk4" else (2, 3, "euler")
        lengths = [1024, 1, 0, 2, 300, 77, 1000] if d == 4 else [4096, 5, 2048, 33]
        p = synth.massaction(len(lengths), d, R, 1, seed=21 + d, dt=0.01, integrator=integ)

        def od(b):
            return odyn.MassAction(p["topology"][b:b + 1], p["params"][b:b + 1], p["dt"],
                                   integ, d=d)
        dyn = deer.Dynamics.massaction(_t(p["topology"], torch.int32), _t(p["params"], dt), d,
                                       p["dt"], integ)
        return lengths, p["s0"], od, dyn, None
    if name == "langevin1":
        T = 4096
        p = synth.two_well(2, T, 1, seed=5)
        x = p["x"]
        return ([T, T], p["s0"],
                lambda b: odyn.TwoWellLangevin(p["params"], p["dt"], x[b:b + 1], d=1),
                deer.Dynamics.langevin_2well(_t(p["params"], dt), p["dt"]),
                _t(x.reshape(-1, 1), dt))
    if name == "rnn4":
        T = 900
        p = synth.mean_field_rnn(3, T, 4, 0.8, seed=6)
        return ([T] * 3, p["s0"], lambda b: odyn.MeanFieldRNN(p["W"], p["x"][b:b + 1]),
                deer.Dynamics.rnn_tanh(_t(p["W"], dt)), _t(p["x"].reshape(-1, 4), dt))
    raise KeyError(name)


def _solve(name, dt=torch.float64, **opts):
    deer = _deer()
    lengths, s0, od, dyn, x = _problem(name, dt)
    off = synth.offsets_from_lengths(lengths)
    s, info = deer.deer_solve_batched(dyn, _t(s0, dt), off, x, **opts)
    return s.cpu().numpy(), info, lengths, off, s0, od


@pytest.mark.parametrize("name", ["brusselator", "ma4_rk4", "ma2_euler", "langevin1", "rnn4"])
@pytest.mark.parametrize("block", [True, False])
def test_fp64_solve_reaches_rollout(name, block):
    s, info, lengths, off, s0, od = _solve(name, jac="full", tol=1e-12, init="s0", reset=True,
                                           block_solve=block)
    assert bool(info.converged.all()), info
    for b, n in enumerate(lengths):
        if n == 0:  # an empty sequence (converged at once, nothing to compare)
            continue
        roll = onewton.rollout(od(b), s0[b:b + 1], n)[0]
        assert _relerr(s[off[b]:off[b + 1]], roll) <= 1e-10, (b, n)


@pytest.mark.parametrize("name", ["brusselator", "ma4_rk4", "langevin1"])
def test_two_iterations_equal_the_oracle(name):
    """Two Newton iterations from s_0: the block solve's and the multi-kernel loop's
    iterates both equal two forward-substitution steps of the oracle."""
    for block in (True, False):
        s, info, lengths, off, s0, od = _solve(name, jac="full", tol=0.0, max_iters=2,
                                               init="s0", block_solve=block)
        # (sequences of one or two steps are exact after one or two iterations)
        assert info.status == 1 and max(info.iters.tolist()) == 2
        for b, n in enumerate(lengths):
            if n == 0:
                continue
            ref = onewton.initial_guess(od(b), s0[b:b + 1], n, "s0")
            for _ in range(2):
                ref = onewton.quasi_newton_step(od(b), s0[b:b + 1], ref, "full")
            tol = 1e-10 if name == "langevin1" else 1e-11
            assert _relerr(s[off[b]:off[b + 1]], ref[0]) <= tol, (block, b)


def test_fp32_reaches_the_fp64_rollout():
    """float32 (mass action d = 2, Euler; no compensated state at this size) reaches the
    float64 rollout within 1e-5 on both loops. (Their iteration counts may differ by a few:
    near the float32 rounding floor the scaled residual sits close to the tolerance, and
    the two scans round differently.)"""
    opts = dict(jac="full", tol=5e-7, confirm=2, prec="fp32", init="zeros", reset=True)
    for block in (True, False):
        s, info, lengths, off, s0, od = _solve("ma2_euler", torch.float32, block_solve=block,
                                               **opts)
        assert bool(info.converged.all()), (block, info)
        for b, n in enumerate(lengths):
            roll = onewton.rollout(od(b), s0[b:b + 1], n)[0]
            assert _relerr(s[off[b]:off[b + 1]], roll) <= 1e-5, (block, b)


def test_linear_recurrence_in_one_iteration():
    deer = _deer()
    lds = synth.linear_lds(B=2, T=2000, d=2, seed=8)
    dyn = deer.Dynamics.linear(_t(lds["A"]))
    s, info = deer.deer_solve(dyn, _t(lds["s0"]), 2000, _t(lds["x"].reshape(-1, 2)),
                              jac="full", tol=1e-9, init="zeros")
    assert info.iters.tolist() == [1, 1]
    roll = onewton.rollout(odyn.Linear(lds["A"], lds["x"]), lds["s0"], 2000)
    assert _relerr(s.cpu().numpy(), roll.reshape(-1, 2)) <= 1e-10


def test_one_launch_and_fallback_past_the_block_size():
    """The Brusselator at T = 1024 is the sequence tables, the initial guess, the
    active-set pass and one whole-solve launch; at T = 8193 (past the 8192 steps a cluster holds for d = 2) the
    multi-kernel loop takes over and still reaches the rollout."""
    deer = _deer()
    p = synth.brusselator(T=8193)
    dyn = deer.Dynamics.brusselator(_t(p["params"]), p["dt"])
    s0 = _t(p["s0"])
    n0 = deer.kernel_launch_count()
    _, info = deer.deer_solve(dyn, s0, 1024, jac="full", tol=1e-12, reset=True)
    torch.cuda.synchronize()
    assert deer.kernel_launch_count() - n0 == 4 and bool(info.converged.all())
    n1 = deer.kernel_launch_count()
    s, info = deer.deer_solve(dyn, s0, 8193, jac="full", tol=1e-12, reset=True)
    torch.cuda.synchronize()
    assert deer.kernel_launch_count() - n1 > 4 + 2 * int(info.iters[0])
    roll = onewton.rollout(odyn.Brusselator(p["params"], p["dt"]), p["s0"], 8193)[0]
    assert bool(info.converged.all()) and _relerr(s.cpu().numpy(), roll) <= 1e-10


def test_iteration_cap_and_status():
    s, info, lengths, off, s0, od = _solve("brusselator", jac="full", tol=1e-30, max_iters=3,
                                           init="s0", reset=True)
    assert info.status == 1 and not bool(info.converged.any())
    assert info.iters.tolist() == [3]


@pytest.mark.parametrize("k", [0.3, 0.7])
def test_scale_damping_iterates_equal_the_oracle(k):
    """Scale damping (A_t scaled by 1 - k) inside the whole-solve kernel: two iterations equal
    the oracle's damped forward-substitution steps, and the damped iteration still reaches
    the rollout."""
    s, info, lengths, off, s0, od = _solve("ma4_rk4", jac="full", damp="scale", damp_param=k,
                                           tol=0.0, max_iters=2, init="s0")
    for b, n in enumerate(lengths):
        if n == 0:
            continue
        ref = onewton.initial_guess(od(b), s0[b:b + 1], n, "s0")
        for _ in range(2):
            ref = onewton.quasi_newton_step(od(b), s0[b:b + 1], ref, "full", damp="scale",
                                            damp_param=k)
        assert _relerr(s[off[b]:off[b + 1]], ref[0]) <= 1e-11, b
    s, info, lengths, off, s0, od = _solve("ma4_rk4", jac="full", damp="scale", damp_param=k,
                                           tol=1e-12, init="s0", max_iters=4000)
    assert bool(info.converged.all()), info.iters.max()
    for b, n in enumerate(lengths):
        if n == 0:
            continue
        roll = onewton.rollout(od(b), s0[b:b + 1], n)[0]
        assert _relerr(s[off[b]:off[b + 1]], roll) <= 1e-10, b
