"""The initial guesses of Sec. 3.3.3 on the GPU (one Jacobi step from zero, iid normal
draws) and the per-iteration history record, compared with the FP64 oracle through the
C ABI binding."""
import numpy as np
import pytest
import torch

import synth
from oracle import dynamics as odyn
from oracle import newton as onewton

pytestmark = pytest.mark.gpu


def _t(a, dt=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


def _relerr(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return np.max(np.abs(got - ref)) / max(np.max(np.abs(ref)), 1e-300)


@pytest.mark.parametrize("init,seed", [("jacobi", 0), ("randn", 11), ("randn", 2 ** 63 + 5)])
@pytest.mark.parametrize("case", ["massaction_full", "gru_diag"])
def test_initial_guess_iterates_match_oracle(init, seed, case):
    """With a cap of k iterations the GPU iterate equals k oracle steps taken from the
    oracle's own initial guess (one Jacobi step f_t(0), or the counter-based N(0, 1)
    draws), for a ragged-tailed length spanning several chunks; run to convergence, the
    fixed point is the sequential rollout whatever the guess."""
    import paper_2603_16850_gb300 as deer
    B, T = 3, 333
    if case == "massaction_full":
        p = synth.massaction(B, 8, 12, T, seed=21)
        od = odyn.MassAction(p["topology"], p["params"], p["dt"], "rk4", d=8)
        dyn = deer.Dynamics.massaction(_t(p["topology"], torch.int32), _t(p["params"]), 8,
                                       p["dt"])
        s0, x, jac, d = p["s0"], None, "full", 8
    else:
        g = synth.gru(B, T, 8, 8, seed=5)
        od = odyn.GRU(g["W"], g["U"], g["x"])
        dyn = deer.Dynamics.gru(_t(g["W"]), _t(g["U"]))
        s0, x, jac, d = g["s0"], _t(g["x"].reshape(-1, 8)), "diag", 8
    for k in (1, 2):
        s, info = deer.deer_solve(dyn, _t(s0), T, x, jac=jac, tol=0.0, max_iters=k, init=init,
                                  seed=seed, prec="fp64")
        assert info.status == 1 and info.iters.tolist() == [k] * B
        ref = onewton.initial_guess(od, s0, T, init, seed=seed)
        for _ in range(k):
            ref = onewton.quasi_newton_step(od, s0, ref, jac)
        assert _relerr(s.cpu().numpy(), ref.reshape(-1, d)) <= 1e-11
    s, info = deer.deer_solve(dyn, _t(s0), T, x, jac=jac, tol=1e-12, init=init, seed=seed,
                              prec="fp64", reset=True)
    assert bool(info.converged.all())
    roll = onewton.rollout(od, s0, T).reshape(-1, d)
    assert _relerr(s.cpu().numpy(), roll) <= 1e-10


def test_randn_guess_is_the_documented_draw():
    """One iteration from the random guess on a recurrence with A~ = 0 (Jacobi mode) keeps
    nothing of the guess; with the identity (Picard) mode the first iterate's first row is
    f_1(s_0) and the rest shift by the guess, so the guess itself can be read back:
    s^(1)_t - s^(1)_{t-1} = f_t(s^(0)_{t-1}) - s^(0)_{t-1} for the affine recurrence with
    A = 0 and x = 0 gives -s^(0)_{t-1}. Compared with the oracle's generator entry by
    entry (float32 and float64 buffers)."""
    import paper_2603_16850_gb300 as deer
    from oracle import rng
    B, T, d = 2, 700, 4
    # the read-back differences of a running sum of ~|s| <= 60 carry its rounding
    for prec, dt, tol in (("fp64", torch.float64, 1e-13), ("fp32", torch.float32, 1e-6)):
        A = torch.zeros((d, d), dtype=dt, device="cuda")
        dyn = deer.Dynamics.linear(A)
        s0 = torch.zeros((B, d), dtype=dt, device="cuda")
        s, info = deer.deer_solve(dyn, s0, T, jac="identity", tol=0.0, max_iters=1,
                                  init="randn", seed=99, prec=prec)
        g = rng.randn_guess(99, B * T, d).reshape(B, T, d)
        sv = s.double().cpu().numpy().reshape(B, T, d)
        # Picard step: s^(1)_t = f_t(s^(0)_{t-1}) + (s^(1)_{t-1} - s^(0)_{t-1}), f = 0
        steps = sv[:, 1:] - sv[:, :-1]
        # the scan's prefix sums of |s| <= 60 round to a few ulps of that magnitude
        ulp = float(np.spacing(np.array(np.max(np.abs(sv)), dtype=np.float32 if prec == "fp32"
                                        else np.float64)))
        assert np.max(np.abs(steps + g[:, :-1])) <= max(tol, 16 * ulp)
        assert np.max(np.abs(sv[:, 0])) == 0.0


def test_history_records_each_convergence_test():
    """The history buffer holds, per convergence test, the iteration index, the merit
    1/2 ||r||^2 and the largest scaled residual of the sequences tested, and the number of
    sequences still active; for one Brusselator trajectory in FP64 these equal the oracle's
    record of Algorithm alg:deer, and rows after the last test stay untouched."""
    import paper_2603_16850_gb300 as deer
    T = 300
    p = synth.brusselator(T=T)
    od = odyn.Brusselator(p["params"], p["dt"])
    dyn = deer.Dynamics.brusselator(_t(p["params"]), p["dt"])
    hist = torch.full((64, 4), -7.0, dtype=torch.float64, device="cuda")
    s, info = deer.deer_solve(dyn, _t(p["s0"]), T, jac="full", tol=1e-12, init="s0",
                              prec="fp64", reset=True, history=hist)
    ref = onewton.solve(od, p["s0"], T, "full", tol=1e-12, init="s0", reset=True,
                        record=True)
    n = len(ref["history"])
    assert int(info.iters[0]) == int(ref["iters"][0]) == n - 1
    h = hist.cpu().numpy()
    assert np.array_equal(h[:n, 0], np.arange(n))
    for i, (mr, mer) in enumerate(ref["history"]):
        assert abs(h[i, 2] - mr[0]) <= 1e-9 * max(mr[0], 1e-300) + 1e-14
        # at convergence the residual is at rounding level (merit ~1e-16) and its last bits
        # differ between the two orders of evaluation
        assert abs(h[i, 1] - mer[0]) <= 1e-9 * max(mer[0], 1e-300) + 1e-20
    assert np.array_equal(h[:n, 3], [1.0] * (n - 1) + [0.0])
    assert np.all(h[n:] == -7.0)
