"""The thesis's second workloads on the CUDA path, against the float64 oracle: the
mean-field RNN of the predictability threshold (Sec. ssc:exp_thresh), Langevin dynamics
in a two-well potential (Sec. ssc:2well, sec:WellExp), Lorenz-96 stepped by the
Dormand-Prince method (Sec. elk_exps) and the group word problem as an input-selected
permutation (Sec. sec:GrpWordProb, Prop. cayley).

Parity: FP64 iterates equal the oracle's forward-substitution iterates to 1e-11
(normwise), converged trajectories equal the sequential rollout to 1e-10 (FP64) and 1e-5
(FP32); the word problem moves exact small integers and is compared bit for bit. Beyond
parity, the iteration counts reproduce the qualitative claims of those sections."""
import numpy as np
import pytest
import torch

import synth
from oracle import dynamics as odyn
from oracle import elk as oelk
from oracle import lle as olle
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


def _case(kind, B, T, d, seed, dt=torch.float64, g=0.5):
    """(problem, oracle dynamics, GPU dynamics, GPU inputs or None)."""
    deer = _deer()
    if kind == "rnn":
        p = synth.mean_field_rnn(B, T, d, g, seed)
        return (p, odyn.MeanFieldRNN(p["W"], p["x"]), deer.Dynamics.rnn_tanh(_t(p["W"], dt)),
                _t(p["x"].reshape(-1, d), dt))
    if kind == "langevin":
        p = synth.two_well(B, T, d, seed)
        return (p, odyn.TwoWellLangevin(p["params"], p["dt"], p["x"], d=d),
                deer.Dynamics.langevin_2well(_t(p["params"], dt), p["dt"]),
                _t(p["x"].reshape(-1, d), dt))
    if kind == "lorenz":
        p = synth.lorenz96(B, d, seed)
        return (p, odyn.Lorenz96(p["params"], p["dt"], d),
                deer.Dynamics.lorenz96(_t(p["params"], dt), d, p["dt"]), None)
    if kind == "permute":
        p = synth.word_problem(B, T, seed, d=d)
        return (p, odyn.Permute(p["x"]), deer.Dynamics.permute(d, dt, DEV),
                _t(p["x"].reshape(-1, d), dt))
    raise ValueError(kind)


ITER_CASES = [("rnn", 8, "full"), ("rnn", 32, "diag"), ("rnn", 16, "full"),
              ("langevin", 2, "full"), ("langevin", 4, "diag"), ("langevin", 2, "identity"),
              ("lorenz", 5, "full"), ("lorenz", 5, "diag"), ("lorenz", 8, "full"),
              ("lorenz", 4, "full"), ("permute", 5, "full"), ("permute", 5, "diag"),
              ("permute", 8, "zero")]


# Iterate tolerance per kind. The Langevin step evaluates exp/log (last-bit differences
# between the device and host math libraries) and its linearisation expands between the
# wells; Lorenz-96 is chaotic. Both amplify rounding along the sequence, so their iterates
# get a factor of ten over the association-order bound of the other kinds.
ITER_TOL = {"rnn": 1e-11, "permute": 1e-11, "langevin": 1e-10, "lorenz": 1e-10}


@pytest.mark.parametrize("kind,d,jac", ITER_CASES)
def test_iterates_match_oracle(kind, d, jac):
    """Two iterations from the same start equal two oracle forward-substitution steps
    (T = 300: several scan chunks and a ragged tail), then the solve reaches the
    sequential rollout."""
    deer = _deer()
    B, T = 3, (60 if kind == "lorenz" else 300)
    p, od, dyn, x = _case(kind, B, T, d, seed=7)
    s0 = _t(p["s0"])
    s2, info2 = deer.deer_solve(dyn, s0, T, x, jac=jac, tol=0.0, max_iters=2, init="s0")
    # the word problem is linear: one Newton iteration leaves a residual of exactly zero
    assert info2.status == (0 if (kind, jac) == ("permute", "full") else 1)
    ref = onewton.initial_guess(od, p["s0"], T, "s0")
    for _ in range(2):
        ref = onewton.quasi_newton_step(od, p["s0"], ref, jac)
    assert _relerr(s2.cpu().numpy(), ref.reshape(-1, d)) <= ITER_TOL[kind]
    s, info = deer.deer_solve(dyn, s0, T, x, jac=jac, tol=1e-12, init="s0", reset=True)
    assert bool(info.converged.all()), info.iters
    roll = onewton.rollout(od, p["s0"], T)
    for b in range(B):
        assert _relerr(s.cpu().numpy()[b * T:(b + 1) * T], roll[b]) <= 1e-10


@pytest.mark.parametrize("kind,d,T", [("rnn", 32, 2000), ("langevin", 2, 3000),
                                      ("langevin", 16, 1000), ("lorenz", 8, 80)])
def test_fp32_converges_to_the_fp64_rollout(kind, d, T):
    deer = _deer()
    B = 4
    p, od, dyn, x = _case(kind, B, T, d, seed=11, dt=torch.float32)
    s, info = deer.deer_solve(dyn, _t(p["s0"], torch.float32), T, x, jac="full", tol=5e-7,
                              confirm=2, prec="fp32", init="zeros", reset=True, window=True)
    assert bool(info.converged.all()), info.iters
    roll = onewton.rollout(od, p["s0"], T)
    for b in range(B):
        assert _relerr(s.cpu().numpy()[b * T:(b + 1) * T], roll[b]) <= 1e-5


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_word_problem_one_newton_iteration_bit_exact(prec):
    """Sec. sec:GrpWordProb: one Newton iteration solves the S5 word problem (the result
    equals the group product bit for bit: small integers are exact in both precisions),
    while quasi-DEER is still far from converged after 50 iterations."""
    deer = _deer()
    tdt = torch.float32 if prec == "fp32" else torch.float64
    B, T, d = 8, 4096, 5
    p, od, dyn, x = _case("permute", B, T, d, seed=3, dt=tdt)
    s, info = deer.deer_solve(dyn, _t(p["s0"], tdt), T, x, jac="full", tol=1e-12,
                              prec=prec, init="zeros")
    assert bool(info.converged.all()) and info.iters.tolist() == [1] * B
    roll = onewton.rollout(od, p["s0"], T)
    assert np.array_equal(s.cpu().numpy().astype(np.float64), roll.reshape(-1, d))
    _, iq = deer.deer_solve(dyn, _t(p["s0"], tdt), T, x, jac="diag", tol=1e-12, prec=prec,
                            init="zeros", max_iters=50)
    assert iq.status == 1 and not bool(iq.converged.any())


def test_mean_field_rnn_threshold_on_gpu():
    """Sec. ssc:exp_thresh on the GPU: below the threshold (g = 0.5, negative LLE) DEER
    converges in a handful of iterations, above it (g = 2, positive LLE) it needs an order
    of magnitude more; the counts agree with the oracle's and the LLE signs with its
    estimates."""
    deer = _deer()
    T, d = 200, 16
    res = {}
    for g in (0.5, 2.0):
        p, od, dyn, x = _case("rnn", 1, T, d, seed=1, g=g)
        s0 = _t(p["s0"])
        s, info = deer.deer_solve(dyn, s0, T, x, jac="full", tol=1e-10, init="zeros")
        o = onewton.solve(od, p["s0"], T, mode="full", tol=1e-10, init="zeros")
        assert bool(info.converged[0]) and o["converged"][0]
        gi, oi = int(info.iters[0]), int(o["iters"][0])
        assert abs(gi - oi) <= 1 + oi // 10
        lle = float(deer.deer_lle(dyn, s0, T, s, x=x)[0])
        roll = onewton.rollout(od, p["s0"], T)
        ref = float(olle.lle_estimate(od, p["s0"], roll, np.full((1, d), d ** -0.5))[0])
        assert abs(lle - ref) <= 1e-8
        res[g] = (gi, lle)
    assert res[0.5][1] < 0.0 < res[2.0][1]
    assert res[0.5][0] <= 5 and res[2.0][0] >= 10 * res[0.5][0]


def test_langevin_two_well_iterations_and_lle():
    """Sec. ssc:2well: from a random (iid standard normal) initial guess DEER converges in
    a few iterations although the dynamics expand between the wells; the LLE of the
    trajectory is negative; Jacobi needs all T iterations."""
    deer = _deer()
    B, T, d = 4, 1000, 2
    p, od, dyn, x = _case("langevin", B, T, d, seed=0)
    guess = synth.targets_noise((B * T, d), seed=5)
    s0 = _t(p["s0"])
    s, info = deer.deer_solve(dyn, s0, T, x, s_init=_t(guess), jac="full", tol=1e-10)
    assert bool(info.converged.all()) and int(info.iters.max()) <= 20
    o = onewton.solve(od, p["s0"], T, mode="full", tol=1e-10, init="user",
                      user=guess.reshape(B, T, d))
    assert np.all(np.abs(info.iters.numpy() - o["iters"]) <= 1)
    lle = deer.deer_lle(dyn, s0, T, s, x=x).cpu().numpy()
    ref = olle.lle_estimate(od, p["s0"], onewton.rollout(od, p["s0"], T),
                            np.full((B, d), d ** -0.5))
    assert np.abs(lle - ref).max() <= 1e-8 and np.all(lle < 0.0)
    _, ij = deer.deer_solve(dyn, s0, T, x, jac="zero", tol=1e-10, init="zeros")
    assert ij.iters.tolist() == [T] * B


@pytest.mark.parametrize("d,jac", [(8, "full"), (5, "diag")])
def test_lorenz96_elk_iterates_and_fixed_point(d, jac):
    """Lorenz-96 (chaotic, Sec. elk_exps) with the Kalman-filter step: dense ELK (d = 8)
    and quasi-ELK (d = 5); two iterations equal the oracle's filtered means and the
    damped iteration reaches the rollout."""
    deer = _deer()
    B, T, lam = 2, 100, 1.0
    p, od, dyn, x = _case("lorenz", B, T, d, seed=4)
    s0 = _t(p["s0"])
    s2, _ = deer.deer_solve(dyn, s0, T, x, jac=jac, damp="elk", damp_param=lam, tol=0.0,
                            max_iters=2, init="s0")
    ref = onewton.initial_guess(od, p["s0"], T, "s0")
    for _ in range(2):
        ref = oelk.elk_filter_step(od, p["s0"], ref, jac, lam)
    assert _relerr(s2.cpu().numpy(), ref.reshape(-1, d)) <= ITER_TOL["lorenz"]
    s, info = deer.deer_solve(dyn, s0, T, x, jac=jac, damp="elk", damp_param=lam, tol=1e-12,
                              init="s0", max_iters=5000)
    assert bool(info.converged.all()), info.iters
    roll = onewton.rollout(od, p["s0"], T)
    for b in range(B):
        assert _relerr(s.cpu().numpy()[b * T:(b + 1) * T], roll[b]) <= 1e-10


@pytest.mark.parametrize("kind,d", [("rnn", 32), ("langevin", 4), ("lorenz", 5),
                                    ("permute", 5)])
def test_lle_matches_oracle(kind, d):
    """deer_lle on the new kinds (d = 5 walks a padded group of eight lanes)."""
    deer = _deer()
    B, T = 3, 400
    p, od, dyn, x = _case(kind, B, T, d, seed=9)
    roll = onewton.rollout(od, p["s0"], T)
    u0 = np.random.default_rng(2).standard_normal((B, d))
    u0 /= np.linalg.norm(u0, axis=1, keepdims=True)
    got = deer.deer_lle(dyn, _t(p["s0"]), T, _t(roll.reshape(-1, d)), _t(u0), x=x)
    ref = olle.lle_estimate(od, p["s0"], roll, u0)
    assert np.abs(got.cpu().numpy() - ref).max() <= 1e-9


def test_rnn_adjoint_ds0_matches_bptt():
    """dl/ds0 through deer_grad for a kind without trainable parameters, against the
    oracle's reverse recursion (BPTT) on the same trajectory."""
    from oracle import adjoint as oadj
    deer = _deer()
    B, T, d = 2, 300, 8
    p, od, dyn, x = _case("rnn", B, T, d, seed=5)
    roll = onewton.rollout(od, p["s0"], T)
    y = roll + 0.1 * synth.targets_noise(roll.shape, seed=6)
    g = oadj.sq_loss_cotangent(roll, y)
    _, ds0 = deer.deer_grad(dyn, _t(p["s0"]), T, _t(roll.reshape(-1, d)),
                            _t(g.reshape(-1, d)), x=x)
    _, ref, _ = oadj.adjoint_grad(od, p["s0"], roll, g)
    assert _relerr(ds0.cpu().numpy(), ref) <= 1e-10


def test_bad_permutation_index_is_reported():
    """An index outside [0, d) yields NaN for that entry (the kernel never reads outside
    the state), which the solver reports as a non-finite residual."""
    deer = _deer()
    B, T, d = 1, 64, 5
    p, od, dyn, _ = _case("permute", B, T, d, seed=0)
    xb = p["x"].copy()
    xb[0, 10, 2] = 7.0
    with pytest.raises(RuntimeError, match="non-finite"):
        deer.deer_solve(dyn, _t(p["s0"]), T, _t(xb.reshape(-1, d)), jac="full", tol=1e-12,
                        init="zeros")


@pytest.mark.parametrize("kind,d", [("rnn", 32), ("rnn", 8), ("langevin", 2), ("lorenz", 5),
                                    ("permute", 5)])
def test_sequential_rollout_matches_oracle(kind, d):
    """The GPU sequential baseline (warp per trajectory for the RNN, a thread per
    trajectory otherwise) on a ragged batch whose groups share warps."""
    deer = _deer()
    lengths = [300, 1, 77, 250, 5]
    off = synth.offsets_from_lengths(lengths)
    B, T = len(lengths), max(lengths)
    p, od, dyn, _ = _case(kind, B, T, d, seed=13)
    x = None
    if "x" in p:
        x = _t(np.concatenate([p["x"][b, :n] for b, n in enumerate(lengths)]).reshape(-1, d))
    s = deer.deer_rollout(dyn, _t(p["s0"]), 0, x, offsets=_t(off, torch.int64))
    roll = onewton.rollout(od, p["s0"], T)
    sn = s.cpu().numpy()
    for b, n in enumerate(lengths):
        assert _relerr(sn[off[b]:off[b + 1]], roll[b, :n]) <= 1e-12


def test_full_size_single_trajectory_rnn_fp32():
    """The single-trajectory workload timed by the benchmark (mean-field RNN d = 32,
    T = 100000, g = 0.5, FP32, sliding window, chunk length 256) against the float64
    oracle rollout over the whole trajectory."""
    deer = _deer()
    T, d = 100000, 32
    p = synth.mean_field_rnn(1, T, d, 0.5, seed=0)
    dyn = deer.Dynamics.rnn_tanh(_t(p["W"], torch.float32))
    x = _t(p["x"].reshape(-1, d), torch.float32)
    s, info = deer.deer_solve(dyn, _t(p["s0"], torch.float32), T, x, jac="full", tol=1e-5,
                              prec="fp32", init="zeros", reset=True, window=True,
                              max_iters=300, chunk=256)
    assert bool(info.converged[0]) and int(info.iters[0]) <= 5
    roll = onewton.rollout(odyn.MeanFieldRNN(p["W"], p["x"]), p["s0"], T)[0]
    assert _relerr(s.cpu().numpy(), roll) <= 1e-5
