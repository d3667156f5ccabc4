"""Parity with the FP64 oracle at the full sizes of the benchmarked workloads, in the
launch configurations bench.py times. Every trajectory that the plain C oracle can roll
out in seconds is compared (normwise per sequence: max |s_gpu - s_ref| / max |s_ref|);
the adjoint gradient is compared with the oracle's reverse recursion (Eq. bptt) and with
central finite differences of the oracle's loss."""
import numpy as np
import pytest
import torch

import synth
from oracle import cma
from oracle import dynamics as odyn
from oracle import newton as onewton

pytestmark = pytest.mark.gpu


def _t(a, dt=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


def _per_seq_err(got, ref, off):
    """normwise error of every sequence of a packed batch"""
    got = np.asarray(got, dtype=np.float64)
    out = np.empty(len(off) - 1)
    for b in range(len(off) - 1):
        seg = slice(int(off[b]), int(off[b + 1]))
        if off[b + 1] == off[b]:
            out[b] = 0.0
            continue
        out[b] = np.max(np.abs(got[seg] - ref[seg])) / max(np.max(np.abs(ref[seg])), 1e-300)
    return out


def test_massaction_d8_B4096_T16384_fp32_every_trajectory():
    """The headline workload as bench.py runs it (B=4096 networks, d=8, 12 reactions, RK4
    dt=1e-3, T=16384, full-Jacobian Newton in FP32 with the compensated state, guess s_0,
    scaled residual 5e-8 on two consecutive iterates, sliding window): all 4096 converged
    trajectories equal the FP64 rollout within 1e-5. (With a plain float32 state the
    float32 rounding of the near-equilibrium increments leaves 37 % of them above 1e-5, as
    it does the float32 sequential rollout; with the compensated state but a scaled
    residual of 5e-7, the residual left in each of 16384 rows adds up to 1e-4 along the
    conserved directions on a few of them.)"""
    import paper_2603_16850_gb300 as deer
    B, d, R, T = 4096, 8, 12, 16384
    p = synth.massaction(B, d, R, T, seed=0)
    dyn = deer.Dynamics.massaction(_t(p["topology"], torch.int32),
                                   _t(p["params"], torch.float32), d, p["dt"])
    s, info = deer.deer_solve(dyn, _t(p["s0"], torch.float32), T, jac="full", tol=5e-8,
                              confirm=2, prec="fp32", init="s0", reset=True, window=True)
    assert bool(info.converged.all())
    off = cma.uniform_offsets(B, T)
    ref = cma.Batch(p["topology"], p["params"], p["dt"], "rk4", d=d).rollout(p["s0"], off)
    err = _per_seq_err(s.cpu().numpy(), ref, off)
    worst = np.argsort(-info.iters.numpy())[:8]
    assert np.all(err[worst] <= 1e-5), (err[worst], info.iters.numpy()[worst])
    assert err.max() <= 1e-5, (err.max(), int(err.argmax()), int(info.iters[int(err.argmax())]))


def test_massaction_d8_B4096_T16384_fp64_every_trajectory():
    """The same workload in FP64 mode (scaled residual 1e-12 on two consecutive iterates):
    all 4096 trajectories equal the FP64 rollout within 1e-10."""
    import paper_2603_16850_gb300 as deer
    B, d, R, T = 4096, 8, 12, 16384
    p = synth.massaction(B, d, R, T, seed=0)
    dyn = deer.Dynamics.massaction(_t(p["topology"], torch.int32), _t(p["params"]), d,
                                   p["dt"])
    s, info = deer.deer_solve(dyn, _t(p["s0"]), T, jac="full", tol=1e-12, confirm=2,
                              prec="fp64", init="zeros", reset=True, window=True)
    assert bool(info.converged.all())
    off = cma.uniform_offsets(B, T)
    ref = cma.Batch(p["topology"], p["params"], p["dt"], "rk4", d=d).rollout(p["s0"], off)
    err = _per_seq_err(s.cpu().numpy(), ref, off)
    assert err.max() <= 1e-10, (err.max(), int(err.argmax()))


def test_gru_d64_B64_T65536_quasi_deer_every_trajectory():
    """C3 as bench.py runs it (GRU d=64, inputs 64, T=65536, B=64, weights N(0,1/d), inputs
    N(0,1), quasi-DEER on the tensor-core linearisation, FP32, tol 1e-5 twice, zero guess):
    all 64 trajectories equal the FP64 oracle rollout within 1e-5."""
    import paper_2603_16850_gb300 as deer
    B, T, d = 64, 65536, 64
    g = synth.gru(B, T, d, d, seed=0, dtype=np.float32)
    dyn = deer.Dynamics.gru(_t(g["W"], torch.float32), _t(g["U"], torch.float32))
    x = torch.tensor(g["x"].reshape(-1, d), device="cuda")
    s, info = deer.deer_solve(dyn, _t(g["s0"], torch.float32), T, x, jac="diag", tol=1e-5,
                              confirm=2, prec="fp32", init="zeros")
    assert bool(info.converged.all())
    ref = onewton.rollout(odyn.GRU(g["W"], g["U"], g["x"].astype(np.float64)), g["s0"], T)
    off = cma.uniform_offsets(B, T)
    err = _per_seq_err(s.cpu().numpy(), ref.reshape(-1, d), off)
    assert err.max() <= 1e-5, (err.max(), int(err.argmax()))


def test_adjoint_d32_B256_T32768_against_oracle_and_fd():
    """C4 as bench.py runs it: d=32 networks (48 reactions), B=256, T=32768, RK4 dt=1e-3,
    FP32 solve (compensated state, scaled residual 5e-8 twice), loss sum_t ||s_t - y_t||^2 with y the rollout at rate constants
    k exp(0.1 eps); the adjoint gradient w.r.t. the rate constants of 8 trajectories
    (including the one with the most Newton iterations) equals the FP64 oracle's reverse
    recursion within 1e-3 normwise, and 8 of its entries equal central differences
    (h = 1e-6) of the FP64 oracle loss. The converged trajectories of those 8 equal the
    FP64 rollout within 1e-5."""
    import paper_2603_16850_gb300 as deer
    B, d, R, T = 256, 32, 48, 32768
    p = synth.massaction(B, d, R, T, seed=3)
    kp = synth.perturbed_rates(p["params"], seed=4)
    off = cma.uniform_offsets(B, T)
    y = cma.Batch(p["topology"], kp, p["dt"], "rk4", d=d).rollout(p["s0"], off)
    dyn = deer.Dynamics.massaction(_t(p["topology"], torch.int32),
                                   _t(p["params"], torch.float32), d, p["dt"])
    s0 = _t(p["s0"], torch.float32)
    s, info = deer.deer_solve(dyn, s0, T, jac="full", tol=5e-8, confirm=2, prec="fp32",
                              init="zeros", reset=True)
    assert bool(info.converged.all())
    g = 2.0 * (s - _t(y, torch.float32))
    dk, _ = deer.deer_grad(dyn, s0, T, s, g.contiguous(), prec="fp32")
    dk = dk.double().cpu().numpy()
    rng = np.random.default_rng(7)
    pick = np.unique(np.concatenate([[int(info.iters.argmax())],
                                     rng.choice(B, size=7, replace=False)]))
    sub_off = cma.uniform_offsets(len(pick), T)
    sub = cma.Batch(p["topology"][pick], p["params"][pick], p["dt"], "rk4", d=d)
    sref = sub.rollout(p["s0"][pick], sub_off)
    yp = y.reshape(B, T, d)[pick].reshape(-1, d)
    sv = s.view(B, T, d)[torch.as_tensor(pick, device="cuda")].reshape(-1, d).cpu().numpy()
    assert _per_seq_err(sv, sref, sub_off).max() <= 1e-5
    dk_ref, _ = sub.adjoint(p["s0"][pick], sref, 2.0 * (sref - yp), sub_off)
    for i, b in enumerate(pick):
        e = np.max(np.abs(dk[b] - dk_ref[i])) / np.max(np.abs(dk_ref[i]))
        assert e <= 1e-3, (b, e)
    # central differences of the oracle loss for 4 rate constants of 2 trajectories
    h = 1e-6
    for i in range(2):
        b = int(pick[i])
        one = cma.uniform_offsets(1, T)
        yb = y.reshape(B, T, d)[b]
        for j in rng.choice(R, size=4, replace=False):
            ks = []
            for sgn in (1.0, -1.0):
                kk = p["params"][b:b + 1].copy()
                kk[0, j] += sgn * h
                sb = cma.Batch(p["topology"][b:b + 1], kk, p["dt"], "rk4", d=d).rollout(
                    p["s0"][b:b + 1], one)
                ks.append(np.sum((sb - yb) ** 2))
            fd = (ks[0] - ks[1]) / (2 * h)
            assert abs(dk[b, j] - fd) <= 1e-3 * np.max(np.abs(dk_ref[i])), (b, j, dk[b, j], fd)


def test_ragged_mixed_d16_group_of_1000_every_trajectory():
    """C5's group as bench.py runs it (1000 ragged d=16 networks, 24 reactions, lengths
    uniform on [1000, 100000], RK4 dt=1e-3, bf16 Jacobians with float32 scan accumulation,
    float64 state and residual, scaled residual 1e-12, sliding window, chunk length 256):
    every trajectory, the longest included, equals the float64 rollout within 1e-9. (At a
    scaled residual of 1e-10 the residual left at convergence adds up along the conserved
    directions to 1e-7 over 1e5 steps.)"""
    import paper_2603_16850_gb300 as deer
    B, d, R = 1000, 16, 24
    lengths = synth.ragged_lengths(B, 1000, 100000, seed=5)
    off = synth.offsets_from_lengths(lengths)
    p = synth.massaction(B, d, R, 1, seed=6)
    dyn = deer.Dynamics.massaction(_t(p["topology"], torch.int32), _t(p["params"]), d,
                                   p["dt"])
    s, info = deer.deer_solve_batched(dyn, _t(p["s0"]), off, jac="full", tol=1e-12,
                                      prec="mixed_bf16", init="zeros", reset=True, window=True,
                                      chunk=256)
    assert bool(info.converged.all())
    ref = cma.Batch(p["topology"], p["params"], p["dt"], "rk4", d=d).rollout(p["s0"], off)
    err = _per_seq_err(s.cpu().numpy(), ref, off)
    longest = int(np.argmax(lengths))
    assert err[longest] <= 1e-9, (err[longest], lengths[longest])
    assert err.max() <= 1e-9, (err.max(), int(err.argmax()), lengths[int(err.argmax())])
