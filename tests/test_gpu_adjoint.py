"""Adjoint gradient (deer_grad) against the FP64 oracle: the reverse recursion of BPTT,
forward sensitivities and central finite differences (h = 1e-6)."""
import numpy as np
import pytest
import torch

import synth
from oracle import adjoint as oadj
from oracle import dynamics as odyn
from oracle import newton as onewton

pytestmark = pytest.mark.gpu


def _t(a, dt=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


def _setup(B, d, R, T, seed, dt=1e-2):
    p = synth.massaction(B, d, R, T, seed, dt=dt)
    od = odyn.MassAction(p["topology"], p["params"], dt, "rk4", d=d)
    s = onewton.rollout(od, p["s0"], T)
    kp = synth.perturbed_rates(p["params"], seed=seed + 100)
    y = onewton.rollout(odyn.MassAction(p["topology"], kp, dt, "rk4", d=d), p["s0"], T)
    return p, od, s, y


def _relerr(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


@pytest.mark.parametrize("d,R,T", [(4, 6, 300), (8, 12, 200)])
def test_adjoint_fp64_matches_oracle(d, R, T):
    import paper_2603_16850_gb300 as deer
    B = 3
    p, od, s, y = _setup(B, d, R, T, seed=d)
    g = oadj.sq_loss_cotangent(s, y)
    dth, ds0, _ = oadj.adjoint_grad(od, p["s0"], s, g)
    dyn = deer.Dynamics.massaction(_t(p["topology"], torch.int32), _t(p["params"]), d, p["dt"])
    gp, gs0 = deer.deer_grad(dyn, _t(p["s0"]), T, _t(s.reshape(-1, d)), _t(g.reshape(-1, d)))
    assert _relerr(gp.cpu().numpy(), dth) <= 1e-10
    assert _relerr(gs0.cpu().numpy(), ds0) <= 1e-10
    # independent routes: forward sensitivities and central differences
    fth, _ = oadj.forward_sensitivity_grad(od, p["s0"], s, g)
    assert _relerr(gp.cpu().numpy(), fth) <= 1e-10
    mk = lambda k: odyn.MassAction(p["topology"], k, p["dt"], "rk4", d=d)
    idx = [(0, 0), (1, R - 1), (2, R // 2)]
    fd = oadj.fd_grad(mk, p["params"], p["s0"], T, y, idx, h=1e-6)
    got = np.array([gp.cpu().numpy()[b, j] for b, j in idx])
    assert np.allclose(got, fd, rtol=1e-5, atol=1e-9)


def test_adjoint_fp32_d32_against_fp64():
    """d = 32 network (48 reactions), FP32 adjoint vs the FP64 oracle gradient: <= 1e-3
    normwise (float32 accumulation over T rows)."""
    import paper_2603_16850_gb300 as deer
    B, d, R, T = 2, 32, 48, 256
    p, od, s, y = _setup(B, d, R, T, seed=5, dt=1e-3)
    g = oadj.sq_loss_cotangent(s, y)
    dth, ds0, _ = oadj.adjoint_grad(od, p["s0"], s, g)
    dyn = deer.Dynamics.massaction(_t(p["topology"], torch.int32),
                                   _t(p["params"], torch.float32), d, p["dt"])
    gp, gs0 = deer.deer_grad(dyn, _t(p["s0"], torch.float32), T,
                             _t(s.reshape(-1, d), torch.float32),
                             _t(g.reshape(-1, d), torch.float32), prec="fp32")
    for b in range(B):
        assert _relerr(gp.cpu().numpy()[b], dth[b]) <= 1e-3
    assert _relerr(gs0.cpu().numpy(), ds0) <= 1e-3


def test_autograd_function_end_to_end():
    """DeerFunction: forward solve, backward adjoint; gradients of the loss w.r.t. the
    rate constants equal the oracle's."""
    import paper_2603_16850_gb300 as deer
    B, d, R, T = 2, 4, 6, 150
    p, od, s, y = _setup(B, d, R, T, seed=11)
    topo = _t(p["topology"], torch.int32)
    k = _t(p["params"]).requires_grad_(True)
    dyn = deer.Dynamics.massaction(topo, k.detach(), d, p["dt"])
    sol = deer.DeerFunction.apply(k, _t(p["s0"]), dyn, T, None,
                                  dict(jac="full", tol=1e-12, init="s0"))
    loss = ((sol - _t(y.reshape(-1, d))) ** 2).sum()
    loss.backward()
    dth, _, _ = oadj.adjoint_grad(od, p["s0"], s, oadj.sq_loss_cotangent(s, y))
    assert _relerr(k.grad.cpu().numpy(), dth) <= 1e-9


def _input_case(kind, B, T, d, seed):
    import paper_2603_16850_gb300 as deer
    if kind == "gru":
        p = synth.gru(B, T, d, d, seed)
        s0 = np.random.default_rng(seed).standard_normal((B, d)) * 0.5
        return (odyn.GRU(p["W"], p["U"], p["x"]), deer.Dynamics.gru(_t(p["W"]), _t(p["U"])),
                p["x"], s0)
    if kind == "rnn":
        p = synth.mean_field_rnn(B, T, d, 0.9, seed)
        return odyn.MeanFieldRNN(p["W"], p["x"]), deer.Dynamics.rnn_tanh(_t(p["W"])), p["x"], p["s0"]
    if kind == "langevin":
        p = synth.two_well(B, T, d, seed)
        return (odyn.TwoWellLangevin(p["params"], p["dt"], p["x"], d=d),
                deer.Dynamics.langevin_2well(_t(p["params"]), p["dt"]), p["x"], p["s0"])
    p = synth.linear_lds(B, T, d, seed)
    return odyn.Linear(p["A"], p["x"]), deer.Dynamics.linear(_t(p["A"])), p["x"], p["s0"]


@pytest.mark.parametrize("kind,d", [("gru", 8), ("rnn", 16), ("rnn", 32), ("langevin", 4),
                                    ("linear", 4)])
def test_input_gradient_matches_oracle(kind, d):
    """dl/dx_t = lambda_t^T df_t/dx_t (deer_grad_ex) against the oracle's adjoint states and
    input derivatives, FP64, on a 300-step trajectory (several scan chunks, ragged tail)."""
    import paper_2603_16850_gb300 as deer
    B, T = 2, 300
    od, dyn, x, s0 = _input_case(kind, B, T, d, seed=6)
    s = onewton.rollout(od, s0, T)
    y = s + 0.2 * synth.targets_noise(s.shape, seed=7)
    g = oadj.sq_loss_cotangent(s, y)
    _, ds0_ref, lam = oadj.adjoint_grad(od, s0, s, g)
    dx_ref = oadj.input_grad(od, s0, s, lam)
    _, ds0, dx = deer.deer_grad(dyn, _t(s0), T, _t(s.reshape(-1, d)), _t(g.reshape(-1, d)),
                                x=_t(x.reshape(-1, x.shape[-1])), want_dx=True)
    assert _relerr(dx.cpu().numpy().reshape(dx_ref.shape), dx_ref) <= 1e-10
    assert _relerr(ds0.cpu().numpy(), ds0_ref) <= 1e-10


def test_autograd_reaches_the_gru_inputs():
    """DeerFunction: the gradient of a loss of the solved GRU trajectory with respect to its
    input sequence equals deer_grad_ex's dl/dx at the same fixed point."""
    import paper_2603_16850_gb300 as deer
    B, T, d = 2, 200, 8
    p = synth.gru(B, T, d, d, seed=9)
    dyn = deer.Dynamics.gru(_t(p["W"]), _t(p["U"]))
    x = _t(p["x"].reshape(-1, d)).requires_grad_(True)
    s0 = torch.zeros((B, d), dtype=torch.float64, device="cuda")
    s = deer.DeerFunction.apply(dyn.params, s0, dyn, T, x,
                                dict(jac="full", tol=1e-12, init="zeros"))
    loss = (s ** 2).sum()
    loss.backward()
    _, _, dx = deer.deer_grad(dyn, s0, T, s.detach(), (2 * s).detach(), x=x.detach(),
                              want_dx=True)
    assert torch.allclose(x.grad, dx, rtol=0, atol=0)


@pytest.mark.parametrize("d,R,T,prec", [(8, 12, 1000, "fp64"), (32, 48, 700, "fp32"),
                                        (16, 24, 513, "fp64")])
def test_memory_bounded_adjoint_equals_stored(d, R, T, prec):
    """With a Jacobian memory bound the reverse recursion runs over time windows from the
    end (each window's Jacobians formed when it is reached): the gradient w.r.t. the rate
    constants and s0 equals the all-stored one and the FP64 oracle's (C reverse
    recursion), for windows that do not divide T (a ragged earliest window), and the
    workspace shrinks."""
    import paper_2603_16850_gb300 as deer
    from oracle import cma
    B = 3
    dt = torch.float64 if prec == "fp64" else torch.float32
    p = synth.massaction(B, d, R, T, seed=d + 1, dt=1e-2)
    off = cma.uniform_offsets(B, T)
    cb = cma.Batch(p["topology"], p["params"], p["dt"], "rk4", d=d)
    s = cb.rollout(p["s0"], off)
    kp = synth.perturbed_rates(p["params"], seed=d + 101)
    y = cma.Batch(p["topology"], kp, p["dt"], "rk4", d=d).rollout(p["s0"], off)
    g = 2.0 * (s - y)
    dk_ref, ds0_ref = cb.adjoint(p["s0"], s, g, off)
    dyn = deer.Dynamics.massaction(_t(p["topology"], torch.int32), _t(p["params"], dt), d,
                                   p["dt"])
    args = (dyn, _t(p["s0"], dt), T, _t(s, dt), _t(g, dt))
    full_k, full_s0 = deer.deer_grad(*args, prec=prec)
    W = 77
    rs = 8 if prec == "fp64" else 4
    budget = W * B * d * d * rs
    win_k, win_s0 = deer.deer_grad(*args, prec=prec, jac_bytes_max=budget)
    tol = 1e-12 if prec == "fp64" else 1e-5
    assert _relerr(win_k.double().cpu().numpy(), full_k.double().cpu().numpy()) <= tol
    assert _relerr(win_s0.double().cpu().numpy(), full_s0.double().cpu().numpy()) <= tol
    otol = 1e-10 if prec == "fp64" else 1e-4
    assert _relerr(win_k.double().cpu().numpy(), dk_ref) <= otol
    assert _relerr(win_s0.double().cpu().numpy(), ds0_ref) <= otol
    from paper_2603_16850_gb300 import _native as N
    import ctypes as C
    lib = N.load()
    o_full = deer._options(**deer._opt_defaults(dict(prec=prec)))
    o_win = deer._options(**deer._opt_defaults(dict(prec=prec, jac_bytes_max=budget)))
    cd = dyn.c_struct()
    assert lib.deer_grad_workspace_bytes(C.byref(cd), B, T, C.byref(o_win)) < \
        lib.deer_grad_workspace_bytes(C.byref(cd), B, T, C.byref(o_full))


def test_memory_bounded_adjoint_input_gradient():
    """The windowed adjoint also gives the gradient w.r.t. the inputs curried into f_t
    (GRU, d = 8): equal to the all-stored one and to the oracle's lambda_t^T df_t/dx_t."""
    import paper_2603_16850_gb300 as deer
    B, T, d = 2, 600, 8
    gp = synth.gru(B, T, d, d, seed=3)
    og = odyn.GRU(gp["W"], gp["U"], gp["x"])
    s = onewton.rollout(og, gp["s0"], T)
    y = np.sin(np.arange(B * T * d)).reshape(B, T, d) * 0.1
    g = 2.0 * (s - y)
    _, ds0_ref, lam = oadj.adjoint_grad(og, gp["s0"], s, g)
    dx_ref = oadj.input_grad(og, gp["s0"], s, lam)
    dyn = deer.Dynamics.gru(_t(gp["W"]), _t(gp["U"]))
    x = _t(gp["x"].reshape(-1, d))
    args = (dyn, _t(gp["s0"]), T, _t(s.reshape(-1, d)), _t(g.reshape(-1, d)), x)
    _, ds0_f, dx_f = deer.deer_grad(*args, want_dx=True)
    _, ds0_w, dx_w = deer.deer_grad(*args, want_dx=True, jac_bytes_max=61 * B * d * d * 8)
    assert _relerr(dx_w.cpu().numpy(), dx_f.cpu().numpy()) <= 1e-12
    assert _relerr(ds0_w.cpu().numpy(), ds0_f.cpu().numpy()) <= 1e-12
    assert _relerr(dx_w.cpu().numpy().reshape(B, T, d), dx_ref) <= 1e-10
    assert _relerr(ds0_w.cpu().numpy(), ds0_ref) <= 1e-10
