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
