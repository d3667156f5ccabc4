"""deer_lle (largest Lyapunov exponent along a trajectory, Algorithm alg:LLE_estimate)
against the float64 oracle on the same trajectory and start vectors, for every dynamics
kind; the GPU stores the step Jacobians and walks each sequence with a group of d lanes."""
import numpy as np
import pytest
import torch

import synth
from oracle import dynamics as odyn
from oracle import lle as olle
from oracle import newton as onewton

pytestmark = pytest.mark.gpu


def _t(a, dt=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


def _unit(B, d, seed):
    u = np.random.default_rng(seed).standard_normal((B, d))
    return u / np.linalg.norm(u, axis=1, keepdims=True)


@pytest.mark.parametrize("case", ["bruss", "ma4", "ma8", "ma16", "ma32", "gru8", "linear4",
                                  "ma8_fp32"])
def test_lle_matches_oracle(case):
    import paper_2603_16850_gb300 as deer
    prec = "fp32" if case.endswith("fp32") else "fp64"
    tdt = torch.float32 if prec == "fp32" else torch.float64
    x = None
    if case == "bruss":
        p = synth.brusselator(T=700)
        od = odyn.Brusselator(p["params"], p["dt"])
        dyn = deer.Dynamics.brusselator(_t(p["params"], tdt), p["dt"])
        s0, B, T, d = p["s0"], 1, 700, 2
    elif case.startswith("ma"):
        d = int(case[2:].split("_")[0])
        B, T = 3, 500
        p = synth.massaction(B, d, {4: 6, 8: 12, 16: 24, 32: 48}[d], T, seed=40 + d)
        od = odyn.MassAction(p["topology"], p["params"], p["dt"], "rk4", d=d)
        dyn = deer.Dynamics.massaction(_t(p["topology"], torch.int32), _t(p["params"], tdt), d,
                                       p["dt"])
        s0 = p["s0"]
    elif case == "gru8":
        B, T, d = 2, 600, 8
        g = synth.gru(B, T, d, d, seed=41, weight_scale=1.2 / np.sqrt(8))
        od = odyn.GRU(g["W"], g["U"], g["x"])
        dyn = deer.Dynamics.gru(_t(g["W"], tdt), _t(g["U"], tdt))
        x = _t(g["x"].reshape(-1, d), tdt)
        s0 = g["s0"]
    else:
        B, T, d = 2, 400, 4
        rng = np.random.default_rng(42)
        A = rng.standard_normal((d, d)) * 0.6
        od = odyn.Linear(A)
        dyn = deer.Dynamics.linear(_t(A, tdt))
        s0 = rng.standard_normal((B, d))
    traj = onewton.rollout(od, s0, T)
    u0 = _unit(B, d, 7)
    want = olle.lle_estimate(od, s0, traj, u0)
    got = deer.deer_lle(dyn, _t(s0, tdt), T, _t(traj.reshape(-1, d), tdt), _t(u0, tdt), x,
                        prec=prec).cpu().numpy()
    tol = 1e-10 if prec == "fp64" else 2e-5
    assert np.all(np.abs(got - want) <= tol * np.maximum(1.0, np.abs(want))), (got, want)


def test_lle_rejects_unsupported_sizes():
    import paper_2603_16850_gb300 as deer
    from paper_2603_16850_gb300 import _native as N
    g = synth.gru(1, 4, 64, 64, seed=1)
    dyn = deer.Dynamics.gru(_t(g["W"]), _t(g["U"]))
    s0 = _t(g["s0"])
    with pytest.raises(N.DeerError):
        deer.deer_lle(dyn, s0, 4, _t(np.zeros((4, 64))), None, _t(g["x"].reshape(-1, 64)))
