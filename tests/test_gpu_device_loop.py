"""The device-resident Newton loop (deer_options.device_loop): the iterations after the
first run as one CUDA graph (a gate node and a conditional while node whose body is one
iteration), every kernel reading the active-set sizes from device memory with grids sized
for the whole problem. On every path family it must return what the host-driven loop
returns: the same trajectory bit for bit, the same per-sequence iteration counts,
largest residuals, convergence flags and status, and the same per-iteration history up to
the merit sums, which the float32 kernels form per thread block (the device loop's grids
differ, so the partial sums round differently: relative 1e-5 is allowed).
"""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

DEV = "cuda"


def _deer():
    import paper_2603_16850_gb300 as deer
    return deer


def _t(a, dt=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dt, device=DEV)


def _ma_dyn(p, dtype):
    deer = _deer()
    return deer.Dynamics.massaction(_t(p["topology"], torch.int32), _t(p["params"], dtype),
                                    p["d"], p["dt"], p["kind"].split("_")[1])


def _case(name):
    """(solve(**extra) -> (s, info), expect_converged) for one path family."""
    deer = _deer()
    if name == "fused_fp32_window":
        # the batched kinetics path: lane-per-species fused kernel, compensated state,
        # sliding window
        p = synth.massaction(16, 8, 12, 3000, seed=11)
        dyn = _ma_dyn(p, torch.float32)
        s0 = _t(p["s0"], torch.float32)
        opts = dict(jac="full", tol=5e-8, confirm=2, prec="fp32", init="zeros", reset=True,
                    window=True)
        return (lambda **e: deer.deer_solve(dyn, s0, 3000, **opts, **e)), True
    if name == "brusselator_fp64":
        p = synth.brusselator(T=1024)
        dyn = deer.Dynamics.brusselator(_t(p["params"]), p["dt"])
        s0 = _t(p["s0"])
        # reset heuristic on: undamped Newton overflows on the way at this horizon; the
        # multi-kernel loop (a sequence this short otherwise runs whole in one block)
        return (lambda **e: deer.deer_solve(dyn, s0, 1024, jac="full", tol=1e-12,
                                            prec="fp64", reset=True, block_solve=False,
                                            **e)), True
    if name == "gru_diag_lookback_fp32":
        g = synth.gru(4, 4096, 64, 64, seed=2, dtype=np.float32)
        dyn = deer.Dynamics.gru(_t(g["W"], torch.float32), _t(g["U"], torch.float32))
        x = _t(g["x"].reshape(-1, 64), torch.float32)
        s0 = torch.zeros((4, 64), dtype=torch.float32, device=DEV)
        return (lambda **e: deer.deer_solve(dyn, s0, 4096, x, jac="diag", tol=1e-5, confirm=2,
                                            prec="fp32", init="zeros", **e)), True
    if name == "gru_diag_lookback_window_fp32":
        # the look-back scan with the sliding window (sequence-major tile order)
        g = synth.gru(3, 3000, 16, 16, seed=5, dtype=np.float32)
        dyn = deer.Dynamics.gru(_t(g["W"], torch.float32), _t(g["U"], torch.float32))
        x = _t(g["x"].reshape(-1, 16), torch.float32)
        s0 = torch.zeros((3, 16), dtype=torch.float32, device=DEV)
        return (lambda **e: deer.deer_solve(dyn, s0, 3000, x, jac="diag", tol=1e-5, confirm=2,
                                            prec="fp32", init="zeros", window=True, **e)), True
    if name == "gru_quasi_elk_fp64":
        g = synth.gru(3, 700, 8, 8, seed=4)
        dyn = deer.Dynamics.gru(_t(g["W"]), _t(g["U"]))
        x = _t(g["x"].reshape(-1, 8))
        s0 = _t(g["s0"])
        return (lambda **e: deer.deer_solve(dyn, s0, 700, x, jac="diag", damp="elk",
                                            damp_param=0.5, tol=1e-11, init="zeros",
                                            max_iters=4000, **e)), True
    if name in ("mixed_stored", "mixed_recompute"):
        lengths = [1500, 333, 4000, 1]
        off = synth.offsets_from_lengths(lengths)
        p = synth.massaction(len(lengths), 16, 24, 1, seed=12)
        dyn = _ma_dyn(p, torch.float64)
        s0 = _t(p["s0"])
        jb = 0 if name == "mixed_stored" else 1
        return (lambda **e: deer.deer_solve_batched(dyn, s0, off, jac="full", tol=1e-12,
                                                    prec="mixed_bf16", init="s0", reset=True,
                                                    max_iters=500, jac_bytes_max=jb,
                                                    **e)), True
    if name == "dense_elk_parallel_covariance":
        p = synth.massaction(2, 8, 12, 5000, seed=13, dt=0.01)
        dyn = _ma_dyn(p, torch.float64)
        s0 = _t(p["s0"])
        # a fixed number of damped iterations: the cap is reached (status 1) on both loops
        return (lambda **e: deer.deer_solve(dyn, s0, 5000, jac="full", damp="elk",
                                            damp_param=1.0, tol=1e-14, init="s0",
                                            max_iters=6, chunk=128, **e)), False
    if name == "rnn_d32_wide":
        pr = synth.mean_field_rnn(2, 3000, 32, 0.5, seed=1)
        dyn = deer.Dynamics.rnn_tanh(_t(pr["W"], torch.float32))
        x = _t(pr["x"].reshape(-1, 32), torch.float32)
        s0 = _t(pr["s0"], torch.float32)
        return (lambda **e: deer.deer_solve(dyn, s0, 3000, x, jac="full", tol=5e-7,
                                            confirm=2, prec="fp32", init="zeros", reset=True,
                                            window=True, chunk=128, **e)), True
    if name == "ragged_fp64_d4":
        lengths = [900, 17, 2500, 64, 1200]
        off = synth.offsets_from_lengths(lengths)
        p = synth.massaction(len(lengths), 4, 6, 1, seed=14)
        dyn = _ma_dyn(p, torch.float64)
        s0 = _t(p["s0"])
        return (lambda **e: deer.deer_solve_batched(dyn, s0, off, jac="full", tol=1e-12,
                                                    init="zeros", reset=True, window=True,
                                                    **e)), True
    if name == "word_problem_one_iteration":
        pw = synth.word_problem(3, 800, seed=1)
        dyn = deer.Dynamics.permute(5, torch.float32, DEV)
        x = _t(pw["x"].reshape(-1, 5), torch.float32)
        s0 = _t(pw["s0"], torch.float32)
        return (lambda **e: deer.deer_solve(dyn, s0, 800, x, jac="full", tol=1e-6,
                                            prec="fp32", init="zeros", **e)), True
    raise KeyError(name)


CASES = ["fused_fp32_window", "brusselator_fp64", "gru_diag_lookback_fp32",
         "gru_diag_lookback_window_fp32",
         "gru_quasi_elk_fp64", "mixed_stored", "mixed_recompute",
         "dense_elk_parallel_covariance", "rnn_d32_wide", "ragged_fp64_d4",
         "word_problem_one_iteration"]


@pytest.mark.parametrize("name", CASES)
def test_device_loop_matches_host_loop(name):
    deer = _deer()
    solve, converges = _case(name)
    hist_h = torch.zeros((64, 4), dtype=torch.float64, device=DEV)
    hist_d = torch.zeros((64, 4), dtype=torch.float64, device=DEV)
    s_h, info_h = solve(device_loop=False, history=hist_h)
    torch.cuda.synchronize()
    n0 = deer.kernel_launch_count()
    s_d, info_d = solve(device_loop=True, history=hist_d)
    torch.cuda.synchronize()
    n_dev = deer.kernel_launch_count() - n0
    assert torch.equal(s_h, s_d), name
    assert info_h.iters.tolist() == info_d.iters.tolist(), (info_h.iters, info_d.iters)
    assert info_h.converged.tolist() == info_d.converged.tolist()
    assert bool(info_d.converged.all()) == converges, info_d
    assert info_h.status == info_d.status
    assert torch.equal(info_h.max_resid, info_d.max_resid)
    assert torch.allclose(info_h.merit, info_d.merit, rtol=1e-5, atol=0.0)
    # history rows: iteration and active count exactly, the merit sum up to its order
    hh, hd = hist_h.cpu().numpy(), hist_d.cpu().numpy()
    assert np.array_equal(hh[:, [0, 2, 3]], hd[:, [0, 2, 3]]), (hh[:4], hd[:4])
    assert np.allclose(hh[:, 1], hd[:, 1], rtol=1e-5, atol=0.0)
    assert n_dev >= 3  # iteration 0, the gate, and the counted graph bodies


@pytest.mark.parametrize("name", ["brusselator_fp64", "fused_fp32_window"])
def test_device_loop_launch_count(name):
    """On paths whose launches per iteration do not depend on the active set, the device
    loop runs the host loop's kernels plus the gate."""
    deer = _deer()
    solve, _ = _case(name)
    n0 = deer.kernel_launch_count()
    solve(device_loop=False)
    torch.cuda.synchronize()
    n1 = deer.kernel_launch_count()
    solve(device_loop=True)
    torch.cuda.synchronize()
    n2 = deer.kernel_launch_count()
    assert (n2 - n1) == (n1 - n0) + 1, (n1 - n0, n2 - n1)
