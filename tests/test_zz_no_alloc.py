"""deer_solve_noalloc: the entry point for callers that cannot allocate device memory when
they solve (it runs inside a fixed per-device scratch array). Called through the C ABI and
compared with deer_solve on the same inputs, twice in a row, since every call reuses the
scratch left behind by the previous one. This file sorts last so that a run that stops at
the first failure has already run every other test."""
import ctypes as C

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


def _t(a, dt=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


def _call_noalloc(lib, N, dyn, B, T, s0, x, opts):
    import paper_2603_16850_gb300 as deer
    o = deer._options(**deer._opt_defaults(opts))
    out = torch.full((B * T, dyn.d), float("nan"), dtype=s0.dtype, device="cuda")
    infos = (N.deer_info * B)()
    st = lib.deer_solve_noalloc(C.byref(dyn.c_struct()), B, T, s0.data_ptr(),
                                0 if x is None else x.data_ptr(), out.data_ptr(), C.byref(o),
                                torch.cuda.current_stream().cuda_stream, infos)
    return st, out, [infos[i].iters for i in range(B)], [bool(infos[i].converged) for i in range(B)]


CASES = ["brusselator_fp64", "massaction_fp32", "gru_diag_lookback_fp32",
         "massaction_d2_diag_chunked_fp64", "gru_quasi_elk_fp32"]


def _case(case):
    """(dynamics, s0, x, T, B, tolerance against deer_solve, options) of one test case:
    full-Jacobian paths (Brusselator fp64, mass action fp32) and the diagonal family
    (the single-pass look-back scan, the three-pass chunked scan for d not a multiple of 4,
    and the Kalman-damped quasi-ELK scan)."""
    import paper_2603_16850_gb300 as deer
    if case == "brusselator_fp64":
        p = synth.brusselator(T=1024)
        dyn = deer.Dynamics.brusselator(_t(p["params"]), p["dt"])
        return dyn, _t(p["s0"]), None, 1024, 1, 1e-10, dict(
            jac="full", tol=1e-12, prec="fp64", init="s0", reset=True)
    if case == "massaction_fp32":
        p = synth.massaction(4, 8, 12, 700, seed=8)
        dyn = deer.Dynamics.massaction(_t(p["topology"], torch.int32),
                                       _t(p["params"], torch.float32), 8, p["dt"])
        # compared with deer_solve on the same plain float32 state (the fixed scratch keeps
        # no compensation terms)
        return dyn, _t(p["s0"], torch.float32), None, 700, 4, 1e-5, dict(
            jac="full", tol=5e-7, confirm=2, prec="fp32", init="s0", reset=True,
            compensate=False)
    if case == "massaction_d2_diag_chunked_fp64":
        p = synth.massaction(3, 2, 3, 900, seed=9)
        dyn = deer.Dynamics.massaction(_t(p["topology"], torch.int32), _t(p["params"]), 2,
                                       p["dt"])
        return dyn, _t(p["s0"]), None, 900, 3, 1e-10, dict(
            jac="diag", tol=1e-12, prec="fp64", init="s0")
    g = synth.gru(3, 2500, 8, 8, seed=2)
    dyn = deer.Dynamics.gru(_t(g["W"], torch.float32), _t(g["U"], torch.float32))
    x = _t(g["x"].reshape(-1, 8), torch.float32)
    s0 = torch.zeros((3, 8), dtype=torch.float32, device="cuda")
    opts = dict(jac="diag", tol=1e-6, confirm=2, prec="fp32", init="zeros")
    if case == "gru_quasi_elk_fp32":
        opts.update(damp="elk", damp_param=0.5)
    return dyn, s0, x, 2500, 3, 1e-5, opts


@pytest.mark.parametrize("case", CASES)
def test_noalloc_matches_deer_solve_twice(case):
    """Two calls in a row (the second reuses the scratch the first left behind) give
    deer_solve's trajectory and iteration counts."""
    import paper_2603_16850_gb300 as deer
    from paper_2603_16850_gb300 import _native as N
    lib = N.load()
    dyn, s0, x, T, B, tol_err, opts = _case(case)
    ref, rinfo = deer.deer_solve(dyn, s0, T, x, **opts)
    assert bool(rinfo.converged.all())
    scale = float(ref.abs().max())
    for _ in range(2):
        st, out, iters, conv = _call_noalloc(lib, N, dyn, B, T, s0, x, opts)
        torch.cuda.synchronize()
        assert st == N.DEER_OK
        assert all(conv)
        err = float((out - ref).abs().max()) / scale
        assert err <= tol_err, err
        assert iters == rinfo.iters.tolist()


def test_noalloc_rejects_problems_larger_than_its_scratch():
    import paper_2603_16850_gb300 as deer
    from paper_2603_16850_gb300 import _native as N
    lib = N.load()
    cap = lib.deer_noalloc_scratch_bytes()
    p = synth.massaction(64, 8, 12, 1, seed=1)
    dyn = deer.Dynamics.massaction(_t(p["topology"], torch.int32), _t(p["params"], torch.float32),
                                   8, p["dt"])
    s0 = _t(p["s0"], torch.float32)
    T = 1 << 14  # 64 x 16384 rows of 8x8 float32 Jacobians: far more than the scratch
    assert deer.deer_workspace_bytes(dyn, 64, 64 * T, prec="fp32") > cap
    o = deer._options(**deer._opt_defaults(dict(prec="fp32")))
    st = lib.deer_solve_noalloc(C.byref(dyn.c_struct()), 64, T, s0.data_ptr(), 0,
                                s0.data_ptr(), C.byref(o), 0, None)
    assert st == N.DEER_ERR_WORKSPACE
    assert b"scratch" in lib.deer_last_cuda_error()
