"""Mixed precision without stored Jacobians (d = 16, deer_options.jac_bytes_max below the
bf16 Jacobians of all rows): the chunk aggregates are formed while linearising and the
scan's final pass linearises again, from the same iterate, with float32 Jacobians composed
to float32 accuracy (tf32 MMAs with the three-term split). A Newton step therefore equals
the oracle's exact-Jacobian step to float32 accuracy (the stored-Jacobian path rounds the
Jacobians to bf16), and the fixed point is the float64 rollout."""
import ctypes as C

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


@pytest.mark.parametrize("window", [False, True])
def test_recomputing_mixed_path(window):
    import paper_2603_16850_gb300 as deer
    lengths = [700, 1, 0, 2049, 333, 64]
    off = synth.offsets_from_lengths(lengths)
    B = len(lengths)
    p = synth.massaction(B, 16, 24, 1, seed=31)
    dyn = deer.Dynamics.massaction(_t(p["topology"], torch.int32), _t(p["params"]), 16,
                                   p["dt"])
    base = dict(jac="full", prec="mixed_bf16", init="s0", reset=True, window=window, chunk=64)
    # one Newton step from the constant guess against the oracle's exact-Jacobian step
    one, _ = deer.deer_solve_batched(dyn, _t(p["s0"]), off, jac_bytes_max=1 << 16,
                                     **dict(base, tol=0.0, max_iters=1))
    one = one.cpu().numpy()
    for b, L in enumerate(lengths):
        if L == 0:
            continue
        od = odyn.MassAction(p["topology"][b:b + 1], p["params"][b:b + 1], p["dt"], "rk4", d=16)
        guess = onewton.initial_guess(od, p["s0"][b:b + 1], L, "s0")
        ref = onewton.quasi_newton_step(od, p["s0"][b:b + 1], guess, "full")[0]
        got = one[off[b]:off[b + 1]]
        err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
        # the first step evaluates the residual in float32 (far from convergence), whose
        # rounding the correction sums over the sequence
        assert err <= 5e-5, (b, err)
    s_rc, i_rc = deer.deer_solve_batched(dyn, _t(p["s0"]), off, jac_bytes_max=1 << 16,
                                         **dict(base, tol=1e-12, max_iters=600))
    s_st, i_st = deer.deer_solve_batched(dyn, _t(p["s0"]), off, **dict(base, tol=1e-12,
                                                                       max_iters=600))
    assert bool(i_rc.converged.all()) and bool(i_st.converged.all())
    # float32 Jacobians converge at least as fast as bf16 ones
    assert max(i_rc.iters.tolist()) <= max(i_st.iters.tolist())
    ref = cma.Batch(p["topology"], p["params"], p["dt"], "rk4", d=16).rollout(p["s0"], off)
    got = s_rc.cpu().numpy()
    for b in range(B):
        lo, hi = off[b], off[b + 1]
        if hi > lo:
            err = np.max(np.abs(got[lo:hi] - ref[lo:hi])) / np.max(np.abs(ref[lo:hi]))
            assert err <= 1e-9, (b, err)
    from paper_2603_16850_gb300 import _native as N
    lib = N.load()
    cd = dyn.c_struct()
    big = deer._options(**deer._opt_defaults(dict(base)))
    small = deer._options(**deer._opt_defaults(dict(base, jac_bytes_max=1 << 16)))
    n = int(off[-1])
    assert lib.deer_workspace_bytes(C.byref(cd), B, n, C.byref(small)) < \
        lib.deer_workspace_bytes(C.byref(cd), B, n, C.byref(big)) - n * 16 * 16 * 2 // 2


def test_tcgen05_block_diagonal_chunk_pass():
    """The d = 16 mixed-precision chunk products as tcgen05 MMAs (tensor-core mode 2: 8
    chunks per CTA stacked block-diagonally, the products accumulated in tensor memory)
    give the aggregates of the warp-level MMA pass up to the bf16 rounding of the chain,
    so the solve reaches the same fixed point (the float64 rollout within 1e-9), on a
    ragged batch whose tiles mix chunks of different lengths and end part-full."""
    import paper_2603_16850_gb300 as deer
    lengths = [700, 1, 0, 2049, 333, 64, 65, 1000, 17]
    off = synth.offsets_from_lengths(lengths)
    B = len(lengths)
    p = synth.massaction(B, 16, 24, 1, seed=33)
    dyn = deer.Dynamics.massaction(_t(p["topology"], torch.int32), _t(p["params"]), 16,
                                   p["dt"])
    opts = dict(jac="full", tol=1e-12, prec="mixed_bf16", init="zeros", reset=True, chunk=64)
    out = {}
    try:
        for mode in (1, 2):
            deer.set_tensor_cores(mode)
            it1, _ = deer.deer_solve_batched(dyn, _t(p["s0"]), off, **dict(opts, tol=0.0,
                                                                          max_iters=1))
            s, info = deer.deer_solve_batched(dyn, _t(p["s0"]), off, **opts)
            assert bool(info.converged.all()), mode
            out[mode] = (it1.cpu().numpy(), s.cpu().numpy())
    finally:
        deer.set_tensor_cores(1)
    # one iteration from the same guess: the chunk products round P to bf16 at every row in
    # both forms, in different orders of accumulation
    d1 = np.max(np.abs(out[1][0] - out[2][0])) / np.max(np.abs(out[1][0]))
    assert d1 <= 2e-2, d1
    ref = cma.Batch(p["topology"], p["params"], p["dt"], "rk4", d=16).rollout(p["s0"], off)
    for mode in (1, 2):
        got = out[mode][1]
        for b in range(B):
            lo, hi = off[b], off[b + 1]
            if hi > lo:
                err = np.max(np.abs(got[lo:hi] - ref[lo:hi])) / np.max(np.abs(ref[lo:hi]))
                assert err <= 1e-9, (mode, b, err)
