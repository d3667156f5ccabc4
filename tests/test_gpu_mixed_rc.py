"""Mixed precision without stored Jacobians (d = 16, deer_options.jac_bytes_max below the
bf16 Jacobians of all rows): the chunk aggregates are formed while linearising and the
scan's final pass linearises again. The recomputed Jacobians and residuals are the same
arithmetic from the same iterate, so the iterates equal those of the stored-Jacobian path
bit for bit, and the fixed point is the float64 rollout."""
import ctypes as C

import numpy as np
import pytest
import torch

import synth
from oracle import cma

pytestmark = pytest.mark.gpu


def _t(a, dt=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


@pytest.mark.parametrize("window,iters", [(False, 3), (True, 0), (False, 0)])
def test_recomputing_mixed_path_equals_stored(window, iters):
    import paper_2603_16850_gb300 as deer
    lengths = [700, 1, 0, 2049, 333, 64]
    off = synth.offsets_from_lengths(lengths)
    B = len(lengths)
    p = synth.massaction(B, 16, 24, 1, seed=31)
    dyn = deer.Dynamics.massaction(_t(p["topology"], torch.int32), _t(p["params"]), 16,
                                   p["dt"])
    opts = dict(jac="full", tol=1e-12 if iters == 0 else 0.0, prec="mixed_bf16", init="zeros",
                reset=True, window=window, chunk=64, max_iters=iters if iters else 600)
    s_ref, i_ref = deer.deer_solve_batched(dyn, _t(p["s0"]), off, **opts)
    s_rc, i_rc = deer.deer_solve_batched(dyn, _t(p["s0"]), off, jac_bytes_max=1 << 16, **opts)
    assert torch.equal(s_rc, s_ref)
    assert i_rc.iters.tolist() == i_ref.iters.tolist()
    assert i_rc.converged.tolist() == i_ref.converged.tolist()
    if iters == 0:
        assert bool(i_rc.converged.all())
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
    big = deer._options(**deer._opt_defaults(dict(opts)))
    small = deer._options(**deer._opt_defaults(dict(opts, jac_bytes_max=1 << 16)))
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
