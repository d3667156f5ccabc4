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
