"""Host-side checks of the C ABI (no GPU needed): the library builds, loads and exports
every function include/deer.h declares; argument validation and workspace sizing run
without touching the device."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2603_16850_gb300 import _build, _native
    _build.build()
    return _native.load()


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(deer_\w+)\s*\(", text):
            names.add(m.group(1))
    return names


def test_every_declared_symbol_is_exported(lib):
    from paper_2603_16850_gb300 import _native
    declared = _declared_functions()
    assert "deer_solve" in declared and "deer_grad" in declared and "deer_solve_batched" in declared
    for name in declared:
        assert hasattr(lib, name), name
    # the Python binding covers the same set
    assert declared <= set(_native.SIGNATURES), declared - set(_native.SIGNATURES)


def test_defaults_and_strings(lib):
    from paper_2603_16850_gb300 import _native as N
    o = N.deer_options()
    lib.deer_default_options(C.byref(o))
    assert o.tol == 1e-10 and o.jac == 0 and o.init == 1 and o.prec == 0
    assert lib.deer_status_string(0) == b"ok"
    assert b"invalid" in lib.deer_status_string(-1)
    assert lib.deer_version() >= 1


def _dyn(N, kind="massaction_rk4", d=8, R=12, params=1, topo=1):
    return N.deer_dynamics(N.KIND[kind], d, 0, R, 1e-3, params, R, topo, 4 * R)


def test_workspace_sizes_and_validation(lib):
    from paper_2603_16850_gb300 import _native as N
    o = N.deer_options()
    lib.deer_default_options(C.byref(o))
    o.prec = N.PREC["fp32"]
    dyn = _dyn(N)
    b = lib.deer_workspace_bytes(C.byref(dyn), 4096, 4096 * 16384, C.byref(o))
    # the dense Jacobians dominate: 4096*16384 rows * 8*8 float32
    assert b >= 4096 * 16384 * 64 * 4
    o.jac = N.JAC["diag"]
    bd = lib.deer_workspace_bytes(C.byref(dyn), 4096, 4096 * 16384, C.byref(o))
    assert 0 < bd < b
    # unsupported state size / invalid combination -> 0
    bad = _dyn(N, d=3)
    assert lib.deer_workspace_bytes(C.byref(bad), 1, 10, C.byref(o)) == 0
    # dense ELK: the full-Jacobian Kalman step is built for d <= 16 only
    o.jac = N.JAC["full"]
    o.damp = N.DAMP["elk"]
    assert lib.deer_workspace_bytes(C.byref(dyn), 1, 10, C.byref(o)) > 0
    assert lib.deer_workspace_bytes(C.byref(_dyn(N, d=16)), 1, 10, C.byref(o)) > 0
    assert lib.deer_workspace_bytes(C.byref(_dyn(N, d=32)), 1, 10, C.byref(o)) == 0


def test_invalid_arguments_fail_without_device_work(lib):
    from paper_2603_16850_gb300 import _native as N
    o = N.deer_options()
    lib.deer_default_options(C.byref(o))
    dyn = _dyn(N)
    info = (N.deer_info * 1)()
    # empty batch: nothing to do
    assert lib.deer_solve(C.byref(dyn), 0, 10, None, None, None, C.byref(o), None, 0, None,
                          info) == 0
    # null state pointers
    assert lib.deer_solve(C.byref(dyn), 1, 10, None, None, None, C.byref(o), None, 0, None,
                          info) == N.DEER_ERR_INVALID
    # bad enum
    o.jac = 9
    assert lib.deer_solve(C.byref(dyn), 1, 10, 8, None, 8, C.byref(o), None, 0, None,
                          info) == N.DEER_ERR_INVALID
    lib.deer_default_options(C.byref(o))
    # decreasing offsets
    off = (C.c_int64 * 3)(0, 5, 3)
    assert lib.deer_solve_batched(C.byref(dyn), 2, off, 8, None, 8, C.byref(o), None, 0, None,
                                  info) == N.DEER_ERR_INVALID
    # missing topology for mass action
    nd = _dyn(N, topo=0)
    assert lib.deer_solve(C.byref(nd), 1, 10, 8, None, 8, C.byref(o), None, 0, None,
                          info) == N.DEER_ERR_INVALID
    # workspace too small (checked before any device call)
    assert lib.deer_solve(C.byref(dyn), 1, 10, 8, None, 8, C.byref(o), 256, 16, None,
                          info) == N.DEER_ERR_WORKSPACE
    # a history length without a buffer, an unknown initial guess
    o.history_len = 4
    assert lib.deer_solve(C.byref(dyn), 1, 10, 8, None, 8, C.byref(o), None, 0, None,
                          info) == N.DEER_ERR_INVALID
    lib.deer_default_options(C.byref(o))
    o.init = 5
    assert lib.deer_solve(C.byref(dyn), 1, 10, 8, None, 8, C.byref(o), None, 0, None,
                          info) == N.DEER_ERR_INVALID
    lib.deer_default_options(C.byref(o))
    # sizes whose products would overflow are rejected before any arithmetic on them
    assert lib.deer_solve(C.byref(dyn), 1 << 40, 1 << 40, 8, None, 8, C.byref(o), None, 0,
                          None, info) == N.DEER_ERR_INVALID
    assert lib.deer_workspace_bytes(C.byref(dyn), 1, 1 << 62, C.byref(o)) == 0
    assert lib.deer_grad_workspace_bytes(C.byref(dyn), 1 << 40, 1 << 40, C.byref(o)) == 0
    assert lib.deer_solve_noalloc(C.byref(dyn), 1 << 40, 1 << 40, 8, None, 8, C.byref(o),
                                  None, info) == N.DEER_ERR_INVALID


def test_second_workload_kinds_sizes_and_checks(lib):
    """Supported sizes of the mean-field RNN, two-well Langevin, Lorenz-96 and permutation
    kinds, and their argument checks (all host-side: no device work)."""
    from paper_2603_16850_gb300 import _native as N
    o = N.deer_options()
    lib.deer_default_options(C.byref(o))

    def ws(kind, d, dt=0.01, stride=0, jac="full", damp="none"):
        o.jac, o.damp = N.JAC[jac], N.DAMP[damp]
        dyn = N.deer_dynamics(N.KIND[kind], d, d, 0, dt, 8, stride, 0, 0)
        return lib.deer_workspace_bytes(C.byref(dyn), 2, 200, C.byref(o))

    assert ws("rnn_tanh", 32) > 0 and ws("rnn_tanh", 64) == 0 and ws("rnn_tanh", 5) == 0
    assert ws("langevin_2well", 2) > 0 and ws("langevin_2well", 16, jac="diag") > 0
    assert ws("lorenz96_dp5", 5) > 0 and ws("lorenz96_dp5", 8) > 0
    assert ws("lorenz96_dp5", 2) == 0 and ws("lorenz96_dp5", 16) == 0
    assert ws("permute", 5) > 0 and ws("permute", 32) > 0 and ws("permute", 1) == 0
    # dense ELK keeps its register sizes (1, 2, 4, 8); quasi-ELK takes any size
    assert ws("lorenz96_dp5", 8, damp="elk") > 0 and ws("lorenz96_dp5", 5, damp="elk") == 0
    assert ws("lorenz96_dp5", 5, jac="diag", damp="elk") > 0
    # a time step is required where f integrates an ODE or scales the noise
    assert ws("lorenz96_dp5", 5, dt=0.0) == 0 and ws("langevin_2well", 2, dt=-1.0) == 0
    # per-sequence parameter strides below one block of parameters are rejected
    assert ws("langevin_2well", 2, stride=9) == 0 and ws("langevin_2well", 2, stride=10) > 0
    assert ws("rnn_tanh", 4, stride=15) == 0 and ws("rnn_tanh", 4, stride=16) > 0
    # the permutation needs its inputs: a solve without x fails before any device work
    lib.deer_default_options(C.byref(o))
    info = (N.deer_info * 1)()
    pd = N.deer_dynamics(N.KIND["permute"], 5, 5, 0, 0.0, 8, 0, 0, 0)
    assert lib.deer_solve(C.byref(pd), 1, 10, 8, None, 8, C.byref(o), 256, 1 << 20, None,
                          info) == N.DEER_ERR_INVALID


def test_host_output_buffer_checked_before_any_work():
    """deer_solve with host inputs validates the caller's output buffer (shape, dtype,
    host residency) before touching the device."""
    import torch

    import paper_2603_16850_gb300 as deer
    dyn = deer.Dynamics.lorenz96(torch.full((1,), 8.0), 5, 0.01)
    s0 = torch.full((2, 5), 8.0, dtype=torch.float64)
    for bad in (torch.empty((2 * 7, 5)),                         # wrong dtype
                torch.empty((2 * 6, 5), dtype=torch.float64),    # wrong shape
                torch.empty((5, 2 * 7), dtype=torch.float64).t()):  # not contiguous
        with pytest.raises(ValueError, match="out must be"):
            deer.deer_solve(dyn, s0, 7, out=bad, jac="full")


def test_dynamics_factories_describe_the_registry_layouts():
    """The Python factories of the second-workload kinds fill the C struct the way the
    header documents (kind, d, input size, per-sequence parameter stride)."""
    import torch

    import paper_2603_16850_gb300 as deer
    from paper_2603_16850_gb300 import _native as N
    W1 = torch.zeros(8, 8)
    W3 = torch.zeros(3, 8, 8)
    r1, r3 = deer.Dynamics.rnn_tanh(W1), deer.Dynamics.rnn_tanh(W3)
    assert (r1.kind, r1.d, r1.d_in, r1.params_stride) == ("rnn_tanh", 8, 8, 0)
    assert r3.params_stride == 64 and r3.params.numel() == 3 * 64
    lw = deer.Dynamics.langevin_2well(torch.zeros(5, 4 * 2 + 2), 0.01)
    assert (lw.d, lw.d_in, lw.params_stride, lw.dt) == (2, 2, 10, 0.01)
    l96 = deer.Dynamics.lorenz96(torch.full((4,), 8.0), 5, 0.01)
    assert (l96.d, l96.d_in, l96.params_stride) == (5, 0, 1)
    pm = deer.Dynamics.permute(5, torch.float32, "cpu")
    assert (pm.d, pm.d_in, pm.params.dtype) == (5, 5, torch.float32)
    assert [N.KIND[k] for k in ("rnn_tanh", "langevin_2well", "lorenz96_dp5", "permute")] == \
        [5, 6, 7, 8]


def test_options_struct_layout_matches_the_header(lib):
    """deer_default_options writes exactly the struct the binding declares: every field
    reads back its documented default and the bytes past the ctypes struct stay untouched
    (a larger C struct would overwrite them)."""
    from paper_2603_16850_gb300 import _native as N
    size = C.sizeof(N.deer_options)
    buf = (C.c_ubyte * (size + 64))(*([0xAB] * (size + 64)))
    o = N.deer_options.from_buffer(buf)
    lib.deer_default_options(C.byref(o))
    assert (o.max_iters, o.tol, o.jac, o.damp, o.damp_param, o.init, o.prec, o.reset,
            o.chunk, o.confirm, o.window, o.seed, o.history, o.history_len, o.compensate,
            o.jac_bytes_max, o.device_loop, o.no_block_solve) == \
        (0, 1e-10, 0, 0, 0.0, 1, 0, 0, 0, 1, 0, 0, None, 0, 1, 0, 0, 0)
    assert all(b == 0xAB for b in bytes(buf)[size:])


def test_binding_enums_match_the_header():
    """Every enumerator of include/deer.h's kind, Jacobian, damping, initial-guess and
    precision enums has the same value in the Python binding's maps."""
    import re

    from paper_2603_16850_gb300 import _native as N
    hdr = open(os.path.join(ROOT, "include", "deer.h")).read()
    vals = {m.group(1): int(m.group(2))
            for m in re.finditer(r"\b(DEER_[A-Z0-9_]+)\s*=\s*(-?\d+)", hdr)}
    maps = {"DEER_F_": (N.KIND, {"brusselator_euler": "BRUSSELATOR_EULER",
                                 "massaction_euler": "MASSACTION_EULER",
                                 "massaction_rk4": "MASSACTION_RK4", "gru": "GRU",
                                 "linear": "LINEAR", "rnn_tanh": "RNN_TANH",
                                 "langevin_2well": "LANGEVIN_2WELL",
                                 "lorenz96_dp5": "LORENZ96_DP5", "permute": "PERMUTE"}),
            "DEER_JAC_": (N.JAC, {"full": "FULL", "diag": "DIAG", "identity": "IDENTITY",
                                  "zero": "ZERO"}),
            "DEER_DAMP_": (N.DAMP, {"none": "NONE", "elk": "ELK", "scale": "SCALE",
                                    "clip": "CLIP"}),
            "DEER_INIT_": (N.INIT, {"zeros": "ZEROS", "s0": "S0", "jacobi": "JACOBI",
                                    "user": "USER", "randn": "RANDN"}),
            "DEER_": (N.PREC, {"fp64": "FP64", "fp32": "FP32", "mixed_bf16": "MIXED_BF16"})}
    for prefix, (pymap, names) in maps.items():
        assert set(pymap) == set(names), prefix
        for py, c in names.items():
            assert pymap[py] == vals[prefix + c], (prefix, py)
    kinds = {k for k in vals if k.startswith("DEER_F_")}
    assert len(kinds) == len(N.KIND)


def test_binding_options_map_the_loop_forms():
    """The Python options reach the C struct: device_loop, and block_solve inverted into
    no_block_solve, beside the defaults of everything else."""
    import paper_2603_16850_gb300 as deer
    o = deer._options(**deer._opt_defaults({}))
    assert (o.device_loop, o.no_block_solve, o.compensate) == (0, 0, 1)
    o = deer._options(**deer._opt_defaults(dict(device_loop=True, block_solve=False)))
    assert (o.device_loop, o.no_block_solve) == (1, 1)
