"""GB300-native parallel Newton (DEER / quasi-DEER / ELK) for nonlinear recurrences.

Python binding of the C ABI in include/deer.h. The functions below carry the C names
(``deer_solve``, ``deer_solve_batched``, ``deer_grad``, ``deer_rollout``) and only
marshal arguments: PyTorch provides device memory and the current CUDA stream; every
step of the solver runs in the hand-written sm_103a kernels of ``libdeer.so``.

Inputs given as CPU tensors are copied to the GPU and the result back (the end-to-end
path a host-side caller uses); CUDA tensors are used in place.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass
from typing import Optional

import torch

from . import _native as N

__all__ = [
    "Dynamics", "deer_solve", "deer_solve_batched", "deer_rollout", "deer_grad",
    "deer_workspace_bytes", "DeerFunction", "SolveInfo", "kernel_launch_count",
]


@dataclass
class Dynamics:
    """A built-in recurrence f (the registry of include/deer.h) and its parameters."""
    kind: str
    d: int
    params: torch.Tensor
    d_in: int = 0
    n_reactions: int = 0
    dt: float = 0.0
    params_stride: int = 0
    topology: Optional[torch.Tensor] = None
    topology_stride: int = 0

    @staticmethod
    def brusselator(params: torch.Tensor, dt: float) -> "Dynamics":
        """params [B][2] = (a, b) per sequence (or [2] shared)."""
        stride = 2 if params.dim() == 2 and params.shape[0] > 1 else 0
        return Dynamics("brusselator_euler", 2, params, dt=dt, params_stride=stride)

    @staticmethod
    def massaction(topology: torch.Tensor, k: torch.Tensor, d: int, dt: float,
                   integrator: str = "rk4") -> "Dynamics":
        """topology int32 [B][R][4] (or [R][4] shared), rate constants k [B][R] (or [R])."""
        R = k.shape[-1]
        ps = R if k.dim() == 2 and k.shape[0] > 1 else 0
        ts = 4 * R if topology.dim() == 3 and topology.shape[0] > 1 else 0
        return Dynamics(f"massaction_{integrator}", d, k, n_reactions=R, dt=dt,
                        params_stride=ps, topology=topology, topology_stride=ts)

    @staticmethod
    def gru(W: torch.Tensor, U: torch.Tensor) -> "Dynamics":
        """W [3][d][d_in], U [3][d][d] (gate order z, r, h); shared by the batch."""
        d, d_in = W.shape[1], W.shape[2]
        params = torch.cat([W.reshape(-1), U.reshape(-1)]).contiguous()
        return Dynamics("gru", d, params, d_in=d_in)

    @staticmethod
    def linear(A: torch.Tensor) -> "Dynamics":
        """s_t = A s_{t-1} + x_t with A [d][d] shared by the batch."""
        return Dynamics("linear", A.shape[0], A.contiguous(), d_in=A.shape[0])

    @staticmethod
    def rnn_tanh(W: torch.Tensor) -> "Dynamics":
        """Mean-field RNN s_t = W tanh(s_{t-1}) + u_t; W [d][d] shared or [B][d][d] per
        sequence; the inputs u_t are the rows of x (or none)."""
        d = W.shape[-1]
        stride = d * d if W.dim() == 3 and W.shape[0] > 1 else 0
        return Dynamics("rnn_tanh", d, W.reshape(-1).contiguous(), d_in=d, params_stride=stride)

    @staticmethod
    def langevin_2well(params: torch.Tensor, eps: float) -> "Dynamics":
        """Langevin step of size eps in the two-Gaussian potential; params [4d+2] shared or
        [B][4d+2] = m1 | m2 | v1 | v2 | w1 | w2; the noise draws are the rows of x."""
        n = params.shape[-1]
        d = (n - 2) // 4
        stride = n if params.dim() == 2 and params.shape[0] > 1 else 0
        return Dynamics("langevin_2well", d, params.reshape(-1).contiguous(), d_in=d, dt=eps,
                        params_stride=stride)

    @staticmethod
    def lorenz96(F: torch.Tensor, d: int, dt: float) -> "Dynamics":
        """Lorenz-96 with forcing F ([1] shared or [B]), one Dormand-Prince step dt per step."""
        stride = 1 if F.numel() > 1 else 0
        return Dynamics("lorenz96_dp5", d, F.reshape(-1).contiguous(), dt=dt,
                        params_stride=stride)

    @staticmethod
    def permute(d: int, dtype=torch.float64, device="cuda") -> "Dynamics":
        """Input-selected permutation s_t[i] = s_{t-1}[x_t[i]] (x holds the indices)."""
        return Dynamics("permute", d, torch.zeros(1, dtype=dtype, device=device), d_in=d)

    def to(self, device) -> "Dynamics":
        return Dynamics(self.kind, self.d, self.params.to(device), self.d_in, self.n_reactions,
                        self.dt, self.params_stride,
                        None if self.topology is None else self.topology.to(device),
                        self.topology_stride)

    def c_struct(self) -> N.deer_dynamics:
        _check_dev(self.params, "params")
        if self.topology is not None:
            _check_dev(self.topology, "topology")
            if self.topology.dtype != torch.int32:
                raise ValueError("topology must be int32")
        return N.deer_dynamics(
            N.KIND[self.kind], self.d, self.d_in, self.n_reactions, float(self.dt),
            self.params.data_ptr(), self.params_stride,
            0 if self.topology is None else self.topology.data_ptr(), self.topology_stride)


@dataclass
class SolveInfo:
    status: int
    iters: torch.Tensor       # [B] int32
    converged: torch.Tensor   # [B] bool
    merit: torch.Tensor       # [B] float64
    max_resid: torch.Tensor   # [B] float64


def _check_dev(t: torch.Tensor, name: str):
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def _ptr(t):
    return 0 if t is None else t.data_ptr()


def _dtype(prec: str):
    return torch.float32 if prec == "fp32" else torch.float64


def _options(jac, damp, damp_param, tol, max_iters, init, prec, reset, chunk,
             confirm=1, window=False, seed=0, history=None,
             compensate=True, jac_bytes_max=0, device_loop=False,
             block_solve=True) -> N.deer_options:
    o = N.deer_options()
    o.max_iters = int(max_iters)
    o.tol = float(tol)
    o.jac = N.JAC[jac]
    o.damp = N.DAMP[damp]
    o.damp_param = float(damp_param)
    o.init = N.INIT[init]
    o.prec = N.PREC[prec]
    o.reset = int(bool(reset))
    o.chunk = int(chunk)
    o.confirm = int(confirm)
    o.window = int(bool(window))
    o.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    o.compensate = int(bool(compensate))
    o.jac_bytes_max = int(jac_bytes_max)
    o.device_loop = int(bool(device_loop))
    o.no_block_solve = 0 if block_solve else 1
    if history is not None:
        _check_dev(history, "history")
        if history.dtype != torch.float64 or history.dim() != 2 or history.shape[1] != 4:
            raise ValueError("history must be a float64 CUDA tensor [n][4]")
        o.history = history.data_ptr()
        o.history_len = history.shape[0]
    return o


def _stream_handle(stream) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def kernel_launch_count() -> int:
    return int(N.load().deer_kernel_launch_count())


def set_tensor_cores(on) -> None:
    """Select the tensor-core kernels where a step has one (deer_set_tensor_cores): False /
    0 SIMT, True / 1 the default tensor-core kernels, 2 the tcgen05 block-diagonal form of
    the d = 16 mixed-precision chunk products."""
    N.load().deer_set_tensor_cores(int(on))


def tensor_cores() -> int:
    """The current selection of set_tensor_cores (deer_get_tensor_cores): 0, 1 or 2."""
    return int(N.load().deer_get_tensor_cores())


def deer_workspace_bytes(dyn: Dynamics, batch: int, total_steps: int, **opts) -> int:
    o = _options(**_opt_defaults(opts))
    return int(N.load().deer_workspace_bytes(C.byref(dyn.c_struct()), batch, total_steps,
                                             C.byref(o)))


def _opt_defaults(opts):
    base = dict(jac="full", damp="none", damp_param=0.0, tol=1e-10, max_iters=0, init="s0",
                prec="fp64", reset=False, chunk=0, confirm=1, window=False, seed=0,
                history=None, compensate=True, jac_bytes_max=0, device_loop=False,
                block_solve=True)
    base.update(opts)
    return base


def _run_solve(dyn, B, T, offsets, s0, x, s_init, opts, stream, workspace, device,
               explicit=()):
    lib = N.load()
    # the autotuner's cached configuration for this GPU and problem class, if any: its
    # chunk length where the caller left chunk = 0, its loop forms where the caller did not
    # choose them (``explicit``: the option names the caller passed)
    from . import autotune
    Tmax = T if offsets is None else max(
        (int(offsets[i + 1]) - int(offsets[i]) for i in range(B)), default=0)
    tuned = autotune.cached_options(dyn, Tmax, opts["jac"], opts["prec"],
                                    gpu=torch.cuda.get_device_name(device))
    if tuned:
        upd = {k: v for k, v in tuned.items()
               if (k == "chunk" and int(opts.get("chunk", 0)) == 0)
               or (k != "chunk" and k not in explicit)}
        opts = dict(opts, **upd)
    o = _options(**opts)
    dt = _dtype(opts["prec"])
    N_rows = int(offsets[-1]) if offsets is not None else B * T
    for name, t in (("s0", s0), ("x", x)):
        if t is not None:
            _check_dev(t, name)
            if t.dtype != dt:
                raise ValueError(f"{name} must be {dt} for prec={opts['prec']}")
    if dyn.params.dtype != dt:
        raise ValueError(f"params must be {dt} for prec={opts['prec']}")
    if s_init is not None:
        s = s_init.to(device=device, dtype=dt).contiguous().clone()
        o.init = N.INIT["user"]
    else:
        s = torch.empty((N_rows, dyn.d), dtype=dt, device=device)
    cdyn = dyn.c_struct()
    need = lib.deer_workspace_bytes(C.byref(cdyn), B, N_rows, C.byref(o))
    if need == 0 and B > 0:
        raise N.DeerError(N.DEER_ERR_UNSUPPORTED, "deer_workspace_bytes")
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(max(need, 256), dtype=torch.uint8, device=device)
    infos = (N.deer_info * max(B, 1))()
    sh = _stream_handle(stream)
    if offsets is None:
        st = lib.deer_solve(C.byref(cdyn), B, T, _ptr(s0), _ptr(x), _ptr(s), C.byref(o),
                            _ptr(workspace), workspace.numel(), sh, infos)
    else:
        off = (C.c_int64 * (B + 1))(*[int(v) for v in offsets])
        st = lib.deer_solve_batched(C.byref(cdyn), B, off, _ptr(s0), _ptr(x), _ptr(s),
                                    C.byref(o), _ptr(workspace), workspace.numel(), sh, infos)
    if st not in (N.DEER_OK, N.DEER_NOT_CONVERGED):
        raise N.DeerError(st, "deer_solve")
    info = SolveInfo(
        status=st,
        iters=torch.tensor([infos[i].iters for i in range(B)], dtype=torch.int32),
        converged=torch.tensor([bool(infos[i].converged) for i in range(B)]),
        merit=torch.tensor([infos[i].merit for i in range(B)], dtype=torch.float64),
        max_resid=torch.tensor([infos[i].max_resid for i in range(B)], dtype=torch.float64))
    return s, info


def deer_solve(dyn: Dynamics, s0: torch.Tensor, T: int, x: Optional[torch.Tensor] = None, *,
               s_init: Optional[torch.Tensor] = None, stream=None, workspace=None, out=None,
               **opts):
    """Solve ``B = s0.shape[0]`` sequences of length T. Returns (s [B*T][d], SolveInfo).

    Options (see deer_options in include/deer.h): jac ('full'|'diag'|'identity'|'zero'),
    damp ('none'|'elk'|'scale'|'clip'), damp_param, tol, max_iters, init
    ('zeros'|'s0'|'jacobi'|'randn'|'user'), seed (for 'randn'), prec
    ('fp64'|'fp32'|'mixed_bf16'), reset, chunk, confirm, window (sliding window: freeze the
    converged prefix of each sequence), history (a float64 CUDA tensor [n][4] that receives
    (iteration, merit, max scaled residual, active sequences) of each convergence test),
    compensate (fp32 mass-action kinetics with the full Jacobian: keep a compensated
    two-float state, default True), device_loop (run the iterations after the first as one
    CUDA graph with a conditional while node, no host synchronisation between them),
    block_solve (default True: short sequences run the whole loop in one kernel, one
    thread block per sequence; False keeps the multi-kernel loop).
    Host inputs are copied to the GPU and the result back to the host, into ``out`` when
    given (a preallocated, ideally pinned, host tensor [B*T][d]).
    """
    explicit = frozenset(opts)
    opts = _opt_defaults(opts)
    host = not s0.is_cuda
    device = torch.device("cuda") if host else s0.device
    if host:
        _check_out(out, (s0.shape[0] * int(T), dyn.d), _dtype(opts["prec"]))
        dyn, s0, x = _to_device(dyn, s0, x, device)
    s, info = _run_solve(dyn, s0.shape[0], int(T), None, s0, x, s_init, opts, stream,
                         workspace, device, explicit)
    return (_to_host(s, out) if host else s), info


def deer_solve_batched(dyn: Dynamics, s0: torch.Tensor, offsets, x: Optional[torch.Tensor] = None,
                       *, s_init=None, stream=None, workspace=None, out=None, **opts):
    """Ragged batch: sequence b owns rows offsets[b]..offsets[b+1]-1 of the packed output."""
    explicit = frozenset(opts)
    opts = _opt_defaults(opts)
    offsets = [int(v) for v in (offsets.tolist() if hasattr(offsets, "tolist") else offsets)]
    host = not s0.is_cuda
    device = torch.device("cuda") if host else s0.device
    if host:
        _check_out(out, (int(offsets[-1]), dyn.d), _dtype(opts["prec"]))
        dyn, s0, x = _to_device(dyn, s0, x, device)
    s, info = _run_solve(dyn, s0.shape[0], 0, offsets, s0, x, s_init, opts, stream, workspace,
                         device, explicit)
    return (_to_host(s, out) if host else s), info


def deer_rollout(dyn: Dynamics, s0: torch.Tensor, T: int = 0, x=None, *, offsets=None,
                 prec="fp64", stream=None):
    """Sequential rollout on the GPU (comparison baseline). offsets: CUDA int64 [B+1] or
    None for B sequences of length T."""
    lib = N.load()
    B = s0.shape[0]
    _check_dev(s0, "s0")
    n = int(offsets[-1].item()) if offsets is not None else B * T
    s = torch.empty((n, dyn.d), dtype=s0.dtype, device=s0.device)
    cdyn = dyn.c_struct()
    st = lib.deer_rollout(C.byref(cdyn), B, int(T), _ptr(offsets), _ptr(s0), _ptr(x), _ptr(s),
                          N.PREC[prec], _stream_handle(stream))
    if st != N.DEER_OK:
        raise N.DeerError(st, "deer_rollout")
    return s


def deer_grad(dyn: Dynamics, s0, T, s_star, dl_ds, x=None, *, prec="fp64", chunk=0,
              stream=None, workspace=None, want_ds0=True, want_dx=False, jac_bytes_max=0):
    """Adjoint gradient at the converged trajectory. Returns (dl/dparams [B][P], dl/ds0),
    plus dl/dx (the layout of x) when ``want_dx`` (deer_grad_ex: GRU, affine, mean-field
    RNN and Langevin inputs); dl/dparams is None for kinds without per-sequence trainable
    parameters (only the Brusselator's (a, b) and the mass-action rate constants are
    differentiated). ``jac_bytes_max`` > 0 bounds the memory of the stored step Jacobians
    (the reverse scan then runs over time windows, see deer_options.jac_bytes_max)."""
    lib = N.load()
    B = s0.shape[0]
    dt = _dtype(prec)
    o = _options(**_opt_defaults(dict(prec=prec, chunk=chunk, jac_bytes_max=jac_bytes_max)))
    cdyn = dyn.c_struct()
    P = dyn.params_stride if dyn.params_stride else dyn.params.numel()
    trainable = dyn.kind in ("brusselator_euler", "massaction_euler", "massaction_rk4")
    dparams = torch.zeros((B, P), dtype=dt, device=s0.device) if trainable else None
    ds0 = torch.zeros((B, dyn.d), dtype=dt, device=s0.device) if want_ds0 else None
    need = lib.deer_grad_workspace_bytes(C.byref(cdyn), B, int(T), C.byref(o))
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(max(need, 256), dtype=torch.uint8, device=s0.device)
    dx = None
    if want_dx:
        if x is None:
            raise ValueError("want_dx needs the inputs x")
        dx = torch.empty_like(x)
    st = lib.deer_grad_ex(C.byref(cdyn), B, int(T), _ptr(s0), _ptr(x), _ptr(s_star),
                          _ptr(dl_ds), _ptr(dparams), _ptr(ds0), _ptr(dx), C.byref(o),
                          _ptr(workspace), workspace.numel(), _stream_handle(stream))
    if st != N.DEER_OK:
        raise N.DeerError(st, "deer_grad")
    return (dparams, ds0, dx) if want_dx else (dparams, ds0)


def selftest_wait_timeout(stream=None) -> int:
    """Run the library's bounded-wait self-test (deer_selftest_wait_timeout): a look-back
    scan whose predecessor tile never publishes. Returns the status: DEER_ERR_TIMEOUT (-5)
    is the designed outcome."""
    return int(N.load().deer_selftest_wait_timeout(_stream_handle(stream)))


def deer_lle(dyn: Dynamics, s0, T: int, s, u0=None, x=None, *, prec="fp64", stream=None,
             workspace=None):
    """Largest Lyapunov exponent estimate along trajectories (deer_lle): s [B*T][d] (a
    rollout or a converged solve), u0 [B][d] unit start vectors (default: the normalised
    all-ones vector). Returns a float64 tensor [B]."""
    lib = N.load()
    B = s0.shape[0]
    dt = _dtype(prec)
    if u0 is None:
        u0 = torch.full((B, dyn.d), dyn.d ** -0.5, dtype=dt, device=s0.device)
    for name, t in (("s0", s0), ("s", s), ("u0", u0), ("x", x)):
        if t is not None:
            _check_dev(t, name)
            if t.dtype != dt:
                raise ValueError(f"{name} must be {dt} for prec={prec}")
    out = torch.empty(B, dtype=torch.float64, device=s0.device)
    cdyn = dyn.c_struct()
    need = lib.deer_lle_workspace_bytes(C.byref(cdyn), B, int(T), N.PREC[prec])
    if need == 0 and B > 0:
        raise N.DeerError(N.DEER_ERR_UNSUPPORTED, "deer_lle_workspace_bytes")
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(max(need, 256), dtype=torch.uint8, device=s0.device)
    st = lib.deer_lle(C.byref(cdyn), B, int(T), _ptr(s0), _ptr(x), _ptr(s), _ptr(u0),
                      _ptr(out), N.PREC[prec], _ptr(workspace), workspace.numel(),
                      _stream_handle(stream))
    if st != N.DEER_OK:
        raise N.DeerError(st, "deer_lle")
    return out


def _to_device(dyn, s0, x, device):
    nb = True
    dyn = Dynamics(dyn.kind, dyn.d, dyn.params.to(device, non_blocking=nb), dyn.d_in,
                   dyn.n_reactions, dyn.dt, dyn.params_stride,
                   None if dyn.topology is None else dyn.topology.to(device, non_blocking=nb),
                   dyn.topology_stride)
    s0 = s0.to(device, non_blocking=nb)
    x = None if x is None else x.to(device, non_blocking=nb)
    return dyn, s0, x


def _to_host(s, out=None):
    """Copy a device result to the host: into ``out`` (a host tensor of the same shape and
    dtype; pinned for full copy bandwidth) or into a newly pinned buffer. Pinning gigabytes
    takes longer than the copy itself, so callers that solve repeatedly pass ``out``."""
    if out is None:
        out = torch.empty(s.shape, dtype=s.dtype, pin_memory=True)
    _check_out(out, tuple(s.shape), s.dtype)
    out.copy_(s)
    return out


def _check_out(out, shape, dtype):
    if out is not None and (out.is_cuda or tuple(out.shape) != tuple(shape) or
                            out.dtype != dtype or not out.is_contiguous()):
        raise ValueError(f"out must be a contiguous host tensor {tuple(shape)} {dtype}")


class DeerFunction(torch.autograd.Function):
    """Differentiable solve: forward = deer_solve (any mode; the result is the fixed point),
    backward = deer_grad (reverse adjoint scan at the fixed point, implicit
    differentiation, no unrolled Newton history). Gradients flow to the per-sequence
    parameters, to s0 and, for the kinds with differentiable inputs, to x."""

    @staticmethod
    def forward(ctx, params, s0, dyn: Dynamics, T: int, x, opts: dict):
        d2 = Dynamics(dyn.kind, dyn.d, params.detach().contiguous(), dyn.d_in, dyn.n_reactions,
                      dyn.dt, dyn.params_stride, dyn.topology, dyn.topology_stride)
        xd = None if x is None else x.detach().contiguous()
        s, info = deer_solve(d2, s0.detach().contiguous(), T, xd, **opts)
        ctx.dyn, ctx.T, ctx.x, ctx.prec = d2, T, xd, opts.get("prec", "fp64")
        ctx.save_for_backward(s0.detach(), s)
        ctx.info = info
        return s

    @staticmethod
    def backward(ctx, g):
        s0, s = ctx.saved_tensors
        want_dx = ctx.x is not None and ctx.needs_input_grad[4]
        out = deer_grad(ctx.dyn, s0, ctx.T, s, g.contiguous(), ctx.x, prec=ctx.prec,
                        want_dx=want_dx)
        dp, ds0 = out[0], out[1]
        dx = out[2] if want_dx else None
        return (None if dp is None else dp.reshape(ctx.dyn.params.shape)), ds0, None, None, \
            dx, None
