"""ctypes binding of the C ABI declared in include/deer.h (argument marshalling only).

The shared library is the in-tree ``libdeer.so``; importing this module fails loudly when
it is missing (there is no CPU fallback: every step of the solver runs in the CUDA
kernels of the library).
"""
from __future__ import annotations

import ctypes as C
import os

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libdeer.so")

# enums (mirror deer.h)
DEER_OK, DEER_NOT_CONVERGED = 0, 1
DEER_ERR_INVALID, DEER_ERR_CUDA, DEER_ERR_NONFINITE = -1, -2, -3
DEER_ERR_WORKSPACE, DEER_ERR_TIMEOUT, DEER_ERR_UNSUPPORTED = -4, -5, -6

KIND = {"brusselator_euler": 0, "massaction_euler": 1, "massaction_rk4": 2, "gru": 3, "linear": 4,
        "rnn_tanh": 5, "langevin_2well": 6, "lorenz96_dp5": 7, "permute": 8}
JAC = {"full": 0, "diag": 1, "identity": 2, "zero": 3}
DAMP = {"none": 0, "elk": 1, "scale": 2, "clip": 3}
INIT = {"zeros": 0, "s0": 1, "jacobi": 2, "user": 3, "randn": 4}
PREC = {"fp64": 0, "fp32": 1, "mixed_bf16": 2}


class deer_dynamics(C.Structure):
    _fields_ = [
        ("kind", C.c_int32), ("d", C.c_int32), ("d_in", C.c_int32), ("n_reactions", C.c_int32),
        ("dt", C.c_double), ("params", C.c_void_p), ("params_stride", C.c_int64),
        ("topology", C.c_void_p), ("topology_stride", C.c_int64),
    ]


class deer_options(C.Structure):
    _fields_ = [
        ("max_iters", C.c_int32), ("tol", C.c_double), ("jac", C.c_int32), ("damp", C.c_int32),
        ("damp_param", C.c_double), ("init", C.c_int32), ("prec", C.c_int32),
        ("reset", C.c_int32), ("chunk", C.c_int32), ("confirm", C.c_int32),
        ("window", C.c_int32), ("seed", C.c_uint64), ("history", C.c_void_p),
        ("history_len", C.c_int32), ("compensate", C.c_int32),
        ("jac_bytes_max", C.c_int64), ("device_loop", C.c_int32), ("no_block_solve", C.c_int32),
    ]


class deer_info(C.Structure):
    _fields_ = [("iters", C.c_int32), ("converged", C.c_int32), ("merit", C.c_double),
                ("max_resid", C.c_double)]


class deer_profile(C.Structure):
    _fields_ = [("launches", C.c_int64 * 4), ("ms", C.c_double * 4), ("rows", C.c_int64 * 4)]


PHASES = ("setup", "linearize", "check", "scan")

# Every exported symbol with its argument and return types.
SIGNATURES = {
    "deer_default_options": (None, [C.POINTER(deer_options)]),
    "deer_workspace_bytes": (C.c_size_t, [C.POINTER(deer_dynamics), C.c_int64, C.c_int64,
                                          C.POINTER(deer_options)]),
    "deer_solve": (C.c_int32, [C.POINTER(deer_dynamics), C.c_int64, C.c_int64, C.c_void_p,
                               C.c_void_p, C.c_void_p, C.POINTER(deer_options), C.c_void_p,
                               C.c_size_t, C.c_void_p, C.POINTER(deer_info)]),
    "deer_solve_batched": (C.c_int32, [C.POINTER(deer_dynamics), C.c_int64,
                                       C.POINTER(C.c_int64), C.c_void_p, C.c_void_p,
                                       C.c_void_p, C.POINTER(deer_options), C.c_void_p,
                                       C.c_size_t, C.c_void_p, C.POINTER(deer_info)]),
    "deer_grad_workspace_bytes": (C.c_size_t, [C.POINTER(deer_dynamics), C.c_int64, C.c_int64,
                                               C.POINTER(deer_options)]),
    "deer_grad": (C.c_int32, [C.POINTER(deer_dynamics), C.c_int64, C.c_int64, C.c_void_p,
                              C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                              C.POINTER(deer_options), C.c_void_p, C.c_size_t, C.c_void_p]),
    "deer_grad_ex": (C.c_int32, [C.POINTER(deer_dynamics), C.c_int64, C.c_int64, C.c_void_p,
                                 C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                 C.c_void_p, C.POINTER(deer_options), C.c_void_p, C.c_size_t,
                                 C.c_void_p]),
    "deer_rollout": (C.c_int32, [C.POINTER(deer_dynamics), C.c_int64, C.c_int64, C.c_void_p,
                                 C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]),
    "deer_solve_noalloc": (C.c_int32, [C.POINTER(deer_dynamics), C.c_int64, C.c_int64,
                                       C.c_void_p, C.c_void_p, C.c_void_p,
                                       C.POINTER(deer_options), C.c_void_p,
                                       C.POINTER(deer_info)]),
    "deer_noalloc_scratch_bytes": (C.c_size_t, []),
    "deer_kernel_launch_count": (C.c_int64, []),
    "deer_measure_peak": (C.c_int32, [C.c_int32, C.c_void_p, C.POINTER(C.c_double)]),
    "deer_selftest_wait_timeout": (C.c_int32, [C.c_void_p]),
    "deer_profile_enable": (None, [C.c_int32]),
    "deer_set_tensor_cores": (None, [C.c_int32]),
    "deer_lle_workspace_bytes": (C.c_size_t, [C.POINTER(deer_dynamics), C.c_int64, C.c_int64,
                                              C.c_int32]),
    "deer_lle": (C.c_int32, [C.POINTER(deer_dynamics), C.c_int64, C.c_int64, C.c_void_p,
                             C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32,
                             C.c_void_p, C.c_size_t, C.c_void_p]),
    "deer_get_tensor_cores": (C.c_int32, []),
    "deer_profile_reset": (None, []),
    "deer_profile_read": (None, [C.POINTER(deer_profile)]),
    "deer_status_string": (C.c_char_p, [C.c_int32]),
    "deer_last_cuda_error": (C.c_char_p, []),
    "deer_version": (C.c_int32, []),
}

_lib = None


def lib_path() -> str:
    return _LIB_PATH


def load():
    """Load libdeer.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError(
            f"{_LIB_PATH} is missing: build it first (python -c 'import __graft_entry__ as g; "
            "g.build()'); the solver has no CPU fallback")
    lib = C.CDLL(_LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class DeerError(RuntimeError):
    def __init__(self, status: int, where: str):
        lib = load()
        msg = lib.deer_status_string(status).decode()
        if status == DEER_ERR_CUDA:
            msg += ": " + lib.deer_last_cuda_error().decode()
        super().__init__(f"{where}: {msg} (status {status})")
        self.status = status
