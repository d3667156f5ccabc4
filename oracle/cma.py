"""Float64 mass-action oracle in plain C (oracle/c/massaction.c), for full-size checks.

Test infrastructure only. The same functions as ``dynamics.MassAction`` with
``newton.rollout`` and ``adjoint.adjoint_grad`` (Sec. 2.1; Eq. lil_j; Eq. bptt /
unrolled_bwds), computed one trajectory and one step at a time in C. A batch is split over
host threads (the C calls release the interpreter lock); ``threads`` defaults to every
core of the host. The library is built on first use (``oracle.build``).
"""
from __future__ import annotations

import ctypes as C
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from . import build as _build

_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(_build.build())
        p64, pi32, pd = C.POINTER(C.c_int64), C.POINTER(C.c_int32), C.POINTER(C.c_double)
        common = [C.c_int, C.c_int, C.c_int, C.c_double, p64, pi32, C.c_int64, pd, C.c_int64,
                  pd]
        lib.ora_ma_rollout.argtypes = common + [pd, C.c_int64, C.c_int64]
        lib.ora_ma_step_jacobians.argtypes = common + [pd, pd, C.c_int64, C.c_int64]
        lib.ora_ma_adjoint.argtypes = common + [pd, pd, pd, pd, C.c_int64, C.c_int64]
        for fn in (lib.ora_ma_rollout, lib.ora_ma_step_jacobians, lib.ora_ma_adjoint):
            fn.restype = C.c_int
        _lib = lib
    return _lib


def cores() -> int:
    return os.cpu_count() or 1


def _arr(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def _ptr(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


class Batch:
    """A batch of mass-action systems: topology [B][R][4] int, rate constants k [B][R],
    integrator 'euler' or 'rk4' with step dt, state size d."""

    def __init__(self, topology, k, dt, integrator="rk4", d=None):
        self.topo = _arr(topology, np.int32)
        self.k = _arr(k, np.float64)
        self.B, self.R = self.k.shape
        self.d = int(self.topo.max()) + 1 if d is None else int(d)
        self.dt = float(dt)
        self.rk4 = 1 if integrator == "rk4" else 0

    def _common(self, off):
        return (self.d, self.R, self.rk4, self.dt, _ptr(off, C.c_int64),
                _ptr(self.topo, C.c_int32), 4 * self.R, _ptr(self.k, C.c_double), self.R)

    def _split(self, fn, threads):
        threads = max(1, min(threads or cores(), self.B))
        edges = np.linspace(0, self.B, threads + 1).astype(np.int64)
        with ThreadPoolExecutor(max_workers=threads) as ex:
            rcs = list(ex.map(lambda i: fn(int(edges[i]), int(edges[i + 1])), range(threads)))
        if any(rc != 0 for rc in rcs):
            raise MemoryError("oracle work buffers")

    def rollout(self, s0, offsets, threads=None):
        """s_t = f(s_{t-1}) from s0 [B][d] over the packed rows of `offsets` [B+1] ->
        [N][d]."""
        lib = _load()
        off = _arr(offsets, np.int64)
        s0 = _arr(s0, np.float64)
        out = np.empty((int(off[-1]), self.d))
        args = self._common(off) + (_ptr(s0, C.c_double), _ptr(out, C.c_double))
        self._split(lambda lo, hi: lib.ora_ma_rollout(*args, lo, hi), threads)
        return out

    def step_jacobians(self, s0, s, offsets, threads=None):
        """A_t = df/ds at s_{t-1} for every packed row -> [N][d][d]."""
        lib = _load()
        off = _arr(offsets, np.int64)
        s0, s = _arr(s0, np.float64), _arr(s, np.float64)
        A = np.empty((int(off[-1]), self.d, self.d))
        args = self._common(off) + (_ptr(s0, C.c_double), _ptr(s, C.c_double),
                                    _ptr(A, C.c_double))
        self._split(lambda lo, hi: lib.ora_ma_step_jacobians(*args, lo, hi), threads)
        return A

    def adjoint(self, s0, s, g, offsets, threads=None):
        """dl/dk [B][R] and dl/ds0 [B][d] for cotangents g = dl/ds [N][d] at s [N][d]."""
        lib = _load()
        off = _arr(offsets, np.int64)
        s0, s, g = _arr(s0, np.float64), _arr(s, np.float64), _arr(g, np.float64)
        dk = np.empty((self.B, self.R))
        ds0 = np.empty((self.B, self.d))
        args = self._common(off) + (_ptr(s0, C.c_double), _ptr(s, C.c_double),
                                    _ptr(g, C.c_double), _ptr(dk, C.c_double),
                                    _ptr(ds0, C.c_double))
        self._split(lambda lo, hi: lib.ora_ma_adjoint(*args, lo, hi), threads)
        return dk, ds0


def uniform_offsets(B, T):
    return np.arange(B + 1, dtype=np.int64) * int(T)
