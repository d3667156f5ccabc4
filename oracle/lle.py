"""Largest Lyapunov exponent along a trajectory, float64 (test infrastructure only; see
the package docstring).

The thesis estimates the LLE of a recurrence by pushing a unit vector through the
Jacobians of the trajectory and renormalising it every step (Algorithm alg:LLE_estimate,
Ch. 5): u_t = J_t u_{t-1}, lambda_t = ||u_t||, u_t <- u_t / lambda_t, and the estimate is
(1/T) sum_t log lambda_t. J_t = df_t/ds evaluated at s_{t-1} (Eq. lil_j), s_0 the given
initial state. The loop below follows those steps one time step at a time.
"""
from __future__ import annotations

import numpy as np


def lle_estimate(dyn, s0, s, u0):
    """dyn: oracle dynamics; s0 [B, d]; s [B, T, d] the trajectory; u0 [B, d] unit
    vectors. Returns the estimate for every sequence, [B]."""
    s0 = np.asarray(s0, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64)
    u = np.asarray(u0, dtype=np.float64).copy()
    B, T, d = s.shape
    acc = np.zeros(B)
    prev = s0
    for t in range(1, T + 1):
        J = dyn.jac(t, prev)                      # [B, d, d] at s_{t-1}
        u = np.einsum("bij,bj->bi", J, u)         # evolved vector
        lam = np.linalg.norm(u, axis=1)           # stretch factor
        u = u / lam[:, None]                      # renormalise
        acc += np.log(lam)                        # accumulate the log stretch
        prev = s[:, t - 1]
    return acc / T
