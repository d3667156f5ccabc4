"""Gradients through the recurrence at its fixed point, float64.

Test infrastructure only. For a loss l(s_{1:T}) with cotangents g_t = dl/ds_t:

* ``adjoint_grad``  - the reverse recursion of BPTT (Eq. bptt, bptt_lds, unrolled in
  Eq. unrolled_bwds): lambda_T = g_T, lambda_{t-1} = g_{t-1} + A_t^T lambda_t;
  dl/dtheta = sum_t lambda_t^T df_t/dtheta(s_{t-1}); dl/ds_0 = A_1^T lambda_1.
* ``forward_sensitivity_grad`` - Eq. bptt_lds run forward: S_t = A_t S_{t-1} +
  df_t/dtheta, dl/dtheta = sum_t g_t^T S_t (an independent route to the same number).
* ``fd_grad`` - central finite differences of the loss of the rollout.
* ``input_grad`` - dl/dx_t = lambda_t^T df_t/dx_t for inputs curried into f_t, pinned by
  ``fd_input_grad`` (central differences with respect to single input entries).
"""
from __future__ import annotations

import numpy as np

from .newton import rollout


def sq_loss(s, y):
    """l = sum_t ||s_t - y_t||^2 per sequence [B]."""
    return np.sum((s - y) ** 2, axis=(1, 2))


def sq_loss_cotangent(s, y):
    """g_t = dl/ds_t = 2 (s_t - y_t)."""
    return 2.0 * (s - y)


def adjoint_grad(dyn, s0, s, g):
    """Reverse-time adjoint recursion at the trajectory s (= s*), cotangents g [B,T,d].
    Returns (dl/dtheta [B, P], dl/ds0 [B, d], lambda [B, T, d])."""
    B, T, d = s.shape
    lam = np.empty_like(s)
    dtheta = np.zeros((B, dyn.n_params))
    cur = g[:, T - 1].copy()
    for t in range(T, 0, -1):
        prev = s[:, t - 2] if t >= 2 else s0
        lam[:, t - 1] = cur
        if dyn.n_params:
            dtheta += np.einsum("bi,bip->bp", cur, dyn.dparams(t, prev))
        back = np.einsum("bij,bi->bj", dyn.jac(t, prev), cur)           # A_t^T lambda_t
        cur = back + (g[:, t - 2] if t >= 2 else 0.0)
    ds0 = back
    return dtheta, ds0, lam


def input_grad(dyn, s0, s, lam):
    """dl/dx_t = lambda_t^T d f_t / d x_t (s_{t-1}) for every step, from the adjoint
    states lambda [B, T, d] of ``adjoint_grad`` (the inputs are curried into f_t,
    Sec. 2.1). Returns [B, T, d_in]."""
    B, T, d = s.shape
    out = []
    for t in range(1, T + 1):
        prev = s[:, t - 2] if t >= 2 else s0
        out.append(np.einsum("bi,bik->bk", lam[:, t - 1], dyn.dinputs(t, prev)))
    return np.stack(out, axis=1)


def fd_input_grad(make_dyn, x, s0, T, y, indices, h=1e-6):
    """Central differences of the rollout loss with respect to single input entries
    x[b, t, k] (indices (b, t, k)); make_dyn(x) -> dynamics."""
    out = []
    for (b, t, k) in indices:
        xp = np.array(x, dtype=np.float64, copy=True)
        xm = np.array(x, dtype=np.float64, copy=True)
        xp[b, t, k] += h
        xm[b, t, k] -= h
        lp = sq_loss(rollout(make_dyn(xp), s0, T), y)[b]
        lm = sq_loss(rollout(make_dyn(xm), s0, T), y)[b]
        out.append((lp - lm) / (2.0 * h))
    return np.array(out)


def forward_sensitivity_grad(dyn, s0, s, g):
    """dl/dtheta and dl/ds0 by forward sensitivities dS_t = A_t dS_{t-1} + df_t/dtheta."""
    B, T, d = s.shape
    P = dyn.n_params
    S = np.zeros((B, d, P))
    S0 = np.broadcast_to(np.eye(d), (B, d, d)).copy()
    dtheta = np.zeros((B, P))
    ds0 = np.zeros((B, d))
    prev = s0
    for t in range(1, T + 1):
        A = dyn.jac(t, prev)
        S = A @ S + (dyn.dparams(t, prev) if P else 0.0)
        S0 = A @ S0
        dtheta += np.einsum("bi,bip->bp", g[:, t - 1], S)
        ds0 += np.einsum("bi,bij->bj", g[:, t - 1], S0)
        prev = s[:, t - 1]
    return dtheta, ds0


def fd_grad(make_dyn, params, s0, T, y, indices, h=1e-6):
    """Central differences (l(theta + h e_j) - l(theta - h e_j)) / 2h of the rollout loss,
    for the parameter indices given as (b, j) pairs. make_dyn(params) -> dynamics."""
    out = []
    for (b, j) in indices:
        pp = np.array(params, dtype=np.float64, copy=True)
        pm = np.array(params, dtype=np.float64, copy=True)
        pp[b, j] += h
        pm[b, j] -= h
        lp = sq_loss(rollout(make_dyn(pp), s0, T), y)[b]
        lm = sq_loss(rollout(make_dyn(pm), s0, T), y)[b]
        out.append((lp - lm) / (2.0 * h))
    return np.array(out)
