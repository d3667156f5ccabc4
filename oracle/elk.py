"""Damped (trust-region) steps: Levenberg-Marquardt and its Kalman forms, float64.

Test infrastructure only. For one iteration with current iterate s^{(i)} the LDS
has transition A~_t (per mode, at s^{(i)}_{t-1}) and offset
b_t = f_t(s^{(i)}_{t-1}) - A~_t s^{(i)}_{t-1} (Sec. 4.3, "Derivation").

* ``lm_step_dense``     - Delta s = -(J^T J + lambda I)^{-1} J^T r (Sec. 4.1), dense.
* ``elk_filter_step``   - the Kalman filter of Sec. 4.3: process noise I, emission
                          s_t^{(i)} ~ N(s_t, sigma^2 I) with sigma^2 = 1/lambda, prior
                          mu_0 = s_0, Sigma_0 = 0 (s_0 is known; Eq. lgssm). The filtered
                          means are the next iterate (the paper runs ELK as a filter).
* ``elk_smoother_step`` - RTS smoother of the same LGSSM; its means are the MAP, i.e.
                          the LM step (Prop. ELK).
"""
from __future__ import annotations

import numpy as np

from .newton import transition


def _lds_terms(dyn, s0, s, mode):
    """A~_t and b_t of the linearised dynamics for t = 1..T, [B, T, d, d] and [B, T, d]."""
    B, T, d = s.shape
    A = np.empty((B, T, d, d))
    b = np.empty((B, T, d))
    prev = s0
    for t in range(1, T + 1):
        At = transition(dyn, t, prev, mode)
        A[:, t - 1] = At
        b[:, t - 1] = dyn.f(t, prev) - np.einsum("bij,bj->bi", At, prev)
        prev = s[:, t - 1]
    return A, b


def kalman_filter(A, b, y, s0, lam):
    """Filtered means/covariances and one-step predictions of the LGSSM
    s_t = A_t s_{t-1} + b_t + N(0, I), y_t = s_t + N(0, I/lam), s_0 known.
    lam = 0 means no observation (the predict step alone: the DEER LDS)."""
    B, T, d = b.shape
    I = np.eye(d)
    mu = np.asarray(s0, dtype=np.float64)
    P = np.zeros((B, d, d))
    mus = np.empty((B, T, d))
    Ps = np.empty((B, T, d, d))
    mu_pred = np.empty((B, T, d))
    P_pred = np.empty((B, T, d, d))
    for t in range(T):
        At = A[:, t]
        m = np.einsum("bij,bj->bi", At, mu) + b[:, t]                 # predict mean
        S = At @ P @ np.swapaxes(At, 1, 2) + I                          # predict covariance
        mu_pred[:, t] = m
        P_pred[:, t] = S
        if lam > 0:
            sigma2 = 1.0 / lam
            K = S @ np.linalg.inv(S + sigma2 * I)                       # gain
            mu = m + np.einsum("bij,bj->bi", K, y[:, t] - m)            # update
            P = S - K @ S
        else:
            mu, P = m, S
        mus[:, t] = mu
        Ps[:, t] = P
    return mus, Ps, mu_pred, P_pred


def elk_filter_step(dyn, s0, s, mode="full", lam=1.0, active=None, reset=False,
                    reset_threshold=1e30):
    """One (quasi-)ELK iteration as the paper runs it: the filtered means of the
    LGSSM whose emissions are the previous iterate (Sec. 4.2 implementation details)."""
    A, b = _lds_terms(dyn, s0, s, mode)
    mus, _, _, _ = kalman_filter(A, b, s, s0, lam)
    if reset:
        from .newton import reset_overflow
        mus = reset_overflow(mus, reset_threshold)
    if active is not None:
        mus = np.where(active[:, None, None], mus, s)
    return mus


def elk_smoother_step(dyn, s0, s, mode="full", lam=1.0):
    """Rauch-Tung-Striebel smoothed means of the same LGSSM (the MAP, Prop. ELK)."""
    A, b = _lds_terms(dyn, s0, s, mode)
    mus, Ps, mu_pred, P_pred = kalman_filter(A, b, s, s0, lam)
    B, T, d = s.shape
    out = mus.copy()
    for t in range(T - 2, -1, -1):
        G = Ps[:, t] @ np.swapaxes(A[:, t + 1], 1, 2) @ np.linalg.inv(P_pred[:, t + 1])
        out[:, t] = mus[:, t] + np.einsum("bij,bj->bi", G, out[:, t + 1] - mu_pred[:, t + 1])
    return out


def lm_step_dense(dyn, s0, s, mode="full", lam=1.0):
    """Levenberg-Marquardt step for ONE sequence (s [T, d]) by dense linear algebra:
    s + Delta, Delta = -(J^T J + lambda I)^{-1} J^T r (Sec. 4.1)."""
    from .newton import dense_jacobian, residual

    T, d = s.shape
    r = residual(dyn, s0[None], s[None])[0].reshape(-1)
    J = dense_jacobian(dyn, s0, s, mode)
    H = J.T @ J + lam * np.eye(T * d)
    return s - np.linalg.solve(H, J.T @ r).reshape(T, d)


# --- the covariance recursion as an associative scan ------------------------------------
# Sarkka and Garcia-Fernandez ("Temporal parallelization of Bayesian smoothers", IEEE TAC
# 2021) write one filtering step as an element (A, C, J) acting on the incoming covariance
# P by P -> A (I + P J)^{-1} P A^T + C, with an associative combination, so the filtered
# covariances of all steps are a prefix scan. For this LGSSM (transition F_t = A~_t,
# process noise I, emission y_t = s_t + N(0, sigma^2 I), sigma^2 = 1/lambda) the step's
# element is A = c F_t, C = c I, J = lambda c F_t^T F_t with c = 1 / (1 + lambda).

def cov_element(F, lam):
    """Element (A, C, J) of one filtering step with transition F [B, d, d]."""
    B, d, _ = F.shape
    c = 1.0 / (1.0 + lam)
    return (c * F, np.broadcast_to(c * np.eye(d), (B, d, d)).copy(),
            lam * c * np.swapaxes(F, 1, 2) @ F)


def cov_combine(ei, ej):
    """e_i then e_j: A = A_j N A_i, C = A_j N C_i A_j^T + C_j, J = A_i^T N^T J_j A_i + J_i
    with N = (I + C_i J_j)^{-1}."""
    Ai, Ci, Ji = ei
    Aj, Cj, Jj = ej
    d = Ai.shape[-1]
    N = np.linalg.inv(np.eye(d) + Ci @ Jj)
    At = np.swapaxes
    return (Aj @ N @ Ai, Aj @ N @ Ci @ At(Aj, 1, 2) + Cj,
            At(Ai, 1, 2) @ At(N, 1, 2) @ Jj @ Ai + Ji)


def cov_apply(e, P):
    """The covariance after the steps of element e, entered with covariance P."""
    A, C, J = e
    d = A.shape[-1]
    return A @ np.linalg.inv(np.eye(d) + P @ J) @ P @ np.swapaxes(A, 1, 2) + C
