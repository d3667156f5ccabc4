"""Sequential rollout and textbook (quasi-)Newton iterations, float64.

Test infrastructure only. Nothing here is blocked, fused or reordered: every
loop over t runs forward, one step at a time, exactly as the paper writes it.

Transition modes (Table fxd_pt_sum): 'full' (Newton / DEER, A_t = df_t/ds),
'diag' (quasi-Newton, diag[A_t], Eq. quasi_lds), 'identity' (Picard, A~=I),
'zero' (Jacobi, A~=0). Damping: 'scale' multiplies A~ by (1-k) (scale-ELK,
Sec. 4.5.1), 'clip' clips the diagonal of A~ to [-rho, rho] (clip-ELK,
Sec. 4.5.2), 'elk' replaces the LDS solve by the Kalman filter of Sec. 4.3
(see ``oracle.elk``).
"""
from __future__ import annotations

import numpy as np


def rollout(dyn, s0, T):
    """The plain definition of the answer: s*_t = f_t(s*_{t-1}), t = 1..T (Sec. 2.1).
    s0 [B, d] -> s [B, T, d]."""
    s0 = np.asarray(s0, dtype=np.float64)
    B, d = s0.shape
    out = np.empty((B, T, d))
    prev = s0
    for t in range(1, T + 1):
        prev = dyn.f(t, prev)
        out[:, t - 1] = prev
    return out


def residual(dyn, s0, s):
    """r_t(s) = s_t - f_t(s_{t-1}) for t = 1..T with s_0 fixed (Eq. r_def). [B, T, d]."""
    B, T, d = s.shape
    r = np.empty_like(s)
    prev = s0
    for t in range(1, T + 1):
        r[:, t - 1] = s[:, t - 1] - dyn.f(t, prev)
        prev = s[:, t - 1]
    return r


def transition(dyn, t, s_prev, mode="full", damp="none", damp_param=0.0):
    """The transition matrix A~_t of the LDS that one iteration solves, evaluated at
    s_{t-1} (Eq. lil_j; Table fxd_pt_sum; scale-/clip-ELK of Sec. 4.5). [B, d, d]."""
    B, d = s_prev.shape
    if mode == "full":
        A = dyn.jac(t, s_prev)
    elif mode == "diag":
        J = dyn.jac(t, s_prev)
        A = np.zeros_like(J)
        idx = np.arange(d)
        A[:, idx, idx] = J[:, idx, idx]
    elif mode == "identity":
        A = np.broadcast_to(np.eye(d), (B, d, d)).copy()
    elif mode == "zero":
        A = np.zeros((B, d, d))
    else:
        raise ValueError(mode)
    if damp == "scale":
        A = (1.0 - damp_param) * A
    elif damp == "clip":
        if mode == "full":
            raise ValueError("clip-ELK applies to the diagonal approximation only")
        idx = np.arange(d)
        A[:, idx, idx] = np.clip(A[:, idx, idx], -damp_param, damp_param)
    return A


def quasi_newton_step(dyn, s0, s, mode="full", damp="none", damp_param=0.0,
                      reset=False, reset_threshold=1e30, active=None):
    """One application of the LDS operator of Eq. gen_qdeer, written in the
    correction form of Eq. qdeer_lds and solved by forward substitution:

        s^{(i+1)}_t = f_t(s^{(i)}_{t-1}) + A~_t (s^{(i+1)}_{t-1} - s^{(i)}_{t-1}),  s_0 fixed.

    With mode='full' this is the DEER/Newton update (Eq. deer_lds / lin_rr).
    ``reset`` applies the reset heuristic (Sec. 3.2: overflowed entries may be set
    to a fixed value, here zero). ``active`` [B] bool limits the update to some
    sequences (others are returned unchanged)."""
    B, T, d = s.shape
    new = s.copy()
    new_prev = np.asarray(s0, dtype=np.float64)
    old_prev = np.asarray(s0, dtype=np.float64)
    for t in range(1, T + 1):
        F = dyn.f(t, old_prev)
        A = transition(dyn, t, old_prev, mode, damp, damp_param)
        v = F + np.einsum("bij,bj->bi", A, new_prev - old_prev)
        if active is not None:
            v = np.where(active[:, None], v, s[:, t - 1])
        new[:, t - 1] = v
        old_prev = s[:, t - 1]
        new_prev = v
    if reset:
        new = reset_overflow(new, reset_threshold)
    return new


def reset_overflow(s, threshold):
    """Reset heuristic (Sec. 3.2): entries of the new iterate that are non-finite or whose
    magnitude exceeds ``threshold`` are set to zero. Applied to the whole iterate once the
    linear recurrence has been solved (entries of the exact prefix are never touched)."""
    bad = ~np.isfinite(s) | (np.abs(s) > threshold)
    return np.where(bad, 0.0, s)


def scaled_residual_max(r, s):
    """max_t,i |r_t,i| / max(1, |s_t,i|) per sequence: the convergence measure. It is the
    absolute residual of Eq. r_def wherever |s| <= 1 and the relative one elsewhere."""
    return np.max(np.abs(r) / np.maximum(1.0, np.abs(s)), axis=(1, 2))


def initial_guess(dyn, s0, T, init="s0", user=None, seed=0):
    """s^{(0)} (Sec. 3.3.3): 'zeros'; 's0' (s_0 broadcast over t); 'jacobi' (one Jacobi
    step from zero, s_t^{(0)} = f_t(0)); 'randn' (iid N(0, 1) entries of the packed
    [B*T][d] state from the counter-based generator of ``oracle.rng``); 'user' (given)."""
    s0 = np.asarray(s0, dtype=np.float64)
    B, d = s0.shape
    if init == "zeros":
        return np.zeros((B, T, d))
    if init == "randn":
        from .rng import randn_guess
        return randn_guess(seed, B * T, d).reshape(B, T, d)
    if init == "s0":
        return np.repeat(s0[:, None, :], T, axis=1)
    if init == "jacobi":
        z = np.zeros((B, d))
        return np.stack([dyn.f(t, z) for t in range(1, T + 1)], axis=1)
    if init == "user":
        return np.array(user, dtype=np.float64, copy=True)
    raise ValueError(init)


def solve(dyn, s0, T, mode="full", damp="none", damp_param=0.0, tol=1e-10, max_iters=None,
          init="s0", user=None, reset=False, reset_threshold=1e30, record=False, confirm=1,
          seed=0):
    """Algorithm alg:deer (ParallelNewton), per sequence of the batch.

    Iteration i evaluates r(s^{(i)}); a sequence whose scaled residual
    max_t,i |r_t,i| / max(1, |s_t,i|) is <= tol is converged and keeps s^{(i)} (the error
    test of the algorithm, applied to the current iterate). Otherwise one LDS solve gives s^{(i+1)}. ``iters`` counts the LDS
    solves. The cap defaults to T, which suffices by Prop. global_convergence.
    With ``confirm`` > 1 a sequence converges only after that many consecutive iterates
    pass the test.
    """
    from . import elk as _elk

    s0 = np.asarray(s0, dtype=np.float64)
    B, d = s0.shape
    if max_iters is None:
        max_iters = T
    s = initial_guess(dyn, s0, T, init, user, seed)
    iters = np.zeros(B, dtype=np.int64)
    converged = np.zeros(B, dtype=bool)
    hist = []
    max_resid = np.full(B, np.inf)
    merit = np.full(B, np.inf)
    passes = np.zeros(B, dtype=np.int64)
    for i in range(max_iters + 1):
        r = residual(dyn, s0, s)
        mr = scaled_residual_max(r, s)
        mer = 0.5 * np.sum(r * r, axis=(1, 2))
        upd = ~converged
        max_resid[upd] = mr[upd]
        merit[upd] = mer[upd]
        if record:
            hist.append((mr.copy(), mer.copy()))
        passes = np.where(mr <= tol, passes + 1, 0)
        converged |= passes >= max(confirm, 1)
        if np.all(converged) or i == max_iters:
            break
        active = ~converged
        if damp == "elk":
            s = _elk.elk_filter_step(dyn, s0, s, mode=mode, lam=damp_param, active=active,
                                     reset=reset, reset_threshold=reset_threshold)
        else:
            s = quasi_newton_step(dyn, s0, s, mode, damp, damp_param, reset, reset_threshold, active)
        iters[active] += 1
    return {"s": s, "iters": iters, "converged": converged, "max_resid": max_resid,
            "merit": merit, "history": hist}


# --- brute force on tiny problems ----------------------------------------------

def dense_jacobian(dyn, s0, s, mode="full", damp="none", damp_param=0.0):
    """The TD x TD residual Jacobian of Eq. big_j for ONE sequence (s [T, d]):
    identity blocks on the diagonal, -A~_t on the block sub-diagonal (t = 2..T)."""
    T, d = s.shape
    J = np.eye(T * d)
    for t in range(2, T + 1):
        A = transition(dyn, t, s[None, t - 2], mode, damp, damp_param)[0]
        J[(t - 1) * d:t * d, (t - 2) * d:(t - 1) * d] = -A
    return J


def dense_newton_step(dyn, s0, s, mode="full", damp="none", damp_param=0.0):
    """s - J^{-1} r (Eq. deer_full_update) with J built densely and solved by LU (numpy),
    for ONE sequence. The reference for the forward-substitution update."""
    T, d = s.shape
    r = residual(dyn, s0[None], s[None])[0].reshape(-1)
    J = dense_jacobian(dyn, s0, s, mode, damp, damp_param)
    return s - np.linalg.solve(J, r).reshape(T, d)
