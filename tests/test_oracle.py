"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test pins the oracle to something other than itself: printed values of a
worked example, closed forms, exact-arithmetic theorems, brute force on tiny
inputs, textbook special cases and finite differences.
"""
import json
import math
import os

import numpy as np
import pytest

import synth
from oracle import adjoint, dynamics, elk, newton

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _small_massaction(B=3, d=4, R=6, seed=0, integrator="rk4", dt=1e-2):
    p = synth.massaction(B, d, R, T=1, seed=seed, dt=dt, integrator=integrator)
    return dynamics.MassAction(p["topology"], p["params"], dt, integrator, d=d), p


def _small_gru(B=2, T=12, d=4, seed=0):
    p = synth.gru(B, T, d, d, seed)
    return dynamics.GRU(p["W"], p["U"], p["x"]), p


def _fd_jac(f, s, h=1e-6):
    B, d = s.shape
    J = np.empty((B, d, d))
    for j in range(d):
        e = np.zeros(d)
        e[j] = h
        J[:, :, j] = (f(s + e) - f(s - e)) / (2 * h)
    return J


# --- worked example (Appendix A) ----------------------------------------------

def test_worked_example_tang():
    g = json.load(open(os.path.join(GOLDEN, "tang_example.json")))
    dyn = dynamics.Linear(np.array([[2.0]]))
    s0 = np.array([[g["s0"]]])
    T = g["T"]
    s_star = newton.rollout(dyn, s0, T)[0, :, 0]
    assert np.array_equal(s_star, g["s_star"])
    s = np.array(g["s_init"]).reshape(1, T, 1)
    r = newton.residual(dyn, s0, s)[0, :, 0]
    assert np.array_equal(r, g["r_init"])
    # the update s - G r with the non-lower-triangular G of the counterexample
    G = np.array(g["G_not_lower_triangular"])
    cur = np.array(g["s_init"])
    for expect in g["update_iterates"]:
        rr = newton.residual(dyn, s0, cur.reshape(1, T, 1))[0, :, 0]
        cur = cur - G @ rr
        assert np.array_equal(cur, expect)
    # DEER (G = J^{-1}) from the same start reaches s* in one iteration
    one = newton.quasi_newton_step(dyn, s0, s, "full")[0, :, 0]
    assert np.array_equal(one, g["s_star"])
    out = newton.solve(dyn, s0, T, "full", tol=0.0, init="user", user=s)
    assert out["iters"][0] == 1 and out["converged"][0]


# --- dynamics pinned by closed forms / invariants / finite differences ------------

def test_brusselator_stationary_point_and_textbook_jacobian():
    a, b = 1.0, 3.0
    dyn = dynamics.Brusselator(np.array([[a, b]]), 0.01)
    fp = np.array([[a, b / a]])
    assert np.allclose(dyn.rhs(fp), 0.0, atol=1e-15)
    # textbook linearisation of the Brusselator at (a, b/a): [[b-1, a^2], [-b, -a^2]]
    assert np.allclose(dyn.rhs_jac(fp)[0], [[b - 1, a * a], [-b, -a * a]], atol=1e-14)
    s = np.array([[0.7, 2.1]])
    assert np.allclose(dyn.jac(1, s), _fd_jac(lambda v: dyn.f(1, v), s), rtol=1e-8, atol=1e-10)
    # explicit Euler: f(s) = s + dt g(s)
    assert np.allclose(dyn.f(1, s), s + 0.01 * dyn.rhs(s), rtol=0, atol=1e-15)


@pytest.mark.parametrize("integrator", ["euler", "rk4"])
def test_massaction_conservation_and_jacobian_fd(integrator):
    dyn, p = _small_massaction(B=4, d=6, R=9, seed=3, integrator=integrator)
    rng = np.random.default_rng(0)
    c = rng.uniform(0.1, 1.0, size=(4, 6))
    m = p["masses"].astype(np.float64)
    # every reaction conserves sum_i m_i c_i
    assert np.allclose(np.sum(m * dyn.rhs(c), axis=1), 0.0, atol=1e-12)
    assert np.allclose(np.sum(m * dyn.f(1, c), axis=1), np.sum(m * c, axis=1), atol=1e-12)
    assert np.allclose(dyn.rhs_jac(c), _fd_jac(dyn.rhs, c), rtol=1e-7, atol=1e-9)
    assert np.allclose(dyn.jac(1, c), _fd_jac(lambda v: dyn.f(1, v), c), rtol=1e-7, atol=1e-9)
    # d f / d k by central differences on each rate constant
    P = dyn.dparams(1, c)
    for r in range(p["R"]):
        kp = p["params"].copy(); kp[:, r] += 1e-6
        km = p["params"].copy(); km[:, r] -= 1e-6
        fp_ = dynamics.MassAction(p["topology"], kp, dyn.dt, integrator, d=6).f(1, c)
        fm_ = dynamics.MassAction(p["topology"], km, dyn.dt, integrator, d=6).f(1, c)
        assert np.allclose(P[:, :, r], (fp_ - fm_) / 2e-6, rtol=1e-6, atol=1e-10)


def test_rk4_is_quartic_taylor_on_linear_network():
    """On a conversion-only network g(c) = M c, so one classical RK4 step equals
    the degree-4 Taylor polynomial of exp(hM) applied to s; its error against the
    exact flow shrinks ~2^5 per halving of h (local order 5)."""
    from scipy.linalg import expm
    net = synth.linear_conversion_network(d=5, R=8, seed=1)
    d = 5
    for h in (0.05, 0.1):
        dyn = dynamics.MassAction(net["topology"], net["params"], h, "rk4", d=d)
        M = np.stack([dyn.rhs(np.eye(d)[j][None])[0] for j in range(d)], axis=1)  # columns g(e_j)
        hM = h * M
        P4 = np.eye(d) + hM + hM @ hM / 2 + hM @ hM @ hM / 6 + hM @ hM @ hM @ hM / 24
        s = net["s0"]
        assert np.allclose(dyn.f(1, s)[0], P4 @ s[0], rtol=1e-13, atol=1e-15)
    errs = []
    for h in (0.2, 0.1):
        dyn = dynamics.MassAction(net["topology"], net["params"], h, "rk4", d=d)
        M = np.stack([dyn.rhs(np.eye(d)[j][None])[0] for j in range(d)], axis=1)
        errs.append(np.linalg.norm(dyn.f(1, net["s0"])[0] - expm(h * M) @ net["s0"][0]))
    ratio = errs[0] / errs[1]
    assert 20 < ratio < 45


def test_gru_special_cases_and_jacobian():
    d = 4
    rng = np.random.default_rng(5)
    h = rng.uniform(-0.9, 0.9, size=(1, d))
    x = rng.standard_normal((1, 1, d))
    zero = np.zeros((3, d, d))
    # W = U = 0: z = r = 1/2, h~ = 0, so h' = h / 2
    g0 = dynamics.GRU(zero, zero, x)
    assert np.allclose(g0.f(1, h), 0.5 * h, atol=1e-15)
    # update gate saturated open (W_z x = +50) and U = 0: h' = tanh(W_h x)
    W = np.zeros((3, d, d))
    W[0] = np.eye(d) * (50.0 / x[0, 0])[:, None]
    W[2] = rng.standard_normal((d, d))
    g1 = dynamics.GRU(W, zero, x)
    assert np.allclose(g1.f(1, h), np.tanh(W[2] @ x[0, 0]), atol=1e-12)
    # update gate saturated closed (W_z x = -50): h' = h
    W[0] = -W[0]
    g2 = dynamics.GRU(W, zero, x)
    assert np.allclose(g2.f(1, h), h, atol=1e-12)
    dyn, _ = _small_gru(B=3, T=2, d=5, seed=2)
    s = np.random.default_rng(1).uniform(-0.8, 0.8, size=(3, 5))
    assert np.allclose(dyn.jac(1, s), _fd_jac(lambda v: dyn.f(1, v), s), rtol=1e-7, atol=1e-9)


# --- Prop. global_convergence (exact-arithmetic, bitwise in correction form) -------

class _RandomTransition:
    """Wraps a dynamics object but reports an arbitrary (random) matrix as its Jacobian,
    so that mode='full' runs Eq. gen_qdeer with arbitrary A~_t."""

    def __init__(self, dyn, seed):
        self.dyn, self.d, self.rng = dyn, dyn.d, np.random.default_rng(seed)
        self.n_params = 0

    def f(self, t, s):
        return self.dyn.f(t, s)

    def jac(self, t, s):
        return 0.3 * self.rng.standard_normal((s.shape[0], self.d, self.d))


@pytest.mark.parametrize("mode", ["full", "diag", "identity", "zero", "random"])
def test_prefix_exactness_and_T_iterations(mode):
    dyn, p = _small_massaction(B=2, d=4, R=6, seed=7)
    T = 24
    s0 = p["s0"]
    if mode == "random":
        dyn, mode = _RandomTransition(dyn, 11), "full"
    s_star = newton.rollout(dyn, s0, T)
    s = newton.initial_guess(dyn, s0, T, "zeros")
    for i in range(1, T + 1):
        s = newton.quasi_newton_step(dyn, s0, s, mode)
        # after iteration i the first i states are exactly the rollout
        assert np.array_equal(s[:, :i], s_star[:, :i])
    assert np.array_equal(s, s_star)
    out = newton.solve(dyn, s0, T, mode, tol=0.0, init="zeros")
    assert np.all(out["converged"]) and np.all(out["iters"] <= T)


def test_linear_recurrence_converges_in_one_iteration():
    lds = synth.linear_lds(B=3, T=40, d=5, seed=2)
    dyn = dynamics.Linear(lds["A"], lds["x"])
    out = newton.solve(dyn, lds["s0"], 40, "full", tol=1e-11, init="zeros")
    assert np.all(out["iters"] == 1)
    assert np.allclose(out["s"], newton.rollout(dyn, lds["s0"], 40), rtol=1e-12, atol=1e-12)
    # diagonal linear dynamics: quasi-DEER is exact, also one iteration
    ldd = synth.linear_lds(B=2, T=40, d=4, seed=3, diagonal=True)
    dd = dynamics.Linear(ldd["A"], ldd["x"])
    assert np.all(newton.solve(dd, ldd["s0"], 40, "diag", tol=1e-11, init="zeros")["iters"] == 1)
    # a permutation LDS (group word problem, Sec. 6.4): one Newton iteration
    perm = np.eye(5)[np.random.default_rng(0).permutation(5)]
    dp = dynamics.Linear(perm, lds["x"][:, :, :5])
    assert np.all(newton.solve(dp, lds["s0"], 40, "full", tol=1e-11, init="zeros")["iters"] == 1)


@pytest.mark.parametrize("which", ["massaction", "gru", "brusselator"])
@pytest.mark.parametrize("mode", ["full", "diag"])
def test_forward_substitution_equals_dense_lu(which, mode):
    """One (quasi-)Newton update by forward substitution equals s - J~^{-1} r with the
    block-bidiagonal J~ of Eq. big_j built explicitly and LU-solved (T d <= 256)."""
    if which == "massaction":
        dyn, p = _small_massaction(B=1, d=4, R=6, seed=1)
        s0, T = p["s0"], 40
    elif which == "gru":
        dyn, p = _small_gru(B=1, T=32, d=6, seed=4)
        s0, T = p["s0"], 32
    else:
        pb = synth.brusselator(T=64)
        dyn, s0, T = dynamics.Brusselator(pb["params"], pb["dt"]), pb["s0"], 64
    s = newton.initial_guess(dyn, s0, T, "zeros") + 0.3 * np.random.default_rng(0).standard_normal((1, T, dyn.d))
    a = newton.quasi_newton_step(dyn, s0, s, mode)[0]
    b = newton.dense_newton_step(dyn, s0[0], s[0], mode)
    assert np.allclose(a, b, rtol=1e-11, atol=1e-12)


def test_J_inverse_blocks_are_products():
    """Eq. J_inv: block (t, tau) of J^{-1} is A_t A_{t-1} ... A_{tau+1}."""
    dyn, p = _small_massaction(B=1, d=3, R=5, seed=2)
    T, d = 4, 3
    s = np.random.default_rng(1).uniform(0, 1, size=(T, d))
    Jinv = np.linalg.inv(newton.dense_jacobian(dyn, p["s0"][0], s))
    A = [None] + [dyn.jac(t, s[None, t - 2])[0] for t in range(2, T + 1)]
    for t in range(1, T + 1):
        for tau in range(1, t + 1):
            blk = Jinv[(t - 1) * d:t * d, (tau - 1) * d:tau * d]
            prod = np.eye(d)
            for k in range(tau + 1, t + 1):
                prod = A[k - 1] @ prod
            assert np.allclose(blk, prod, atol=1e-13)
    for t in range(1, T + 1):
        for tau in range(t + 1, T + 1):
            assert np.all(Jinv[(t - 1) * d:t * d, (tau - 1) * d:tau * d] == 0)


def test_jacobi_error_closed_form_and_slope():
    """s_{t+1} = alpha s_t, Jacobi from zeros: e_t^{(i)} = 0 for t <= i and -alpha^t s_0
    otherwise, so log10 ||e^{(i)}|| falls with slope log10(alpha) (Sec. 6.3)."""
    alpha, T = 0.5, 60
    dyn = dynamics.Linear(np.eye(2) * alpha)
    s0 = np.array([[1.0, -2.0]])
    s_star = newton.rollout(dyn, s0, T)
    s = np.zeros((1, T, 2))
    norms = []
    for i in range(1, 30):
        s = newton.quasi_newton_step(dyn, s0, s, "zero")
        e = s - s_star
        t = np.arange(1, T + 1)
        expect = np.where((t <= i)[:, None], 0.0, -(alpha ** t)[:, None] * s0[0][None])
        assert np.allclose(e[0], expect, rtol=1e-14, atol=0)
        norms.append(np.linalg.norm(e))
    slope = np.polyfit(np.arange(1, 30), np.log10(norms), 1)[0]
    assert abs(slope - math.log10(alpha)) < 1e-6


@pytest.mark.parametrize("T", [3, 5, 10, 33])
def test_picard_inverse_norm_closed_form(T):
    """Lemma PicardNorm: ||J~_P^{-1}||_2 = 1 / (2 sin(pi / (2 (2T + 1))))."""
    dyn = dynamics.Linear(np.eye(2) * 0.3)
    J = newton.dense_jacobian(dyn, np.zeros(2), np.zeros((T, 2)), mode="identity")
    got = np.linalg.norm(np.linalg.inv(J), 2)
    assert abs(got - 1.0 / (2.0 * math.sin(math.pi / (2 * (2 * T + 1))))) < 1e-10 * got


def test_picard_is_prefix_sum_of_euler_increments():
    """Prop. picard on an Euler ODE: s_{t+1}^{(i+1)} = s_0 + sum_{tau<=t} g(s_tau^{(i)}) dt."""
    pb = synth.brusselator(T=50)
    dyn = dynamics.Brusselator(pb["params"], pb["dt"])
    s0 = pb["s0"]
    s = 1.0 + 0.1 * np.random.default_rng(2).standard_normal((1, 50, 2))
    got = newton.quasi_newton_step(dyn, s0, s, "identity")[0]
    prev = np.concatenate([s0, s[0, :-1]], axis=0)
    incr = pb["dt"] * dyn.rhs(prev)
    expect = s0[0] + np.cumsum(incr, axis=0)
    assert np.allclose(got, expect, rtol=1e-13, atol=1e-13)


# --- fixed point, rates ------------------------------------------------------

@pytest.mark.parametrize("mode", ["full", "diag", "identity", "zero"])
def test_fixed_point_is_rollout_nonlinear(mode):
    dyn, p = _small_gru(B=2, T=48, d=4, seed=9)
    out = newton.solve(dyn, p["s0"], 48, mode, tol=1e-13, init="zeros")
    assert np.all(out["converged"])
    assert np.allclose(out["s"], newton.rollout(dyn, p["s0"], 48), rtol=0, atol=1e-12)


def _order(r):
    """Observed order of convergence: slope of log r_{i+1} against log r_i."""
    r = np.log(np.asarray(r))
    return np.polyfit(r[:-1], r[1:], 1)[0]


def test_newton_tail_is_quadratic_and_quasi_is_linear():
    """Basin of quadratic convergence (Thm. basin_size): ||r^+|| <= (L/2mu) ||r||^2 for
    Newton; the diagonal quasi-Newton update converges only linearly."""
    pb = synth.brusselator(T=256)
    dyn = dynamics.Brusselator(pb["params"], pb["dt"])
    full = newton.solve(dyn, pb["s0"], 256, "full", tol=1e-300, max_iters=40, init="s0", record=True)
    r = np.array([h[0][0] for h in full["history"]])
    r = r[r > 1e-13][-3:]
    assert _order(r) > 1.7
    md, pd = _small_massaction(B=1, d=4, R=6, seed=3, dt=0.05)
    quasi = newton.solve(md, pd["s0"], 200, "diag", tol=1e-300, max_iters=60, init="s0", record=True)
    rq = np.array([h[0][0] for h in quasi["history"]])
    rq = rq[(rq > 1e-13) & (rq < 1e-4)]
    assert len(rq) >= 8
    assert 0.8 < _order(rq) < 1.25


def test_reset_heuristic_keeps_global_convergence():
    """An expanding linearisation overflows; resetting overflowed entries to zero still
    converges within T iterations (Sec. 3.2)."""
    dyn = dynamics.Linear(np.array([[3.0]]))
    rng = np.random.default_rng(0)
    dyn.x = rng.standard_normal((1, 40, 1))
    T = 40
    tiny = _RandomTransition(dyn, 3)
    tiny.jac = lambda t, s: np.full((s.shape[0], 1, 1), 1e12)
    out = newton.solve(tiny, np.zeros((1, 1)), T, "full", tol=0.0, init="zeros", reset=True,
                       reset_threshold=1e30)
    assert out["converged"][0] and out["iters"][0] <= T
    assert np.array_equal(out["s"], newton.rollout(dyn, np.zeros((1, 1)), T))


# --- damped (ELK) --------------------------------------------------------------

@pytest.mark.parametrize("mode", ["full", "diag"])
def test_lm_step_is_kalman_smoother_mean(mode):
    dyn, p = _small_gru(B=1, T=24, d=3, seed=6)
    s = 0.5 * np.random.default_rng(3).standard_normal((1, 24, 3))
    lam = 2.5
    lm = elk.lm_step_dense(dyn, p["s0"][0], s[0], mode, lam)
    sm = elk.elk_smoother_step(dyn, p["s0"], s, mode, lam)[0]
    assert np.allclose(lm, sm, rtol=1e-10, atol=1e-11)
    filt = elk.elk_filter_step(dyn, p["s0"], s, mode, lam)[0]
    assert np.allclose(filt[-1], sm[-1], rtol=1e-10, atol=1e-11)
    assert not np.allclose(filt[0], sm[0], atol=1e-6)


def test_elk_limits_and_scale_clip_reductions():
    dyn, p = _small_gru(B=2, T=20, d=3, seed=8)
    s = 0.5 * np.random.default_rng(4).standard_normal((2, 20, 3))
    s0 = p["s0"]
    deer = newton.quasi_newton_step(dyn, s0, s, "full")
    # lambda -> 0 (sigma^2 -> inf): the ELK filter step is the DEER step
    assert np.allclose(elk.elk_filter_step(dyn, s0, s, "full", lam=0.0), deer, rtol=1e-12, atol=1e-12)
    assert np.allclose(elk.elk_filter_step(dyn, s0, s, "full", lam=1e-12), deer, rtol=1e-8, atol=1e-9)
    # huge lambda: the step stays at the previous iterate (vanishing trust region)
    assert np.allclose(elk.elk_filter_step(dyn, s0, s, "full", lam=1e12), s, atol=1e-9)
    # scale-ELK: k = 0 is DEER, k = 1 is Jacobi
    assert np.allclose(newton.quasi_newton_step(dyn, s0, s, "full", "scale", 0.0), deer, atol=1e-14)
    assert np.allclose(newton.quasi_newton_step(dyn, s0, s, "full", "scale", 1.0),
                       newton.quasi_newton_step(dyn, s0, s, "zero"), atol=1e-14)
    # clip-ELK equals quasi-DEER when the clip bound is never active
    prev = np.concatenate([s0[:, None], s[:, :-1]], axis=1)
    amax = max(np.max(np.abs(np.diagonal(dyn.jac(t, prev[:, t - 1]), axis1=1, axis2=2)))
               for t in range(1, 21))
    assert np.allclose(newton.quasi_newton_step(dyn, s0, s, "diag", "clip", amax + 1e-9),
                       newton.quasi_newton_step(dyn, s0, s, "diag"), atol=1e-14)
    assert not np.allclose(newton.quasi_newton_step(dyn, s0, s, "diag", "clip", 0.5 * amax),
                           newton.quasi_newton_step(dyn, s0, s, "diag"), atol=1e-6)
    # ... and with rho = 0 it is Jacobi
    assert np.allclose(newton.quasi_newton_step(dyn, s0, s, "diag", "clip", 0.0),
                       newton.quasi_newton_step(dyn, s0, s, "zero"), atol=1e-14)


def test_elk_attenuation_bound():
    """Sec. 4.3: the filtered mean is an LDS with transition Gamma_t A_t and
    ||Gamma_t||_2 <= 1 / (1 + lambda). Check the scalar case numerically."""
    lam = 3.0
    sigma2 = 1.0 / lam
    rng = np.random.default_rng(0)
    a = rng.uniform(-2, 2, size=100)
    P = 0.0
    for at in a:
        Pm = at * at * P + 1.0
        gamma = sigma2 / (Pm + sigma2)
        assert gamma <= 1.0 / (1.0 + lam) + 1e-15
        P = gamma * Pm


# --- adjoint -----------------------------------------------------------------

def test_adjoint_equals_forward_sensitivity_and_fd():
    dyn, p = _small_massaction(B=2, d=4, R=6, seed=5, dt=1e-2)
    T = 30
    s0 = p["s0"]
    s = newton.rollout(dyn, s0, T)
    kp = synth.perturbed_rates(p["params"], seed=1)
    y = newton.rollout(dynamics.MassAction(p["topology"], kp, dyn.dt, "rk4", d=4), s0, T)
    g = adjoint.sq_loss_cotangent(s, y)
    dth, ds0, _ = adjoint.adjoint_grad(dyn, s0, s, g)
    fth, fs0 = adjoint.forward_sensitivity_grad(dyn, s0, s, g)
    assert np.allclose(dth, fth, rtol=1e-10, atol=1e-14)
    assert np.allclose(ds0, fs0, rtol=1e-10, atol=1e-14)
    mk = lambda k: dynamics.MassAction(p["topology"], k, dyn.dt, "rk4", d=4)
    idx = [(0, 0), (0, 3), (1, 2), (1, 5)]
    fd = adjoint.fd_grad(mk, p["params"], s0, T, y, idx, h=1e-6)
    got = np.array([dth[b, j] for b, j in idx])
    assert np.allclose(got, fd, rtol=1e-5, atol=1e-9)


# ---------------------------------------------------------------------------
# Largest Lyapunov exponent (Algorithm alg:LLE_estimate)
# ---------------------------------------------------------------------------
def test_lle_diagonal_linear_closed_form():
    """For a constant diagonal Jacobian the renormalised products telescope:
    the estimate is (1/T) log ||A^T u0|| = (1/(2T)) log sum_i a_i^(2T) u0_i^2."""
    from oracle import lle
    rng = np.random.default_rng(3)
    d, T, B = 5, 60, 3
    a = rng.uniform(0.4, 1.6, size=d) * rng.choice([-1.0, 1.0], size=d)
    u0 = rng.standard_normal((B, d))
    u0 /= np.linalg.norm(u0, axis=1, keepdims=True)
    dyn = dynamics.Linear(np.diag(a))
    s = newton.rollout(dyn, np.zeros((B, d)), T)
    got = lle.lle_estimate(dyn, np.zeros((B, d)), s, u0)
    want = 0.5 * np.log((a[None, :] ** (2 * T) * u0 ** 2).sum(axis=1)) / T
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-14)


def test_lle_linear_tends_to_log_spectral_radius():
    """A constant non-normal Jacobian with known eigenvalues: the estimate approaches
    log of the spectral radius at the rate 1/T."""
    from oracle import lle
    rng = np.random.default_rng(4)
    d = 4
    lam = np.array([0.9, -1.3, 0.5, 0.2])
    Q = rng.standard_normal((d, d)) + 2 * np.eye(d)
    A = Q @ np.diag(lam) @ np.linalg.inv(Q)
    dyn = dynamics.Linear(A)
    u0 = rng.standard_normal((2, d))
    u0 /= np.linalg.norm(u0, axis=1, keepdims=True)
    errs = []
    for T in (250, 2000):
        s = newton.rollout(dyn, np.zeros((2, d)), T)
        errs.append(np.abs(lle.lle_estimate(dyn, np.zeros((2, d)), s, u0) - np.log(1.3)).max())
    assert errs[1] < 2e-3 and errs[1] < errs[0] / 4


def test_lle_mass_action_bounded_below_by_conservation():
    """A mass-conserving network: m^T J_t = m^T for every step Jacobian, so
    ||J_T..J_1 u0|| >= |m^T u0| / ||m|| and the estimate is at least
    (1/T) log(|m^T u0| / ||m||); it is also at most 0 up to O(1/T) for these relaxing
    networks (the mass direction is neutral, every other mode decays)."""
    from oracle import lle
    p = synth.massaction(3, 6, 9, 800, seed=5)
    dyn = dynamics.MassAction(p["topology"], p["params"], p["dt"], "rk4", d=6)
    s = newton.rollout(dyn, p["s0"], 800)
    rng = np.random.default_rng(6)
    u0 = rng.standard_normal((3, 6))
    u0 /= np.linalg.norm(u0, axis=1, keepdims=True)
    got = lle.lle_estimate(dyn, p["s0"], s, u0)
    m = p["masses"].astype(np.float64)  # per system
    lower = np.log(np.abs((u0 * m).sum(axis=1)) / np.linalg.norm(m, axis=1)) / 800
    assert np.all(got >= lower - 1e-12)
    assert np.all(got <= 0.05)


# --- second workloads: mean-field RNN, two-well Langevin, Lorenz-96, word problem ------

def test_rnn_jacobian_matches_fd_and_has_zero_diagonal():
    """A = W diag(1 - tanh^2) against central differences; with W_ii = 0 (no
    self-coupling, Sec. ssc:exp_thresh) the diagonal of every step Jacobian is zero, so
    quasi-DEER coincides with Jacobi on this family."""
    p = synth.mean_field_rnn(3, 4, 6, 1.5, seed=2)
    dyn = dynamics.MeanFieldRNN(p["W"], p["x"])
    s = np.random.default_rng(3).standard_normal((3, 6))
    J = dyn.jac(2, s)
    assert np.abs(J - _fd_jac(lambda v: dyn.f(2, v), s)).max() < 1e-8
    assert np.all(np.diagonal(J, axis1=1, axis2=2) == 0.0)


def test_rnn_without_coupling_returns_its_input():
    """g = 0 gives W = 0: s_t = u_t exactly."""
    p = synth.mean_field_rnn(2, 20, 4, 0.0, seed=0)
    s = newton.rollout(dynamics.MeanFieldRNN(p["W"], p["x"]), p["s0"], 20)
    assert np.array_equal(s, p["x"])


def test_rnn_threshold_between_predictable_and_chaotic():
    """Sec. ssc:exp_thresh: the LLE rises with the gain g and changes sign; DEER needs a
    handful of iterations for the predictable network and an order of magnitude more
    for the chaotic one (Theorem PL-LLE)."""
    from oracle import lle
    u0 = np.ones((1, 16)) / 4.0
    lles, its = [], []
    for g in (0.5, 1.0, 2.0, 3.0):
        p = synth.mean_field_rnn(1, 200, 16, g, seed=1)
        dyn = dynamics.MeanFieldRNN(p["W"], p["x"])
        s = newton.rollout(dyn, p["s0"], 200)
        lles.append(float(lle.lle_estimate(dyn, p["s0"], s, u0)[0]))
        if g in (0.5, 2.0):
            its.append(int(newton.solve(dyn, p["s0"], 200, mode="full", tol=1e-10,
                                        init="zeros")["iters"][0]))
    assert all(a < b for a, b in zip(lles, lles[1:]))
    assert lles[0] < 0.0 < lles[2]
    assert its[0] <= 5 and its[1] >= 10 * its[0]


def _mixture_potential(dyn, s):
    """-log(w1 N(s; m1, v1) + w2 N(s; m2, v2)) straight from the Gaussian densities."""
    def dens(m, v):
        return np.exp(-0.5 * np.sum(np.log(2 * np.pi * v) + (s - m) ** 2 / v, axis=1))
    return -np.log(dyn.w1 * dens(dyn.m1, dyn.v1) + dyn.w2 * dens(dyn.m2, dyn.v2))


def test_langevin_gradient_and_jacobian_match_fd():
    """grad phi against central differences of the potential written from the densities,
    and A = I - eps Hess phi against central differences of f."""
    p = synth.two_well(4, 3, 3, seed=1)
    dyn = dynamics.TwoWellLangevin(p["params"], p["dt"], p["x"], d=3)
    s = np.random.default_rng(2).standard_normal((4, 3)) * 1.5
    h = 1e-5
    fd = np.stack([(_mixture_potential(dyn, s + h * e) - _mixture_potential(dyn, s - h * e))
                   / (2 * h) for e in np.eye(3)], axis=1)
    assert np.abs(dyn.grad_phi(s) - fd).max() < 1e-8
    J = dyn.jac(1, s)
    assert np.abs(J - _fd_jac(lambda v: dyn.f(1, v), s)).max() < 1e-9
    assert np.allclose(J, np.transpose(J, (0, 2, 1)))  # I - eps Hess is symmetric


def test_langevin_one_component_is_ornstein_uhlenbeck():
    """With w2 = 0 the potential is one Gaussian: f is affine with the constant Jacobian
    I - eps diag(1/v1), so DEER converges in one iteration and Jacobi needs T."""
    p = synth.two_well(2, 40, 2, seed=3)
    prm = p["params"].copy()
    prm[-1] = 0.0
    dyn = dynamics.TwoWellLangevin(prm, p["dt"], p["x"], d=2)
    s = np.random.default_rng(4).standard_normal((2, 2)) * 3.0
    assert np.allclose(dyn.jac(1, s), np.diag(1.0 - p["dt"] / prm[4:6])[None], atol=1e-15)
    exp = s - p["dt"] * (s - prm[0:2]) / prm[4:6] + np.sqrt(2 * p["dt"]) * p["x"][:, 0]
    assert np.allclose(dyn.f(1, s), exp, rtol=1e-14, atol=1e-14)
    r = newton.solve(dyn, p["s0"], 40, mode="full", tol=1e-12, init="zeros")
    assert list(r["iters"]) == [1, 1]
    rj = newton.solve(dyn, p["s0"], 40, mode="zero", tol=1e-12, init="zeros")
    assert list(rj["iters"]) == [40, 40]


def test_langevin_unstable_between_wells_contracting_inside():
    """Sec. ssc:2well: the step is expanding between the wells (negative curvature of
    phi) and contracting at the bottom of a well."""
    p = synth.two_well(1, 1, 2, seed=0)
    dyn = dynamics.TwoWellLangevin(p["params"], p["dt"], d=2)
    mid = np.array([[0.0, 0.1]])
    well = np.array([[0.0, 1.6]])
    assert np.linalg.norm(dyn.jac(1, mid)[0], 2) > 1.0
    assert np.linalg.norm(dyn.jac(1, well)[0], 2) < 1.0


def test_langevin_deer_converges_fast_jacobi_needs_T():
    """Sec. ssc:2well / sec:WellExp: from a random initial guess DEER converges in a few
    iterations, growing sublinearly in T; Picard takes far fewer than T and Jacobi
    exactly T."""
    its = {}
    for T in (100, 400):
        p = synth.two_well(1, T, 2, seed=0)
        dyn = dynamics.TwoWellLangevin(p["params"], p["dt"], p["x"], d=2)
        guess = synth.targets_noise((1, T, 2), seed=5)
        its[T] = {m: int(newton.solve(dyn, p["s0"], T, mode=m, tol=1e-10, init="user",
                                      user=guess)["iters"][0])
                  for m in ("full", "identity", "zero")}
    assert its[100]["full"] <= 10 and its[400]["full"] <= 2 * its[100]["full"]
    assert its[400]["identity"] < 400 // 2
    assert its[100]["zero"] == 100 and its[400]["zero"] == 400


def test_dp5_tableau_satisfies_the_order_conditions():
    """Every coefficient of the Dormand-Prince tableau is pinned by the row-sum condition
    c = A 1 and by the 17 Butcher order conditions up to order five (rooted trees)."""
    A, b, c = dynamics.DP5_A, dynamics.DP5_B, dynamics.DP5_C
    assert np.allclose(A.sum(axis=1), c, atol=1e-15)
    Ac, Ac2, Ac3 = A @ c, A @ c ** 2, A @ c ** 3
    conds = [
        (b.sum(), 1.0), (b @ c, 1 / 2),
        (b @ c ** 2, 1 / 3), (b @ Ac, 1 / 6),
        (b @ c ** 3, 1 / 4), (b @ (c * Ac), 1 / 8), (b @ Ac2, 1 / 12), (b @ (A @ Ac), 1 / 24),
        (b @ c ** 4, 1 / 5), (b @ (c ** 2 * Ac), 1 / 10), (b @ (c * Ac2), 1 / 15),
        (b @ (c * (A @ Ac)), 1 / 30), (b @ (Ac * Ac), 1 / 20), (b @ Ac3, 1 / 20),
        (b @ (A @ (c * Ac)), 1 / 40), (b @ (A @ Ac2), 1 / 60), (b @ (A @ (A @ Ac)), 1 / 120),
    ]
    for got, want in conds:
        assert abs(got - want) < 1e-14


def test_lorenz96_step_order_equilibrium_and_jacobian():
    """One DP5 step has local error O(h^6) against a tight reference integration (the
    ratio for h and h/2 approaches 64); x = F 1 is an equilibrium (f leaves it
    unchanged); the stage chain-rule Jacobian matches central differences."""
    from scipy.integrate import solve_ivp
    p = synth.lorenz96(1, 5, seed=0)
    errs = []
    for h in (0.02, 0.01):
        dyn = dynamics.Lorenz96(p["params"], h, 5)
        ref = solve_ivp(lambda t, x: dyn.rhs(x[None])[0], (0.0, h), p["s0"][0], method="DOP853",
                        rtol=1e-13, atol=1e-13).y[:, -1]
        errs.append(np.abs(dyn.f(1, p["s0"]) - ref).max())
    assert errs[0] / errs[1] > 40.0
    dyn = dynamics.Lorenz96(p["params"], 0.01, 5)
    eq = np.full((1, 5), 8.0)
    assert np.array_equal(dyn.f(1, eq), eq)
    s = p["s0"] + np.random.default_rng(1).standard_normal((1, 5))
    assert np.abs(dyn.jac(1, s) - _fd_jac(lambda v: dyn.f(1, v), s)).max() < 1e-8


def test_word_problem_rollout_is_the_group_product():
    """Prop. cayley: s_t is s_0 permuted by the running product of the step
    permutations (composed here as index arrays, not through f), so s_T is a
    permutation of s_0; every step Jacobian is the permutation matrix of its input."""
    p = synth.word_problem(3, 50, seed=0)
    dyn = dynamics.Permute(p["x"])
    s = newton.rollout(dyn, p["s0"], 50)
    for b in range(3):
        idx = np.arange(5)
        for t in range(50):
            idx = idx[p["x"][b, t].astype(int)]
            assert np.array_equal(s[b, t], p["s0"][b, idx])
        assert np.array_equal(np.sort(s[b, -1]), np.sort(p["s0"][b]))
    J = dyn.jac(7, s[:, 5])
    assert np.array_equal(J.sum(axis=1), np.ones((3, 5)))
    assert np.array_equal(J.sum(axis=2), np.ones((3, 5)))
    assert np.array_equal(np.einsum("bij,bj->bi", J, s[:, 5]), dyn.f(7, s[:, 5]))


def test_word_problem_newton_one_iteration_others_near_T():
    """Sec. sec:GrpWordProb: the recursion is linear, so one Newton iteration solves it;
    quasi-Newton, Picard and Jacobi need a number of iterations close to T."""
    T = 32
    p = synth.word_problem(2, T, seed=1)
    dyn = dynamics.Permute(p["x"])
    its = {m: newton.solve(dyn, p["s0"], T, mode=m, tol=1e-12, init="zeros")["iters"]
           for m in ("full", "diag", "identity", "zero")}
    assert list(its["full"]) == [1, 1]
    for m in ("diag", "identity", "zero"):
        assert np.all(its[m] >= T // 2)


@pytest.mark.parametrize("kind", ["gru", "rnn", "langevin", "linear"])
def test_input_gradient_matches_finite_differences(kind):
    """dl/dx_t from the adjoint states (lambda_t^T df_t/dx_t) against central differences
    of the rollout loss in single input entries; the GRU's input derivative goes through
    all three gates."""
    B, T, d = 2, 12, 4
    if kind == "gru":
        p = synth.gru(B, T, d, d, seed=3)
        x = p["x"]
        mk = lambda xx: dynamics.GRU(p["W"], p["U"], xx)  # noqa: E731
        s0 = np.random.default_rng(1).standard_normal((B, d)) * 0.5
    elif kind == "rnn":
        p = synth.mean_field_rnn(B, T, d, 1.2, seed=3)
        x = p["x"]
        mk = lambda xx: dynamics.MeanFieldRNN(p["W"], xx)  # noqa: E731
        s0 = p["s0"]
    elif kind == "langevin":
        p = synth.two_well(B, T, d, seed=3)
        x = p["x"]
        mk = lambda xx: dynamics.TwoWellLangevin(p["params"], p["dt"], xx, d=d)  # noqa: E731
        s0 = p["s0"]
    else:
        p = synth.linear_lds(B, T, d, seed=3)
        x = p["x"]
        mk = lambda xx: dynamics.Linear(p["A"], xx)  # noqa: E731
        s0 = p["s0"]
    dyn = mk(x)
    s = newton.rollout(dyn, s0, T)
    y = s + 0.3 * synth.targets_noise(s.shape, seed=4)
    g = adjoint.sq_loss_cotangent(s, y)
    _, _, lam = adjoint.adjoint_grad(dyn, s0, s, g)
    gx = adjoint.input_grad(dyn, s0, s, lam)
    idx = [(0, 0, 1), (1, 5, 0), (0, 11, 3), (1, 7, 2)]
    fd = adjoint.fd_input_grad(mk, x, s0, T, y, idx, h=1e-6)
    got = np.array([gx[b, t, k] for (b, t, k) in idx])
    assert np.allclose(got, fd, rtol=1e-6, atol=1e-7)


def test_lorenz96_elk_stays_bounded_where_deer_overflows():
    """Sec. elk_exps: on the chaotic Lorenz-96 system (F = 8, D = 5) undamped DEER from the
    constant guess leaves the attractor within one iteration and overflows after the
    next, while the Kalman-damped step (ELK, lambda = 1) keeps every iterate on the
    attractor's scale."""
    T = 200
    p = synth.lorenz96(2, 5, seed=0)
    dyn = dynamics.Lorenz96(p["params"], p["dt"], 5)
    with np.errstate(all="ignore"):
        s = newton.initial_guess(dyn, p["s0"], T, "s0")
        for _ in range(3):
            s = newton.quasi_newton_step(dyn, p["s0"], s, "full")
        assert not np.all(np.isfinite(s)) or np.max(np.abs(s)) > 1e6
        e = newton.initial_guess(dyn, p["s0"], T, "s0")
        for _ in range(40):
            e = elk.elk_filter_step(dyn, p["s0"], e, "full", 1.0)
            assert np.all(np.isfinite(e)) and np.max(np.abs(e)) < 50.0


def test_rnn_iterations_flat_in_T_when_predictable_growing_when_chaotic():
    """Theorem PL-LLE's two regimes on the mean-field RNN (d = 16): with a negative LLE
    (g = 0.5) the DEER iteration count does not grow with the sequence length; with a
    positive one (g = 3) it grows roughly in proportion to T."""
    its = {}
    for g in (0.5, 3.0):
        for T in (50, 150):
            p = synth.mean_field_rnn(1, T, 16, g, seed=1)
            dyn = dynamics.MeanFieldRNN(p["W"], p["x"])
            its[g, T] = int(newton.solve(dyn, p["s0"], T, mode="full", tol=1e-10,
                                         init="zeros")["iters"][0])
    assert its[0.5, 150] <= its[0.5, 50] + 1
    assert its[3.0, 150] >= 2 * its[3.0, 50]


def test_randn_guess_generator_pins():
    """The counter-based generator behind the random initial guess (Sec. 3.3.3): its
    SplitMix64 stream reproduces the published reference outputs of the algorithm for seed
    1234567, and the Box-Muller draws are standard normal (moments, a Kolmogorov-Smirnov
    test against the normal CDF, no correlation between neighbouring entries), differ
    between seeds and are stable under repacking of the same entry index."""
    from scipy import stats

    from oracle import rng
    ref = [6457827717110365317, 3203168211198807973, 9817491932198370423,
           4593380528125082431, 16408922859458223821]
    assert [int(v) for v in rng.splitmix64(1234567, np.arange(1, 6))] == ref
    x = rng.randn_guess(7, 1 << 14, 16).ravel()
    n = x.size
    assert abs(x.mean()) < 5 / np.sqrt(n)
    assert abs(x.var() - 1.0) < 5 * np.sqrt(2.0 / n)
    assert abs(stats.skew(x)) < 5 * np.sqrt(6.0 / n)
    assert stats.kstest(x, "norm").pvalue > 1e-4
    assert abs(np.corrcoef(x[:-1], x[1:])[0, 1]) < 5 / np.sqrt(n)
    y = rng.randn_guess(8, 1 << 14, 16).ravel()
    assert abs(np.corrcoef(x, y)[0, 1]) < 5 / np.sqrt(n)
    # entry e depends on e only: the same entries in another [rows][d] shape are equal
    assert np.array_equal(rng.randn_guess(7, 1 << 13, 32).ravel(), x[: (1 << 13) * 32])


@pytest.mark.parametrize("d,R,integ", [(4, 6, "euler"), (8, 12, "rk4"), (16, 24, "rk4"),
                                       (32, 48, "rk4")])
def test_c_oracle_equals_numpy_oracle(d, R, integ):
    """The plain C mass-action oracle (used where the numpy loops are too slow: full-size
    parity and the timed CPU baseline) computes what the pinned numpy oracle computes: the
    rollout (Sec. 2.1), the step Jacobians (Eq. lil_j) and the adjoint gradient (Eq. bptt)
    on a ragged batch, to rounding; and its rollout conserves mass like the networks do."""
    from oracle import adjoint as oadj
    from oracle import cma
    lengths = [37, 1, 0, 50]
    off = synth.offsets_from_lengths(lengths)
    B = len(lengths)
    p = synth.massaction(B, d, R, 1, seed=4, integrator=integ)
    cb = cma.Batch(p["topology"], p["params"], p["dt"], integ, d=d)
    s = cb.rollout(p["s0"], off, threads=2)
    A = cb.step_jacobians(p["s0"], s, off, threads=2)
    rng = np.random.default_rng(1)
    g = rng.standard_normal(s.shape)
    dk, ds0 = cb.adjoint(p["s0"], s, g, off, threads=3)
    for b, L in enumerate(lengths):
        sub = dynamics.MassAction(p["topology"][b:b + 1], p["params"][b:b + 1], p["dt"], integ,
                              d=d)
        if L == 0:
            assert np.all(dk[b] == 0.0) and np.all(ds0[b] == 0.0)
            continue
        ref = newton.rollout(sub, p["s0"][b:b + 1], L)[0]
        seg = slice(off[b], off[b + 1])
        assert np.max(np.abs(s[seg] - ref)) <= 1e-14 * max(1.0, np.max(np.abs(ref)))
        An = np.stack([sub.jac(t, ref[None, t - 2] if t >= 2 else p["s0"][b:b + 1])[0]
                       for t in range(1, L + 1)])
        assert np.max(np.abs(A[seg] - An)) <= 1e-13 * max(1.0, np.max(np.abs(An)))
        dkn, ds0n, _ = oadj.adjoint_grad(sub, p["s0"][b:b + 1], ref[None], g[None, seg])
        assert np.max(np.abs(dk[b] - dkn[0])) <= 1e-12 * max(1.0, np.max(np.abs(dkn)))
        assert np.max(np.abs(ds0[b] - ds0n[0])) <= 1e-12 * max(1.0, np.max(np.abs(ds0n)))
        # mass conservation (masses m_i in {1, 2}): sum_i m_i s_t,i is constant
        m = p["masses"][b] if "masses" in p else None
        if m is not None:
            tot = ref @ m
            assert np.max(np.abs(s[seg] @ m - tot)) <= 1e-12 * np.max(np.abs(tot))


def test_filter_covariance_as_associative_elements():
    """The covariance recursion of the ELK filter (Sec. 4.3: predict with process noise I,
    update with emission variance 1/lambda, Sigma_0 = 0) is a prefix scan of per-step
    elements: one element applied to P is one filter step; combining elements is
    associative; the in-order prefix combinations, applied to the zero prior, give every
    filtered covariance of elk.kalman_filter; and splitting a sequence into chunks
    (aggregate per chunk, carry across chunks, re-run inside) gives them too."""
    rng = np.random.default_rng(3)
    B, T, d, lam = 2, 23, 4, 0.7
    F = rng.standard_normal((B, T, d, d)) * 0.5 + np.eye(d)
    _, Ps, _, _ = elk.kalman_filter(F, np.zeros((B, T, d)), np.zeros((B, T, d)),
                                     np.zeros((B, d)), lam)
    # one element = one step
    P = rng.standard_normal((B, d, d))
    P = P @ np.swapaxes(P, 1, 2)
    Pm = F[:, 0] @ P @ np.swapaxes(F[:, 0], 1, 2) + np.eye(d)
    step = np.linalg.inv(np.eye(d) + lam * Pm) @ Pm
    assert np.allclose(elk.cov_apply(elk.cov_element(F[:, 0], lam), P), step, atol=1e-12)
    # associativity
    e = [elk.cov_element(F[:, t], lam) for t in range(3)]
    l = elk.cov_combine(elk.cov_combine(e[0], e[1]), e[2])
    r = elk.cov_combine(e[0], elk.cov_combine(e[1], e[2]))
    for x, y in zip(l, r):
        assert np.allclose(x, y, atol=1e-12)
    # prefix scan from the zero prior = the filter's covariances
    Z = np.zeros((B, d, d))
    acc = elk.cov_element(F[:, 0], lam)
    for t in range(T):
        if t > 0:
            acc = elk.cov_combine(acc, elk.cov_element(F[:, t], lam))
        assert np.allclose(elk.cov_apply(acc, Z), Ps[:, t], atol=1e-12)
    # chunked: aggregates of chunks of 5, carried, then the sequential recursion inside
    P_in = Z
    for c0 in range(0, T, 5):
        agg = elk.cov_element(F[:, c0], lam)
        for t in range(c0 + 1, min(c0 + 5, T)):
            agg = elk.cov_combine(agg, elk.cov_element(F[:, t], lam))
        Pt = P_in
        for t in range(c0, min(c0 + 5, T)):
            Pm = F[:, t] @ Pt @ np.swapaxes(F[:, t], 1, 2) + np.eye(d)
            Pt = np.linalg.inv(np.eye(d) + lam * Pm) @ Pm
            assert np.allclose(Pt, Ps[:, t], atol=1e-12)
        P_in = elk.cov_apply(agg, P_in)
        assert np.allclose(P_in, Pt, atol=1e-12)


# --- convergence measure, reset heuristic, loss, offsets ------------------------
def test_scaled_residual_is_absolute_below_one_relative_above():
    """The convergence measure (the residual of Eq. r_def scaled by max(1, |s|), the
    reading of the paper's unspecified error test) on values worked by hand: where
    |s| <= 1 the residual counts as it is, above 1 it is divided by |s|; the maximum runs
    over steps and coordinates, separately per sequence."""
    r = np.zeros((2, 3, 2))
    s = np.zeros((2, 3, 2))
    r[0, 0, 0], s[0, 0, 0] = 0.5, 0.1      # absolute: 0.5
    r[0, 1, 0], s[0, 1, 0] = 3.0, 10.0     # relative: 0.3
    r[0, 2, 1], s[0, 2, 1] = -0.2, -1.0    # |s| = 1: 0.2
    r[1, 0, 1], s[1, 0, 1] = -4.0, -2.0    # relative: 2.0
    r[1, 2, 0], s[1, 2, 0] = 1e-3, 0.0     # absolute: 1e-3
    got = newton.scaled_residual_max(r, s)
    assert got.shape == (2,)
    assert got[0] == pytest.approx(0.5, abs=0)
    assert got[1] == pytest.approx(2.0, abs=0)
    # large states: a residual of 1e-6 relative to a state of 1e6 is 1e-12
    r2 = np.full((1, 4, 1), 1.0)
    s2 = np.full((1, 4, 1), 1e12)
    assert newton.scaled_residual_max(r2, s2)[0] == pytest.approx(1e-12, rel=1e-15)


def test_reset_zeroes_only_non_finite_and_overflowing_entries():
    """The reset heuristic (Sec. 3.2): entries that are NaN, infinite or above the
    threshold in magnitude become zero; every other entry, including one just below the
    threshold and negative ones, is left exactly as it was."""
    s = np.array([[[1.0, np.nan, np.inf], [-2e31, 1e29, -np.inf], [-0.5, 1e30, -1e30]]])
    got = newton.reset_overflow(s, 1e30)
    want = np.array([[[1.0, 0.0, 0.0], [0.0, 1e29, 0.0], [-0.5, 1e30, -1e30]]])
    assert np.array_equal(got, want)
    assert np.isnan(s[0, 0, 1])          # the input is not modified


def test_squared_loss_cotangent_is_its_gradient():
    """The adjoint's test loss and its cotangent: the cotangent equals the central
    difference of the loss in every entry (exact up to rounding: the loss is quadratic),
    and the loss of a trajectory equal to its target is zero."""
    rng = np.random.default_rng(3)
    s = rng.standard_normal((2, 5, 3))
    y = rng.standard_normal((2, 5, 3))
    g = adjoint.sq_loss_cotangent(s, y)
    h = 1e-3
    for b in range(2):
        for t in range(5):
            for i in range(3):
                e = np.zeros_like(s)
                e[b, t, i] = h
                fd = (adjoint.sq_loss(s + e, y)[b] - adjoint.sq_loss(s - e, y)[b]) / (2 * h)
                assert fd == pytest.approx(g[b, t, i], abs=1e-9)
    assert np.array_equal(adjoint.sq_loss(y, y), np.zeros(2))


def test_uniform_offsets_are_the_ragged_heads_of_equal_lengths():
    """Equal-length batches as the ragged layout: sequence b occupies rows
    [b T, (b + 1) T) of the packed state."""
    from oracle import cma
    off = cma.uniform_offsets(4, 7)
    assert off.dtype == np.int64
    assert off.tolist() == [0, 7, 14, 21, 28]
    assert cma.uniform_offsets(0, 7).tolist() == [0]
