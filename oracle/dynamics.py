"""Recurrences s_t = f_t(s_{t-1}) used by the oracle (float64, batched over B).

Test infrastructure only (see the package docstring). Each class exposes

    f(t, s)      -> [B, d]      one step of the recurrence, t = 1..T
    jac(t, s)    -> [B, d, d]   A_t = d f_t / d s_{t-1} at s (Eq. lil_j)
    dparams(t, s)-> [B, d, P]   d f_t / d theta at s (used by the adjoint)

where s is the previous state s_{t-1} of every sequence in the batch.
Inputs are curried into f_t (Sec. 2.1: f_t(s) := f(s, u_t)).
"""
from __future__ import annotations

import numpy as np


def _sigmoid(v):
    return 1.0 / (1.0 + np.exp(-v))


class Brusselator:
    """Textbook Brusselator kinetics dx/dt = a - (b+1) x + x^2 y, dy/dt = b x - x^2 y,
    discretised by explicit Euler (an explicit ODE solver is an SSM, Table ssm_examples).
    params [B][2] = (a, b)."""

    def __init__(self, params, dt):
        self.p = np.asarray(params, dtype=np.float64)
        self.dt = float(dt)
        self.d = 2
        self.n_params = 2

    def rhs(self, s):
        a, b = self.p[:, 0], self.p[:, 1]
        x, y = s[:, 0], s[:, 1]
        return np.stack([a - (b + 1.0) * x + x * x * y, b * x - x * x * y], axis=1)

    def rhs_jac(self, s):
        b = self.p[:, 1]
        x, y = s[:, 0], s[:, 1]
        J = np.empty((s.shape[0], 2, 2))
        J[:, 0, 0] = -(b + 1.0) + 2.0 * x * y
        J[:, 0, 1] = x * x
        J[:, 1, 0] = b - 2.0 * x * y
        J[:, 1, 1] = -x * x
        return J

    def f(self, t, s):
        return s + self.dt * self.rhs(s)

    def jac(self, t, s):
        return np.eye(2)[None] + self.dt * self.rhs_jac(s)

    def dparams(self, t, s):
        x = s[:, 0]
        out = np.zeros((s.shape[0], 2, 2))
        out[:, 0, 0] = self.dt            # d f_x / d a
        out[:, 0, 1] = -self.dt * x       # d f_x / d b
        out[:, 1, 1] = self.dt * x        # d f_y / d b
        return out


class MassAction:
    """Mass-action kinetics of a reaction network, integrated by explicit Euler or
    classical RK4. topology [B][R][4] = (i1, i2, p1, p2), -1 = absent; rate
    constants k [B][R]. The rate of reaction r is k_r c_{i1} c_{i2} (c_{i2} -> 1 when
    unimolecular); it consumes its reactants and produces its products."""

    def __init__(self, topology, k, dt, integrator="rk4", d=None):
        self.topo = np.asarray(topology, dtype=np.int64)
        self.k = np.asarray(k, dtype=np.float64)
        self.B, self.R, _ = self.topo.shape
        self.dt = float(dt)
        self.integrator = integrator
        self.d = int(self.topo.max()) + 1 if d is None else int(d)
        self.n_params = self.R
        self._bi = np.arange(self.B)

    # --- right-hand side g(c), its Jacobian G(c) and d g / d k -----------------
    def _phi(self, c, r):
        """Mass-action monomial of reaction r (without k_r), per batch member."""
        i1, i2 = self.topo[:, r, 0], self.topo[:, r, 1]
        v = c[self._bi, i1]
        second = np.where(i2 >= 0, c[self._bi, np.maximum(i2, 0)], 1.0)
        return v * second

    def _stoich_add(self, out, r, vals):
        """out[b, species] += nu_r[species] * vals[b] for reaction r (vals [B] or [B, m])."""
        i1, i2, p1, p2 = (self.topo[:, r, j] for j in range(4))
        bi = self._bi
        out[bi, i1] -= vals
        m = i2 >= 0
        out[bi[m], i2[m]] -= vals[m]
        out[bi, p1] += vals
        m = p2 >= 0
        out[bi[m], p2[m]] += vals[m]

    def rhs(self, c):
        out = np.zeros((self.B, self.d))
        for r in range(self.R):
            self._stoich_add(out, r, self.k[:, r] * self._phi(c, r))
        return out

    def rhs_jac(self, c):
        """G[b, i, j] = d g_i / d c_j = sum_r nu_r[i] * d(rate_r)/d c_j."""
        G = np.zeros((self.B, self.d, self.d))
        bi = self._bi
        for r in range(self.R):
            i1, i2 = self.topo[:, r, 0], self.topo[:, r, 1]
            kr = self.k[:, r]
            grad = np.zeros((self.B, self.d))
            bim = i2 >= 0
            # d(k c_i1 c_i2)/d c_i1 = k c_i2 ; d/d c_i2 = k c_i1 (adds up for i1 == i2)
            grad[bi, i1] += np.where(bim, kr * c[bi, np.maximum(i2, 0)], kr)
            grad[bi[bim], i2[bim]] += kr[bim] * c[bi[bim], i1[bim]]
            self._stoich_add(G, r, grad)
        return G

    def rhs_dk(self, c):
        """d g_i / d k_r = nu_r[i] * phi_r(c); shape [B, d, R]."""
        out = np.zeros((self.B, self.d, self.R))
        for r in range(self.R):
            col = np.zeros((self.B, self.d))
            self._stoich_add(col, r, self._phi(c, r))
            out[:, :, r] = col
        return out

    # --- one integrator step and its derivatives ------------------------------
    def f(self, t, s):
        h = self.dt
        if self.integrator == "euler":
            return s + h * self.rhs(s)
        k1 = self.rhs(s)
        k2 = self.rhs(s + 0.5 * h * k1)
        k3 = self.rhs(s + 0.5 * h * k2)
        k4 = self.rhs(s + h * k3)
        return s + (h / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)

    def jac(self, t, s):
        """Exact Jacobian of one step, by the chain rule through the RK4 stages."""
        h = self.dt
        I = np.eye(self.d)[None]
        if self.integrator == "euler":
            return I + h * self.rhs_jac(s)
        k1 = self.rhs(s)
        s2 = s + 0.5 * h * k1
        k2 = self.rhs(s2)
        s3 = s + 0.5 * h * k2
        k3 = self.rhs(s3)
        s4 = s + h * k3
        K1 = self.rhs_jac(s)
        K2 = self.rhs_jac(s2) @ (I + 0.5 * h * K1)
        K3 = self.rhs_jac(s3) @ (I + 0.5 * h * K2)
        K4 = self.rhs_jac(s4) @ (I + h * K3)
        return I + (h / 6.0) * (K1 + 2.0 * K2 + 2.0 * K3 + K4)

    def dparams(self, t, s):
        """d f / d k [B, d, R], chain rule through the stages (k enters every stage)."""
        h = self.dt
        if self.integrator == "euler":
            return h * self.rhs_dk(s)
        k1 = self.rhs(s)
        s2 = s + 0.5 * h * k1
        k2 = self.rhs(s2)
        s3 = s + 0.5 * h * k2
        k3 = self.rhs(s3)
        s4 = s + h * k3
        P1 = self.rhs_dk(s)
        P2 = self.rhs_dk(s2) + self.rhs_jac(s2) @ (0.5 * h * P1)
        P3 = self.rhs_dk(s3) + self.rhs_jac(s3) @ (0.5 * h * P2)
        P4 = self.rhs_dk(s4) + self.rhs_jac(s4) @ (h * P3)
        return (h / 6.0) * (P1 + 2.0 * P2 + 2.0 * P3 + P4)


class GRU:
    """Gated recurrent unit (Cho et al. 2014 form, zero biases):
        z = sigma(W_z x + U_z h), r = sigma(W_r x + U_r h),
        h~ = tanh(W_h x + U_h (r * h)), h' = (1 - z) * h + z * h~.
    W [3][d][d_in], U [3][d][d] (gate order z, r, h), x [B][T][d_in].
    The inputs are curried into f_t (Sec. 2.1)."""

    def __init__(self, W, U, x):
        self.W = np.asarray(W, dtype=np.float64)
        self.U = np.asarray(U, dtype=np.float64)
        self.x = np.asarray(x, dtype=np.float64)
        self.d = self.U.shape[1]
        self.n_params = 0

    def _gates(self, t, h):
        xt = self.x[:, t - 1]
        Wz, Wr, Wh = self.W
        Uz, Ur, Uh = self.U
        z = _sigmoid(xt @ Wz.T + h @ Uz.T)
        r = _sigmoid(xt @ Wr.T + h @ Ur.T)
        ht = np.tanh(xt @ Wh.T + (r * h) @ Uh.T)
        return z, r, ht

    def f(self, t, h):
        z, r, ht = self._gates(t, h)
        return (1.0 - z) * h + z * ht

    def jac(self, t, h):
        """Full Jacobian d h' / d h, term by term from the product/chain rules."""
        z, r, ht = self._gates(t, h)
        Uz, Ur, Uh = self.U
        d = self.d
        dz = (z * (1.0 - z))[:, :, None] * Uz[None]                       # dz_i/dh_j
        dr = (r * (1.0 - r))[:, :, None] * Ur[None]                       # dr_m/dh_j
        # d a_i / d h_j with a = W_h x + U_h (r*h): U_h[i,j] r_j + sum_m U_h[i,m] h_m dr_m/dh_j
        da = Uh[None] * r[:, None, :] + np.einsum("im,bm,bmj->bij", Uh, h, dr)
        dht = (1.0 - ht * ht)[:, :, None] * da
        J = np.zeros((h.shape[0], d, d))
        J += (1.0 - z)[:, :, None] * np.eye(d)[None]
        J += (ht - h)[:, :, None] * dz
        J += z[:, :, None] * dht
        return J


    def dinputs(self, t, h):
        """d h' / d x_t [B, d, d_in] at h, through the three gates (chain rule)."""
        z, r, ht = self._gates(t, h)
        Wz, Wr, Wh = self.W
        Uz, Ur, Uh = self.U
        dz = (z * (1.0 - z))[:, :, None] * Wz[None]                       # dz_i/dx_k
        dr = (r * (1.0 - r))[:, :, None] * Wr[None]                       # dr_m/dx_k
        # a = W_h x + U_h (r * h): da_i/dx_k = W_h[i,k] + sum_m U_h[i,m] h_m dr_m/dx_k
        da = Wh[None] + np.einsum("im,bm,bmk->bik", Uh, h, dr)
        return (ht - h)[:, :, None] * dz + (z * (1.0 - ht * ht))[:, :, None] * da


class Linear:
    """Affine recurrence s_t = A s_{t-1} + x_t (an LDS, Eq. lds), A [d][d] shared,
    x [B][T][d] (x may be None for s_t = A s_{t-1})."""

    def __init__(self, A, x=None):
        self.A = np.asarray(A, dtype=np.float64)
        self.d = self.A.shape[0]
        self.x = None if x is None else np.asarray(x, dtype=np.float64)
        self.n_params = 0

    def f(self, t, s):
        out = s @ self.A.T
        if self.x is not None:
            out = out + self.x[:, t - 1]
        return out

    def jac(self, t, s):
        return np.broadcast_to(self.A, (s.shape[0], self.d, self.d)).copy()

    def dinputs(self, t, s):
        """d f / d x_t = I."""
        return np.broadcast_to(np.eye(self.d), (s.shape[0], self.d, self.d)).copy()


class MeanFieldRNN:
    """Mean-field RNN of the predictability-threshold experiment (Sec. ssc:exp_thresh):
        s_t = W tanh(s_{t-1}) + u_t,   A_t = W diag(1 - tanh(s_{t-1})^2).
    W [d][d] shared or [B][d][d] per sequence; u [B][T][d] (None for u = 0)."""

    def __init__(self, W, u=None):
        self.W = np.asarray(W, dtype=np.float64)
        self.d = self.W.shape[-1]
        self.u = None if u is None else np.asarray(u, dtype=np.float64)
        self.n_params = 0

    def f(self, t, s):
        th = np.tanh(s)
        if self.W.ndim == 2:
            out = th @ self.W.T
        else:
            out = np.einsum("bij,bj->bi", self.W, th)
        if self.u is not None:
            out = out + self.u[:, t - 1]
        return out

    def jac(self, t, s):
        sech2 = 1.0 - np.tanh(s) ** 2
        W = np.broadcast_to(self.W, (s.shape[0], self.d, self.d))
        return W * sech2[:, None, :]

    def dinputs(self, t, s):
        """d f / d u_t = I (the input enters additively)."""
        return np.broadcast_to(np.eye(self.d), (s.shape[0], self.d, self.d)).copy()


class TwoWellLangevin:
    """Discretised Langevin dynamics (Eq. langevin) for the potential
        phi(s) = -log( w1 N(s; m1, diag v1) + w2 N(s; m2, diag v2) ),
        s_t = s_{t-1} - eps grad phi(s_{t-1}) + sqrt(2 eps) xi_t,
    with xi_t the standard normal draws in ``noise`` [B][T][d] (None: no noise).
    The Jacobian is I - eps Hess phi (Sec. ssc:2well).
    params [4d+2] shared or [B][4d+2]: m1 | m2 | v1 | v2 | w1 | w2."""

    def __init__(self, params, eps, noise=None, d=None):
        p = np.atleast_2d(np.asarray(params, dtype=np.float64))
        self.d = (p.shape[1] - 2) // 4 if d is None else d
        d = self.d
        self.m1, self.m2 = p[:, :d], p[:, d:2 * d]
        self.v1, self.v2 = p[:, 2 * d:3 * d], p[:, 3 * d:4 * d]
        self.w1, self.w2 = p[:, 4 * d], p[:, 4 * d + 1]
        self.eps = float(eps)
        self.noise = None if noise is None else np.asarray(noise, dtype=np.float64)
        self.n_params = 0

    def _resp(self, s):
        """Responsibilities of the two components at s (posterior weights)."""
        with np.errstate(divide="ignore", over="ignore"):  # w_k = 0 or far from a well
            l1 = np.log(self.w1) - 0.5 * np.sum(np.log(self.v1) + (s - self.m1) ** 2 / self.v1,
                                                axis=1)
            l2 = np.log(self.w2) - 0.5 * np.sum(np.log(self.v2) + (s - self.m2) ** 2 / self.v2,
                                                axis=1)
            g1 = 1.0 / (1.0 + np.exp(l2 - l1))
            g2 = 1.0 / (1.0 + np.exp(l1 - l2))
        return g1, g2

    def grad_phi(self, s):
        g1, g2 = self._resp(s)
        return g1[:, None] * (s - self.m1) / self.v1 + g2[:, None] * (s - self.m2) / self.v2

    def hess_phi(self, s):
        """sum_k g_k diag(1/v_k) minus the covariance of the component scores."""
        g1, g2 = self._resp(s)
        sc1 = -(s - self.m1) / self.v1          # score of component 1
        sc2 = -(s - self.m2) / self.v2
        H = np.zeros((s.shape[0], self.d, self.d))
        idx = np.arange(self.d)
        H[:, idx, idx] = g1[:, None] / self.v1 + g2[:, None] / self.v2
        diff = sc1 - sc2
        H -= (g1 * g2)[:, None, None] * diff[:, :, None] * diff[:, None, :]
        return H

    def f(self, t, s):
        out = s - self.eps * self.grad_phi(s)
        if self.noise is not None:
            out = out + np.sqrt(2.0 * self.eps) * self.noise[:, t - 1]
        return out

    def jac(self, t, s):
        return np.eye(self.d)[None] - self.eps * self.hess_phi(s)

    def dinputs(self, t, s):
        """d f / d xi_t = sqrt(2 eps) I (the noise draws are the inputs)."""
        return np.broadcast_to(np.sqrt(2.0 * self.eps) * np.eye(self.d),
                               (s.shape[0], self.d, self.d)).copy()


# Dormand-Prince 5(4) pair (Dormand & Prince, 1980): nodes, stage matrix and the weights
# of the fifth-order solution; the seventh (FSAL) stage has zero weight there.
DP5_C = np.array([0.0, 1 / 5, 3 / 10, 4 / 5, 8 / 9, 1.0])
DP5_A = np.array([
    [0, 0, 0, 0, 0, 0],
    [1 / 5, 0, 0, 0, 0, 0],
    [3 / 40, 9 / 40, 0, 0, 0, 0],
    [44 / 45, -56 / 15, 32 / 9, 0, 0, 0],
    [19372 / 6561, -25360 / 2187, 64448 / 6561, -212 / 729, 0, 0],
    [9017 / 3168, -355 / 33, 46732 / 5247, 49 / 176, -5103 / 18656, 0],
])
DP5_B = np.array([35 / 384, 0.0, 500 / 1113, 125 / 192, -2187 / 6784, 11 / 84])


class Lorenz96:
    """Lorenz-96, dx_i/dt = (x_{i+1} - x_{i-2}) x_{i-1} - x_i + F (cyclic indices), one
    fixed step h of an explicit Runge-Kutta method (default: the fifth-order
    Dormand-Prince solution) per time step (the Lorenz-96 experiment of Sec. elk_exps
    evaluates it with the Dormand-Prince solver).
    F scalar or [B]."""

    def __init__(self, F, dt, d, tableau=None):
        self.F = np.asarray(F, dtype=np.float64).reshape(-1, 1)
        self.dt = float(dt)
        self.d = d
        self.A, self.b = (DP5_A, DP5_B) if tableau is None else tableau
        self.n_params = 0

    def rhs(self, x):
        return (np.roll(x, -1, axis=1) - np.roll(x, 2, axis=1)) * np.roll(x, 1, axis=1) - x + self.F

    def rhs_jac(self, x):
        B, d = x.shape
        G = np.zeros((B, d, d))
        for i in range(d):
            ip, im, im2 = (i + 1) % d, (i - 1) % d, (i - 2) % d
            G[:, i, ip] += x[:, im]
            G[:, i, im2] -= x[:, im]
            G[:, i, im] += x[:, ip] - x[:, im2]
            G[:, i, i] -= 1.0
        return G

    def _stages(self, s):
        h = self.dt
        Y, K = [], []
        for k in range(len(self.b)):
            y = s.copy()
            for j in range(k):
                y = y + h * self.A[k, j] * K[j]
            Y.append(y)
            K.append(self.rhs(y))
        return Y, K

    def f(self, t, s):
        Y, K = self._stages(s)
        return s + self.dt * sum(bk * kk for bk, kk in zip(self.b, K))

    def jac(self, t, s):
        """Chain rule through the stages: dK_k = G(Y_k) (I + h sum_j a_kj dK_j)."""
        h = self.dt
        Y, _ = self._stages(s)
        I = np.eye(self.d)[None]
        dK = []
        for k in range(len(self.b)):
            M = I.copy()
            for j in range(k):
                M = M + h * self.A[k, j] * dK[j]
            dK.append(self.rhs_jac(Y[k]) @ M)
        return I + h * sum(bk * dk for bk, dk in zip(self.b, dK))


class Permute:
    """The group word problem as a time-varying LDS (Prop. cayley):
        s_t[i] = s_{t-1}[p_t[i]],  A_t = the permutation matrix with A_t[i, p_t[i]] = 1,
    p [B][T][d] integer source indices (one permutation per step)."""

    def __init__(self, perms):
        self.p = np.asarray(perms).astype(np.int64)
        self.d = self.p.shape[2]
        self.n_params = 0

    def f(self, t, s):
        return np.take_along_axis(s, self.p[:, t - 1], axis=1)

    def jac(self, t, s):
        B = s.shape[0]
        J = np.zeros((B, self.d, self.d))
        rows = np.arange(self.d)
        for b in range(B):
            J[b, rows, self.p[b, t - 1]] = 1.0
        return J


def from_problem(prob: dict):
    """Build the oracle dynamics for a problem dict made by ``synth``."""
    kind = prob["kind"]
    if kind == "brusselator_euler":
        return Brusselator(prob["params"], prob["dt"])
    if kind.startswith("massaction"):
        integ = kind.split("_", 1)[1]
        return MassAction(prob["topology"], prob["params"], prob["dt"], integ, d=prob["d"])
    if kind == "gru":
        return GRU(prob["W"], prob["U"], prob["x"])
    if kind == "linear":
        return Linear(prob["A"], prob["x"])
    if kind == "rnn_tanh":
        return MeanFieldRNN(prob["W"], prob["x"])
    if kind == "langevin_2well":
        return TwoWellLangevin(prob["params"], prob["dt"], prob["x"], d=prob["d"])
    if kind == "lorenz96_dp5":
        return Lorenz96(prob["params"], prob["dt"], prob["d"])
    if kind == "permute":
        return Permute(prob["x"])
    raise ValueError(kind)
