"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module draws random numbers and builds problem *structure* only
(reaction-network topology, rate constants, weights, inputs, sequence
lengths). It holds none of the parallel-Newton arithmetic, no dynamics
evaluation and no Jacobians: both sides of every parity test receive the
arrays made here and nothing else.

All generators use ``numpy.random.default_rng(seed)`` and return float64
arrays; callers cast to the precision they run in.

Workload shapes follow the synthetic problems of the build (the paper runs
none of them; they are stand-ins for its kinetic-ODE and GRU settings):

* Brusselator kinetics, d=2 (explicit Euler).
* Random mass-action reaction networks with mass-conserving uni- and
  bimolecular reactions (explicit Euler or classical RK4).
* Untrained GRU cells with weights N(0, 1/d) and inputs N(0, 1)
  (Sec. 3.3 of the paper evaluates untrained GRUs the same way).
* Ragged batches with lengths uniform on an integer range.
* The second workloads of the thesis (its experiments' settings, synthetic):
  mean-field RNN weights N(0, g^2/d) with zero diagonal and sinusoidal inputs,
  a two-well Gaussian-mixture potential with Langevin noise draws, Lorenz-96
  initial points, and uniformly random permutations for the S_d word problem.
"""
from __future__ import annotations

import numpy as np

# Reaction encoding: one row (i1, i2, p1, p2) per reaction, -1 = absent slot.
#   conversion   X -> Y      : (X, -1, Y, -1)   with m_X == m_Y
#   association  X + Y -> Z  : (X,  Y, Z, -1)   with m_X + m_Y == m_Z
#   dissociation Z -> X + Y  : (Z, -1, X,  Y)   with m_Z == m_X + m_Y
# The mass-action rate of reaction r is k_r * c[i1] * (c[i2] if i2 >= 0 else 1).


def brusselator(a: float = 1.0, b: float = 3.0, s0=(1.0, 1.0), dt: float = 0.01,
                T: int = 1024) -> dict:
    """Brusselator problem: params [B=1][2] = (a, b), s0 [1][2]."""
    return {
        "kind": "brusselator_euler",
        "d": 2,
        "dt": float(dt),
        "T": int(T),
        "params": np.array([[a, b]], dtype=np.float64),
        "s0": np.array([s0], dtype=np.float64),
    }


def _one_network(rng: np.random.Generator, d: int, R: int, max_tries: int = 1000):
    """Draw one mass-conserving network on d species with R reactions."""
    if d < 2:
        raise ValueError("mass-action networks need d >= 2")
    for _ in range(max_tries):
        masses = rng.integers(1, 3, size=d)  # m_i in {1, 2}
        if d >= 3 and (np.all(masses == 1) or np.all(masses == 2)):
            continue
        light = np.flatnonzero(masses == 1)
        heavy = np.flatnonzero(masses == 2)
        classes = [c for c in (light, heavy) if len(c) >= 2]
        topo = np.full((R, 4), -1, dtype=np.int32)
        ok = True
        for r in range(R):
            kinds = []
            if classes:
                kinds.append(0)
            if len(light) >= 1 and len(heavy) >= 1:
                kinds += [1, 2]
            if not kinds:
                ok = False
                break
            kind = kinds[rng.integers(len(kinds))]
            if kind == 0:
                cls = classes[rng.integers(len(classes))]
                x, y = rng.choice(cls, size=2, replace=False)
                topo[r] = (x, -1, y, -1)
            elif kind == 1:
                x, y = rng.choice(light, size=2, replace=True)
                z = rng.choice(heavy)
                topo[r] = (x, y, z, -1)
            else:
                z = rng.choice(heavy)
                x, y = rng.choice(light, size=2, replace=True)
                topo[r] = (z, -1, x, y)
        if not ok:
            continue
        used = np.unique(topo[topo >= 0])
        if len(used) == d:
            return topo, masses
    raise RuntimeError(f"could not draw a network covering all {d} species with {R} reactions")


def massaction(B: int, d: int, R: int, T: int, seed: int, dt: float = 1e-3,
               integrator: str = "rk4", k_range=(1e-2, 1e1), shared_topology: bool = False) -> dict:
    """B random mass-action systems: topology [B][R][4] int32, rates k [B][R], s0 [B][d].

    Rate constants are log-uniform on ``k_range``; s0 is uniform on [0, 1]^d.
    With ``shared_topology`` every system uses the first drawn network.
    """
    rng = np.random.default_rng(seed)
    topo = np.empty((B, R, 4), dtype=np.int32)
    masses = np.empty((B, d), dtype=np.int64)
    for b in range(B):
        if shared_topology and b > 0:
            topo[b] = topo[0]
            masses[b] = masses[0]
            continue
        topo[b], masses[b] = _one_network(rng, d, R)
    lo, hi = np.log(k_range[0]), np.log(k_range[1])
    k = np.exp(rng.uniform(lo, hi, size=(B, R)))
    s0 = rng.uniform(0.0, 1.0, size=(B, d))
    return {
        "kind": f"massaction_{integrator}",
        "d": d,
        "R": R,
        "dt": float(dt),
        "T": int(T),
        "topology": topo,
        "masses": masses,
        "params": k,
        "s0": s0,
    }


def linear_conversion_network(d: int, R: int, seed: int, dt: float = 1e-2) -> dict:
    """A single network with conversions X -> Y only (a linear ODE); used to pin
    integrators against the matrix exponential's Taylor polynomial."""
    rng = np.random.default_rng(seed)
    topo = np.full((1, R, 4), -1, dtype=np.int32)
    for r in range(R):
        x, y = rng.choice(d, size=2, replace=False)
        topo[0, r] = (x, -1, y, -1)
    k = np.exp(rng.uniform(np.log(0.1), np.log(2.0), size=(1, R)))
    s0 = rng.uniform(0.0, 1.0, size=(1, d))
    return {"d": d, "R": R, "dt": dt, "topology": topo, "params": k, "s0": s0}


def perturbed_rates(k: np.ndarray, seed: int, scale: float = 0.1) -> np.ndarray:
    """k * exp(scale * eps), eps ~ N(0, 1): rate constants of the loss targets."""
    rng = np.random.default_rng(seed)
    return k * np.exp(scale * rng.standard_normal(k.shape))


def gru(B: int, T: int, d: int, d_in: int, seed: int, weight_scale: float | None = None,
        dtype=np.float64) -> dict:
    """Untrained GRU: W [3][d][d_in], U [3][d][d] iid N(0, 1/d) (gate order z, r, h),
    zero biases, inputs x [B][T][d_in] iid N(0, 1), s0 = 0."""
    rng = np.random.default_rng(seed)
    std = np.sqrt(1.0 / d) if weight_scale is None else weight_scale
    W = rng.standard_normal((3, d, d_in)) * std
    U = rng.standard_normal((3, d, d)) * std
    x = rng.standard_normal((B, T, d_in), dtype=np.float64 if dtype == np.float64 else np.float32)
    return {
        "kind": "gru",
        "d": d,
        "d_in": d_in,
        "T": int(T),
        "W": W,
        "U": U,
        "x": x,
        "s0": np.zeros((B, d)),
    }


def linear_lds(B: int, T: int, d: int, seed: int, spectral_radius: float = 0.9,
               diagonal: bool = False) -> dict:
    """Affine recurrence s_t = A s_{t-1} + x_t with a fixed random A per problem
    (scaled to the given spectral radius) and inputs x ~ N(0, 1)."""
    rng = np.random.default_rng(seed)
    if diagonal:
        A = np.diag(rng.uniform(-spectral_radius, spectral_radius, size=d))
    else:
        A = rng.standard_normal((d, d))
        rho = np.max(np.abs(np.linalg.eigvals(A)))
        A = A * (spectral_radius / rho)
    x = rng.standard_normal((B, T, d))
    s0 = rng.standard_normal((B, d))
    return {"kind": "linear", "d": d, "d_in": d, "T": int(T), "A": A, "x": x, "s0": s0}


def mean_field_rnn(B: int, T: int, d: int, g: float, seed: int, amp: float = 0.1,
                   period: float = 50.0) -> dict:
    """Mean-field RNN of the threshold experiment: W_ij iid N(0, g^2/d) with W_ii = 0
    (shared by the batch), mild sinusoidal inputs u[b, t, i] = amp sin(2 pi t / period +
    phase[b, i]) with uniform phases, and s0 ~ N(0, 1)."""
    rng = np.random.default_rng(seed)
    W = rng.standard_normal((d, d)) * (g / np.sqrt(d))
    np.fill_diagonal(W, 0.0)
    phase = rng.uniform(0.0, 2.0 * np.pi, size=(B, 1, d))
    t = np.arange(1, T + 1, dtype=np.float64).reshape(1, T, 1)
    x = amp * np.sin(2.0 * np.pi * t / period + phase)
    s0 = rng.standard_normal((B, d))
    return {"kind": "rnn_tanh", "d": d, "T": int(T), "W": W, "x": x, "s0": s0, "g": g}


def two_well(B: int, T: int, d: int, seed: int, eps: float = 0.01) -> dict:
    """Two-well potential of the Langevin experiment: a mixture of two diagonal
    Gaussians with equal weights centred at -1.4 and +1.6 on the separating axis
    (coordinate 1, or 0 when d = 1) and 0 elsewhere; variances 0.5 on that axis and 1.0
    on the others (anisotropic). Standard normal noise draws x [B][T][d], s0 ~ N(0, 1).
    params [4d+2] = m1 | m2 | v1 | v2 | w1 | w2."""
    rng = np.random.default_rng(seed)
    ax = 1 if d >= 2 else 0
    m1 = np.zeros(d)
    m2 = np.zeros(d)
    m1[ax], m2[ax] = -1.4, 1.6
    v = np.ones(d)
    v[ax] = 0.5
    params = np.concatenate([m1, m2, v, v, [0.5, 0.5]])
    x = rng.standard_normal((B, T, d))
    s0 = rng.standard_normal((B, d))
    return {"kind": "langevin_2well", "d": d, "T": int(T), "params": params, "dt": eps,
            "x": x, "s0": s0}


def lorenz96(B: int, d: int, seed: int, F: float = 8.0, dt: float = 0.01,
             spread: float = 1.0) -> dict:
    """Lorenz-96 with forcing F: initial points F + spread * N(0, 1) per coordinate."""
    rng = np.random.default_rng(seed)
    s0 = F + spread * rng.standard_normal((B, d))
    return {"kind": "lorenz96_dp5", "d": d, "params": np.full(B, F), "dt": dt, "s0": s0}


def word_problem(B: int, T: int, seed: int, d: int = 5) -> dict:
    """Group word problem in S_d: one uniformly random permutation of range(d) per step
    (as source indices, x [B][T][d]) and the distinct vocabulary s0 = (1, ..., d)."""
    rng = np.random.default_rng(seed)
    x = np.ascontiguousarray(
        rng.permuted(np.broadcast_to(np.arange(d), (B, T, d)), axis=2).astype(np.float64))
    s0 = np.broadcast_to(np.arange(1, d + 1, dtype=np.float64), (B, d)).copy()
    return {"kind": "permute", "d": d, "T": int(T), "x": x, "s0": s0}


def ragged_lengths(B: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """Sequence lengths uniform on the integers [lo, hi]."""
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi + 1, size=B).astype(np.int64)


def offsets_from_lengths(lengths) -> np.ndarray:
    """CSR offsets [B+1] of a packed ragged batch."""
    lengths = np.asarray(lengths, dtype=np.int64)
    out = np.zeros(len(lengths) + 1, dtype=np.int64)
    np.cumsum(lengths, out=out[1:])
    return out


def targets_noise(shape, seed: int) -> np.ndarray:
    """Standard normal draws (e.g. for random initial guesses passed in as inputs)."""
    return np.random.default_rng(seed).standard_normal(shape)
