"""The random initial guess of Sec. 3.3.3 (iid standard normal entries), float64.

Test infrastructure only. The guess is drawn by a counter-based generator so that any
entry can be computed on its own: entry e of the packed state (e = row * d + i) takes
outputs 2e+1 and 2e+2 of the SplitMix64 stream started at the seed (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014: output n, n >= 1,
is the 64-bit mix of seed + n * gamma with the golden-ratio gamma), and the Box-Muller
transform turns the two into one normal draw:

    u1 = ((z1 >> 11) + 1) 2^-53 in (0, 1],   u2 = (z2 >> 11) 2^-53 in [0, 1),
    x  = sqrt(-2 ln u1) cos(2 pi u2).
"""
from __future__ import annotations

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
M1 = 0xBF58476D1CE4E5B9
M2 = 0x94D049BB133111EB


def splitmix64(seed, n):
    """Output n (n >= 1, array) of the SplitMix64 stream started at `seed`: the mix of
    seed + n * GAMMA, all arithmetic modulo 2^64."""
    n = np.asarray(n, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + n * np.uint64(GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(M1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(M2)
        return z ^ (z >> np.uint64(31))


def randn_guess(seed, n_rows, d):
    """Initial guess s^(0) [n_rows, d] of iid N(0, 1) entries for the packed state."""
    e = np.arange(n_rows * d, dtype=np.uint64)
    z1 = splitmix64(seed, np.uint64(2) * e + np.uint64(1))
    z2 = splitmix64(seed, np.uint64(2) * e + np.uint64(2))
    u1 = ((z1 >> np.uint64(11)) + np.uint64(1)).astype(np.float64) * 2.0 ** -53
    u2 = (z2 >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    return (np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)).reshape(n_rows, d)
