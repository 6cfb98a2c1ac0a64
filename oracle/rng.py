"""Counter-based SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014; the 64-bit finaliser published
with it) used for the random initial angles theta_init of Sec. IV-B.

The value for restart b and spin i is the generator's output after
counter + 1 increments from ``seed``, with counter = (b << 32) | i, mapped to
[-1, 1) with 53 random bits. The initial angle is theta = asin(x0), so the
initial relaxed spin sin(theta) is the uniform draw itself.
"""

from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
M1 = np.uint64(0xBF58476D1CE4E5B9)
M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, counter) -> np.ndarray:
    """Output number ``counter`` (0-based) of SplitMix64 started at ``seed``."""
    c = np.asarray(counter, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (c + np.uint64(1)) * GAMMA
        z = (z ^ (z >> np.uint64(30))) * M1
        z = (z ^ (z >> np.uint64(27))) * M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform_pm1(seed: int, restarts: int, n: int) -> np.ndarray:
    """x0[i, b] uniform in [-1, 1), shape (n, restarts), float64."""
    b = np.arange(restarts, dtype=np.uint64)[None, :]
    i = np.arange(n, dtype=np.uint64)[:, None]
    z = splitmix64(seed, (b << np.uint64(32)) | i)
    u = (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return 2.0 * u - 1.0


def theta_init(seed: int, restarts: int, n: int) -> np.ndarray:
    """theta_init = asin(x0), shape (n, restarts)."""
    return np.arcsin(uniform_pm1(seed, restarts, n))
