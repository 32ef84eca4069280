"""Counter-based SplitMix64 generator and the particle templates drawn from it.

SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014): state_{n} = seed + n * 0x9E3779B97F4A7C15, output =
mix(state_{n}) with the published two multiply/xor-shift rounds.  Because the
n-th output depends only on (seed, n), any slice of the stream can be
regenerated independently and the generator is bit-identical on every machine.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Outputs offset .. offset+count-1 of the SplitMix64 stream of `seed` (uint64)."""
    with np.errstate(over="ignore"):
        n = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed) + n * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of each SplitMix64 output."""
    return (splitmix64(seed, count, offset) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def templates(k_max: int, seed: int = 0) -> np.ndarray:
    """Pre-drawn delta-pose templates u_k in [-1, 1]^6, float32, shape (k_max, 6).

    Row k = (rx, ry, rz, tx, ty, tz): a rotation vector in units of the search
    size's omega (degrees) and a translation in units of its v (centimetres).
    Row 0 is all zeros, so particle 0 is always the current pose itself; the
    other rows are uniform on the cube (Sec. III-B samples delta poses
    uniformly within the search size).  The same rows are reused in every
    iteration and frame, and a search with K particles uses rows 0..K-1.
    """
    if k_max < 1:
        raise ValueError("k_max must be >= 1")
    u = uniform01(seed, 6 * k_max).reshape(k_max, 6) * 2.0 - 1.0
    u[0, :] = 0.0
    return u.astype(np.float32)
