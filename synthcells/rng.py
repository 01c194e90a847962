"""Counter-based random numbers (splitmix64) for the synthetic inputs.

splitmix64 is Steele, Lea and Flood, "Fast splittable pseudorandom number
generators" (OOPSLA 2014): state advances by the golden-ratio increment
0x9E3779B97F4A7C15 and each output is the 64-bit finaliser applied to the
state.  Here the state for draw number ``i`` of stream ``key`` is
``key * 0x9E3779B97F4A7C15 + (i + 1) * 0x9E3779B97F4A7C15`` so that any draw
can be regenerated from (key, i) alone.

This module holds no arithmetic of the J/K method; it only makes numbers.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

MASTER_SEED = 2410022278


def _mix(z: np.ndarray) -> np.ndarray:
    z = z.copy()
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


class Stream:
    """A sequential reader over the counter-based generator for one key."""

    def __init__(self, key: int):
        self.key = np.uint64(key & 0xFFFFFFFFFFFFFFFF)
        self.counter = 0

    def bits(self, n: int) -> np.ndarray:
        with np.errstate(over="ignore"):
            idx = np.arange(self.counter + 1, self.counter + 1 + n, dtype=np.uint64)
            z = self.key * _GOLDEN + idx * _GOLDEN
            out = _mix(z)
        self.counter += n
        return out

    def uniform(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        """Uniform doubles in [lo, hi) from the top 53 bits."""
        u = (self.bits(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u

    def normal(self, n: int) -> np.ndarray:
        """Standard normals by the Box-Muller transform (two uniforms each)."""
        u1 = self.uniform(n)
        u2 = self.uniform(n)
        u1 = np.maximum(u1, 1e-300)
        return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)

    def loguniform(self, n: int, lo: float, hi: float) -> np.ndarray:
        return np.exp(self.uniform(n, np.log(lo), np.log(hi)))

    def integers(self, n: int, lo: int, hi: int) -> np.ndarray:
        """Integers uniform in [lo, hi] inclusive."""
        u = self.uniform(n)
        return (lo + np.floor(u * (hi - lo + 1))).astype(np.int64)


def stream(config_index: int, purpose: int = 0) -> Stream:
    """The stream for one synthetic config: master seed + config index, then a
    purpose tag so that geometry, basis and orbitals draw independent numbers."""
    return Stream(((MASTER_SEED + config_index) << 8) ^ purpose)
