"""Counter-free seeded random numbers for the synthetic workloads.

SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014; the 64-bit finaliser constants are the ones Vigna
published with xoshiro): state advances by the golden-ratio increment and each
output is a bijective mix of the state.  Uniforms take the top 53 bits;
normals use the Box-Muller transform.  Nothing here belongs to the method: it
only draws the parameters of the initial conditions.
"""
from __future__ import annotations

import math

_MASK = (1 << 64) - 1
_GOLDEN = 0x9E3779B97F4A7C15
_MIX1 = 0xBF58476D1CE4E5B9
_MIX2 = 0x94D049BB133111EB


class SplitMix64:
    """Seeded 64-bit generator; identical stream for identical seed."""

    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + _GOLDEN) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * _MIX1) & _MASK
        z = ((z ^ (z >> 27)) * _MIX2) & _MASK
        return z ^ (z >> 31)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        """U[lo, hi) from the top 53 bits."""
        u = (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u

    def randint(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi] (inclusive)."""
        span = hi - lo + 1
        return lo + int(self.uniform() * span)

    def normal(self, mean: float = 0.0, std: float = 1.0) -> float:
        """One N(mean, std^2) draw by Box-Muller (the cosine branch only)."""
        u1 = self.uniform()
        u2 = self.uniform()
        r = math.sqrt(-2.0 * math.log(1.0 - u1))
        return mean + std * r * math.cos(2.0 * math.pi * u2)
