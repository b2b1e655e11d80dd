"""SplitMix64 counter generator (oracle side; test infrastructure only).

Steele, Lea & Flood, "Fast splittable pseudorandom number generators" (OOPSLA
2014): the state advances by the golden gamma 0x9E3779B97F4A7C15 and each
output is the state passed through the variant-13 finaliser.  The i-th output
of a stream seeded with s is therefore mix(s + (i+1)*gamma).  The oracle uses it
for the Lanczos start vector, which the method draws itself; the CUDA library
implements the same published generator on its own.
"""
from __future__ import annotations

import numpy as np

_MASK = (1 << 64) - 1
_GAMMA = 0x9E3779B97F4A7C15


def _mix(z: int) -> int:
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
    return z ^ (z >> 31)


def splitmix64(seed: int, count: int) -> list[int]:
    """First `count` outputs of SplitMix64 seeded with `seed`."""
    return [_mix((seed + (i + 1) * _GAMMA) & _MASK) for i in range(count)]


def uniform_pm1(seed: int, n: int) -> np.ndarray:
    """n values in [-1, 1): 2 * (top 53 bits of output i) * 2^-53 - 1."""
    out = np.empty(n)
    for i, z in enumerate(splitmix64(seed, n)):
        out[i] = 2.0 * ((z >> 11) * 2.0 ** -53) - 1.0
    return out
