"""SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014), written from its published definition.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Counter form used by the densification initial mask: the i-th output of the
generator seeded with `seed` is mix(seed + (i + 1) * GAMMA) (mod 2^64), with
the finaliser
  z ^= z >> 30; z *= 0xBF58476D1CE4E5B9; z ^= z >> 27; z *= 0x94D049BB133111EB;
  z ^= z >> 31.
"""

from __future__ import annotations

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
M1 = 0xBF58476D1CE4E5B9
M2 = 0x94D049BB133111EB
MASK64 = (1 << 64) - 1


def splitmix64_scalar(seed: int, i: int) -> int:
    """Plain-integer reference of one output (slow, for pins)."""
    z = (seed + (i + 1) * GAMMA) & MASK64
    z ^= z >> 30
    z = (z * M1) & MASK64
    z ^= z >> 27
    z = (z * M2) & MASK64
    z ^= z >> 31
    return z


def splitmix64(seed: int, idx: np.ndarray) -> np.ndarray:
    """Vectorised outputs for counters idx (uint64 arithmetic wraps mod 2^64)."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed & MASK64) + (idx.astype(np.uint64) + np.uint64(1)) * np.uint64(GAMMA)
        z ^= z >> np.uint64(30)
        z *= np.uint64(M1)
        z ^= z >> np.uint64(27)
        z *= np.uint64(M2)
        z ^= z >> np.uint64(31)
    return z
