"""Seeded random streams for synthetic CVRPSD workloads.

Two generators, both defined by their published algorithms so that any other
implementation (the CUDA scenario generator included) can reproduce them bit
for bit:

* SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
  generators", OOPSLA 2014; the 64-bit finaliser as given by Vigna) drives the
  host-side instance draws: coordinates, mean demands, tours, tour sizes.
* Philox4x32-10 (Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as
  easy as 1, 2, 3", SC 2011) is a counter-based generator: the random words
  for demand (customer i, scenario s) are a pure function of (key, counter),
  so any subset of scenarios can be produced without generating the rest.

This module holds no Split arithmetic.
"""
from __future__ import annotations

import numpy as np

MASK64 = (1 << 64) - 1

# SplitMix64 constants (golden-ratio increment and the two finaliser
# multipliers of the published generator).
_SM_GAMMA = 0x9E3779B97F4A7C15
_SM_M1 = 0xBF58476D1CE4E5B9
_SM_M2 = 0x94D049BB133111EB


class SplitMix64:
    """SplitMix64 stream with unbiased bounded draws and Fisher-Yates."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + _SM_GAMMA) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * _SM_M1) & MASK64
        z = ((z ^ (z >> 27)) * _SM_M2) & MASK64
        return z ^ (z >> 31)

    def below(self, m: int) -> int:
        """Uniform integer in [0, m) by rejection (no modulo bias)."""
        if m <= 0:
            raise ValueError("m must be positive")
        limit = (1 << 64) - ((1 << 64) % m)
        while True:
            x = self.next_u64()
            if x < limit:
                return x % m

    def integers(self, lo: int, hi: int, count: int) -> np.ndarray:
        """`count` uniform integers in the closed range [lo, hi]."""
        span = hi - lo + 1
        return np.array([lo + self.below(span) for _ in range(count)], dtype=np.int64)

    def permutation(self, values) -> np.ndarray:
        """Fisher-Yates shuffle (Durstenfeld's in-place form) of `values`."""
        a = list(values)
        for k in range(len(a) - 1, 0, -1):
            j = self.below(k + 1)
            a[k], a[j] = a[j], a[k]
        return np.array(a, dtype=np.int64)


def derive_seed(*parts: int) -> int:
    """Combine integers into one 64-bit seed by chaining SplitMix64 outputs."""
    h = 0
    for p in parts:
        h = SplitMix64((h ^ (p & MASK64)) & MASK64).next_u64()
    return h


# Philox4x32-10 constants from the Random123 paper: the two round multipliers
# and the two Weyl key increments.
PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85
_M32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0: int, k1: int):
    """Vectorised Philox4x32 with 10 rounds.

    Counters are arrays (broadcast together) of uint32 values; the key is two
    Python ints. Returns four uint32 arrays.
    """
    c0, c1, c2, c3 = np.broadcast_arrays(
        *(np.asarray(c, dtype=np.uint64) & _M32 for c in (c0, c1, c2, c3)))
    c0 = c0.copy(); c1 = c1.copy(); c2 = c2.copy(); c3 = c3.copy()
    m0 = np.uint64(PHILOX_M0)
    m1 = np.uint64(PHILOX_M1)
    key0 = k0 & 0xFFFFFFFF
    key1 = k1 & 0xFFFFFFFF
    for r in range(10):
        if r > 0:
            key0 = (key0 + PHILOX_W0) & 0xFFFFFFFF
            key1 = (key1 + PHILOX_W1) & 0xFFFFFFFF
        p0 = m0 * c0            # exact: both factors < 2^32
        p1 = m1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _M32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _M32
        n0 = hi1 ^ c1 ^ np.uint64(key0)
        n2 = hi0 ^ c3 ^ np.uint64(key1)
        c0, c1, c2, c3 = n0, lo1, n2, lo0
    return (c0.astype(np.uint32), c1.astype(np.uint32),
            c2.astype(np.uint32), c3.astype(np.uint32))
