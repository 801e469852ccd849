"""Seeded forest-pair subsample for the distortion matrix (Section 2.2: D is
computed with "a small subset" of forest pairs; the paper gives neither the
fraction nor the rule).

Reading: an independent Bernoulli(p) draw per unordered forest pair (a, b),
a < b, made reproducible by hashing the pair:

    key  = a * 2^32 + b
    h    = SplitMix64 output for state (seed XOR key)
    keep = (p >= 1) or h < floor(p * 2^64)

SplitMix64 is the generator of Steele, Lea and Flood (OOPSLA 2014): one step
adds the constant 0x9E3779B97F4A7C15 to the state, then mixes with
z ^= z >> 30; z *= 0xBF58476D1CE4E5B9; z ^= z >> 27; z *= 0x94D049BB133111EB;
z ^= z >> 31.  ``splitmix64`` returns that first output.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(state) -> np.ndarray:
    """First SplitMix64 output for each 64-bit starting state (wrapping arithmetic)."""
    z = np.asarray(state, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = z + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def threshold(p: float) -> int:
    """floor(p * 2^64) for 0 <= p < 1 (exact: scaling a double by 2^64)."""
    return int(float(p) * 18446744073709551616.0)


def keep_pairs(a, b, seed: int, p: float) -> np.ndarray:
    """Boolean mask of the forest pairs kept in the subsample."""
    a = np.asarray(a, dtype=np.int64)
    b = np.asarray(b, dtype=np.int64)
    if p >= 1.0:
        return np.ones(a.shape, dtype=bool)
    if p <= 0.0:
        return np.zeros(a.shape, dtype=bool)
    lo = np.minimum(a, b).astype(np.uint64)
    hi = np.maximum(a, b).astype(np.uint64)
    key = (lo << np.uint64(32)) | hi
    h = splitmix64(np.uint64(seed) ^ key)
    return h < np.uint64(threshold(p))


def subsample(pair_list, seed: int, p: float):
    a, b = pair_list
    m = keep_pairs(a, b, seed, p)
    return np.asarray(a)[m], np.asarray(b)[m]
