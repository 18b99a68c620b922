"""Counter-based SplitMix64 random numbers (vectorised, numpy).

SplitMix64 is the generator of Steele, Lea & Flood, "Fast splittable
pseudorandom number generators" (OOPSLA 2014): the k-th output of a stream
is the 64-bit finaliser ``mix64`` applied to ``base + (k + 1) * GAMMA`` with
``GAMMA = 0x9E3779B97F4A7C15`` (the odd integer nearest 2^64 / phi).  Because
each output depends only on (base, k) the generator is counter-based: any
draw can be produced independently of every other, so rejection loops can be
vectorised over particles while staying bit-for-bit reproducible.

This module draws the synthetic inputs only; it holds none of the N-body
method's arithmetic.
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
# Odd constant used to spread stream identifiers before mixing them into a key.
_STREAM_SPREAD = np.uint64(0xD1342543DE82EF95)
_TWO_M53 = 1.0 / 9007199254740992.0  # 2^-53


def mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output finaliser on uint64 arrays (wrap-around arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream_key(seed: int, stream: int) -> np.uint64:
    """Base value of the sub-stream ``stream`` of generator ``seed``."""
    s = np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
    t = np.array([stream & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
    return mix64(mix64(s) + (t + np.uint64(1)) * _STREAM_SPREAD)[0]


def bits(seed: int, stream: int, counter: np.ndarray) -> np.ndarray:
    """Raw 64-bit outputs number ``counter`` of sub-stream ``stream``."""
    c = np.asarray(counter, dtype=np.uint64)
    return mix64(stream_key(seed, stream) + (c + np.uint64(1)) * GAMMA)


def uniform(seed: int, stream: int, counter: np.ndarray) -> np.ndarray:
    """Doubles in [0, 1): the top 53 bits of each output times 2^-53."""
    return (bits(seed, stream, counter) >> np.uint64(11)).astype(np.float64) * _TWO_M53


def uniform_open(seed: int, stream: int, counter: np.ndarray) -> np.ndarray:
    """Doubles in (0, 1): (top 53 bits + 0.5) times 2^-53."""
    return ((bits(seed, stream, counter) >> np.uint64(11)).astype(np.float64) + 0.5) * _TWO_M53
