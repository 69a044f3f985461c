"""Counter-based random numbers for the seeded synthetic inputs.

Every draw is a pure function of (seed, stream, index): the SplitMix64
finaliser (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) applied to a Weyl sequence keyed by the seed and the
stream.  Because no state is carried between draws, a vectorised numpy draw of
a whole array and a scalar draw of one element give the same bits, and the
result does not depend on chunking or thread count.

This module holds no arithmetic of the evaluation method; it only makes
inputs.
"""
from __future__ import annotations

import numpy as np

MASK64 = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB


def mix64_scalar(x: int) -> int:
    """SplitMix64 finaliser on a Python int (mod 2**64)."""
    x &= MASK64
    x = ((x ^ (x >> 30)) * _M1) & MASK64
    x = ((x ^ (x >> 27)) * _M2) & MASK64
    return x ^ (x >> 31)


def mix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser on a uint64 array (wrapping arithmetic)."""
    x = np.asarray(x, dtype=np.uint64)
    x = (x ^ (x >> np.uint64(30))) * np.uint64(_M1)
    x = (x ^ (x >> np.uint64(27))) * np.uint64(_M2)
    return x ^ (x >> np.uint64(31))


def stream_key(seed: int, stream: int) -> int:
    """Key of one named sub-stream of a seed."""
    return mix64_scalar(mix64_scalar(seed * GOLDEN + 0x1234567) ^ (stream * 0xD1B54A32D192ED03))


def u64(seed: int, stream: int, idx: np.ndarray) -> np.ndarray:
    """Raw 64-bit draws number ``idx`` of sub-stream ``stream``."""
    key = np.uint64(stream_key(seed, stream))
    idx = np.asarray(idx, dtype=np.uint64)
    return mix64(key + (idx + np.uint64(1)) * np.uint64(GOLDEN))


def uniform(seed: int, stream: int, idx: np.ndarray) -> np.ndarray:
    """float64 draws uniform on [0, 1) (53 random bits)."""
    return (u64(seed, stream, idx) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


def uniform_range(seed: int, stream: int, n: int, start: int = 0) -> np.ndarray:
    return uniform(seed, stream, np.arange(start, start + n, dtype=np.uint64))


def randint(seed: int, stream: int, idx: np.ndarray, hi: int) -> np.ndarray:
    """Integers uniform on [0, hi) by the multiply-shift (Lemire) reduction of 32 bits."""
    r = u64(seed, stream, idx) >> np.uint64(32)
    return ((r * np.uint64(hi)) >> np.uint64(32)).astype(np.int64)


def normal(seed: int, stream: int, n: int) -> np.ndarray:
    """Standard normal draws by the Box-Muller transform of two uniform streams."""
    i = np.arange(n, dtype=np.uint64)
    u1 = uniform(seed, stream, i * np.uint64(2))
    u2 = uniform(seed, stream, i * np.uint64(2) + np.uint64(1))
    u1 = np.maximum(u1, 1e-300)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


class Rng:
    """Sequential scalar view of one sub-stream (draw k is u64(seed, stream, k))."""

    __slots__ = ("key", "k")

    def __init__(self, seed: int, stream: int):
        self.key = stream_key(seed, stream)
        self.k = 0

    def next_u64(self) -> int:
        self.k += 1
        return mix64_scalar(self.key + self.k * GOLDEN)

    def random(self) -> float:
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))

    def randint(self, lo: int, hi: int) -> int:
        """Uniform integer on [lo, hi] inclusive."""
        span = hi - lo + 1
        return lo + (((self.next_u64() >> 32) * span) >> 32)

    def choice(self, seq):
        return seq[self.randint(0, len(seq) - 1)]
