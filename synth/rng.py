"""Counter-based SplitMix64 streams (Steele, Lea & Flood, OOPSLA 2014).

The i-th output of the stream with key K is mix64(K + (i + 1) * GOLDEN), where
mix64 is the published SplitMix64 finaliser.  Everything here is integer
arithmetic modulo 2**64, so the words are identical on every platform; doubles
are formed as (word >> 11) * 2**-53, which is exact.

This module draws the synthetic inputs only (networks and cell conditions).  It
holds none of the chemistry: both the oracle and the CUDA library receive the
arrays it produces.
"""
from __future__ import annotations

import numpy as np

M64 = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15
_C1 = 0xBF58476D1CE4E5B9
_C2 = 0x94D049BB133111EB
INV2_53 = 1.0 / 9007199254740992.0


def mix64(z: int) -> int:
    z &= M64
    z = ((z ^ (z >> 30)) * _C1) & M64
    z = ((z ^ (z >> 27)) * _C2) & M64
    return z ^ (z >> 31)


def stream_key(seed: int, stream: int) -> int:
    """Key of an independent sub-stream (e.g. one per input array)."""
    return mix64((seed & M64) ^ mix64((stream * 0xD1B54A32D192ED03) & M64))


class SplitMix64:
    """Sequential view of one counter-based stream."""

    def __init__(self, key: int):
        self.key = key & M64
        self.i = 0

    def next_u64(self) -> int:
        self.i += 1
        return mix64((self.key + self.i * GOLDEN) & M64)

    def uniform(self) -> float:
        """Uniform double in [0, 1)."""
        return (self.next_u64() >> 11) * INV2_53

    def below(self, n: int) -> int:
        """Integer in [0, n) by 32x32 multiply-shift (Lemire, no rejection)."""
        return ((self.next_u64() >> 32) * n) >> 32

    def weighted(self, weights) -> int:
        """Index drawn with probability proportional to integer weights."""
        total = int(sum(weights))
        r = self.below(total)
        acc = 0
        for idx, w in enumerate(weights):
            acc += int(w)
            if r < acc:
                return idx
        raise AssertionError("unreachable")


def uniform_array(key: int, n: int, offset: int = 0) -> np.ndarray:
    """Vectorised stream: outputs offset+1 .. offset+n of the stream with key."""
    i = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(key) + i * np.uint64(GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(_C1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(_C2)
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * INV2_53
