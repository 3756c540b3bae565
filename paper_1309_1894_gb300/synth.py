"""Seeded synthetic inputs: a counter-based splitmix64 stream, host side.

This module holds the input generators only and none of the WXPY arithmetic;
tests and the benchmark use it to build the inputs that both the oracle and the
CUDA path consume.  The library's device-side fill kernel implements the same
generator separately from the same published definition, and the GPU tests
compare the two at sampled indices.

Generator (splitmix64; G. Steele, D. Lea, C. Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014, in the 64-bit form of
S. Vigna's public-domain reference):

    mix64(z):  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9
               z = (z ^ (z >> 27)) * 0x94D049BB133111EB
               return z ^ (z >> 31)             (all arithmetic mod 2^64)

The k-th output (k = 0, 1, ...) of the generator seeded with s is
mix64(s + (k + 1) * 0x9E3779B97F4A7C15), which is what makes it counter based.

Streams.  Every quantity draws from its own stream: the stream key for
(seed, tag) is output number ``tag`` of the generator seeded with ``seed``,
and element i of the stream is output number i of the generator seeded with
that key.

Doubles.  u = (bits >> 11) * 2^-53 is uniform on [0, 1) with 53 random bits;
U(-1, 1) is 2u - 1 and U(-2, 2) is 4u - 2.  Both are exact in binary64, so any
correct implementation reproduces them bit for bit.
"""
from __future__ import annotations

import numpy as np

MASK64 = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15
MIX1 = 0xBF58476D1CE4E5B9
MIX2 = 0x94D049BB133111EB

# Stream tags: one per drawn quantity.
TAG_X = 1
TAG_Y = 2
TAG_ALPHA = 3
TAG_LEN = 4
TAG_ARRIVAL = 5

# Base seed of the synthetic workloads (the paper's arXiv date, 2013-09-07).
BASE_SEED = 20130907


def mix64_int(z: int) -> int:
    """splitmix64's output function on a Python int (mod 2^64)."""
    z &= MASK64
    z = ((z ^ (z >> 30)) * MIX1) & MASK64
    z = ((z ^ (z >> 27)) * MIX2) & MASK64
    return z ^ (z >> 31)


def splitmix64_sequence(seed: int, count: int) -> list[int]:
    """The first ``count`` outputs of splitmix64 seeded with ``seed``."""
    return [mix64_int(seed + (k + 1) * GOLDEN) for k in range(count)]


def stream_key(seed: int, tag: int) -> int:
    """Key of stream ``tag``: output number ``tag`` of the generator at ``seed``."""
    return mix64_int(seed + (tag + 1) * GOLDEN)


def _mix64_array(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(MIX1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(MIX2)
        return z ^ (z >> np.uint64(31))


def bits(seed: int, tag: int, start: int, count: int) -> np.ndarray:
    """Raw 64-bit outputs start .. start+count-1 of stream (seed, tag)."""
    key = np.uint64(stream_key(seed, tag))
    k = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = key + k * np.uint64(GOLDEN)
    return _mix64_array(z)


def u01(seed: int, tag: int, start: int, count: int) -> np.ndarray:
    """Uniform [0, 1) doubles with 53 random bits: (bits >> 11) * 2^-53."""
    b = bits(seed, tag, start, count) >> np.uint64(11)
    return b.astype(np.float64) * (2.0 ** -53)


def uniform_pm1(seed: int, tag: int, count: int, start: int = 0) -> np.ndarray:
    """U(-1, 1) values 2u - 1 (exact in binary64)."""
    return 2.0 * u01(seed, tag, start, count) - 1.0


def uniform_pm2(seed: int, tag: int, count: int, start: int = 0) -> np.ndarray:
    """U(-2, 2) values 4u - 2 (exact in binary64)."""
    return 4.0 * u01(seed, tag, start, count) - 2.0


def bits_at(seed: int, tag: int, idx: np.ndarray) -> np.ndarray:
    """Raw outputs of stream (seed, tag) at arbitrary indices ``idx``."""
    key = np.uint64(stream_key(seed, tag))
    with np.errstate(over="ignore"):
        z = key + (np.asarray(idx).astype(np.uint64) + np.uint64(1)) * np.uint64(GOLDEN)
    return _mix64_array(z)


def uniform_pm1_at(seed: int, tag: int, idx: np.ndarray) -> np.ndarray:
    """U(-1, 1) values of stream (seed, tag) at arbitrary indices ``idx``."""
    b = bits_at(seed, tag, idx) >> np.uint64(11)
    return 2.0 * (b.astype(np.float64) * (2.0 ** -53)) - 1.0


def alpha_scalar(seed: int, index: int = 0) -> float:
    """One alpha ~ U(-2, 2) from stream TAG_ALPHA at ``index``."""
    return float(uniform_pm2(seed, TAG_ALPHA, 1, start=index)[0])


def log_uniform_lengths(seed: int, count: int, lo: int, hi: int) -> np.ndarray:
    """Lengths log-uniform on [lo, hi]: floor(2^(log2 lo + u*(log2(hi+1) - log2 lo))),
    clamped to [lo, hi].  Host-only (it uses exp2/log2), never regenerated on a GPU."""
    if lo < 1 or hi < lo:
        raise ValueError("need 1 <= lo <= hi")
    u = u01(seed, TAG_LEN, 0, count)
    a, b = np.log2(float(lo)), np.log2(float(hi) + 1.0)
    n = np.floor(np.exp2(a + u * (b - a))).astype(np.int64)
    return np.clip(n, lo, hi)


def vectors(seed: int, n: int) -> tuple[float, np.ndarray, np.ndarray]:
    """(alpha, x, y) of one synthetic VecWXPY call: alpha ~ U(-2,2), x, y ~ U(-1,1)."""
    return (alpha_scalar(seed), uniform_pm1(seed, TAG_X, n),
            uniform_pm1(seed, TAG_Y, n))


def poisson_gaps(seed: int, rate: float, count: int) -> np.ndarray:
    """Exponential inter-arrival gaps (seconds) of a Poisson process of ``rate``/s."""
    u = u01(seed, TAG_ARRIVAL, 0, count)
    return -np.log1p(-u) / rate
