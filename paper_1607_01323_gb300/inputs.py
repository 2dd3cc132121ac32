"""Seeded synthetic inputs shared by the tests, the bench and the oracle runs.

This module holds none of the method's arithmetic: it only draws numbers.
Every value is a pure function of (seed, stream name, global index), so a
value never depends on how an array is laid out or chunked.

Generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), used in counter mode:

    key   = mix(seed XOR fnv1a64(stream))
    u64_i = mix(key + (i + 1) * 0x9E3779B97F4A7C15)

with mix the SplitMix64 output function
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9
    z = (z ^ (z >> 27)) * 0x94D049BB133111EB
    z ^ (z >> 31).

uniform[-1, 1) = 2 * (u64 >> 11) * 2^-53 - 1;  normal(0, 1) by Box-Muller on
the pair of indices (2j, 2j+1).
"""
import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z):
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _fnv1a64(name):
    h = 0xCBF29CE484222325
    for ch in name.encode():
        h ^= ch
        h = (h * 0x100000001B3) & 0xFFFFFFFFFFFFFFFF
    return np.uint64(h)


def u64(seed, stream, start, count):
    """Raw 64-bit draws for global indices start .. start+count-1."""
    key = _mix(np.uint64(seed) ^ _fnv1a64(stream))
    idx = np.arange(start, start + count, dtype=np.uint64) + np.uint64(1)
    with np.errstate(over="ignore"):
        return _mix(key + idx * _GOLDEN)


def uniform(seed, stream, n, start=0):
    """n draws from uniform[-1, 1) (float64)."""
    u = u64(seed, stream, start, n)
    return 2.0 * (u >> np.uint64(11)).astype(np.float64) * 2.0 ** -53 - 1.0


def normal(seed, stream, n, start=0):
    """n draws from N(0, 1) (float64); index i uses the Box-Muller pair of i // 2."""
    j0 = start // 2
    npairs = (start + n + 1) // 2 - j0
    u = u64(seed, stream, 2 * j0, 2 * npairs)
    u1 = ((u[0::2] >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53  # (0, 1]
    u2 = (u[1::2] >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    r = np.sqrt(-2.0 * np.log(u1))
    g = np.empty(2 * npairs)
    g[0::2] = r * np.cos(2.0 * np.pi * u2)
    g[1::2] = r * np.sin(2.0 * np.pi * u2)
    off = start - 2 * j0
    return g[off:off + n]
