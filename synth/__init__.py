"""Seeded synthetic inputs shared by the tests, the oracle side and the benchmark.

This module holds no arithmetic of the FFT or of the Navier-Stokes method: it
only turns (seed, field, linear index) into pseudo-random numbers.  Both the
CPU oracle and the CUDA path receive the arrays made here as plain inputs.

Generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), used as a counter-based generator: output
number c of the stream that starts from state 0 is mix64((c + 1) * GAMMA).
The counter of element i of field f for seed s is s * 2**40 + f * 2**36 + i.

* uniform in [-1, 1): u = (x >> 40) * 2**-24, value = 2u - 1 (exact in FP32).
* normal(0, 1): Box-Muller on two consecutive counters 2i and 2i + 1,
  u1 = ((x1 >> 11) + 1) * 2**-53 in (0, 1], u2 = (x2 >> 11) * 2**-53,
  value = sqrt(-2 ln u1) * cos(2 pi u2), in FP64.
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

SEED_SHIFT = 40
FIELD_SHIFT = 36
_CHUNK = 1 << 22


def mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (finaliser) on uint64 arrays, wrapping mod 2**64."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(counter: np.ndarray) -> np.ndarray:
    """Output number `counter` (0-based) of the SplitMix64 stream started at state 0."""
    c = np.asarray(counter, dtype=np.uint64)
    with np.errstate(over="ignore"):
        state = (c + np.uint64(1)) * GAMMA
    return mix64(state)


def counter_base(seed: int, field: int) -> int:
    if not (0 <= seed < (1 << 24)):
        raise ValueError("seed must be in [0, 2**24)")
    if not (0 <= field < 16):
        raise ValueError("field must be in [0, 16)")
    return (seed << SEED_SHIFT) | (field << FIELD_SHIFT)


def uniform_pm1(seed: int, field: int, shape) -> np.ndarray:
    """FP32 values uniform on [-1, 1) with 24-bit resolution."""
    n = int(np.prod(shape))
    base = np.uint64(counter_base(seed, field))
    out = np.empty(n, dtype=np.float32)
    for s in range(0, n, _CHUNK):
        e = min(n, s + _CHUNK)
        x = splitmix64(base + np.arange(s, e, dtype=np.uint64))
        u = (x >> np.uint64(40)).astype(np.float64) * 2.0 ** -24
        out[s:e] = (2.0 * u - 1.0).astype(np.float32)
    return out.reshape(shape)


def normal(seed: int, field: int, shape) -> np.ndarray:
    """FP64 standard normal values (Box-Muller, cosine branch only)."""
    n = int(np.prod(shape))
    if 2 * n > (1 << FIELD_SHIFT):
        raise ValueError("field too large for the counter layout")
    base = np.uint64(counter_base(seed, field))
    out = np.empty(n, dtype=np.float64)
    for s in range(0, n, _CHUNK):
        e = min(n, s + _CHUNK)
        i2 = 2 * np.arange(s, e, dtype=np.uint64)
        x1 = splitmix64(base + i2)
        x2 = splitmix64(base + i2 + np.uint64(1))
        u1 = ((x1 >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53
        u2 = (x2 >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
        out[s:e] = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
    return out.reshape(shape)


def normal_fields(seed: int, nfields: int, shape) -> np.ndarray:
    """`nfields` independent normal fields, field index f = 0 .. nfields-1."""
    return np.stack([normal(seed, f, shape) for f in range(nfields)])
