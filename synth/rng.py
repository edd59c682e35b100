"""Counter-based random numbers for the seeded synthetic inputs.

Every random number is a pure function of (seed, field id, counter), so any
part of a field (one timeslice, one site) can be regenerated on its own and
the same call gives the same bits on every machine.

The integer mixer is the SplitMix64 output function (Steele, Lea & Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014): a Weyl
sequence with increment 0x9e3779b97f4a7c15 fed through two xor-shift-multiply
rounds.  Gaussians come from the Box-Muller transform (Box & Muller, 1958).
All arithmetic is numpy uint64 (wrapping) and float64.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser applied elementwise to a uint64 array."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream_key(seed: int, field_id: int) -> np.uint64:
    """Key of one random stream: mixes the seed and a field id."""
    with np.errstate(over="ignore"):
        k = _mix(np.array([seed], dtype=np.uint64))[0]
        k = _mix(np.array([k ^ (np.uint64(field_id) * _GOLDEN)], dtype=np.uint64))[0]
    return np.uint64(k)


def bits(key: np.uint64, counters: np.ndarray) -> np.ndarray:
    """64 random bits per counter: SplitMix64 of key + (counter + 1) * golden."""
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(key + (c + np.uint64(1)) * _GOLDEN)


def uniform(key: np.uint64, counters: np.ndarray) -> np.ndarray:
    """Uniform doubles in (0, 1]: the top 53 bits plus one, times 2**-53."""
    b = bits(key, counters)
    return ((b >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)


def normal_pairs(key: np.uint64, pair_counters: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Two independent N(0,1) arrays from Box-Muller on counters 2k and 2k+1."""
    k = np.asarray(pair_counters, dtype=np.uint64)
    u1 = uniform(key, k * np.uint64(2))
    u2 = uniform(key, k * np.uint64(2) + np.uint64(1))
    r = np.sqrt(-2.0 * np.log(u1))
    phi = 2.0 * np.pi * u2
    return r * np.cos(phi), r * np.sin(phi)


def complex_normal(key: np.uint64, counters: np.ndarray) -> np.ndarray:
    """Complex Gaussians with E|z|^2 = 1 (real and imaginary parts N(0, 1/2))."""
    re, im = normal_pairs(key, counters)
    return (re + 1j * im) * np.sqrt(0.5)
