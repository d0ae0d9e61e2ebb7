"""Seeded synthetic inputs shared by the GPU path's tests/benchmark and the oracle.

This module holds no arithmetic of the FFT method: it only draws numbers.  The
random stream is SplitMix64 (Steele, Lea, Flood, OOPSLA 2014), written out with
numpy uint64 arithmetic so that the same seed gives the same doubles on every
machine and numpy version.

Distributions:
  * ``uniform``      -- real and imaginary parts i.i.d. U[-1, 1)
  * ``phi``          -- (rand - 0.5) * exp(phi * randn), rand in (0, 1]  (§5.1 of the paper)
  * ``gaussian``     -- parts i.i.d. N(0, 1) (Box-Muller)
  * ``spikes``       -- uniform parts, each replaced with probability 1% by +-1e12
  * ``loguniform``   -- parts +-10^U[-8, 8] with random signs
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, stream: int = 0) -> np.ndarray:
    """count outputs of SplitMix64 started at state = seed + stream * 2^32 (uint64)."""
    with np.errstate(over="ignore"):
        state0 = np.uint64((int(seed) + (int(stream) << 32)) & 0xFFFFFFFFFFFFFFFF)
        z = state0 + _GOLDEN * np.arange(1, count + 1, dtype=np.uint64)
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def unit_open0(seed: int, count: int, stream: int = 0) -> np.ndarray:
    """53-bit uniforms in (0, 1]."""
    u = splitmix64(seed, count, stream) >> np.uint64(11)
    return (u.astype(np.float64) + 1.0) * 2.0 ** -53


def uniform(seed: int, count: int, stream: int = 0, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    u = (splitmix64(seed, count, stream) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    return lo + (hi - lo) * u


def randn(seed: int, count: int, stream: int = 0) -> np.ndarray:
    """Box-Muller standard normals."""
    m = (count + 1) // 2
    u1 = unit_open0(seed, m, 2 * stream + 1)
    u2 = unit_open0(seed, m, 2 * stream + 2)
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.concatenate([r * np.cos(2 * np.pi * u2), r * np.sin(2 * np.pi * u2)])
    return z[:count]


def complex_signal(kind: str, n: int, seed: int, batch: int = 1, phi: float = 0.0) -> np.ndarray:
    """A [batch, n] complex128 array of the named distribution."""
    cnt = batch * n
    if kind == "uniform":
        re, im = uniform(seed, cnt, 0), uniform(seed, cnt, 1)
    elif kind == "phi":
        re = (unit_open0(seed, cnt, 0) - 0.5) * np.exp(phi * randn(seed, cnt, 10))
        im = (unit_open0(seed, cnt, 1) - 0.5) * np.exp(phi * randn(seed, cnt, 11))
    elif kind == "gaussian":
        re, im = randn(seed, cnt, 0), randn(seed, cnt, 1)
    elif kind == "spikes":
        re, im = uniform(seed, cnt, 0), uniform(seed, cnt, 1)
        for part, s in ((re, 2), (im, 3)):
            hit = uniform(seed, cnt, s, 0.0, 1.0) < 0.01
            sign = np.where(uniform(seed, cnt, s + 10, 0.0, 1.0) < 0.5, -1.0, 1.0)
            part[hit] = sign[hit] * 1e12
    elif kind == "loguniform":
        mags_r = 10.0 ** uniform(seed, cnt, 0, -8.0, 8.0)
        mags_i = 10.0 ** uniform(seed, cnt, 1, -8.0, 8.0)
        sr = np.where(uniform(seed, cnt, 2, 0.0, 1.0) < 0.5, -1.0, 1.0)
        si = np.where(uniform(seed, cnt, 3, 0.0, 1.0) < 0.5, -1.0, 1.0)
        re, im = sr * mags_r, si * mags_i
    else:
        raise ValueError(f"unknown distribution {kind!r}")
    return (re + 1j * im).reshape(batch, n)


def uneven_lengths(count: int, seed: int, lo: int = 1000, hi: int = 300000) -> np.ndarray:
    """Lengths drawn log-uniformly from [lo, hi], redrawn while a power of two."""
    out = np.empty(count, dtype=np.int64)
    u = uniform(seed, 4 * count, 0, np.log(lo), np.log(hi))
    j = 0
    for i in range(count):
        while True:
            v = int(round(float(np.exp(u[j])))); j += 1
            v = min(max(v, lo), hi)
            if v & (v - 1):
                break
        out[i] = v
    return out
