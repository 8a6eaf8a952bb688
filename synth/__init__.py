"""Seeded synthetic inputs shared by the CUDA path's tests/benchmark and the oracle.

This module holds random-number generation only -- none of the key-switching
arithmetic.  Moduli are passed in by the caller; nothing here computes primes,
transforms or keys.

Generator: SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014), used counter-style: draw i of a stream with seed s is
mix(s + (i+1) * 0x9E3779B97F4A7C15).  A stream seed is derived from the master
seed and an object name plus an index, so the oracle and the GPU read identical
values for, e.g., limb 5 of the ciphertext polynomial "ct0/a".

Distributions (the paper fixes none of them; the configurations name them):

* ``uniform_residues`` -- uniform in [0, q) per limb, by rejection: take the top
  bits(q) bits of each draw and keep draws < q, in draw order.
* ``ternary`` -- uniform over {-1, 0, 1}: top two bits, reject 3, subtract 1.
* ``gaussian`` -- rounded N(0, sigma^2) by the Box-Muller cosine branch over
  53-bit uniforms, rejecting |e| > bound (default sigma 3.2, bound 19).
* ``small_uniform`` -- uniform integers in [-B, B] by rejection.
"""
from __future__ import annotations

import numpy as np

MASTER_SEED = 2112063960
_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK64 = (1 << 64) - 1


def _mix(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def _mix_int(x: int) -> int:
    return int(_mix(np.array([x & _MASK64], dtype=np.uint64))[0])


def _fnv1a64(s: str) -> int:
    h = 0xCBF29CE484222325
    for byte in s.encode():
        h ^= byte
        h = (h * 0x100000001B3) & _MASK64
    return h


def stream_seed(name: str, index: int = 0, master: int = MASTER_SEED) -> int:
    """Seed of the stream for (name, index) under the master seed."""
    return _mix_int(master ^ _fnv1a64(name) ^ _mix_int(index * 0xD1B54A32D192ED03 + 1))


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Draws offset .. offset+count-1 of the SplitMix64 stream with this seed."""
    i = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & _MASK64) + i * _GAMMA
    return _mix(z)


def _accept(seed: int, n: int, transform, keep):
    """First n accepted values of transform(draw), in draw order."""
    out = []
    have, offset = 0, 0
    batch = max(64, n + n // 4 + 16)
    while have < n:
        d = transform(splitmix64(seed, batch, offset))
        d = d[keep(d)]
        out.append(d)
        have += d.size
        offset += batch
    return np.concatenate(out)[:n]


def uniform_limb(q: int, N: int, seed: int) -> np.ndarray:
    bits = int(q).bit_length()
    shift = np.uint64(64 - bits)
    qq = np.uint64(q)
    return _accept(seed, N, lambda d: d >> shift, lambda x: x < qq).astype(np.uint64)


def uniform_residues(moduli, N: int, name: str, indices=None, master: int = MASTER_SEED) -> np.ndarray:
    """[len(moduli)][N] uniform residues; limb r uses stream (name, indices[r])."""
    if indices is None:
        indices = range(len(moduli))
    out = np.empty((len(moduli), N), dtype=np.uint64)
    for r, (q, idx) in enumerate(zip(moduli, indices)):
        out[r] = uniform_limb(int(q), N, stream_seed(name, int(idx), master))
    return out


def ternary(N: int, name: str, master: int = MASTER_SEED) -> np.ndarray:
    seed = stream_seed(name, 0, master)
    v = _accept(seed, N, lambda d: d >> np.uint64(62), lambda x: x < np.uint64(3))
    return v.astype(np.int64) - 1


def gaussian(N: int, name: str, sigma: float = 3.2, bound: int = 19, master: int = MASTER_SEED) -> np.ndarray:
    seed = stream_seed(name, 0, master)

    def transform(d):
        d = d[: (d.size // 2) * 2].reshape(-1, 2)
        u1 = ((d[:, 0] >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)
        u2 = (d[:, 1] >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
        z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2) * sigma
        return np.floor(z + 0.5).astype(np.int64)

    return _accept(seed, N, transform, lambda x: np.abs(x) <= bound)


def small_uniform(N: int, name: str, bound: int, master: int = MASTER_SEED) -> np.ndarray:
    seed = stream_seed(name, 0, master)
    span = 2 * bound + 1
    bits = max(1, span.bit_length())
    shift = np.uint64(64 - bits)
    v = _accept(seed, N, lambda d: d >> shift, lambda x: x < np.uint64(span))
    return v.astype(np.int64) - bound


def uniform_ints(n: int, lo: int, hi: int, name: str, master: int = MASTER_SEED) -> list[int]:
    """n integers uniform in [lo, hi] (e.g. the levels of a batch), by rejection."""
    seed = stream_seed(name, 0, master)
    span = hi - lo + 1
    bits = max(1, (span - 1).bit_length())
    shift = np.uint64(64 - bits)
    v = _accept(seed, n, lambda d: d >> shift, lambda x: x < np.uint64(span))
    return [int(x) + lo for x in v]


def exponential_gaps(n: int, mean: float, name: str, master: int = MASTER_SEED) -> np.ndarray:
    """n exponential inter-arrival gaps with the given mean (Poisson arrivals)."""
    d = splitmix64(stream_seed(name, 0, master), n)
    u = (d >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))
    return -np.log1p(-u) * mean
