"""Seeded synthetic inputs for the G_{c,d} hash.

This module holds no arithmetic of the hash itself: it only draws key and seed
bits, so both the oracle-side tests and the CUDA side may use it.

Generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), output i of the stream seeded with s being
mix64(s + (i + 1) * 0x9E3779B97F4A7C15) with the published mix constants.

A block of size n is drawn from one stream: ceil(n/64) limbs of x, then as
many of a, then of b (little-endian 64-bit limbs). Bits >= n of the top limb
are cleared, and bit 0 of a is set so that gcd(a, 2) = 1 as the family
requires (Sec. 2.3, Eq. 6). Uniform key bits stand in for a reconciled key:
the paper's timing runs (Sec. 4, Table 2) hash uniform n-bit blocks, and no
dataset is involved.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, start: int, count: int) -> np.ndarray:
    """Outputs start .. start+count-1 of the SplitMix64 stream seeded with ``seed``."""
    with np.errstate(over="ignore"):
        i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def _mask_top(limbs: np.ndarray, nbits: int) -> None:
    r = nbits % 64
    if r:
        limbs[-1] &= np.uint64((1 << r) - 1)


@dataclass
class Block:
    """One hash problem: key x, seeds a (the multiplier c) and b (the addend d)."""

    n: int
    m: int
    x: np.ndarray
    a: np.ndarray
    b: np.ndarray
    seed: int


def make_block(n: int, m: int, seed: int = 1) -> Block:
    """Uniform x, a (odd) and b of n bits from SplitMix64(seed)."""
    if n <= 0 or m <= 0 or m > n:
        raise ValueError(f"invalid sizes n={n} m={m}")
    L = (n + 63) // 64
    s = splitmix64(seed, 0, 3 * L)
    x, a, b = s[:L].copy(), s[L : 2 * L].copy(), s[2 * L :].copy()
    for v in (x, a, b):
        _mask_top(v, n)
    a[0] |= np.uint64(1)
    return Block(n, m, x, a, b, seed)


@dataclass
class ToeplitzBlock:
    """One Toeplitz-hash problem: key x of n bits, seed s of n + m - 1 bits."""

    n: int
    m: int
    x: np.ndarray
    s: np.ndarray
    seed: int


def make_toeplitz_block(n: int, m: int, seed: int = 1) -> ToeplitzBlock:
    """Uniform x (n bits) then s (n + m - 1 bits) from SplitMix64(seed)."""
    if n <= 0 or m <= 0 or m > n:
        raise ValueError(f"invalid sizes n={n} m={m}")
    Lx, Ls = (n + 63) // 64, (n + m - 1 + 63) // 64
    r = splitmix64(seed ^ 0x70E9_0000_0000_0001, 0, Lx + Ls)
    x, s = r[:Lx].copy(), r[Lx:].copy()
    _mask_top(x, n)
    _mask_top(s, n + m - 1)
    return ToeplitzBlock(n, m, x, s, seed)


def uniforms(seed: int, count: int) -> np.ndarray:
    """``count`` doubles in [0, 1) from the top 53 bits of SplitMix64(seed)."""
    return (splitmix64(seed, 0, count) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


def batch_sizes(count: int, n_lo: int, n_hi: int, r_lo: float = 0.1, r_hi: float = 0.5,
                seed: int = 1) -> list[tuple[int, int]]:
    """(n, m) pairs with n = floor(exp(U(ln n_lo, ln n_hi))) and m = floor(n * r),
    r ~ U(r_lo, r_hi): the log-uniform block-size mix of the batched and served
    workloads. Sizes come from a stream seeded apart from the key streams."""
    u = uniforms(seed ^ 0x5A5A_0000_0000_0001, 2 * count)
    out = []
    lo, hi = math.log(n_lo), math.log(n_hi)
    for i in range(count):
        n = int(math.floor(math.exp(lo + (hi - lo) * float(u[2 * i]))))
        n = min(max(n, n_lo), n_hi)
        r = r_lo + (r_hi - r_lo) * float(u[2 * i + 1])
        m = max(1, int(math.floor(n * r)))
        out.append((n, m))
    return out


def make_batch(count: int, n_lo: int, n_hi: int, r_lo: float = 0.1, r_hi: float = 0.5,
               seed: int = 1) -> list[Block]:
    """``count`` independent blocks; block i draws its bits from seed + i."""
    return [make_block(n, m, seed + i) for i, (n, m) in
            enumerate(batch_sizes(count, n_lo, n_hi, r_lo, r_hi, seed))]


def poisson_arrivals(rate_hz: float, duration_s: float, seed: int = 7) -> np.ndarray:
    """Arrival times (seconds) of a Poisson process of the given rate."""
    est = int(rate_hz * duration_s * 1.5 + 64)
    u = uniforms(seed ^ 0x0A11_1BA1_0000_0001, est)
    gaps = -np.log1p(-u) / rate_hz
    t = np.cumsum(gaps)
    return t[t < duration_s]
