"""Toeplitz-hash PA on the GPU (pa_toeplitz, pa_toeplitz_seeded) against the
oracle, bit for bit: y = T x over GF(2), T[i][j] = s[i - j + n - 1]."""
import numpy as np
import pytest

import oracle
from paper_1910_04429_gb300 import binding, inputs
from tests.gpu_util import dev, host

pytestmark = pytest.mark.gpu

# (n, m): single 4096-point tiles (n + m - 1 <= 4096, also exactly 4096), the
# first two-tile length, 3 * 2^k lengths met exactly, strided plans with ragged
# tails, m = 1 and m = n, and the 10^6-bit block (transform 3 * 2^19).
SIZES = [(1, 1), (2, 1), (17, 5), (64, 64), (65, 64), (1000, 333), (2049, 2048), (3000, 1097),
         (3000, 1098), (5000, 5000), (100_000, 96_609), (100_003, 31_337), (262_144, 262_144),
         (1_000_000, 1), (1_000_000, 250_000)]


def _need_gpu():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required")
    return torch


@pytest.mark.parametrize("n,m", SIZES)
def test_matches_oracle(n, m):
    torch = _need_gpu()
    blk = inputs.make_toeplitz_block(n, m, seed=n + 7 * m)
    got = binding.toeplitz(dev(blk.x), dev(blk.s), n, m)
    torch.cuda.synchronize()
    want = oracle.toeplitz(blk.x, blk.s, n, m, threads=oracle.default_threads())
    np.testing.assert_array_equal(host(got), want)


def test_padding_bits_ignored():
    torch = _need_gpu()
    for n, m in [(70, 5), (100_003, 31_337)]:
        blk = inputs.make_toeplitz_block(n, m, seed=5)
        x, s = blk.x.copy(), blk.s.copy()
        x[-1] |= np.uint64(((1 << 64) - 1) ^ ((1 << (n % 64)) - 1))
        s[-1] |= np.uint64(((1 << 64) - 1) ^ ((1 << ((n + m - 1) % 64)) - 1))
        got = binding.toeplitz(dev(x), dev(s), n, m)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(host(got), oracle.toeplitz(blk.x, blk.s, n, m, threads=4))


def _bits(limbs, lo, count):
    b = np.unpackbits(np.ascontiguousarray(limbs, dtype=np.uint64).view(np.uint8), bitorder="little")
    return b[lo: lo + count]


def test_full_size_sampled_rows_unit_key_and_linearity():
    """n = 10^8, m = 2.5e7 (transform 2^27): sampled output bits against the
    oracle's row form; a unit key e_j gives column j of T (seed bits
    n-1-j .. n-2-j+m); and the hash is linear in the key."""
    torch = _need_gpu()
    n, m = 100_000_000, 25_000_000
    blk = inputs.make_toeplitz_block(n, m, seed=1)
    ts = dev(blk.s)
    y = host(binding.toeplitz(dev(blk.x), ts, n, m))
    torch.cuda.synchronize()
    rng = np.random.default_rng(3)
    for i in [0, 1, 63, 64, m // 2, m - 2, m - 1] + [int(v) for v in rng.integers(0, m, 5)]:
        assert (int(y[i // 64]) >> (i % 64)) & 1 == oracle.toeplitz_bit(blk.x, blk.s, n, m, i), i
    for j in (0, 12_345_678, n - 1):
        e = np.zeros_like(blk.x)
        e[j // 64] = np.uint64(1 << (j % 64))
        got = host(binding.toeplitz(dev(e), ts, n, m))
        torch.cuda.synchronize()
        np.testing.assert_array_equal(np.unpackbits(got.view(np.uint8), bitorder="little")[:m],
                                      _bits(blk.s, n - 1 - j, m))
    x2 = inputs.make_toeplitz_block(n, m, seed=2).x
    y2 = host(binding.toeplitz(dev(x2), ts, n, m))
    y12 = host(binding.toeplitz(dev(blk.x ^ x2), ts, n, m))
    torch.cuda.synchronize()
    np.testing.assert_array_equal(y12, y ^ y2)


@pytest.mark.parametrize("n,m", [(1000, 333), (100_003, 31_337), (1_000_000, 250_000)])
def test_seeded_equals_plain(n, m):
    torch = _need_gpu()
    blk = inputs.make_toeplitz_block(n, m, seed=11)
    ts = dev(blk.s)
    s = binding.ToeplitzSeed(ts, n, m)
    try:
        for k in range(3):
            x = inputs.make_toeplitz_block(n, m, seed=100 + k).x
            tx = dev(x)
            got, want = s.hash(tx), binding.toeplitz(tx, ts, n, m)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(host(got), host(want))
            if k == 0:
                np.testing.assert_array_equal(host(got), oracle.toeplitz(x, blk.s, n, m, threads=4))
    finally:
        torch.cuda.synchronize()
        s.close()


def test_seed_kinds_not_mixed():
    torch = _need_gpu()
    import ctypes

    n, m = 1000, 100
    blk = inputs.make_toeplitz_block(n, m, seed=1)
    tx, ts = dev(blk.x), dev(blk.s)
    out = torch.zeros(2, dtype=torch.int64, device="cuda")
    s = binding.ToeplitzSeed(ts, n, m)
    h = binding.Seed(tx, n)
    try:
        lib = binding.raw()
        p = ctypes.c_void_p
        assert lib.pa_hash_seeded(s.handle, p(tx.data_ptr()), p(tx.data_ptr()), 10, p(out.data_ptr()),
                                  None) == binding.PA_EINVAL
        assert lib.pa_toeplitz_seeded(h.handle, p(tx.data_ptr()), p(out.data_ptr()), None) == binding.PA_EINVAL
    finally:
        torch.cuda.synchronize()
        s.close()
        h.close()


def test_toeplitz_autotune_keeps_exact():
    torch = _need_gpu()
    n, m = 300_000, 120_000
    v = binding.toeplitz_autotune(n, m, reps=2)
    assert 0 <= v < 32
    blk = inputs.make_toeplitz_block(n, m, seed=21)
    got = binding.toeplitz(dev(blk.x), dev(blk.s), n, m)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(host(got), oracle.toeplitz(blk.x, blk.s, n, m, threads=8))
