"""Pins of the Toeplitz-hash oracle against things other than itself (no GPU).

The family (random Toeplitz matrices over GF(2), the hash surveyed in Sec. 1 of
the paper): an n + m - 1 bit seed s gives T[i][j] = s[i - j + n - 1] (m x n) and
y = T x over GF(2). Each group targets a different plausible mistake:
  * scipy's Toeplitz constructor + a matrix product  -> the seed indexing (which
    diagonal, which direction), an off-by-one in n - 1
  * numpy integer convolution mod 2                  -> the window of the
    product that is kept
  * Python-int carry-less product                    -> the same, at sizes
    where a matrix no longer fits
  * closed forms (unit key, unit seed, all ones)     -> shifts and masks
  * exhaustive universal_2 count                     -> the family itself
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_1910_04429_gb300 import inputs
from tests.intutil import from_int, to_int


def _bits(limbs, nbits):
    return np.unpackbits(np.ascontiguousarray(limbs, dtype=np.uint64).view(np.uint8),
                         bitorder="little")[:nbits].astype(np.int64)


def _limbs_from_bits(bits):
    bits = np.asarray(bits, dtype=np.uint8)
    pad = (-bits.size) % 64
    packed = np.packbits(np.concatenate([bits, np.zeros(pad, np.uint8)]), bitorder="little")
    return packed.view(np.uint64).copy()


def _rand(rng, nbits):
    return _limbs_from_bits(rng.integers(0, 2, nbits))


def _oracle_bits(x, s, n, m, threads=1):
    return _bits(oracle.toeplitz(x, s, n, m, threads), m)


def test_vs_scipy_toeplitz_matrix():
    linalg = pytest.importorskip("scipy.linalg")
    rng = np.random.default_rng(11)
    cases = [(n, m) for n in range(1, 9) for m in range(1, n + 1)]
    cases += [(int(n), int(rng.integers(1, n + 1))) for n in rng.integers(9, 400, 40)]
    cases += [(64, 64), (65, 1), (128, 63), (129, 65), (300, 300)]
    for n, m in cases:
        x, s = _rand(rng, n), _rand(rng, n + m - 1)
        sb, xb = _bits(s, n + m - 1), _bits(x, n)
        col = sb[n - 1: n - 1 + m]          # T[i][0] = s[i + n - 1]
        row = sb[n - 1::-1][:n]             # T[0][j] = s[n - 1 - j]
        T = linalg.toeplitz(col, row)
        assert T.shape == (m, n)
        want = (T @ xb) % 2
        assert np.array_equal(_oracle_bits(x, s, n, m), want), (n, m)


@pytest.mark.parametrize("n,m", [(1000, 1), (1000, 1000), (4097, 1500), (20000, 6000)])
def test_vs_numpy_convolution(n, m):
    rng = np.random.default_rng(n + m)
    x, s = _rand(rng, n), _rand(rng, n + m - 1)
    full = np.convolve(_bits(s, n + m - 1), _bits(x, n))  # exact integer counts
    want = full[n - 1: n - 1 + m] % 2
    assert np.array_equal(_oracle_bits(x, s, n, m, threads=4), want)


def _clmul(a: int, b: int) -> int:
    r = 0
    while b:
        low = b & -b
        r ^= a << (low.bit_length() - 1)
        b ^= low
    return r


@pytest.mark.parametrize("n,m", [(50_000, 12_500), (65_536, 65_536), (100_003, 31_337)])
def test_vs_python_int_carryless_product(n, m):
    rng = np.random.default_rng(n)
    x, s = _rand(rng, n), _rand(rng, n + m - 1)
    prod = _clmul(to_int(s), to_int(x))
    want = (prod >> (n - 1)) & ((1 << m) - 1)
    assert to_int(oracle.toeplitz(x, s, n, m, threads=8)) == want


@pytest.mark.parametrize("n,m", [(1, 1), (63, 17), (64, 64), (1000, 333)])
def test_closed_forms(n, m):
    rng = np.random.default_rng(n * 7 + m)
    s = _rand(rng, n + m - 1)
    sb = _bits(s, n + m - 1)
    x = _rand(rng, n)
    xb = _bits(x, n)
    for j in sorted({0, n // 2, n - 1}):  # unit key e_j: column j of T
        e = _limbs_from_bits(np.eye(1, n, j, dtype=np.uint8)[0])
        assert np.array_equal(_oracle_bits(e, s, n, m), sb[n - 1 - j: n - 1 - j + m])
    for k in sorted({0, n - 1, n + m - 2}):  # unit seed e_k: y_i = x[i + n - 1 - k]
        e = _limbs_from_bits(np.eye(1, n + m - 1, k, dtype=np.uint8)[0])
        want = [xb[i + n - 1 - k] if 0 <= i + n - 1 - k < n else 0 for i in range(m)]
        assert list(_oracle_bits(x, e, n, m)) == want
    ones_x, ones_s = _limbs_from_bits(np.ones(n, np.uint8)), _limbs_from_bits(np.ones(n + m - 1, np.uint8))
    assert set(_oracle_bits(ones_x, ones_s, n, m)) == {n % 2}
    assert not _oracle_bits(np.zeros_like(x), s, n, m).any()
    assert not _oracle_bits(x, np.zeros_like(s), n, m).any()


def test_linear_in_key_and_seed():
    rng = np.random.default_rng(5)
    n, m = 10_007, 3_001
    x1, x2 = _rand(rng, n), _rand(rng, n)
    s1, s2 = _rand(rng, n + m - 1), _rand(rng, n + m - 1)
    h = lambda x, s: oracle.toeplitz(x, s, n, m, threads=2)  # noqa: E731
    assert np.array_equal(h(x1 ^ x2, s1), h(x1, s1) ^ h(x2, s1))
    assert np.array_equal(h(x1, s1 ^ s2), h(x1, s1) ^ h(x1, s2))


def test_padding_bits_ignored_and_output_masked():
    rng = np.random.default_rng(9)
    for n, m in [(70, 5), (100, 29), (1000, 999)]:
        x, s = _rand(rng, n), _rand(rng, n + m - 1)
        xg, sg = x.copy(), s.copy()
        if n % 64:
            xg[-1] |= np.uint64(~((1 << (n % 64)) - 1) & 0xFFFFFFFFFFFFFFFF)
        if (n + m - 1) % 64:
            sg[-1] |= np.uint64(~((1 << ((n + m - 1) % 64)) - 1) & 0xFFFFFFFFFFFFFFFF)
        y = oracle.toeplitz(x, s, n, m)
        assert np.array_equal(oracle.toeplitz(xg, sg, n, m), y)
        if m % 64:
            assert int(y[-1]) >> (m % 64) == 0


def test_threads_do_not_change_the_result():
    blk = inputs.make_toeplitz_block(200_000, 50_001, seed=3)
    y1 = oracle.toeplitz(blk.x, blk.s, blk.n, blk.m, threads=1)
    y7 = oracle.toeplitz(blk.x, blk.s, blk.n, blk.m, threads=7)
    assert np.array_equal(y1, y7)


def test_row_bits_match_columns_and_numpy_rows():
    blk = inputs.make_toeplitz_block(1_000_000, 250_000, seed=1)
    n, m = blk.n, blk.m
    y = _bits(oracle.toeplitz(blk.x, blk.s, n, m, threads=8), m)
    sb, xb = _bits(blk.s, n + m - 1), _bits(blk.x, n)
    for i in [0, 1, 63, 64, 12345, m // 2, m - 2, m - 1]:
        row = sb[i: i + n][::-1]  # T[i][j] = s[i + n - 1 - j]
        assert int(row @ xb) % 2 == y[i] == oracle.toeplitz_bit(blk.x, blk.s, n, m, i)


@pytest.mark.parametrize("n,m", [(4, 2), (5, 3), (6, 1)])
def test_universal2_exhaustive(n, m):
    """For x1 != x2 exactly 2^(n-1) of the 2^(n+m-1) seeds collide: the family
    is universal_2 with collision probability 2^-m (it is even pairwise
    independent)."""
    seeds = 1 << (n + m - 1)
    table = np.zeros((seeds, 1 << n), dtype=np.int64)
    for sv in range(seeds):
        s = from_int(sv, 1)
        for xv in range(1 << n):
            table[sv, xv] = int(oracle.toeplitz(from_int(xv, 1), s, n, m)[0])
    for x1, x2 in itertools.combinations(range(1 << n), 2):
        assert int((table[:, x1] == table[:, x2]).sum()) == seeds >> m


def test_argument_validation():
    z = np.zeros(4, dtype=np.uint64)
    with pytest.raises(ValueError):
        oracle.toeplitz(z, z, 10, 11)
    with pytest.raises(ValueError):
        oracle.toeplitz(z, z, 0, 0)
    with pytest.raises(ValueError):
        oracle.toeplitz_bit(z, z, 10, 5, 5)
