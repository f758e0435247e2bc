"""Pins of the CPU oracle against things other than itself (no GPU needed).

Each group targets a different plausible mistake:
  * bit-level brute force      -> carry/shift/mask slips in the limb code
  * Python ints                -> independent arbitrary-precision products
  * closed forms               -> the add, the mod 2^n and the extraction
  * universal_2 count (Eq. 5)  -> the family itself (dropping +d, wrong mod)
  * collision statistics       -> the same at a size where counting is impossible
"""
import itertools
import math
import random

import numpy as np
import pytest

import oracle
from oracle import gmp_ref
from paper_1910_04429_gb300 import inputs
from tests.intutil import from_int, hash_int, to_int


def _oracle_int(x, a, b, n, m, threads=1):
    L = (n + 63) // 64
    return to_int(oracle.pa_hash(from_int(x, L), from_int(a, L), from_int(b, L), n, m, threads))


# ---------------------------------------------------------------------------
# bit-level brute force: integers as bit lists, product by shift-and-add with a
# ripple-carry adder, then + b, truncation to n bits and the top-m slice.
# ---------------------------------------------------------------------------

def _bits(v, n):
    return [(v >> i) & 1 for i in range(n)]


def _ripple_add(acc, addend):
    out, c = [], 0
    for p, q in zip(acc, addend):
        s = p + q + c
        out.append(s & 1)
        c = s >> 1
    return out  # carry out of the top bit is dropped: arithmetic mod 2^len


def _brute(x, a, b, n, m):
    xb, ab, bb = _bits(x, n), _bits(a, n), _bits(b, n)
    acc = [0] * n
    for i in range(n):
        if ab[i]:
            shifted = [0] * i + xb[: n - i]
            acc = _ripple_add(acc, shifted)
    acc = _ripple_add(acc, bb)
    top = acc[n - m:]
    return sum(bit << j for j, bit in enumerate(top))


def test_brute_force_exhaustive_tiny():
    for n in range(1, 5):
        for m in range(1, n + 1):
            for x, a, b in itertools.product(range(1 << n), repeat=3):
                assert _oracle_int(x, a, b, n, m) == _brute(x, a, b, n, m), (n, m, x, a, b)


def test_brute_force_random_to_n12():
    rng = random.Random(12)
    for _ in range(3000):
        n = rng.randint(1, 12)
        m = rng.randint(1, n)
        x, a, b = (rng.getrandbits(n) for _ in range(3))
        assert _oracle_int(x, a, b, n, m) == _brute(x, a, b, n, m)


def test_brute_force_random_to_n200():
    rng = random.Random(200)
    for _ in range(300):
        n = rng.randint(13, 200)
        m = rng.randint(1, n)
        x, a, b = (rng.getrandbits(n) for _ in range(3))
        assert _oracle_int(x, a, b, n, m) == _brute(x, a, b, n, m)


# ---------------------------------------------------------------------------
# independent arbitrary precision (Python ints)
# ---------------------------------------------------------------------------

def test_python_int_small_random():
    rng = random.Random(64)
    for _ in range(2000):
        n = rng.randint(1, 130)
        m = rng.randint(1, n)
        # operands wider than n: bits >= n must be ignored
        x, a, b = (rng.getrandbits(((n + 63) // 64) * 64) for _ in range(3))
        assert _oracle_int(x, a, b, n, m) == hash_int(x, a, b, n, m)


@pytest.mark.parametrize("k", [1, 7, 47, 48, 95, 96, 97, 300, 2049])
def test_python_int_every_residue(k):
    """n = 64 (k-1) + r for every r in 1..64, across the schoolbook / Karatsuba
    switch points of the low-half and full products."""
    rng = random.Random(k)
    for r in range(1, 65):
        n = 64 * (k - 1) + r
        m = rng.choice([1, n, max(1, n // 4), rng.randint(1, n)])
        x, a, b = (rng.getrandbits(n) for _ in range(3))
        assert _oracle_int(x, a, b, n, m) == hash_int(x, a, b, n, m), (n, m)


@pytest.mark.parametrize("k", [1, 2, 47, 48, 49, 96, 97, 500, 4096, 5000])
def test_products_vs_python_int(k):
    rng = random.Random(1000 + k)
    a = rng.getrandbits(64 * k)
    b = rng.getrandbits(64 * k)
    A, B = from_int(a, k), from_int(b, k)
    for threads in (1, 9):
        assert to_int(oracle.mul_full(A, B, threads)) == a * b
        assert to_int(oracle.mul_low(A, B, threads)) == (a * b) % (1 << (64 * k))


def test_products_extreme_limbs():
    """All-ones operands maximise every carry in the limb loops."""
    for k in (1, 3, 48, 97, 4100):
        a = (1 << (64 * k)) - 1
        A = from_int(a, k)
        assert to_int(oracle.mul_full(A, A, 4)) == a * a
        assert to_int(oracle.mul_low(A, A, 4)) == (a * a) % (1 << (64 * k))


def test_config1_size_vs_python_int():
    blk = inputs.make_block(1_000_000, 250_000, seed=1)
    got = oracle.pa_hash(blk.x, blk.a, blk.b, blk.n, blk.m, threads=oracle.default_threads())
    want = hash_int(to_int(blk.x), to_int(blk.a), to_int(blk.b), blk.n, blk.m)
    assert to_int(got) == want


@pytest.mark.parametrize("n", [3_000_001, 1_048_576 + 17])
def test_mid_size_vs_python_int(n):
    blk = inputs.make_block(n, n // 3, seed=5)
    got = oracle.pa_hash(blk.x, blk.a, blk.b, blk.n, blk.m, threads=oracle.default_threads())
    want = hash_int(to_int(blk.x), to_int(blk.a), to_int(blk.b), blk.n, blk.m)
    assert to_int(got) == want


@pytest.mark.skipif(not gmp_ref.available(), reason="libgmp not loadable on this host")
def test_vs_gmp_ten_million_bits():
    """GMP's own multiply (the paper's Sec. 3.2 pipeline) as a second
    independent arbitrary-precision implementation."""
    blk = inputs.make_block(10_000_000, 2_500_000, seed=1)
    got = oracle.pa_hash(blk.x, blk.a, blk.b, blk.n, blk.m, threads=oracle.default_threads())
    want = gmp_ref.pa_hash(blk.x, blk.a, blk.b, blk.n, blk.m)
    np.testing.assert_array_equal(got, want)


# ---------------------------------------------------------------------------
# closed forms (expected values need only additions and shifts)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n,m", [(1, 1), (63, 5), (64, 64), (65, 1), (1000, 250),
                                 (1_000_000, 250_000), (1_000_003, 1_000_003)])
def test_closed_forms(n, m):
    L = (n + 63) // 64
    mask = (1 << n) - 1
    blk = inputs.make_block(n, m, seed=n)
    x, b = to_int(blk.x), to_int(blk.b)
    zero = from_int(0, L)
    one = from_int(1, L)
    ones = from_int(mask, L)
    sh = n - m
    T = oracle.default_threads()

    def run(X, A, B):
        return to_int(oracle.pa_hash(X, A, B, n, m, T))

    # x = 0: out = b >> (n - m)
    assert run(zero, blk.a, blk.b) == b >> sh
    # a = 1: out = ((x + b) mod 2^n) >> (n - m)
    assert run(blk.x, one, blk.b) == ((x + b) & mask) >> sh
    # a = 2^k: ((x << k) + b) mod 2^n
    for k in {0, 1, n // 2, n - 1}:
        assert run(blk.x, from_int(1 << k, L), blk.b) == (((x << k) + b) & mask) >> sh
    # a = 2^n - 1 = -1 mod 2^n: (b - x) mod 2^n
    assert run(blk.x, ones, blk.b) == ((b - x) & mask) >> sh
    # all-propagate carry: x = 2^n - 1, a = 1, b = 1 -> y = 0
    assert run(ones, one, one) == 0
    # b = 0, a = 1, x = 2^n - 1 -> all ones
    assert run(ones, one, zero) == (1 << m) - 1


def test_m_equals_n_returns_y():
    n = 5000
    blk = inputs.make_block(n, n, seed=3)
    x, a, b = to_int(blk.x), to_int(blk.a), to_int(blk.b)
    assert _oracle_int(x, a, b, n, n) == (a * x + b) % (1 << n)


def test_linearity_in_b():
    """g(x; a, b1) and g(x; a, b2) with m = n differ by b1 - b2 mod 2^n."""
    n = 777
    L = (n + 63) // 64
    rng = random.Random(9)
    x, a, b1, b2 = (rng.getrandbits(n) for _ in range(4))
    y1 = _oracle_int(x, a, b1, n, n)
    y2 = _oracle_int(x, a, b2, n, n)
    assert (y1 - y2) % (1 << n) == (b1 - b2) % (1 << n)
    assert L == 13


def test_argument_validation():
    assert oracle.raw_hash_rc(0, 1) == -1
    assert oracle.raw_hash_rc(10, 0) == -1
    assert oracle.raw_hash_rc(10, 11) == -1
    assert oracle.raw_hash_rc(10, 10) == 0


# ---------------------------------------------------------------------------
# universal_2 (Sec. 2.3, Eq. 3-6): exhaustive delta counts on tiny alpha
# ---------------------------------------------------------------------------

def _tables(alpha, beta, with_d=True):
    """g_{c,d}(x) for every odd c, every d (or d = 0) and every x, via the oracle."""
    L = 1
    rows = []
    ds = range(1 << alpha) if with_d else [0]
    for c in range(1, 1 << alpha, 2):
        C = from_int(c, L)
        for d in ds:
            D = from_int(d, L)
            rows.append([int(oracle.pa_hash(from_int(x, L), C, D, alpha, beta)[0])
                         for x in range(1 << alpha)])
    return np.array(rows, dtype=np.int64)


def _max_delta(tab):
    # delta_G(x, y) = number of functions with g(x) == g(y), for x != y (Eq. 4)
    eq = (tab[:, :, None] == tab[:, None, :]).sum(axis=0)
    np.fill_diagonal(eq, 0)
    return int(eq.max())


@pytest.mark.parametrize("alpha,beta", [(3, 1), (4, 1), (4, 2), (5, 2), (5, 3), (6, 2), (6, 3)])
def test_universal2_exhaustive(alpha, beta):
    tab = _tables(alpha, beta)
    G = tab.shape[0]
    assert G == 2 ** (2 * alpha - 1)        # |G_{c,d}|: odd c times all d (Eq. 6)
    bound = G // (1 << beta)                # |G| / |B| (Eq. 5)
    assert _max_delta(tab) == bound         # the bound holds, and is attained


@pytest.mark.parametrize("alpha,beta", [(4, 2), (5, 2), (6, 3)])
def test_universal2_fails_without_addend(alpha, beta):
    """Without the addend d the family {g_{c,0}} is not universal_2: some pair
    collides under twice the allowed share of functions. The pin shows that the
    oracle's +d matters to the property."""
    tab = _tables(alpha, beta, with_d=False)
    G = tab.shape[0]
    assert _max_delta(tab) == 2 * (G // (1 << beta))


@pytest.mark.parametrize("m", [4, 8, 12])
def test_collision_rate_statistical(m):
    """n = 64: for fixed x != y, the collision rate over random (c, d) is at
    most 2^-m (Eq. 5 divided by |G|), within a 5-sigma binomial band."""
    n, trials = 64, 20000
    rng = random.Random(m)
    pairs = [(rng.getrandbits(n), None) for _ in range(3)]
    pairs = [(x, x ^ (1 << rng.randrange(n))) for x, _ in pairs]  # one-bit differences
    pairs.append((0, 1 << 63))
    for x, y in pairs:
        hits = 0
        for _ in range(trials):
            c = rng.getrandbits(n) | 1
            d = rng.getrandbits(n)
            hits += _oracle_int(x, c, d, n, m) == _oracle_int(y, c, d, n, m)
        p = 2.0 ** -m
        sigma = math.sqrt(p * (1 - p) / trials)
        assert hits / trials <= p + 5 * sigma, (x, y, hits)
