"""The wrapped product of the modular hash and the digit width, on the CPU.

The hash needs only bits [n-m, n) of a x + b mod 2^n. A cyclic convolution of
the w-bit digits of length N, L <= N < 2L - 1 (L = ceil(n/w)), folds the
linear coefficients t_{k+N} onto c_k for k < W = 2L - 1 - N and leaves every
c_k with k >= W exact. The library drops the coefficients below lo (W rounded
up to even) and certifies the result: the dropped part is below 2^wbits,
wbits = w (lo + 1) + bit_length(lo), so unless limb q - 1 (q = floor((n-m)/64))
of the exact remaining sum Q is all ones -- which needs wbits <= 64 (q - 1) --
the output taken from Q is exact; otherwise the full-length product runs.
A width w is exact when L (2^w - 1)^2 < p; by default the library takes, of
the exact widths 16 .. 20, the one whose product is shortest (the narrowest
of equals).

Here: pa_plan_info / pa_plan_digits (host logic of the library, no device)
against those rules, and an exact-integer model of the fold and of the
certificate against the oracle on small sizes (cyclic lengths of any size, so
that wrapping happens at a few hundred digits), for every width, including
inputs built to fail the certificate.
"""
import random

import numpy as np
import pytest

import oracle
from paper_1910_04429_gb300 import binding, inputs


def _lengths(lo_len, hi_len):
    """Transform lengths of the library (2^k, k >= 12; 3 * 2^j, j >= 12 with
    (j - 12) mod 6 <= 4; 5 * 2^j, j >= 12 with (j - 12) mod 6 <= 3: first radix
    at most 48 or 40), ascending, in [lo_len, hi_len]."""
    out = set()
    for k in range(12, 40):
        if lo_len <= (1 << k) <= hi_len:
            out.add(1 << k)
        if (k - 12) % 6 <= 4 and lo_len <= (3 << k) <= hi_len:
            out.add(3 << k)
        if (k - 12) % 6 <= 3 and lo_len <= (5 << k) <= hi_len:
            out.add(5 << k)
    return sorted(out)


P = (1 << 64) - (1 << 32) + 1
WIDTHS = [16, 17, 18, 19, 20]


def _wbits(lo, w=16):
    return w * (lo + 1) + lo.bit_length()


def _certifiable(N, L, n, m, w=16):
    """(ok, lo) of the rule above for cyclic length N."""
    if N < L or N >= 2 * L - 1:
        return False, 0
    W = 2 * L - 1 - N
    lo = W + (W & 1)
    q = (n - m) // 64
    return q >= 1 and _wbits(lo, w) <= 64 * (q - 1), lo


def _exact(n, w):
    return -(-n // w) * ((1 << w) - 1) ** 2 < P


def _first_length(n, m, w, mode):
    """(first length, dropped) of one width under a wrap mode (the rule above)."""
    L = -(-n // w)
    full = _lengths(max(4096, 2 * L - 1), 1 << 40)[0]
    if mode == 0 or (mode == 1 and full < 1 << 19):
        return full, 0, full
    for N in _lengths(max(4096, L), full - 1):
        ok, lo = _certifiable(N, L, n, m, w)
        if ok:
            return N, lo, full
    return full, 0, full


SIZES = [(1, 1), (64, 1), (5000, 100), (65_536, 1), (65_537, 16_000), (100_000, 25_000), (100_000, 50_000),
         (1_000_000, 100_000), (1_000_000, 250_000), (1_000_000, 500_000), (3_000_017, 300_001),
         (10_000_000, 1_000_000), (10_000_000, 5_000_000), (100_000_000, 10_000_000),
         (100_000_000, 25_000_000), (100_000_000, 50_000_000), (1_000_000_000, 250_000_000),
         (2 ** 31, 2 ** 29), (2 ** 31, 1)]


@pytest.fixture
def width16():
    """16-bit digits for one test (pa_digit_width, a host-side setting)."""
    prev = binding.digit_width(16)
    yield
    binding.digit_width(prev)


@pytest.fixture
def wrap_mode():
    """Sets pa_wrap_mode for one test (a host-side setting, no device)."""
    prev = []

    def set_mode(mode):
        prev.append(binding.wrap_mode(mode))

    yield set_mode
    if prev:
        binding.wrap_mode(prev[0])


@pytest.mark.parametrize("mode", [1, 2, 0])
@pytest.mark.parametrize("n,m", SIZES)
def test_plan_info_follows_the_rule(n, m, mode, wrap_mode, width16):
    """16-bit digits. Mode 1 (default): the rule where the full product has
    >= 2^19 points; mode 2: wherever a shorter length is certifiable; mode 0:
    never."""
    wrap_mode(mode)
    info = binding.plan_info(n, m)
    L = -(-n // 16)
    full = _lengths(max(4096, 2 * L - 1), 1 << 40)[0]
    assert info["full"] == full
    shorter = [N for N in _lengths(max(4096, L), full - 1)]
    ok = [(N, lo) for N in shorter for c, lo in [_certifiable(N, L, n, m)] if c]
    if mode == 0 or (mode == 1 and full < 1 << 19):
        ok = []
    if ok:  # the shortest certifiable length, with its dropped-coefficient count
        assert (info["first"], info["dropped"]) == ok[0]
        assert L <= info["first"] < 2 * L - 1
    else:
        assert (info["first"], info["dropped"]) == (full, 0)


def test_headline_sizes_wrap(wrap_mode, width16):
    """The 10^8-bit block (m = n/4) runs 2^23 points instead of 3 * 2^22, and
    5 * 2^21 at m = n/2; the 10^9-bit block 5 * 2^24 instead of 2^27; the
    10^7-bit block's full product is 5 * 2^18 (2L - 1 = 1249999). The 10^6-bit
    block (2^17 points) stays unwrapped by default and wraps to 5 * 2^14 in
    mode 2."""
    info = binding.plan_info(10 ** 8, 25 * 10 ** 6)
    assert info["first"] == 1 << 23
    # W = 2L - 1 - N = 12,499,999 - 8,388,608 = 4,111,391, rounded up to even
    assert info["dropped"] == 4_111_392 and _wbits(4_111_392) == 65_782_310
    assert binding.plan_info(10 ** 8, 5 * 10 ** 7)["first"] == 5 << 21
    assert binding.plan_info(10 ** 9, 25 * 10 ** 7)["first"] == 5 << 24
    assert binding.plan_info(10 ** 7, 10 ** 6)["full"] == 5 << 18
    assert binding.plan_info(10 ** 6, 250_000)["dropped"] == 0
    wrap_mode(2)
    assert binding.plan_info(10 ** 6, 250_000)["first"] == 5 << 14


@pytest.mark.parametrize("mode", [1, 2, 0])
@pytest.mark.parametrize("n,m", SIZES)
def test_width_choice_follows_the_rule(n, m, mode, wrap_mode):
    """Chosen width (the default): of the exact widths, the one whose first
    product is shortest; of equals an unwrapped one, then the narrowest; its
    lengths as for that width."""
    wrap_mode(mode)
    best = None
    for w in WIDTHS:
        if not _exact(n, w):
            continue
        first, lo, full = _first_length(n, m, w, mode)
        if best is None or first < best[1] or (first == best[1] and best[2] > 0 and lo == 0):
            best = (w, first, lo)
    info = binding.plan_info(n, m)
    assert binding.plan_digits(n, m) == best[0]
    assert (info["first"], info["dropped"]) == best[1:]
    # the full-length (unwrapped) product, at the width chosen without wrapping
    fulls = [(_first_length(n, m, w, 0)[0], w) for w in WIDTHS if _exact(n, w)]
    assert info["full"] == min(fulls)[0]


@pytest.mark.parametrize("w", WIDTHS)
def test_forced_width_where_exact(w):
    prev = binding.digit_width(w)
    try:
        for n in (1000, 10 ** 6, 10 ** 8, 3 * 10 ** 8, 10 ** 9, 2 ** 31):
            assert binding.plan_digits(n, n // 4) == (w if _exact(n, w) else 16)
    finally:
        binding.digit_width(prev)
    with pytest.raises(binding.PaError):
        binding.digit_width(15)
    with pytest.raises(binding.PaError):
        binding.digit_width(21)


def test_headline_widths():
    """20-bit digits are exact up to n = 3.355e8 bits: at n = 10^8 (m = n/4) the
    product is 3 * 2^21 points instead of 2^23 (m = n/2: 18-bit digits, 2^23
    instead of 5 * 2^21); at 10^9 bits 19-bit digits are the widest exact ones
    and certify 2^26 points instead of 5 * 2^24."""
    assert _exact(10 ** 8, 20) and not _exact(4 * 10 ** 8, 20)
    assert _exact(10 ** 9, 19) and not _exact(10 ** 9, 20)
    assert binding.plan_digits(10 ** 8, 25 * 10 ** 6) == 20
    assert binding.plan_info(10 ** 8, 25 * 10 ** 6)["first"] == 3 << 21
    assert binding.plan_digits(10 ** 8, 5 * 10 ** 7) == 18
    assert binding.plan_info(10 ** 8, 5 * 10 ** 7)["first"] == 1 << 23
    assert binding.plan_digits(10 ** 9, 25 * 10 ** 7) == 19
    assert binding.plan_info(10 ** 9, 25 * 10 ** 7)["first"] == 1 << 26


def test_plan_info_rejects_bad_sizes():
    for n, m in [(0, 0), (10, 11), (10, 0), (2 ** 31 + 1, 1)]:
        with pytest.raises(binding.PaError):
            binding.plan_info(n, m)


# ---------------------------------------------------------------------------
# exact-integer model of the wrapped product and its certificate
# ---------------------------------------------------------------------------
def _digits(v, L, w=16):
    return [(v >> (w * i)) & ((1 << w) - 1) for i in range(L)]


def _model(x, a, b, n, m, N, w=16):
    """(output or None, lo): the output taken from the certified sum Q, or None
    when the certificate fails (the library then runs the full product)."""
    L = -(-n // w)
    ok, lo = _certifiable(N, L, n, m, w)
    assert ok
    dx, da = _digits(x, L, w), _digits(a, L, w)
    c = [0] * N
    t = [0] * (2 * L - 1)
    for i in range(L):
        if da[i]:
            for j in range(L):
                c[(i + j) % N] += da[i] * dx[j]
                t[i + j] += da[i] * dx[j]
    # the fold: every c_k with k >= lo is the linear coefficient
    assert all(c[k] == t[k] for k in range(lo, min(N, 2 * L - 1)))
    assert max(t) < P  # the width is exact: every coefficient below p
    T = sum(t[k] << (w * k) for k in range(lo))
    assert T < 1 << _wbits(lo, w)  # the dropped part's bound
    Q = sum(c[k] << (w * k) for k in range(lo, L)) + b
    assert (Q + T) % (1 << n) == (a * x + b) % (1 << n)
    q = (n - m) // 64
    if (Q >> (64 * (q - 1))) & ((1 << 64) - 1) == (1 << 64) - 1:
        return None, lo
    return (Q % (1 << n)) >> (n - m), lo


def _small_case(n, m, w=16):
    """The shortest cyclic length (any integer) that the rule certifies."""
    L = -(-n // w)
    for N in range(L, 2 * L - 1):
        if _certifiable(N, L, n, m, w)[0]:
            return N
    return None


def _to_limbs(v, n):
    return np.array([(v >> (64 * i)) & ((1 << 64) - 1) for i in range(-(-n // 64))], dtype=np.uint64)


def _from_limbs(arr):
    return sum(int(w) << (64 * i) for i, w in enumerate(arr))


@pytest.mark.parametrize("w", WIDTHS)
@pytest.mark.parametrize("n,m", [(1600, 160), (2000, 500), (3001, 750), (4096, 1024), (2500, 250)])
def test_model_matches_oracle_on_random_inputs(n, m, w):
    N = _small_case(n, m, w)
    assert N is not None and N < 2 * (-(-n // w)) - 1
    rng = random.Random(n * 7 + m + w)
    for _ in range(6):
        x, a, b = (rng.getrandbits(n) for _ in range(3))
        got, _ = _model(x, a, b, n, m, N, w)
        want = _from_limbs(oracle.pa_hash(_to_limbs(x, n), _to_limbs(a, n), _to_limbs(b, n), n, m, threads=1))
        assert got is not None  # a uniform b fails the certificate with probability 2^-64
        assert got == want


@pytest.mark.parametrize("w", WIDTHS)
def test_model_certificate_fails_exactly_where_needed(w):
    """Inputs built so that limb q - 1 of Q is all ones fail the certificate:
    x = 0 with b = 2^n - 1; a = 1 with x = 2^n - 1; and b chosen so that the
    low n - m bits of Q are 2^(n-m) - T, where T > 0 is the dropped part. In
    that last case the dropped part carries into the output, so an output
    taken from Q alone would be wrong: the fallback is needed there."""
    n, m = 2000, 500
    s = n - m
    N = _small_case(n, m, w)
    L = -(-n // w)
    lo = _certifiable(N, L, n, m, w)[1]
    full = (1 << n) - 1
    assert _model(0, 5, full, n, m, N, w)[0] is None
    assert _model(full, 1, 0, n, m, N, w)[0] is None
    rng = random.Random(3 + w)
    x, a = rng.getrandbits(n), rng.getrandbits(n) | 1
    t = [0] * (2 * L - 1)
    for i, ai in enumerate(_digits(a, L, w)):
        for j, xj in enumerate(_digits(x, L, w)):
            t[i + j] += ai * xj
    T = sum(t[k] << (w * k) for k in range(lo))
    assert T > 0
    q_target = (rng.getrandbits(m) << s) + ((1 << s) - T)
    b = (q_target - a * x + T) % (1 << n)  # then a x + b = Q + T (mod 2^n) with Q = q_target
    assert _model(x, a, b, n, m, N, w)[0] is None
    want = ((a * x + b) % (1 << n)) >> s
    assert want != (q_target % (1 << n)) >> s
    assert want == _from_limbs(oracle.pa_hash(_to_limbs(x, n), _to_limbs(a, n), _to_limbs(b, n), n, m, threads=1))


def test_inputs_module_blocks_pass_the_certificate():
    """The seeded benchmark blocks (uniform b) pass the certificate in the model."""
    n, m = 2000, 500
    N = _small_case(n, m)
    for seed in range(5):
        blk = inputs.make_block(n, m, seed=seed)
        x, a, b = (_from_limbs(v) for v in (blk.x, blk.a, blk.b))
        got, _ = _model(x, a, b, n, m, N)
        assert got == _from_limbs(oracle.pa_hash(blk.x, blk.a, blk.b, n, m, threads=1))
