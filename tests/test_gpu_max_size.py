"""The largest key the library takes, n = PA_MAX_BITS = 2^31 bits, on the GPU.

The oracle does not finish a 2^31-bit product in seconds, so these tests use
a property that holds at any size. The multiplier a has a few nonzero 16-bit
digits (the lowest, the highest and three at seeded positions). Its transform
is dense, so every pass of the product runs on general data, while x and b are
uniform. Then a x + b is a sum of a few shifted single-digit products, which
Python's integers form exactly in linear time.

Plans at this size with 16-bit digits: the wrapped products at 3 * 2^26 points
(m = n/4) and 5 * 2^25 points (m = 1); the full product, the recomputation and
m = n at 2^28 points, the longest transform (radix 16, 64, 64, then the
4096-point tile). With the default width (17-bit digits here: 18 is the widest
exact one and gives no shorter product) m = n/4 wraps to 5 * 2^25 points and
m = 1 to 2^27.
"""
import numpy as np
import pytest

from paper_1910_04429_gb300 import binding, inputs
from tests.gpu_util import gpu_hash

pytestmark = pytest.mark.gpu

N = 1 << 31


@pytest.fixture(scope="module")
def case():
    assert binding.PA_MAX_BITS == N
    blk = inputs.make_block(N, N // 4, seed=31)
    rng = np.random.default_rng(3131)
    digits = N // 16
    pos = [0, digits - 1] + [int(p) for p in rng.choice(np.arange(1, digits - 1), size=3, replace=False)]
    vals = [int(v) for v in rng.integers(1, 1 << 16, size=len(pos))]
    a16 = np.zeros(digits, dtype="<u2")
    a16[pos] = vals
    a = a16.view("<u8").astype(np.uint64)  # digit k weighs 2^(16k)
    xi = int.from_bytes(blk.x.astype("<u8").tobytes(), "little")
    y = int.from_bytes(blk.b.astype("<u8").tobytes(), "little")
    for p, v in zip(pos, vals):
        y += (xi * v) << (16 * p)
    y &= (1 << N) - 1  # (a x + b) mod 2^n
    return blk.x, a, blk.b, y


@pytest.mark.parametrize("m,mode,width,length,flags", [
    (N // 4, 1, 16, 3 << 26, 0),   # wrapped, certified (16-bit digits)
    (1, 1, 16, 5 << 25, 0),        # wrapped, one output bit
    (N // 4, 0, 16, 1 << 28, 0),   # full product
    (N // 4, 3, 16, 3 << 26, 1),   # wrapped, certificate forced to fail: recomputation at 2^28
    (N, 1, 16, 1 << 28, 0),        # every bit out
    (N // 4, 1, 0, 5 << 25, 0),    # the default width here: 17-bit digits (18 is as short)
    (1, 1, 0, 1 << 27, 0),         # 17-bit digits, one output bit
    (N // 4, 3, 0, 5 << 25, 1),    # 17-bit wrapped product, then the 16-bit recomputation
])
def test_maximum_key_size(case, m, mode, width, length, flags):
    x, a, b, y = case
    prev = binding.wrap_mode(mode)
    prev_w = binding.digit_width(width)
    try:
        assert binding.plan_info(N, m)["first"] == length
        if width == 0:
            assert binding.plan_digits(N, m) == 17
        binding.wrap_flags(clear=True)
        got = gpu_hash(binding, x, a, b, N, m)
        assert binding.wrap_flags() == flags
    finally:
        binding.wrap_mode(prev)
        binding.digit_width(prev_w)
    assert got.size == -(-m // 64)
    assert int.from_bytes(got.astype("<u8").tobytes(), "little") == y >> (N - m)
    assert binding.device_status() == 0
