"""Digit widths 16 .. 20 (the split of Algorithm 1 into w-bit pieces) on the GPU,
bit for bit against the oracle.

Every width is forced in turn (pa_digit_width) over sizes that span the
transform layouts (one tile, one and two strided passes, the 3 * 2^k and 5 * 2^k
families), ragged n and m, and the three product forms: full length, wrapped
wherever certifiable, and wrapped with the certificate forced to fail (so the
16-bit recomputation runs too). The default choice is exercised on mixed
batches (blocks of several widths in one call), seed reuse, host buffers,
operands that are not 16-byte aligned (which take 16-bit digits) and inputs
built so that the certificate fails by itself.
"""
import numpy as np
import pytest

import oracle
from paper_1910_04429_gb300 import binding, inputs
from tests.gpu_util import dev, gpu_hash, host

pytestmark = pytest.mark.gpu

WIDTHS = [16, 17, 18, 19, 20]
# (n, m): 1-tile, [R0], [R0, 64] transforms, 3 * 2^k and 5 * 2^k lengths, ragged sizes
SIZES = [(1, 1), (63, 17), (20_001, 5_003), (100_003, 31_111), (333_337, 150_001), (1_000_000, 250_000),
         (1_234_567, 600_001), (3_000_001, 750_003)]


@pytest.fixture(autouse=True)
def _modes():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    w0, m0 = binding.digit_width(0), binding.wrap_mode(1)
    yield
    binding.digit_width(w0)
    binding.wrap_mode(m0)


def _want(b):
    return oracle.pa_hash(b.x, b.a, b.b, b.n, b.m, threads=oracle.default_threads())


@pytest.mark.parametrize("mode", [0, 2, 3])
@pytest.mark.parametrize("w", WIDTHS)
def test_forced_width_every_form(w, mode):
    binding.digit_width(w)
    binding.wrap_mode(mode)
    binding.wrap_flags(clear=True)
    wrapped = 0
    for i, (n, m) in enumerate(SIZES):
        b = inputs.make_block(n, m, seed=1000 * w + 10 * mode + i)
        wrapped += binding.plan_info(n, m)["dropped"] > 0
        np.testing.assert_array_equal(gpu_hash(binding, b.x, b.a, b.b, n, m), _want(b),
                                      err_msg=f"w={w} mode={mode} n={n} m={m}")
    if mode:
        assert wrapped >= 4
    # mode 3 forces every certificate to fail: each wrapped hash ran the recomputation
    assert binding.wrap_flags() == (wrapped if mode == 3 else 0)
    assert binding.stream_status() == binding.PA_OK


def test_every_residue_of_n_at_width_20():
    """n = 300_000 + r for r < 64 spread over residues mod 20 and mod 64, so the
    top digit and the top limb take every partial size."""
    binding.digit_width(20)
    binding.wrap_mode(2)
    for r in range(0, 64, 3):
        n = 300_000 + r
        b = inputs.make_block(n, n // 5 + r, seed=77 + r)
        np.testing.assert_array_equal(gpu_hash(binding, b.x, b.a, b.b, n, b.m), _want(b), err_msg=f"n={n}")


def test_batch_of_mixed_widths():
    """One batched call whose blocks take different widths (16 .. 20 by size and
    m) and different lengths, wrapped where certifiable, against the oracle."""
    import torch

    binding.wrap_mode(2)
    blks = inputs.make_batch(36, 200_000, 6_000_000, seed=5)
    widths = {binding.plan_digits(b.n, b.m) for b in blks}
    assert len(widths) >= 3, widths
    t = [(dev(b.x), dev(b.a), dev(b.b), b.n, b.m,
          torch.full(((b.m + 63) // 64,), -1, dtype=torch.int64, device="cuda")) for b in blks]
    binding.hash_batched(t)
    torch.cuda.synchronize()
    for b, tt in zip(blks, t):
        np.testing.assert_array_equal(host(tt[5]), _want(b), err_msg=f"n={b.n} m={b.m}")


def test_seed_reuse_across_widths():
    """One seed handle serving outputs of several lengths m, whose products take
    different widths and lengths: each hash equals the oracle."""
    import torch

    binding.wrap_mode(2)
    n = 4_000_003
    base = inputs.make_block(n, 1, seed=41)
    s = binding.Seed(dev(base.a), n)
    try:
        seen = set()
        for i, m in enumerate([400_001, 1_300_007, 2_000_001, 3_999_999]):
            b = inputs.make_block(n, m, seed=50 + i)
            seen.add((binding.plan_digits(n, m), binding.plan_info(n, m)["first"]))
            got = s.hash(dev(b.x), dev(b.b), m)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(host(got), oracle.pa_hash(b.x, base.a, b.b, n, m,
                                                                    threads=oracle.default_threads()))
        assert len(seen) >= 2, seen
    finally:
        s.close()


def test_unaligned_operands_take_16_bit_digits():
    """Key and seed one limb into their tensors (8-byte, not 16-byte, aligned):
    the wide first pass needs aligned rows, so such a hash uses 16-bit digits;
    it is exact either way."""
    import torch

    binding.wrap_mode(2)
    n, m = 2_500_003, 600_001
    b = inputs.make_block(n, m, seed=8)
    assert binding.plan_digits(n, m) > 16
    L = (n + 63) // 64
    bx = torch.zeros(L + 1, dtype=torch.int64, device="cuda")
    ba = torch.zeros(L + 1, dtype=torch.int64, device="cuda")
    bx[1:].copy_(dev(b.x))
    ba[1:].copy_(dev(b.a))
    got = binding.hash(bx[1:], ba[1:], dev(b.b), n, m)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(host(got), _want(b))


def test_host_buffers_at_width_20():
    binding.digit_width(20)
    n, m = 5_000_011, 1_250_003
    b = inputs.make_block(n, m, seed=12)
    np.testing.assert_array_equal(binding.hash_host(b.x, b.a, b.b, n, m), _want(b))


@pytest.mark.parametrize("w", [18, 20])
def test_crafted_inputs_fail_the_certificate_and_stay_exact(w):
    """x = 0 with b all ones, and a = 1 with x all ones: limb q - 1 of the
    certified sum is all ones, the certificate fails, and the 16-bit
    recomputation gives the exact output."""
    binding.digit_width(w)
    binding.wrap_mode(2)
    n, m = 2_000_000, 400_000
    assert binding.plan_info(n, m)["dropped"] > 0 and binding.plan_digits(n, m) == w
    ones = np.full((n + 63) // 64, np.uint64(0xFFFFFFFFFFFFFFFF))
    ones[-1] &= np.uint64((1 << (n % 64)) - 1) if n % 64 else np.uint64(0xFFFFFFFFFFFFFFFF)
    zero = np.zeros_like(ones)
    one = zero.copy()
    one[0] = 1
    binding.wrap_flags(clear=True)
    for x, a, bb in [(zero, inputs.make_block(n, m, seed=3).a, ones), (ones, one, zero)]:
        got = gpu_hash(binding, x, a, bb, n, m)
        np.testing.assert_array_equal(got, oracle.pa_hash(x, a, bb, n, m, threads=oracle.default_threads()))
    assert binding.wrap_flags() == 2
