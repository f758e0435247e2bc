"""Wrapped products on the GPU, bit for bit against the oracle: the shorter
cyclic convolution whose folded low coefficients are dropped, the carry step's
certificate (limb floor((n-m)/64) - 1 of the remaining sum not all ones), and
the exact recomputation (the full product at a power-of-two length, one
cooperative launch) that runs when the certificate fails."""
import numpy as np
import pytest

import oracle
from paper_1910_04429_gb300 import binding, inputs
from tests.gpu_util import dev, gpu_hash, host

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def wrap_wherever_shorter():
    """Mode 2: wrapped products at every size with a shorter length (the
    default, mode 1, leaves full products below 2^19 points unwrapped)."""
    prev = binding.wrap_mode(2)
    yield
    binding.wrap_mode(prev)

# sizes whose hash wraps (checked below): a few tiles, ragged n and m, 2^k,
# 3 * 2^k and 5 * 2^k wrapped lengths, one and two strided passes, and the
# 10^6-bit block
WRAPPED = [(100_000, 25_000), (100_003, 12_345), (1_000_000, 250_000), (1_000_003, 100_001),
           (3_000_017, 300_001), (6_000_000, 600_000), (4_800_000, 240_000), (10_000_000, 1_000_000),
           # floor((n - m)/64) = 10 * 1024: the certificate's limb lies in the carry
           # tile below the first output tile (the carry kernel starts one tile lower),
           # with n - m a multiple of 64 and not
           (819_200, 163_840), (819_200, 163_823)]


def _want(blk):
    return oracle.pa_hash(blk.x, blk.a, blk.b, blk.n, blk.m, threads=oracle.default_threads())


def _limbs(v, n):
    return np.array([(v >> (64 * i)) & ((1 << 64) - 1) for i in range(-(-n // 64))], dtype=np.uint64)


def _int(arr):
    return int.from_bytes(np.ascontiguousarray(arr, dtype=np.uint64).tobytes(), "little")


@pytest.mark.parametrize("n,m", WRAPPED)
def test_wrapped_matches_oracle(n, m):
    info = binding.plan_info(n, m)
    assert info["dropped"] > 0 and info["first"] < info["full"]  # the full product at the width chosen unwrapped
    binding.wrap_flags(clear=True)
    for seed in (1, 2):
        blk = inputs.make_block(n, m, seed=seed)
        np.testing.assert_array_equal(gpu_hash(binding, blk.x, blk.a, blk.b, n, m), _want(blk))
    assert binding.wrap_flags() == 0  # uniform b: the certificate holds


@pytest.mark.parametrize("n,m", WRAPPED[:5])
def test_forced_fallback_matches_oracle(n, m):
    """Mode 3 fails every certificate: the recomputation runs after the
    wrapped product and its output replaces the wrapped one's."""
    blk = inputs.make_block(n, m, seed=5)
    binding.wrap_mode(3)
    binding.wrap_flags(clear=True)
    got = gpu_hash(binding, blk.x, blk.a, blk.b, n, m)
    assert binding.wrap_flags() == 1
    np.testing.assert_array_equal(got, _want(blk))


def test_wrapping_off_matches_oracle():
    n, m = 1_000_003, 100_001
    blk = inputs.make_block(n, m, seed=6)
    binding.wrap_mode(0)
    assert binding.plan_info(n, m)["dropped"] == 0
    np.testing.assert_array_equal(gpu_hash(binding, blk.x, blk.a, blk.b, n, m), _want(blk))


def _dropped_part(x, a, L, lo):
    """T = sum_{k < lo} t_k 2^(16k), t the linear convolution of the digits."""
    dx = np.frombuffer(x.tobytes(), dtype=np.uint16)[:L].astype(np.int64)
    da = np.frombuffer(a.tobytes(), dtype=np.uint16)[:L].astype(np.int64)
    t = np.convolve(da[:lo], dx[:lo])[:lo]  # t_k, k < lo, uses digits below lo only (< 2^63)
    T = 0
    for k in range(lo - 1, -1, -1):
        T = (T << 16) + int(t[k])
    return T


def test_crafted_inputs_take_the_fallback():
    """Inputs whose limb q - 1 of the remaining sum is all ones: x = 0 with
    b = 2^n - 1; a = 1 with x = 2^n - 1; and b built so that the dropped part
    carries into the output (the wrapped product alone would be one off there).
    Each fails the certificate once and comes out exact."""
    n, m = 1_000_000, 250_000
    s = n - m
    L = -(-n // 16)
    lo = binding.plan_info(n, m)["dropped"]
    blk = inputs.make_block(n, m, seed=7)
    ones = _limbs((1 << n) - 1, n)
    zero = np.zeros_like(ones)
    one = zero.copy()
    one[0] = 1
    x, a = blk.x, blk.a
    T = _dropped_part(x, a, L, lo)
    assert T > 0
    xi, ai = _int(x), _int(a)
    q_target = (_int(blk.b) >> s << s) + ((1 << s) - T)
    b_carry = _limbs((q_target - ai * xi + T) % (1 << n), n)
    cases = [(zero, a, ones), (ones, one, zero), (x, a, b_carry)]
    binding.wrap_flags(clear=True)
    for i, (cx, ca, cb) in enumerate(cases):
        want = oracle.pa_hash(cx, ca, cb, n, m, threads=oracle.default_threads())
        np.testing.assert_array_equal(gpu_hash(binding, cx, ca, cb, n, m), want, err_msg=f"case {i}")
        assert binding.wrap_flags() == i + 1, i
    # the last case needed the fallback: the sum without the dropped part is one off
    assert _int(oracle.pa_hash(x, a, b_carry, n, m, threads=4)) == ((q_target >> s) + 1) % (1 << m)


@pytest.mark.parametrize("n,m", [(819_200, 163_840), (819_200, 163_823), (1_000_000, 250_000)])
def test_all_ones_addend_is_flagged(n, m):
    """x = 0, b = 2^n - 1: the sum's limb below the output is all ones, so the
    certificate must fail (also where that limb lies in the tile below the
    first output tile) and the output is b's top m bits."""
    assert binding.plan_info(n, m)["dropped"] > 0
    ones = _limbs((1 << n) - 1, n)
    a = inputs.make_block(n, m, seed=3).a
    binding.wrap_flags(clear=True)
    got = gpu_hash(binding, np.zeros_like(ones), a, ones, n, m)
    assert binding.wrap_flags() == 1
    np.testing.assert_array_equal(got, oracle.pa_hash(np.zeros_like(ones), a, ones, n, m, threads=4))


def test_host_buffers_wrapped_and_forced():
    n, m = 3_000_017, 300_001
    blk = inputs.make_block(n, m, seed=9)
    want = _want(blk)
    np.testing.assert_array_equal(binding.hash_host(blk.x, blk.a, blk.b, n, m), want)
    binding.wrap_mode(3)
    np.testing.assert_array_equal(binding.hash_host(blk.x, blk.a, blk.b, n, m), want)


def test_full_size_wrapped_sampled():
    """n = 10^8, m = 2.5e7 (wrapped length 3 * 2^21 on 20-bit digits): the
    certificate holds, and the output equals the full-length product's and the
    16-bit wrapped product's (2^23 points) bit for bit (the full-length path is
    itself checked against the oracle by the other parity tests)."""
    import torch

    n, m = 100_000_000, 25_000_000
    assert binding.plan_info(n, m)["first"] == 3 << 21 and binding.plan_digits(n, m) == 20
    blk = inputs.make_block(n, m, seed=1)
    tx, ta, tb = dev(blk.x), dev(blk.a), dev(blk.b)
    binding.wrap_flags(clear=True)
    got = host(binding.hash(tx, ta, tb, n, m))
    torch.cuda.synchronize()
    assert binding.wrap_flags() == 0
    binding.wrap_mode(0)
    ref = host(binding.hash(tx, ta, tb, n, m))
    torch.cuda.synchronize()
    binding.wrap_mode(3)  # the recomputation at length 2^24 as well
    forced = host(binding.hash(tx, ta, tb, n, m))
    torch.cuda.synchronize()
    binding.wrap_mode(1)
    prev_w = binding.digit_width(16)
    try:
        assert binding.plan_info(n, m)["first"] == 1 << 23
        w16 = host(binding.hash(tx, ta, tb, n, m))
        torch.cuda.synchronize()
    finally:
        binding.digit_width(prev_w)
    np.testing.assert_array_equal(got, ref)
    np.testing.assert_array_equal(forced, ref)
    np.testing.assert_array_equal(w16, ref)
    assert binding.device_status() == 0  # no bounded wait ran out


def test_batched_forced_fallback_over_several_launches():
    """70 wrapped blocks (two transform lengths) and 3 unwrapped ones in one
    batched call, every certificate failed (mode 3): the recomputation runs in
    two launches of at most 64 jobs, each with its own grid-barrier counter;
    every block comes out exact and only the wrapped ones were flagged."""
    import torch

    wrapped = [inputs.make_block(100_000 + 1009 * i, 25_000 + 7 * i, seed=700 + i) for i in range(70)]
    plain = [inputs.make_block(5_000 + 17 * i, 100 + i, seed=800 + i) for i in range(3)]
    for b in wrapped:  # the batch rule is mode 2's: wrap wherever a shorter length certifies
        assert binding.plan_info(b.n, b.m)["dropped"] > 0
    for b in plain:
        assert binding.plan_info(b.n, b.m)["dropped"] == 0
    blks = wrapped[:40] + plain + wrapped[40:]
    binding.wrap_mode(3)
    binding.wrap_flags(clear=True)
    t = [(dev(b.x), dev(b.a), dev(b.b)) for b in blks]
    outs = [torch.full(((b.m + 63) // 64,), -1, dtype=torch.int64, device="cuda") for b in blks]
    binding.hash_batched([(x, a, bb, b.n, b.m, o) for b, (x, a, bb), o in zip(blks, t, outs)])
    torch.cuda.synchronize()
    assert binding.wrap_flags() == len(wrapped)
    for i, (b, o) in enumerate(zip(blks, outs)):
        np.testing.assert_array_equal(host(o), _want(b), err_msg=f"block {i}")
    assert binding.device_status() == 0
