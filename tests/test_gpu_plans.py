"""Every plan variant the autotuner may pick gives the same bits, and the
tuner's choice (kept in memory and in the PA_TUNE_CACHE file) stays exact."""
import os

import numpy as np
import pytest

import oracle
from paper_1910_04429_gb300 import binding, inputs
from tests.gpu_util import dev, gpu_hash, host

pytestmark = pytest.mark.gpu

# full-product lengths 2^12 (no strided pass), 2^14 ([4]), 2^17 ([32]), 3*2^16
# ([48]), 2^19 ([2, 64]), 3*2^18 ([3, 64]) and 3*2^24 ([3, 64, 64]; with the
# odd radix last, [64, 64, 3], the middle pass has 64 sub-problems of 192 tiles
# each), and the radix-5 family 5*2^12 ([5]), 5*2^13 ([10]), 5*2^14 ([20]),
# 5*2^15 ([40]) and 5*2^18 ([5, 64]); the single-pass lengths also run with
# narrow tiles (variants 8 .. 15). Each size also runs its wrapped length.
SIZES = [1000, 100_003, 1_000_000, 1_536_000, 3_000_001, 4_800_000, 300_000_017,
         163_840, 327_680, 655_360, 1_310_720, 10_485_760]


@pytest.mark.parametrize("w", [16, 20])
@pytest.mark.parametrize("n", SIZES)
def test_every_plan_variant_is_exact(n, w):
    """Each variant of the full-length product (wrapping off) and, where the
    hash wraps, of the wrapped length, on 16-bit and (where exact) 20-bit
    digits."""
    m = n // 3 or 1
    blk = inputs.make_block(n, m, seed=n)
    want = oracle.pa_hash(blk.x, blk.a, blk.b, blk.n, blk.m, threads=oracle.default_threads())
    prev_w = binding.digit_width(w)
    prev = binding.wrap_mode(2)  # wrapped wherever a shorter length exists
    first = binding.plan_info(n, m)["first"]
    binding.wrap_mode(0)
    full = binding.plan_info(n, m)["full"]
    try:
        for v in range(32):
            binding.plan_override_length(full, v)
            np.testing.assert_array_equal(gpu_hash(binding, blk.x, blk.a, blk.b, blk.n, blk.m), want,
                                          err_msg=f"full length {full}, variant {v}")
        binding.plan_override_length(full, -1)
        binding.wrap_mode(2)
        for v in range(32):
            binding.plan_override_length(first, v)
            np.testing.assert_array_equal(gpu_hash(binding, blk.x, blk.a, blk.b, blk.n, blk.m), want,
                                          err_msg=f"first length {first}, variant {v}")
    finally:
        binding.plan_override_length(full, -1)
        binding.plan_override_length(first, -1)
        binding.wrap_mode(prev)
        binding.digit_width(prev_w)


def test_seed_keeps_its_plan():
    import torch

    n, m = 3_000_001, 700_000
    blk = inputs.make_block(n, m, seed=4)
    ta = dev(blk.a)
    binding.plan_override(n, binding_R0_LAST())
    s = binding.Seed(ta, n)
    binding.plan_override(n, -1)
    try:
        got = s.hash(dev(blk.x), dev(blk.b), m)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(host(got), oracle.pa_hash(blk.x, blk.a, blk.b, n, m))
    finally:
        s.close()


def binding_R0_LAST():
    return 1


def test_autotune_choice_is_exact_and_cached(tmp_path):
    n, m = 4_800_000, 1_000_003
    cache = tmp_path / "tune.txt"
    os.environ["PA_TUNE_CACHE"] = str(cache)
    try:
        v = binding.autotune(n, reps=2)
    finally:
        del os.environ["PA_TUNE_CACHE"]
    assert 0 <= v < 32 and not v & 8  # no narrow plan at this length
    lines = cache.read_text().splitlines()
    full = binding.plan_info(n, m)["full"]  # the unwrapped product's length (20-bit digits here)
    assert full == 1 << 19
    assert any(line.split("\t")[1:] == [str(full), str(v)] for line in lines), lines
    blk = inputs.make_block(n, m, seed=8)
    np.testing.assert_array_equal(gpu_hash(binding, blk.x, blk.a, blk.b, n, m),
                                  oracle.pa_hash(blk.x, blk.a, blk.b, n, m, threads=oracle.default_threads()))
