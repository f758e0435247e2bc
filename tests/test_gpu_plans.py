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
# narrow tiles (variants 8 .. 15), and lengths of at most 64 tiles with the tile
# pass on four-CTA clusters (variants 32 .. 63). Each size also runs its wrapped
# length.
SIZES = [1000, 100_003, 1_000_000, 1_536_000, 3_000_001, 4_800_000, 300_000_017,
         163_840, 327_680, 655_360, 1_310_720, 10_485_760]


def _variants(N):
    """The variants that can differ at length N (the cluster bit applies to
    transforms of at most 64 tiles; elsewhere it is masked off)."""
    return [v for v in range(binding.PLAN_VARIANTS) if N <= 64 * 4096 or not v & binding.PLAN_CLUSTER]


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
        for v in _variants(full):
            binding.plan_override_length(full, v)
            np.testing.assert_array_equal(gpu_hash(binding, blk.x, blk.a, blk.b, blk.n, blk.m), want,
                                          err_msg=f"full length {full}, variant {v}")
        binding.plan_override_length(full, -1)
        binding.wrap_mode(2)
        for v in _variants(first):
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


@pytest.mark.parametrize("variant", [32, 32 | 8, 32 | 8 | 2 | 4])
def test_cluster_plan_seeds_graphs_and_toeplitz(variant):
    """Under the cluster plan: seeds made and used (their spectra keep the
    one-CTA order), a one-block captured graph, host buffers, and Toeplitz
    hashes (one-bit digits, a single tile and several) are exact."""
    import torch

    n, m = 1_000_000, 250_000
    blk = inputs.make_block(n, m, seed=variant)
    want = oracle.pa_hash(blk.x, blk.a, blk.b, n, m, threads=oracle.default_threads())
    full = binding.plan_info(n, m)["full"]
    assert full <= 64 * 4096
    binding.plan_override_length(full, variant)
    try:
        s = binding.Seed(dev(blk.a), n)
        try:
            got = s.hash(dev(blk.x), dev(blk.b), m)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(host(got), want)
        finally:
            s.close()
        tx, ta, tb = dev(blk.x), dev(blk.a), dev(blk.b)
        out = torch.full(((m + 63) // 64,), -1, dtype=torch.int64, device="cuda")
        g = binding.Batch([(tx, ta, tb, n, m, out)])
        try:
            for _ in range(2):
                out.fill_(-1)
                g.run()
                torch.cuda.synchronize()
                np.testing.assert_array_equal(host(out), want)
        finally:
            g.close()
        np.testing.assert_array_equal(binding.hash_host(blk.x, blk.a, blk.b, n, m), want)
    finally:
        binding.plan_override_length(full, -1)
    # Toeplitz: n + m - 1 = 250,003 bits (2^18 points, 64 tiles) and 3,001 (one tile)
    for tn, tm, tlen in [(200_003, 50_001, 1 << 18), (2_001, 1_001, 4096)]:
        tbk = inputs.make_toeplitz_block(tn, tm, seed=4)
        twant = oracle.toeplitz(tbk.x, tbk.s, tn, tm, threads=oracle.default_threads())
        binding.plan_override_length(tlen, variant)
        try:
            np.testing.assert_array_equal(host(binding.toeplitz(dev(tbk.x), dev(tbk.s), tn, tm)), twant)
        finally:
            binding.plan_override_length(tlen, -1)


def test_autotune_choice_is_exact_and_cached(tmp_path):
    n, m = 4_800_000, 1_000_003
    cache = tmp_path / "tune.txt"
    os.environ["PA_TUNE_CACHE"] = str(cache)
    try:
        v = binding.autotune(n, reps=2)
    finally:
        del os.environ["PA_TUNE_CACHE"]
    assert 0 <= v < binding.PLAN_VARIANTS and not v & (binding.PLAN_NARROW | binding.PLAN_CLUSTER)  # 128 tiles
    lines = cache.read_text().splitlines()
    full = binding.plan_info(n, m)["full"]  # the unwrapped product's length (20-bit digits here)
    assert full == 1 << 19
    assert any(line.split("\t")[1:] == [str(full), str(v)] for line in lines), lines
    blk = inputs.make_block(n, m, seed=8)
    np.testing.assert_array_equal(gpu_hash(binding, blk.x, blk.a, blk.b, n, m),
                                  oracle.pa_hash(blk.x, blk.a, blk.b, n, m, threads=oracle.default_threads()))
