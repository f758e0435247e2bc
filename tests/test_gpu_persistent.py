"""The persistent batched kernel (pa_batch_mode 1): many blocks' transforms in
one cooperative launch, bit for bit against the oracle.

Cases that exercise its bookkeeping: more blocks than one launch holds (256),
more transform lengths than one launch holds (16), blocks whose plan it does
not take (a single 4096-point tile) or whose operands are not 16-byte aligned
(both run by size class beside it), wrapped products with the recomputation
forced, and the same batch in both modes.
"""
import numpy as np
import pytest

import oracle
from paper_1910_04429_gb300 import binding, inputs
from tests.gpu_util import dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _persistent():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    prev = binding.batch_mode(1)
    yield
    binding.batch_mode(prev)


def _run(blks, tensors=None):
    import torch

    t = tensors or [(dev(b.x), dev(b.a), dev(b.b)) for b in blks]
    outs = [torch.full(((b.m + 63) // 64,), -1, dtype=torch.int64, device="cuda") for b in blks]
    binding.hash_batched([(x, a, bb, b.n, b.m, o) for b, (x, a, bb), o in zip(blks, t, outs)])
    torch.cuda.synchronize()
    return [host(o) for o in outs]


def _check(blks, got):
    th = oracle.default_threads()
    for i, (b, g) in enumerate(zip(blks, got)):
        np.testing.assert_array_equal(g, oracle.pa_hash(b.x, b.a, b.b, b.n, b.m, threads=th),
                                      err_msg=f"block {i}: n={b.n} m={b.m}")


def test_more_blocks_than_one_launch():
    blks = inputs.make_batch(300, 20_000, 300_000, seed=901)
    _check(blks, _run(blks))
    assert binding.device_status() == binding.PA_OK


def _family(lo, hi):
    """The library's transform lengths in [lo, hi] (2^k; 3 * 2^j, 5 * 2^j with
    first radix at most 48 and 40)."""
    out = set()
    for k in range(12, 30):
        for odd, top in ((1, 5), (3, 4), (5, 3)):
            if (k - 12) % 6 <= top and lo <= (odd << k) <= hi:
                out.add(odd << k)
    return sorted(out)


def test_more_lengths_than_one_launch():
    """Twenty transform lengths in one call (16-bit digits, full products:
    n = 8 N - 3 has the full length N), so the kernel needs a second launch."""
    lens = _family(8192, 1 << 21)[:20]
    assert len(lens) == 20
    prev_w, prev_m = binding.digit_width(16), binding.wrap_mode(0)
    try:
        blks = [inputs.make_block(8 * N - 3, (8 * N - 3) // 3, seed=950 + i) for i, N in enumerate(lens)]
        assert [binding.plan_info(b.n, b.m)["first"] for b in blks] == lens
        _check(blks, _run(blks))
    finally:
        binding.digit_width(prev_w)
        binding.wrap_mode(prev_m)


def test_blocks_it_does_not_take_run_beside_it():
    """Single-tile transforms and operands one limb into their tensors (8-byte
    aligned) go by size class on the side streams, in the same call."""
    import torch

    blks = inputs.make_batch(24, 200_000, 3_000_000, seed=33) + [inputs.make_block(5_000, 1_000, seed=34)]
    t = []
    for i, b in enumerate(blks):
        if i % 3 == 0:  # not 16-byte aligned
            L = (b.n + 63) // 64
            xs = torch.zeros(L + 1, dtype=torch.int64, device="cuda")
            as_ = torch.zeros(L + 1, dtype=torch.int64, device="cuda")
            xs[1:].copy_(dev(b.x))
            as_[1:].copy_(dev(b.a))
            t.append((xs[1:], as_[1:], dev(b.b)))
        else:
            t.append((dev(b.x), dev(b.a), dev(b.b)))
    _check(blks, _run(blks, t))


@pytest.mark.parametrize("mode", [2, 3])
def test_wrapped_and_forced_recomputation(mode):
    prev = binding.wrap_mode(mode)
    try:
        binding.wrap_flags(clear=True)
        blks = inputs.make_batch(40, 100_000, 4_000_000, seed=60 + mode)
        wrapped = sum(binding.plan_info(b.n, b.m)["dropped"] > 0 for b in blks)
        _check(blks, _run(blks))
        assert binding.wrap_flags() == (wrapped if mode == 3 else 0)
    finally:
        binding.wrap_mode(prev)


def test_both_modes_agree():
    blks = inputs.make_batch(64, 1_000_000, 10_000_000, seed=5)
    t = [(dev(b.x), dev(b.a), dev(b.b)) for b in blks]
    got1 = _run(blks, t)
    binding.batch_mode(0)
    got0 = _run(blks, t)
    for a, b in zip(got1, got0):
        np.testing.assert_array_equal(a, b)
    _check(blks[:16], got1[:16])


def test_automatic_mode_takes_the_persistent_kernel_for_small_batches():
    """Mode 2 (default): 16 blocks of 1e6 .. 2e6 bits (under 8 tiles per SM)
    run in the persistent kernel; the 256-block workload's tiles do not."""
    binding.batch_mode(2)
    blks = inputs.make_batch(16, 1_000_000, 2_000_000, seed=11)
    binding.profile(True)
    got = _run(blks)
    binding.profile(False)
    names = binding.profile_collect()
    assert "ntt_persistent" in names, names
    _check(blks, got)
    big = inputs.make_batch(64, 1_000_000, 10_000_000, seed=1)
    binding.profile(True)
    _run(big)
    binding.profile(False)
    names = binding.profile_collect()
    assert "ntt_persistent" not in names and "ntt_contig_both" in names, names
