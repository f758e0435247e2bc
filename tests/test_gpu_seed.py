"""Seed reuse: hashing with a stored seed spectrum equals pa_hash (exactly)."""
import numpy as np
import pytest

import oracle
from paper_1910_04429_gb300 import binding, inputs
from tests.gpu_util import dev, host

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [1000, 32768, 100_003, 1_536_000, 3_000_001])
def test_seeded_equals_plain(n):
    import torch

    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required")
    seed_blk = inputs.make_block(n, n, seed=n)
    ta = dev(seed_blk.a)
    s = binding.Seed(ta, n)
    try:
        for i, m in enumerate((1, n // 3 or 1, n)):
            blk = inputs.make_block(n, m, seed=n + 100 + i)   # new key and addend, same multiplier
            tx, tb = dev(blk.x), dev(blk.b)
            got = s.hash(tx, tb, m)
            want = binding.hash(tx, ta, tb, n, m)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(host(got), host(want))
            if i == 1:
                np.testing.assert_array_equal(host(got), oracle.pa_hash(blk.x, seed_blk.a, blk.b, n, m))
    finally:
        torch.cuda.synchronize()
        s.close()


@pytest.mark.parametrize("mode", [2, 3])
@pytest.mark.parametrize("n", [100_003, 3_000_001, 10_000_000])
def test_seeded_wrapped_equals_oracle(n, mode):
    """Wrapped seeded hashes (mode 2: wherever shorter; mode 3: the
    recomputation forced) for several m, hence several wrapped lengths built
    on first use from one handle, against the oracle; the seed's limbs may be
    overwritten after the handle is made (the handle keeps its own copy)."""
    import torch

    seed_blk = inputs.make_block(n, n, seed=n + 5)
    ta = dev(seed_blk.a)
    prev = binding.wrap_mode(mode)
    s = binding.Seed(ta, n)
    try:
        torch.cuda.synchronize()
        ta.zero_()  # the handle must not read the caller's seed again
        binding.wrap_flags(clear=True)
        wrapped = 0
        for i, m in enumerate((n // 10, n // 4, n // 10, n // 3)):
            wrapped += binding.plan_info(n, m)["dropped"] > 0
            blk = inputs.make_block(n, m, seed=n + 200 + i)
            got = s.hash(dev(blk.x), dev(blk.b), m)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(host(got), oracle.pa_hash(blk.x, seed_blk.a, blk.b, n, m,
                                                                     threads=oracle.default_threads()),
                                          err_msg=f"m={m}")
        assert wrapped >= 3
        assert binding.wrap_flags() == (wrapped if mode == 3 else 0)
    finally:
        torch.cuda.synchronize()
        s.close()
        binding.wrap_mode(prev)


def test_seeded_wrapped_spectrum_ordered_across_streams():
    """A wrapped spectrum built on one stream and used right away on another:
    the second stream waits for it (the handle's event)."""
    import torch

    n, m = 10_000_000, 1_000_000
    assert binding.plan_info(n, m)["dropped"] > 0
    seed_blk = inputs.make_block(n, m, seed=77)
    s = binding.Seed(dev(seed_blk.a), n)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    try:
        torch.cuda.synchronize()
        blk = inputs.make_block(n, m, seed=78)
        tx, tb = dev(blk.x), dev(blk.b)
        torch.cuda.synchronize()
        o1 = s.hash(tx, tb, m, stream=s1)   # builds the wrapped spectrum on s1
        o2 = s.hash(tx, tb, m, stream=s2)   # must wait for it
        torch.cuda.synchronize()
        want = oracle.pa_hash(blk.x, seed_blk.a, blk.b, n, m, threads=oracle.default_threads())
        np.testing.assert_array_equal(host(o1), want)
        np.testing.assert_array_equal(host(o2), want)
    finally:
        torch.cuda.synchronize()
        s.close()
