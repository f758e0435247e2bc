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
