"""The carry look-back's bounded wait: when an earlier tile never publishes
(a flag nothing sets, armed on the host), the wait runs out after a short
limit, the kernel finishes, the status word reports PA_ETIMEOUT, and the
context stays usable. Nothing faults or hangs the GPU."""
import numpy as np
import pytest

import oracle
from paper_1910_04429_gb300 import binding, inputs
from tests.gpu_util import gpu_hash

pytestmark = pytest.mark.gpu


def test_lookback_timeout_is_reported_and_recoverable():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required")
    binding.load()
    assert binding.device_status(clear=True) == binding.PA_OK
    blk = inputs.make_block(1_000_000, 250_000, seed=9)   # 16 carry tiles
    binding.fault_inject(binding.PA_FAULT_CARRY_WAIT)
    gpu_hash(binding, blk.x, blk.a, blk.b, blk.n, blk.m)  # its output is not checked
    assert binding.device_status(clear=True) == binding.PA_ETIMEOUT
    assert binding.device_status() == binding.PA_OK
    # the next call is exact again
    got = gpu_hash(binding, blk.x, blk.a, blk.b, blk.n, blk.m)
    np.testing.assert_array_equal(got, oracle.pa_hash(blk.x, blk.a, blk.b, blk.n, blk.m))
    assert binding.device_status() == binding.PA_OK
