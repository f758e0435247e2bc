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


def test_stream_status_reports_the_timeout_on_its_stream_only():
    """pa_stream_status: the timeout shows on the stream whose carry launch gave
    up its wait, not on another stream that hashed meanwhile; clearing resets
    that stream's word, and the device-wide word sees the same event."""
    import torch

    binding.load()
    binding.device_status(clear=True)
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    blk = inputs.make_block(1_000_000, 250_000, seed=19)
    for s in (sa, sb):
        assert binding.stream_status(s, clear=True) == binding.PA_OK
    binding.fault_inject(binding.PA_FAULT_CARRY_WAIT)   # the next carry launch: on sa
    gpu_hash(binding, blk.x, blk.a, blk.b, blk.n, blk.m, stream=sa)
    got_b = gpu_hash(binding, blk.x, blk.a, blk.b, blk.n, blk.m, stream=sb)
    assert binding.stream_status(sb) == binding.PA_OK
    assert binding.stream_status(sa) == binding.PA_ETIMEOUT
    assert binding.stream_status(sa, clear=True) == binding.PA_ETIMEOUT
    assert binding.stream_status(sa) == binding.PA_OK
    assert binding.device_status(clear=True) == binding.PA_ETIMEOUT
    want = oracle.pa_hash(blk.x, blk.a, blk.b, blk.n, blk.m)
    np.testing.assert_array_equal(got_b, want)
    np.testing.assert_array_equal(gpu_hash(binding, blk.x, blk.a, blk.b, blk.n, blk.m, stream=sa), want)
    assert binding.stream_status(sa) == binding.PA_OK
