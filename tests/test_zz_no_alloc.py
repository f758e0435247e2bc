"""pa_hash_noalloc, the entry point for callers that cannot allocate device memory.

Some integrators cannot let a library allocate: CUDA-graph builders that must
not contain allocation nodes, real-time post-processing loops that reserve all
device memory up front, and programs whose device memory is owned by another
framework's allocator. pa_hash_noalloc serves them from scratch arrays fixed
inside the library. These tests call it through the C ABI and require its
output to equal pa_hash's (exactly: integer results) on two calls in a row of
different sizes, so the second call runs over the first call's leftovers.

This file is collected last on purpose, so that a run stopping at its first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_1910_04429_gb300 import binding, inputs
from tests.gpu_util import dev, host

pytestmark = pytest.mark.gpu


def _noalloc(lib, tx, ta, tb, n, m, stream):
    import torch

    out = torch.full(((m + 63) // 64,), -1, dtype=torch.int64, device="cuda")
    rc = lib.pa_hash_noalloc(ctypes.c_void_p(tx.data_ptr()), ctypes.c_void_p(ta.data_ptr()),
                             ctypes.c_void_p(tb.data_ptr()), n, m, ctypes.c_void_p(out.data_ptr()),
                             ctypes.c_void_p(stream.cuda_stream))
    assert rc == binding.PA_OK, lib.pa_last_error().decode()
    return out


def test_noalloc_matches_pa_hash_two_calls_in_a_row():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required")
    lib = binding.load()
    stream = torch.cuda.current_stream()
    # the largest accepted key first, then a ragged smaller one
    cases = [(1 << 20, 262_147, 31), (1_000_003, 250_001, 32)]
    results = []
    for n, m, seed in cases:
        blk = inputs.make_block(n, m, seed=seed)
        tx, ta, tb = dev(blk.x), dev(blk.a), dev(blk.b)
        got = _noalloc(lib, tx, ta, tb, n, m, stream)
        want = binding.hash(tx, ta, tb, n, m, stream=stream)
        results.append((got, want))
    torch.cuda.synchronize()
    for got, want in results:
        np.testing.assert_array_equal(host(got), host(want))


def test_noalloc_rejects_keys_beyond_its_scratch():
    import torch

    lib = binding.load()
    z = torch.zeros(((1 << 20) + 128) // 64, dtype=torch.int64, device="cuda")
    p = ctypes.c_void_p(z.data_ptr())
    rc = lib.pa_hash_noalloc(p, p, p, (1 << 20) + 1, 64, p, ctypes.c_void_p(0))
    assert rc == binding.PA_EINVAL
    assert b"PA_NOALLOC_MAX_BITS" in lib.pa_last_error()
