"""pa_hash_noalloc, the entry point for callers that cannot allocate device memory.

Some integrators cannot let a library allocate: CUDA-graph builders that must
not contain allocation nodes, real-time post-processing loops that reserve all
device memory up front, and programs whose device memory is owned by another
framework's allocator. pa_hash_noalloc serves them from scratch arrays fixed
inside the library. These tests call it through the C ABI and require its
output to equal pa_hash's and the oracle's (exactly: integer results) on two
calls in a row of different sizes, so the second call runs over the first
call's leftovers; and again after pa_shutdown, which makes the next call set
up again.

This file is collected last on purpose, so that a run stopping at its first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import oracle
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


# the largest accepted key first, then a ragged smaller one
CASES = [(1 << 20, 262_147, 31), (1_000_003, 250_001, 32)]


def _two_calls_in_a_row(lib, stream):
    import torch

    results = []
    for n, m, seed in CASES:
        blk = inputs.make_block(n, m, seed=seed)
        tx, ta, tb = dev(blk.x), dev(blk.a), dev(blk.b)
        got = _noalloc(lib, tx, ta, tb, n, m, stream)
        want = binding.hash(tx, ta, tb, n, m, stream=stream)
        results.append((blk, got, want))
    torch.cuda.synchronize()
    for blk, got, want in results:
        exact = oracle.pa_hash(blk.x, blk.a, blk.b, blk.n, blk.m, threads=oracle.default_threads())
        np.testing.assert_array_equal(host(got), host(want))
        np.testing.assert_array_equal(host(got), exact)


def test_noalloc_matches_pa_hash_two_calls_in_a_row():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required")
    _two_calls_in_a_row(binding.load(), torch.cuda.current_stream())


def test_noalloc_sets_up_again_after_shutdown():
    """pa_shutdown forgets the per-device set-up (the scratch addresses and the
    filled twiddle tables); the next calls set up again and stay exact."""
    import torch

    lib = binding.load()
    stream = torch.cuda.current_stream()
    _two_calls_in_a_row(lib, stream)
    torch.cuda.synchronize()
    assert lib.pa_shutdown() == binding.PA_OK
    _two_calls_in_a_row(lib, stream)


def test_noalloc_first_call_on_a_capturing_stream_is_refused():
    """The set-up waits for its table kernels, which would end a capture: a first
    call on a capturing stream returns PA_EINVAL, and the capture it was made in
    still completes (its own work replays)."""
    import torch

    lib = binding.load()
    torch.cuda.synchronize()
    assert lib.pa_shutdown() == binding.PA_OK  # the next call is a first call again
    blk = inputs.make_block(100_003, 20_011, seed=33)
    tx, ta, tb = dev(blk.x), dev(blk.a), dev(blk.b)
    out = torch.full(((blk.m + 63) // 64,), -1, dtype=torch.int64, device="cuda")
    counter = torch.zeros(1, dtype=torch.int64, device="cuda")
    side = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        counter.add_(1)
        rc = lib.pa_hash_noalloc(ctypes.c_void_p(tx.data_ptr()), ctypes.c_void_p(ta.data_ptr()),
                                 ctypes.c_void_p(tb.data_ptr()), blk.n, blk.m,
                                 ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(side.cuda_stream))
    assert rc == binding.PA_EINVAL
    assert b"capturing" in lib.pa_last_error()
    g.replay()
    torch.cuda.synchronize()
    assert int(counter.item()) == 1
    # outside a capture the same first call sets up and is exact
    got = _noalloc(lib, tx, ta, tb, blk.n, blk.m, torch.cuda.current_stream())
    torch.cuda.synchronize()
    np.testing.assert_array_equal(host(got), oracle.pa_hash(blk.x, blk.a, blk.b, blk.n, blk.m))


def test_noalloc_rejects_keys_beyond_its_scratch():
    import torch

    lib = binding.load()
    z = torch.zeros(((1 << 20) + 128) // 64, dtype=torch.int64, device="cuda")
    p = ctypes.c_void_p(z.data_ptr())
    rc = lib.pa_hash_noalloc(p, p, p, (1 << 20) + 1, 64, p, ctypes.c_void_p(0))
    assert rc == binding.PA_EINVAL
    assert b"PA_NOALLOC_MAX_BITS" in lib.pa_last_error()
