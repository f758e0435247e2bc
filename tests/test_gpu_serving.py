"""Batched and served forms: every result equals the block hashed alone and
the oracle.

The served loop admits blocks by device footprint and runs continuously
formed batches on several streams; the tests compare each served result with
the oracle and with pa_hash on the same block alone (exact equality: integer
output), so that a fault the served path shared with the plain path would
still show.
"""
import numpy as np
import pytest

import oracle
from paper_1910_04429_gb300 import binding, inputs
from tests.gpu_util import dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    binding.load()
    yield
    binding.serve_stop()


def _alone(blks):
    import torch

    outs = []
    for b in blks:
        outs.append(binding.hash(dev(b.x), dev(b.a), dev(b.b), b.n, b.m))
    torch.cuda.synchronize()
    return [host(o) for o in outs]


def test_batched_more_blocks_than_one_launch():
    """40 blocks of one transform length: two launches of the batched kernels."""
    import torch

    blks = [inputs.make_block(100_000 + 977 * i, 20_000 + 13 * i, seed=500 + i) for i in range(40)]
    t = [(dev(b.x), dev(b.a), dev(b.b)) for b in blks]
    outs = [torch.empty((b.m + 63) // 64, dtype=torch.int64, device="cuda") for b in blks]
    binding.hash_batched([(x, a, bb, b.n, b.m, o) for b, (x, a, bb), o in zip(blks, t, outs)])
    torch.cuda.synchronize()
    for b, o in zip(blks, outs):
        np.testing.assert_array_equal(host(o), oracle.pa_hash(b.x, b.a, b.b, b.n, b.m))


def test_captured_batch_replays_current_contents():
    """pa_batch_create captures the batched launch sequence once; every replay
    rehashes the blocks from the current contents of their buffers."""
    import torch

    blks = inputs.make_batch(20, 1_000, 2_000_000, seed=61)
    t = [(dev(b.x), dev(b.a), dev(b.b)) for b in blks]
    outs = [torch.empty((b.m + 63) // 64, dtype=torch.int64, device="cuda") for b in blks]
    batch = binding.Batch([(x, a, bb, b.n, b.m, o) for b, (x, a, bb), o in zip(blks, t, outs)])
    try:
        for rnd in range(2):
            if rnd:  # new keys in the same buffers
                blks = [inputs.make_block(b.n, b.m, seed=900 + i) for i, b in enumerate(blks)]
                for b, (x, a, bb) in zip(blks, t):
                    x.copy_(dev(b.x))
                    a.copy_(dev(b.a))
                    bb.copy_(dev(b.b))
            for o in outs:
                o.fill_(-1)
            batch.run()
            torch.cuda.synchronize()
            for b, o in zip(blks, outs):
                np.testing.assert_array_equal(host(o), oracle.pa_hash(b.x, b.a, b.b, b.n, b.m))
    finally:
        batch.close()


def test_served_results_equal_alone():
    """48 small blocks (10^3 to 4e6 bits) with five large ones (10^7 to 10^8 bits,
    the top of the served workload's size range) mixed in: each served result
    equals the oracle and the block hashed alone."""
    import torch

    binding.serve_stop()
    binding.serve_init(max_batch=8, streams=3)
    blks = inputs.make_batch(48, 1_000, 4_000_000, seed=77)
    big = [inputs.make_block(n, int(n * r), seed=300 + i) for i, (n, r) in
           enumerate([(10_000_019, 0.31), (23_456_789, 0.1), (47_000_001, 0.45), (71_234_567, 0.22),
                      (100_000_000, 0.5)])]
    for i, b in enumerate(big):  # spread through the stream of small ones
        blks.insert(5 + 9 * i, b)
    th = oracle.default_threads()
    want = [oracle.pa_hash(b.x, b.a, b.b, b.n, b.m, threads=th) for b in blks]
    alone = _alone(blks)
    for w, a_ in zip(want, alone):
        np.testing.assert_array_equal(a_, w)
    keep, tickets = [], []
    for b in blks:
        x, a, bb = dev(b.x), dev(b.a), dev(b.b)
        o = torch.full(((b.m + 63) // 64,), -1, dtype=torch.int64, device="cuda")
        keep.append((x, a, bb, o))
        tickets.append(binding.submit(x, a, bb, b.n, b.m, o))
    for tk in tickets:
        rc, st = binding.poll(tk, 30_000_000)
        assert rc == binding.PA_OK and st == binding.PA_OK
    torch.cuda.synchronize()
    for b, (x, a, bb, o), w in zip(blks, keep, want):
        np.testing.assert_array_equal(host(o), w, err_msg=f"n={b.n} m={b.m}")
    s = binding.serve_stats()
    assert s["completed"] == len(blks) and s["pending"] == 0
    assert 0 < s["p50_us"] <= s["p99_us"] <= s["max_us"]
    assert s["peak_inflight_bytes"] <= s["hbm_budget_bytes"]
    # a released ticket is unknown afterwards
    assert binding.poll(tickets[0], 0)[0] == binding.PA_EINVAL
    binding.serve_stop()


def test_served_admission_budget():
    """A budget that fits one large block at a time still serves every block,
    never exceeds the budget, and refuses a block that can never fit."""
    import torch

    blks = [inputs.make_block(n, n // 4, seed=n) for n in (3_000_000, 2_500_000, 2_000_000, 1_000_000)]
    fp = max(binding.workspace_bytes(b.n) + 8 * (3 * ((b.n + 63) // 64) + (b.m + 63) // 64)
             for b in blks)
    binding.serve_stop()
    binding.serve_init(max_batch=4, streams=2, hbm_budget_bytes=int(fp * 1.3))
    want = _alone(blks)
    keep, tickets = [], []
    for b in blks:
        x, a, bb = dev(b.x), dev(b.a), dev(b.b)
        o = torch.empty((b.m + 63) // 64, dtype=torch.int64, device="cuda")
        keep.append(o)
        tickets.append(binding.submit(x, a, bb, b.n, b.m, o))
        keep.append((x, a, bb))
    for tk in tickets:
        rc, st = binding.poll(tk, 30_000_000)
        assert (rc, st) == (binding.PA_OK, binding.PA_OK)
    torch.cuda.synchronize()
    for o, w in zip(keep[0::2], want):
        np.testing.assert_array_equal(host(o), w)
    s = binding.serve_stats()
    assert s["peak_inflight_bytes"] <= int(fp * 1.3)
    big = inputs.make_block(20_000_000, 1000, seed=3)
    x = dev(big.x)
    o = torch.empty(16, dtype=torch.int64, device="cuda")
    with pytest.raises(binding.PaError) as e:
        binding.submit(x, x, x, big.n, big.m, o)
    assert e.value.code == binding.PA_EINVAL
    binding.serve_stop()


def test_poll_returns_when_the_result_is_ready():
    """pa_poll wakes when the serving loop marks the result done, not at its
    deadline: each of several lone requests (nothing else in flight to wake the
    poller again) is polled with a 10 s timeout and must come back in well
    under a second."""
    import time

    import torch

    binding.serve_stop()
    binding.serve_init(max_batch=4, streams=2)
    b = inputs.make_block(200_000, 50_000, seed=12)
    x, a, bb = dev(b.x), dev(b.a), dev(b.b)
    o = torch.empty((b.m + 63) // 64, dtype=torch.int64, device="cuda")
    want = _alone([b])[0]
    try:
        for _ in range(5):
            tk = binding.submit(x, a, bb, b.n, b.m, o)
            t0 = time.perf_counter()
            rc, st = binding.poll(tk, 10_000_000)
            waited = time.perf_counter() - t0
            assert (rc, st) == (binding.PA_OK, binding.PA_OK)
            assert waited < 0.5, waited
            torch.cuda.synchronize()
            np.testing.assert_array_equal(host(o), want)
    finally:
        binding.serve_stop()
