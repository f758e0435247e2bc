"""The batched workload at its full shape, against the oracle block by block.

256 independent blocks with n log-uniform in [10^6, 10^7] bits, m = floor(n r),
r ~ U(0.1, 0.5), block i seeded 1 + i (the input recipe of the batched
benchmark). Every block's output is Eq. 7 of its own (x, a, b), so each one is
compared bit for bit with the oracle, for the batched call (pa_hash_batched)
both with the persistent kernel and by size class (pa_batch_mode), and for
the same batch captured once and replayed as a CUDA graph (pa_batch_create /
pa_batch_run).
"""
import numpy as np
import pytest

import oracle
from paper_1910_04429_gb300 import binding, inputs
from tests.gpu_util import dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def batch():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    binding.load()
    blks = inputs.make_batch(256, 1_000_000, 10_000_000, seed=1)
    th = oracle.default_threads()
    want = [oracle.pa_hash(b.x, b.a, b.b, b.n, b.m, threads=th) for b in blks]
    t = [(dev(b.x), dev(b.a), dev(b.b)) for b in blks]
    return blks, t, want


def _outs(blks):
    import torch

    return [torch.full(((b.m + 63) // 64,), -1, dtype=torch.int64, device="cuda") for b in blks]


def test_shape_of_the_workload(batch):
    blks, _, _ = batch
    ns = [b.n for b in blks]
    assert len(blks) == 256 and min(ns) >= 1_000_000 and max(ns) <= 10_000_000
    assert all(0.1 * b.n - 1 <= b.m <= 0.5 * b.n for b in blks)
    assert len({b.seed for b in blks}) == 256 and min(b.seed for b in blks) == 1
    # several transform lengths (size classes) and wrapped products among them
    lens = {binding.plan_info(b.n, b.m)["first"] for b in blks}
    assert len(lens) >= 4


@pytest.mark.parametrize("mode", [2, 1, 0])
def test_batched_call_matches_oracle(batch, mode):
    """Mode 1: the persistent kernel; mode 0: launches by size class; mode 2
    (default): chosen by the batch's tile count (by size class here)."""
    import torch

    blks, t, want = batch
    outs = _outs(blks)
    prev = binding.batch_mode(mode)
    try:
        binding.hash_batched([(x, a, bb, b.n, b.m, o) for b, (x, a, bb), o in zip(blks, t, outs)])
        torch.cuda.synchronize()
    finally:
        binding.batch_mode(prev)
    for b, o, w in zip(blks, outs, want):
        np.testing.assert_array_equal(host(o), w, err_msg=f"n={b.n} m={b.m} seed={b.seed}")
    assert binding.stream_status() == binding.PA_OK


def test_captured_graph_matches_oracle(batch):
    import torch

    blks, t, want = batch
    outs = _outs(blks)
    g = binding.Batch([(x, a, bb, b.n, b.m, o) for b, (x, a, bb), o in zip(blks, t, outs)])
    try:
        for o in outs:
            o.fill_(-1)
        g.run()
        torch.cuda.synchronize()
        for b, o, w in zip(blks, outs, want):
            np.testing.assert_array_equal(host(o), w, err_msg=f"n={b.n} m={b.m} seed={b.seed}")
    finally:
        g.close()
