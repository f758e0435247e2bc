"""Multi-rank host logic of the benchmark on CPU (gloo, world size 2).

Blocks are independent problems, so ranks are replicas: each hashes its own
seeded blocks and only the timings meet in a collective (max over ranks).
"""
import os
import socket

import numpy as np
import pytest

import bench
import oracle
from paper_1910_04429_gb300 import inputs

N_SMALL, M_SMALL = 20_000, 5_000


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist

    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        seeds = bench.rank_seeds(rank)
        outs = []
        for s in seeds:
            b = inputs.make_block(N_SMALL, M_SMALL, seed=s)
            outs.append(oracle.pa_hash(b.x, b.a, b.b, b.n, b.m).tobytes())
        # fake per-rank timings: rank r took 10 + r ms for its steps
        ms = bench.max_over_ranks([10.0 + rank, 1.0 + 2 * rank], world)
        q.put((rank, seeds, outs, ms))
    finally:
        dist.destroy_process_group()


def test_two_ranks_replicas_and_max_timing():
    import torch.multiprocessing as mp

    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    got.sort()
    seeds0, seeds1 = got[0][1], got[1][1]
    assert not set(seeds0) & set(seeds1), "ranks must own disjoint blocks"
    # each rank's results equal a single-process computation of the same blocks
    for rank, seeds, outs, ms in got:
        for s, o in zip(seeds, outs):
            b = inputs.make_block(N_SMALL, M_SMALL, seed=s)
            assert o == oracle.pa_hash(b.x, b.a, b.b, b.n, b.m).tobytes()
        assert ms == [11.0, 3.0]  # the slowest rank's time, on every rank
    # whole-job throughput: both ranks' bits over the slowest rank's time
    assert bench.aggregate_mbps(2, 10, N_SMALL, 11.0) == pytest.approx(2 * 10 * N_SMALL / 0.011 / 1e6)


def test_single_rank_is_identity():
    assert bench.max_over_ranks([3.5, 7.0], 1) == [3.5, 7.0]
    assert bench.rank_seeds(0) == [1, 2, 3, 4]
    assert np.isclose(bench.aggregate_mbps(1, 1, 10**8, 1.0), 1e5)
