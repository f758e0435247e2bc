"""Seeded random sizes against the oracle, bit for bit: key lengths log-uniform
from 1 bit to 3e6 bits with any output length, each under a random plan
variant; small keys with the tile pass forced onto four-CTA clusters, full and
wrapped; random Toeplitz sizes; random mixed batches."""
import math

import numpy as np
import pytest

import oracle
from paper_1910_04429_gb300 import binding, inputs
from tests.gpu_util import dev, gpu_hash, host

pytestmark = pytest.mark.gpu


def _sizes(seed, count, n_max):
    u = inputs.uniforms(seed, 3 * count)
    out = []
    for i in range(count):
        n = max(1, int(math.exp(float(u[3 * i]) * math.log(n_max))))
        m = 1 + int(float(u[3 * i + 1]) * n) if n > 1 else 1
        out.append((n, min(m, n), int(float(u[3 * i + 2]) * binding.PLAN_VARIANTS)))
    return out


@pytest.mark.parametrize("chunk", range(4))
def test_random_sizes_and_plans(chunk):
    for n, m, variant in _sizes(1000 + chunk, 12, 3_000_000):
        blk = inputs.make_block(n, m, seed=n ^ (m << 1))
        binding.plan_override(n, variant)  # masked to what applies at this length
        try:
            got = gpu_hash(binding, blk.x, blk.a, blk.b, n, m)
        finally:
            binding.plan_override(n, -1)
        want = oracle.pa_hash(blk.x, blk.a, blk.b, n, m, threads=oracle.default_threads())
        np.testing.assert_array_equal(got, want, err_msg=f"n={n} m={m} variant={variant}")


@pytest.mark.parametrize("wrap", [1, 2])
def test_random_small_sizes_on_clusters(wrap):
    """Keys up to 2.1e6 bits (transforms of at most 64 tiles, the single tile
    included) with the cluster bit set and the other bits random; wrap mode 2
    wraps wherever a shorter length certifies."""
    prev = binding.wrap_mode(wrap)
    try:
        for n, m, variant in _sizes(2000 + wrap, 16, 2_100_000):
            v = variant | binding.PLAN_CLUSTER
            blk = inputs.make_block(n, m, seed=3 * n + m)
            info = binding.plan_info(n, m)
            for N in {info["first"], info["full"]}:
                binding.plan_override_length(N, v)
            try:
                got = gpu_hash(binding, blk.x, blk.a, blk.b, n, m)
            finally:
                for N in {info["first"], info["full"]}:
                    binding.plan_override_length(N, -1)
            want = oracle.pa_hash(blk.x, blk.a, blk.b, n, m, threads=oracle.default_threads())
            np.testing.assert_array_equal(got, want, err_msg=f"n={n} m={m} variant={v} wrap={wrap}")
    finally:
        binding.wrap_mode(prev)


def test_random_toeplitz_sizes():
    import torch

    for n, m, _ in _sizes(77, 16, 400_000):
        blk = inputs.make_toeplitz_block(n, m, seed=n + m)
        got = binding.toeplitz(dev(blk.x), dev(blk.s), n, m)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(host(got), oracle.toeplitz(blk.x, blk.s, n, m, threads=8),
                                      err_msg=f"n={n} m={m}")


def test_random_batches():
    import torch

    sizes = [(n, m) for n, m, _ in _sizes(555, 40, 2_000_000)]
    blks = [inputs.make_block(n, m, seed=7 + i) for i, (n, m) in enumerate(sizes)]
    tensors = [(dev(b.x), dev(b.a), dev(b.b), b.n, b.m,
                torch.zeros((b.m + 63) // 64, dtype=torch.int64, device="cuda")) for b in blks]
    binding.hash_batched(tensors)
    torch.cuda.synchronize()
    for b, t in zip(blks, tensors):
        want = oracle.pa_hash(b.x, b.a, b.b, b.n, b.m, threads=oracle.default_threads())
        np.testing.assert_array_equal(host(t[5]), want, err_msg=f"n={b.n} m={b.m}")


@pytest.mark.parametrize("mode", [2, 3])
def test_random_sizes_wrapped(mode):
    """Wrapped products at random sizes from 1e5 to 5e6 bits (log-uniform) with
    random m up to 0.6 n (mode 2:
    wherever a shorter length is certifiable; mode 3: the certificate forced to
    fail, so every hash also runs the recomputation), against the oracle; in
    mode 2 no certificate fails on these uniform inputs."""
    prev = binding.wrap_mode(mode)
    try:
        binding.wrap_flags(clear=True)
        wrapped = 0
        u = inputs.uniforms(4242 + mode, 48)
        sizes = [(int(math.exp(math.log(1e5) + float(u[2 * i]) * math.log(50.0))), float(u[2 * i + 1]))
                 for i in range(24)]
        for n, r in sizes:
            m = max(1, int(r * 0.6 * n))
            if binding.plan_info(n, m)["dropped"] == 0:
                continue
            wrapped += 1
            blk = inputs.make_block(n, m, seed=n + 3 * m)
            got = gpu_hash(binding, blk.x, blk.a, blk.b, n, m)
            want = oracle.pa_hash(blk.x, blk.a, blk.b, n, m, threads=oracle.default_threads())
            np.testing.assert_array_equal(got, want, err_msg=f"n={n} m={m} mode={mode}")
        assert wrapped >= 16
        assert binding.wrap_flags() == (wrapped if mode == 3 else 0)
    finally:
        binding.wrap_mode(prev)
