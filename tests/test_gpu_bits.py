"""Bit-string adapters on the GPU against the oracle's conventions, and the
whole pipeline from a reconciled bit string to the final-key bit string."""
import random

import numpy as np
import pytest

import oracle
from paper_1910_04429_gb300 import binding, inputs
from tests.gpu_util import dev, host
from tests.intutil import to_int

pytestmark = pytest.mark.gpu


def _u8(data: bytes):
    import torch

    return torch.frombuffer(bytearray(data), dtype=torch.uint8).cuda()


@pytest.mark.parametrize("nbits", [1, 7, 8, 63, 64, 65, 1000, 1_000_003])
def test_import_export_match_oracle(nbits):
    import torch

    rng = random.Random(nbits)
    for ms in (False, True):
        for mb in (False, True):
            data = bytes(rng.getrandbits(8) for _ in range((nbits + 7) // 8))
            limbs = binding.bits_to_limbs(_u8(data), nbits, ms, mb)
            torch.cuda.synchronize()
            v = oracle.bits_to_int(data, nbits, ms, mb)
            assert to_int(host(limbs)) == v
            back = binding.limbs_to_bits(limbs, nbits, ms, mb)
            torch.cuda.synchronize()
            assert bytes(back.cpu().numpy()) == oracle.int_to_bits(v, nbits, ms, mb)


def test_bit_string_pipeline():
    """MSB-first reconciled string X -> limbs -> hash -> MSB-first final key Y."""
    import torch

    n, m = 1_000_003, 250_001
    rng = random.Random(5)
    xs = bytes(rng.getrandbits(8) for _ in range((n + 7) // 8))
    blk = inputs.make_block(n, m, seed=5)
    xl = binding.bits_to_limbs(_u8(xs), n, True, True)
    y = binding.hash(xl, dev(blk.a), dev(blk.b), n, m)
    ys = binding.limbs_to_bits(y, m, True, True)
    torch.cuda.synchronize()
    x = oracle.bits_to_int(xs, n, True, True)
    L = (n + 63) // 64
    from tests.intutil import from_int
    want = oracle.pa_hash(from_int(x, L), blk.a, blk.b, n, m)
    assert bytes(ys.cpu().numpy()) == oracle.int_to_bits(to_int(want), m, True, True)
