"""Final-key length (Eq. 1), the leftover-hash bound (Definition 2) and the
bit-string conventions: oracle pins and the library's host helpers (no GPU)."""
import math
import random

import numpy as np
import pytest

import oracle
from paper_1910_04429_gb300 import binding


@pytest.mark.parametrize("hmin,k", [(1000, 10), (10**8, 40), (123.75, 3), (5000.5, 1)])
def test_final_key_length_closed_form(hmin, k):
    # eps = 2^-k makes log2(1/eps) exact: r = floor(hmin - 2k)
    assert oracle.final_key_length(hmin, 2.0 ** -k) == math.floor(hmin - 2 * k)
    assert binding.final_key_length(hmin, 2.0 ** -k) == math.floor(hmin - 2 * k)


def test_final_key_length_matches_oracle_random():
    rng = random.Random(1)
    for _ in range(500):
        h = rng.uniform(100, 1e9)
        eps = 10 ** rng.uniform(-30, -1)
        assert binding.final_key_length(h, eps) == oracle.final_key_length(h, eps)


def test_leftover_bound_at_eq1_length():
    """With r from Eq. 1 at eps = 2^-k, Definition 2 gives eps_bar = eps/2 + eps'."""
    for k in (5, 20, 60):
        h = 1000.0 + 2 * k
        r = binding.final_key_length(h, 2.0 ** -k)
        for e2 in (0.0, 1e-12):
            want = 0.5 * 2.0 ** -k + e2
            assert oracle.leftover_epsilon(h, r, e2) == want
            assert binding.leftover_epsilon(h, r, e2) == want


def test_helper_argument_checks():
    for h, eps in ((100, 0.0), (100, 1.0), (100, -1e-3), (10, 1e-9), (float("nan"), 0.5)):
        with pytest.raises(binding.PaError):
            binding.final_key_length(h, eps)
    with pytest.raises(ValueError):
        oracle.final_key_length(10, 1e-9)


def test_bit_conventions_small_cases():
    # "1011" packed msb-first in one byte: 0b1011_0000
    data = bytes([0b10110000])
    assert oracle.bits_to_int(data, 4, msb_string=True, msb_bytes=True) == 0b1011
    assert oracle.bits_to_int(data, 4, msb_string=False, msb_bytes=True) == 0b1101
    # lsb-first packing of the same reading order: byte 0b0000_1101
    assert oracle.bits_to_int(bytes([0b00001101]), 4, msb_string=True, msb_bytes=False) == 0b1011
    # lsb-first string and lsb-first packing = plain little-endian bytes
    v = 0x1234_5678_9ABC_DEF0_0FED
    raw = v.to_bytes(10, "little")
    assert oracle.bits_to_int(raw, 80, False, False) == v


@pytest.mark.parametrize("nbits", [1, 7, 8, 9, 63, 64, 65, 1000, 4097])
def test_bit_round_trip(nbits):
    rng = random.Random(nbits)
    for ms in (False, True):
        for mb in (False, True):
            v = rng.getrandbits(nbits)
            data = oracle.int_to_bits(v, nbits, ms, mb)
            assert len(data) == (nbits + 7) // 8
            assert oracle.bits_to_int(data, nbits, ms, mb) == v


def test_adapter_argument_checks():
    import ctypes

    lib = binding.raw()
    z = np.zeros(16, dtype=np.uint64)
    p = ctypes.c_void_p(z.ctypes.data)
    null = ctypes.c_void_p(0)
    assert lib.pa_bits_to_limbs(null, 8, 0, 0, p, null) == binding.PA_EINVAL
    assert lib.pa_bits_to_limbs(p, 0, 0, 0, p, null) == binding.PA_EINVAL
    assert lib.pa_bits_to_limbs(p, 8, 2, 0, p, null) == binding.PA_EINVAL
    assert lib.pa_limbs_to_bits(p, 8, 0, 3, p, null) == binding.PA_EINVAL
    assert lib.pa_limbs_to_bits(p, 8, 0, 0, null, null) == binding.PA_EINVAL
