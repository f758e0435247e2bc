"""The C-ABI library builds, loads and exports every symbol include/pa.h declares.

No compute calls here (no GPU needed): only symbol presence, constants, the
host-side size arithmetic and the argument checks that return before any
CUDA call.
"""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1910_04429_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_text():
    with open(os.path.join(ROOT, "include", "pa.h")) as f:
        return f.read()


def _declared_functions():
    text = re.sub(r"/\*.*?\*/", "", _header_text(), flags=re.S)
    return sorted(set(re.findall(r"\b(pa_[a-z0-9_]+)\s*\(", text)))


def _exported_symbols(path):
    """Dynamic symbols of the library, read from its ELF .dynsym table."""
    import struct

    with open(path, "rb") as f:
        data = f.read()
    assert data[:4] == b"\x7fELF" and data[4] == 2, "expected a 64-bit ELF"
    shoff, = struct.unpack_from("<Q", data, 0x28)
    shentsize, shnum, _ = struct.unpack_from("<HHH", data, 0x3A)
    secs = [struct.unpack_from("<IIQQQQIIQQ", data, shoff + i * shentsize) for i in range(shnum)]
    names = set()
    for s in secs:
        if s[1] == 11:  # SHT_DYNSYM
            strtab = secs[s[6]]
            for off in range(s[4], s[4] + s[5], s[9]):
                st_name, st_info, _, st_shndx = struct.unpack_from("<IBBH", data, off)
                if st_shndx == 0:  # undefined: imported, not exported
                    continue
                end = data.index(b"\0", strtab[4] + st_name)
                names.add(data[strtab[4] + st_name:end].decode())
    return names


def test_library_builds_and_loads():
    lib = binding.load()
    assert os.path.exists(binding.library_path())
    assert lib.pa_version().decode().startswith("pa_gb300")


def test_every_declared_symbol_is_exported():
    declared = _declared_functions()
    assert "pa_hash" in declared and "pa_hash_batched" in declared
    binding.load()
    exported = _exported_symbols(binding.library_path())
    missing = [s for s in declared if s not in exported]
    assert not missing, f"declared in include/pa.h but not exported: {missing}"
    lib = ctypes.CDLL(binding.library_path())
    for s in declared:
        assert getattr(lib, s) is not None


def test_status_constants_match_header():
    text = _header_text()
    for name in ("PA_OK", "PA_EINVAL", "PA_ENOMEM", "PA_ECUDA", "PA_EAGAIN", "PA_ETIMEOUT"):
        m = re.search(rf"#define {name} \(?(-?\d+)\)?", text)
        assert m, name
        assert int(m.group(1)) == getattr(binding, name)


def test_plan_bits_match_header():
    """The binding's plan-variant bits are the header's PA_PLAN_* values, and
    the variants are exactly the combinations of those bits."""
    text = _header_text()
    bits = {}
    for name in ("R0_LAST", "DIRECT_FWD", "DIRECT_INV", "NARROW", "BULK", "CLUSTER"):
        m = re.search(rf"#define PA_PLAN_{name} (\d+)", text)
        assert m, name
        bits[name] = int(m.group(1))
        assert bits[name] == getattr(binding, "PLAN_" + name)
    assert sorted(bits.values()) == [1 << i for i in range(len(bits))]
    assert binding.PLAN_VARIANTS == 1 << len(bits)
    # the last variant passes the argument check (without a GPU the call then
    # fails on the device; with one it sets an override, cleared again)
    lib = binding.raw()
    rc = lib.pa_plan_override(1000, binding.PLAN_VARIANTS - 1)
    assert rc != binding.PA_EINVAL or b"variant" not in lib.pa_last_error()
    lib.pa_plan_override(1000, -1)


def test_argument_checks_without_gpu():
    lib = binding.raw()
    z = np.zeros(4, dtype=np.uint64)
    p = ctypes.c_void_p(z.ctypes.data)
    null = ctypes.c_void_p(0)
    # sizes: n = 0, m = 0, m > n, n beyond the cap
    for n, m in ((0, 1), (10, 0), (10, 11), (binding.PA_MAX_BITS + 64, 1)):
        assert lib.pa_hash(p, p, p, n, m, p, null) == binding.PA_EINVAL
        assert lib.pa_hash_host(p, p, p, n, m, p, null) == binding.PA_EINVAL
        assert lib.pa_hash_host_async(p, p, p, n, m, p, null) == binding.PA_EINVAL
        assert lib.pa_carry_extract(p, 1, p, n, m, p, null) == binding.PA_EINVAL
    # null pointers
    assert lib.pa_hash(null, p, p, 10, 5, p, null) == binding.PA_EINVAL
    assert lib.pa_hash(p, p, p, 10, 5, null, null) == binding.PA_EINVAL
    assert lib.pa_convolve16(p, p, 0, p, null) == binding.PA_EINVAL
    assert lib.pa_convolve16(p, null, 10, p, null) == binding.PA_EINVAL
    assert b"null" in lib.pa_last_error()
    # batched: one bad block rejects the whole call before any work
    blocks = (binding.PaBlock * 2)()
    blocks[0] = binding.PaBlock(z.ctypes.data, z.ctypes.data, z.ctypes.data, 100, 10, z.ctypes.data)
    blocks[1] = binding.PaBlock(z.ctypes.data, z.ctypes.data, z.ctypes.data, 100, 101, z.ctypes.data)
    assert lib.pa_hash_batched(blocks, 2, null) == binding.PA_EINVAL
    assert b"block 1" in lib.pa_last_error()
    # an empty batch is a no-op (no device touched); a null array with blocks is refused
    assert lib.pa_hash_batched(None, 0, null) == binding.PA_OK
    assert lib.pa_hash_batched(None, 3, null) == binding.PA_EINVAL
    hb = ctypes.c_void_p(0)
    assert lib.pa_batch_create(blocks, 0, ctypes.byref(hb)) == binding.PA_EINVAL
    assert lib.pa_batch_create(blocks, 2, None) == binding.PA_EINVAL
    assert lib.pa_prepare(0) == binding.PA_EINVAL
    assert lib.pa_fault_inject(99) == binding.PA_EINVAL
    assert lib.pa_plan_override(0, 0) == binding.PA_EINVAL
    assert lib.pa_plan_override(1000, binding.PLAN_VARIANTS) == binding.PA_EINVAL
    assert lib.pa_plan_override_length(4096, binding.PLAN_VARIANTS) == binding.PA_EINVAL
    assert lib.pa_plan_override_length(4097, 0) == binding.PA_EINVAL  # not a transform length
    assert lib.pa_autotune(0, 1, None) == binding.PA_EINVAL
    h = ctypes.c_void_p(0)
    assert lib.pa_seed_create(null, 100, null, ctypes.byref(h)) == binding.PA_EINVAL
    assert lib.pa_seed_create(p, 0, null, ctypes.byref(h)) == binding.PA_EINVAL
    assert lib.pa_hash_seeded(null, p, p, 10, p, null) == binding.PA_EINVAL
    assert lib.pa_seed_destroy(null) == binding.PA_OK
    # Toeplitz: 1 <= m <= n, n + m - 1 <= PA_TOEPLITZ_MAX_BITS, non-null pointers
    cap = binding.PA_TOEPLITZ_MAX_BITS
    for n, m in ((0, 1), (10, 0), (10, 11), (cap, 2), (cap + 1, 1)):
        assert lib.pa_toeplitz(p, p, n, m, p, null) == binding.PA_EINVAL
        assert lib.pa_toeplitz_seed_create(p, n, m, null, ctypes.byref(h)) == binding.PA_EINVAL
        assert lib.pa_toeplitz_workspace_bytes(n, m) == 0
    assert lib.pa_toeplitz(p, null, 10, 5, p, null) == binding.PA_EINVAL
    assert lib.pa_toeplitz(p, p, 10, 5, null, null) == binding.PA_EINVAL
    assert lib.pa_toeplitz_seed_create(null, 10, 5, null, ctypes.byref(h)) == binding.PA_EINVAL
    assert lib.pa_toeplitz_seeded(null, p, p, null) == binding.PA_EINVAL
    assert lib.pa_toeplitz_autotune(10, 11, 1, None) == binding.PA_EINVAL
    # the fixed-scratch entry point refuses keys beyond its scratch size
    assert lib.pa_hash_noalloc(p, p, p, (1 << 20) + 1, 1, p, null) == binding.PA_EINVAL
    assert b"PA_NOALLOC_MAX_BITS" in lib.pa_last_error()
    assert lib.pa_hash_noalloc(p, p, p, 10, 11, p, null) == binding.PA_EINVAL
    # serving: bad requests are refused before the loop (or CUDA) is touched
    t = ctypes.c_uint64(0)
    bad = binding.PaBlock(z.ctypes.data, z.ctypes.data, z.ctypes.data, 100, 0, z.ctypes.data)
    assert lib.pa_submit(ctypes.byref(bad), ctypes.byref(t)) == binding.PA_EINVAL
    nul = binding.PaBlock(0, z.ctypes.data, z.ctypes.data, 100, 10, z.ctypes.data)
    assert lib.pa_submit(ctypes.byref(nul), ctypes.byref(t)) == binding.PA_EINVAL
    st = ctypes.c_int(0)
    assert lib.pa_poll(12345, 0, ctypes.byref(st)) == binding.PA_EINVAL
    assert b"unknown ticket" in lib.pa_last_error()


@pytest.mark.parametrize("n,N", [(1, 4096), (32768, 4096), (32769, 8192), (96_000, 1 << 14),
                                 (1_000_000, 1 << 17), (1_536_000, 1 << 18),
                                 (100_000_000, 1 << 24), (1_000_000_000, 1 << 27)])
def test_workspace_bytes(n, N):
    """Two transform buffers of N words, N = the smallest power of two >=
    max(4096, 2 ceil(n/16) - 1): the exact recomputation behind a wrapped
    product runs at that length, which covers the full-length product (2^k or
    3 * 2^k) too; and two carry-state sets (tile states, ticket, flag)."""
    tiles = -(-(-(-n // 64)) // 256)
    assert binding.workspace_bytes(n) == 2 * N * 8 + 2 * 4 * (tiles + 2)
    assert binding.workspace_bytes(0) == 0


@pytest.mark.parametrize("n,m,N", [(1, 1, 4096), (2048, 2049 - 2048, 4096), (3000, 1097, 4096),
                                   (3000, 1098, 8192), (1_000_000, 250_000, 5 << 18),
                                   (1_000_000, 320_000, 3 << 19), (100_000_000, 25_000_000, 1 << 27)])
def test_toeplitz_workspace_bytes(n, m, N):
    """Toeplitz transform length: smallest 2^k, 3 * 2^k (first radix <= 48) or
    5 * 2^k (first radix <= 40) that is >= max(4096, n + m - 1); two N-word
    buffers."""
    assert binding.toeplitz_workspace_bytes(n, m) == 2 * N * 8
