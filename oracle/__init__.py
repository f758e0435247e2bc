"""CPU oracle for the G_{c,d} privacy-amplification hash (arXiv 1910.04429).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers. The product path (the CUDA
library and its Python binding) never imports this package, and this package
never imports the product path.

The oracle computes the plain definition of the hash (Sec. 2.3, Definition 5,
Eq. 6 and Eq. 7):  out = floor(((a*x + b) mod 2^n) / 2^(n-m)),  with plain
schoolbook/Karatsuba limb arithmetic in ``pa_oracle.c``. Arrays are numpy
``uint64`` little-endian limb vectors (bit i of the integer is bit i%64 of limb
i//64), the least-significant-word-first import of Sec. 3.2.1.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pa_oracle.c")
_SRC_TOE = os.path.join(_HERE, "toeplitz.c")
_LIB = os.path.join(_HERE, "libpa_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``pa_oracle.c`` and ``toeplitz.c`` into ``libpa_oracle.so`` next
    to them (plain gcc)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_SRC_TOE))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-o", tmp, _SRC, _SRC_TOE]
        )
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            u64p = ctypes.POINTER(ctypes.c_uint64)
            for name in ("pa_oracle_mul_full", "pa_oracle_mul_low"):
                f = getattr(lib, name)
                f.argtypes = [u64p, u64p, ctypes.c_uint64, u64p, ctypes.c_int]
                f.restype = ctypes.c_int
            f = lib.pa_oracle_hash
            f.argtypes = [u64p, u64p, u64p, ctypes.c_uint64, ctypes.c_uint64, u64p, ctypes.c_int]
            f.restype = ctypes.c_int
            f = lib.pa_oracle_toeplitz
            f.argtypes = [u64p, u64p, ctypes.c_uint64, ctypes.c_uint64, u64p, ctypes.c_int]
            f.restype = ctypes.c_int
            f = lib.pa_oracle_toeplitz_bit
            f.argtypes = [u64p, u64p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
            f.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(arr: np.ndarray):
    return arr.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def _limbs(arr, k: int) -> np.ndarray:
    a = np.ascontiguousarray(arr, dtype=np.uint64)
    if a.ndim != 1 or a.size < k:
        raise ValueError(f"expected a 1-D uint64 array of at least {k} limbs, got shape {a.shape}")
    return a


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def pa_hash(x, a, b, n: int, m: int, threads: int = 1) -> np.ndarray:
    """floor(((a*x + b) mod 2^n) / 2^(n-m)) as ceil(m/64) uint64 limbs (Eq. 7)."""
    if n <= 0 or m <= 0 or m > n:
        raise ValueError(f"invalid sizes n={n} m={m}")
    L = (n + 63) // 64
    xs, as_, bs = _limbs(x, L), _limbs(a, L), _limbs(b, L)
    out = np.zeros((m + 63) // 64, dtype=np.uint64)
    rc = _load().pa_oracle_hash(_ptr(xs), _ptr(as_), _ptr(bs), n, m, _ptr(out), int(threads))
    if rc != 0:
        raise RuntimeError(f"pa_oracle_hash failed with {rc}")
    return out


def mul_full(a, b, threads: int = 1) -> np.ndarray:
    """Full product of two k-limb integers, 2k limbs."""
    a = np.ascontiguousarray(a, dtype=np.uint64)
    b = np.ascontiguousarray(b, dtype=np.uint64)
    if a.shape != b.shape or a.ndim != 1:
        raise ValueError("operands must be 1-D and of equal length")
    out = np.zeros(2 * a.size, dtype=np.uint64)
    rc = _load().pa_oracle_mul_full(_ptr(a), _ptr(b), a.size, _ptr(out), int(threads))
    if rc != 0:
        raise RuntimeError(f"pa_oracle_mul_full failed with {rc}")
    return out


def mul_low(a, b, threads: int = 1) -> np.ndarray:
    """Low k limbs of the product of two k-limb integers."""
    a = np.ascontiguousarray(a, dtype=np.uint64)
    b = np.ascontiguousarray(b, dtype=np.uint64)
    if a.shape != b.shape or a.ndim != 1:
        raise ValueError("operands must be 1-D and of equal length")
    out = np.zeros(a.size, dtype=np.uint64)
    rc = _load().pa_oracle_mul_low(_ptr(a), _ptr(b), a.size, _ptr(out), int(threads))
    if rc != 0:
        raise RuntimeError(f"pa_oracle_mul_low failed with {rc}")
    return out


def toeplitz(x, s, n: int, m: int, threads: int = 1) -> np.ndarray:
    """Toeplitz hash y = T x over GF(2), T[i][j] = s[i - j + n - 1] (m x n, seed of
    n + m - 1 bits), as ceil(m/64) uint64 limbs (the family surveyed in Sec. 1)."""
    if n <= 0 or m <= 0 or m > n:
        raise ValueError(f"invalid sizes n={n} m={m}")
    xs = _limbs(x, (n + 63) // 64)
    ss = _limbs(s, (n + m - 1 + 63) // 64)
    out = np.zeros((m + 63) // 64, dtype=np.uint64)
    rc = _load().pa_oracle_toeplitz(_ptr(xs), _ptr(ss), n, m, _ptr(out), int(threads))
    if rc != 0:
        raise RuntimeError(f"pa_oracle_toeplitz failed with {rc}")
    return out


def toeplitz_bit(x, s, n: int, m: int, i: int) -> int:
    """Output bit i of the Toeplitz hash (row i of T against x), O(n)."""
    xs = _limbs(x, (n + 63) // 64)
    ss = _limbs(s, (n + m - 1 + 63) // 64)
    r = _load().pa_oracle_toeplitz_bit(_ptr(xs), _ptr(ss), n, m, i)
    if r < 0:
        raise ValueError(f"invalid arguments n={n} m={m} i={i}")
    return r


def raw_hash_rc(n: int, m: int) -> int:
    """Return code of the C entry point for sizes (n, m) on dummy operands
    (lets tests check the argument validation without a Python pre-check)."""
    L = max(1, (n + 63) // 64)
    z = np.zeros(L, dtype=np.uint64)
    out = np.zeros(max(1, (m + 63) // 64), dtype=np.uint64)
    return _load().pa_oracle_hash(_ptr(z), _ptr(z), _ptr(z), n, m, _ptr(out), 1)


# ---------------------------------------------------------------------------
# Final-key length and bit strings (plain definitions)
# ---------------------------------------------------------------------------

def final_key_length(hmin_bits: float, eps: float) -> int:
    """Eq. 1 (Sec. 2.2): the largest integer r <= H_min^{eps/2} - 2 log2(1/eps)."""
    import math

    if not (0.0 < eps < 1.0):
        raise ValueError("eps must be in (0, 1)")
    r = math.floor(hmin_bits - 2.0 * math.log2(1.0 / eps))
    if r < 1:
        raise ValueError("no positive key length")
    return r


def leftover_epsilon(hmin_bits: float, r: int, eps: float) -> float:
    """Definition 2 (quantum leftover hash lemma): 1/2 * 2^(-(H_min^eps - r)/2) + eps."""
    return 0.5 * 2.0 ** (-0.5 * (hmin_bits - r)) + eps


def bits_to_int(data: bytes, nbits: int, msb_string: bool, msb_bytes: bool) -> int:
    """The integer a packed bit string denotes: string bit i is bit i % 8 (or
    7 - i % 8 with msb_bytes) of byte i // 8; it weighs 2^i, or 2^(nbits-1-i)
    with msb_string."""
    bits = np.unpackbits(np.frombuffer(bytes(data), dtype=np.uint8),
                         bitorder="big" if msb_bytes else "little")[:nbits]
    if msb_string:
        bits = bits[::-1]
    packed = np.packbits(bits, bitorder="little").tobytes()
    return int.from_bytes(packed, "little")


def int_to_bits(value: int, nbits: int, msb_string: bool, msb_bytes: bool) -> bytes:
    """Inverse of bits_to_int for 0 <= value < 2^nbits (padding bits zero)."""
    raw = value.to_bytes((nbits + 7) // 8, "little")
    bits = np.unpackbits(np.frombuffer(raw, dtype=np.uint8), bitorder="little")[:nbits]
    if msb_string:
        bits = bits[::-1]
    return np.packbits(bits, bitorder="big" if msb_bytes else "little").tobytes()
