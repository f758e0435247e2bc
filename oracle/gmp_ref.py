"""GMP-based G_{c,d} hash, the paper's own CPU pipeline (Sec. 3.2).

TEST INFRASTRUCTURE / CPU BASELINE ONLY. Used by the tests as an independent
arbitrary-precision cross-check of the oracle, and by the benchmark as the
"GMP multiply-based hash" CPU baseline. It is loaded only where a shared
``libgmp`` exists on the host; callers must handle ``available() == False``.

The steps follow Sec. 3.2 in order: data import of the limb arrays
(``mpz_import``, least significant word first, Sec. 3.2.1), y = d + c*x with one
multiply-add (``mpz_addmul``, Sec. 3.2.2), reduction mod 2^n by bit masking
(Sec. 3.2.3 names it ``mpz_mod_2exp``; the documented GMP routine for a
non-negative operand is ``mpz_fdiv_r_2exp``), data export (``mpz_export``,
Sec. 3.2.4), keeping the top m bits of the n-bit field (Sec. 3.2.5) by a
right shift of n - m (``mpz_fdiv_q_2exp``). Prototypes are written from the
GMP manual; the library is called through its exported ``__gmpz_*`` names.
"""
from __future__ import annotations

import ctypes
import ctypes.util
import os

import numpy as np


class _Mpz(ctypes.Structure):
    _fields_ = [("alloc", ctypes.c_int), ("size", ctypes.c_int), ("d", ctypes.c_void_p)]


_gmp = None
_tried = False


def _candidates():
    found = ctypes.util.find_library("gmp")
    if found:
        yield found
    yield "libgmp.so.10"
    yield "libgmp.so"


def _load():
    global _gmp, _tried
    if _tried:
        return _gmp
    _tried = True
    for name in _candidates():
        try:
            lib = ctypes.CDLL(name)
        except OSError:
            continue
        P = ctypes.POINTER(_Mpz)
        sz = ctypes.c_size_t
        lib.__gmpz_init.argtypes = [P]
        lib.__gmpz_clear.argtypes = [P]
        lib.__gmpz_import.argtypes = [P, sz, ctypes.c_int, sz, ctypes.c_int, sz, ctypes.c_void_p]
        lib.__gmpz_export.argtypes = [ctypes.c_void_p, ctypes.POINTER(sz), ctypes.c_int, sz,
                                      ctypes.c_int, sz, P]
        lib.__gmpz_export.restype = ctypes.c_void_p
        lib.__gmpz_set.argtypes = [P, P]
        lib.__gmpz_addmul.argtypes = [P, P, P]
        lib.__gmpz_fdiv_r_2exp.argtypes = [P, P, ctypes.c_ulong]
        lib.__gmpz_fdiv_q_2exp.argtypes = [P, P, ctypes.c_ulong]
        _gmp = lib
        break
    return _gmp


def available() -> bool:
    return _load() is not None


def version() -> str | None:
    lib = _load()
    if lib is None:
        return None
    try:
        return ctypes.c_char_p.in_dll(lib, "__gmp_version").value.decode()
    except (ValueError, AttributeError):
        return "unknown"


def pa_hash(x, a, b, n: int, m: int) -> np.ndarray:
    """floor(((a*x + b) mod 2^n) / 2^(n-m)) computed with GMP (single-threaded)."""
    lib = _load()
    if lib is None:
        raise RuntimeError("libgmp is not available on this host")
    if n <= 0 or m <= 0 or m > n:
        raise ValueError(f"invalid sizes n={n} m={m}")
    L = (n + 63) // 64
    M = (m + 63) // 64
    arrs = [np.ascontiguousarray(v[:L], dtype=np.uint64).copy() for v in (x, a, b)]
    if n % 64:
        for v in arrs:
            v[-1] &= np.uint64((1 << (n % 64)) - 1)
    zx, za, zy = _Mpz(), _Mpz(), _Mpz()
    for z in (zx, za, zy):
        lib.__gmpz_init(ctypes.byref(z))
    try:
        lib.__gmpz_import(ctypes.byref(zx), L, -1, 8, 0, 0, arrs[0].ctypes.data)
        lib.__gmpz_import(ctypes.byref(za), L, -1, 8, 0, 0, arrs[1].ctypes.data)
        lib.__gmpz_import(ctypes.byref(zy), L, -1, 8, 0, 0, arrs[2].ctypes.data)
        lib.__gmpz_addmul(ctypes.byref(zy), ctypes.byref(za), ctypes.byref(zx))
        lib.__gmpz_fdiv_r_2exp(ctypes.byref(zy), ctypes.byref(zy), n)
        lib.__gmpz_fdiv_q_2exp(ctypes.byref(zy), ctypes.byref(zy), n - m)
        out = np.zeros(M + 1, dtype=np.uint64)
        cnt = ctypes.c_size_t(0)
        lib.__gmpz_export(ctypes.c_void_p(out.ctypes.data), ctypes.byref(cnt), -1, 8, 0, 0,
                          ctypes.byref(zy))
        if cnt.value > M:
            raise RuntimeError("GMP result longer than m bits")
        return out[:M].copy()
    finally:
        for z in (zx, za, zy):
            lib.__gmpz_clear(ctypes.byref(z))


def host_cores() -> int:
    return os.cpu_count() or 1
