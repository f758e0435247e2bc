"""Thin ctypes binding of libpa_gb300.so (the C ABI of include/pa.h).

Argument marshalling only: every step of the hash runs in the library's CUDA
kernels. Device operands are torch CUDA tensors of dtype int64 (or uint64)
holding little-endian 64-bit limbs; host operands are numpy uint64 arrays.
There is no CPU fallback: if the library cannot be loaded every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

PA_OK, PA_EINVAL, PA_ENOMEM, PA_ECUDA, PA_EAGAIN, PA_ETIMEOUT = 0, -1, -2, -3, -4, -5
PA_MAX_BITS = 1 << 31
PA_FAULT_CARRY_WAIT = 1
PA_TOEPLITZ_MAX_BITS = 1 << 28

_lock = threading.Lock()
_lib = None

_SIGS = {
    "pa_hash": ([ctypes.c_void_p] * 3 + [ctypes.c_uint64] * 2 + [ctypes.c_void_p] * 2, ctypes.c_int),
    "pa_hash_noalloc": ([ctypes.c_void_p] * 3 + [ctypes.c_uint64] * 2 + [ctypes.c_void_p] * 2, ctypes.c_int),
    "pa_seed_create": ([ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)],
                       ctypes.c_int),
    "pa_hash_seeded": ([ctypes.c_void_p] * 3 + [ctypes.c_uint64] + [ctypes.c_void_p] * 2, ctypes.c_int),
    "pa_seed_destroy": ([ctypes.c_void_p], ctypes.c_int),
    "pa_toeplitz": ([ctypes.c_void_p] * 2 + [ctypes.c_uint64] * 2 + [ctypes.c_void_p] * 2, ctypes.c_int),
    "pa_toeplitz_workspace_bytes": ([ctypes.c_uint64] * 2, ctypes.c_uint64),
    "pa_toeplitz_seed_create": ([ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_void_p,
                                 ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
    "pa_toeplitz_seeded": ([ctypes.c_void_p] * 4, ctypes.c_int),
    "pa_toeplitz_autotune": ([ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, ctypes.POINTER(ctypes.c_int)],
                             ctypes.c_int),
    "pa_bits_to_limbs": ([ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                          ctypes.c_void_p], ctypes.c_int),
    "pa_limbs_to_bits": ([ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                          ctypes.c_void_p], ctypes.c_int),
    "pa_final_key_length": ([ctypes.c_double, ctypes.c_double, ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
    "pa_leftover_epsilon": ([ctypes.c_double, ctypes.c_uint64, ctypes.c_double, ctypes.POINTER(ctypes.c_double)],
                            ctypes.c_int),
    "pa_batch_create": ([ctypes.c_void_p, ctypes.c_uint32, ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
    "pa_batch_run": ([ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "pa_batch_destroy": ([ctypes.c_void_p], ctypes.c_int),
    "pa_autotune": ([ctypes.c_uint64, ctypes.c_int, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "pa_plan_override": ([ctypes.c_uint64, ctypes.c_int], ctypes.c_int),
    "pa_plan_override_length": ([ctypes.c_uint64, ctypes.c_int], ctypes.c_int),
    "pa_hash_host": ([ctypes.c_void_p] * 3 + [ctypes.c_uint64] * 2 + [ctypes.c_void_p] * 2, ctypes.c_int),
    "pa_hash_host_async": ([ctypes.c_void_p] * 3 + [ctypes.c_uint64] * 2 + [ctypes.c_void_p] * 2, ctypes.c_int),
    "pa_convolve16": ([ctypes.c_void_p] * 2 + [ctypes.c_uint64] + [ctypes.c_void_p] * 2, ctypes.c_int),
    "pa_carry_extract": ([ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_uint64,
                          ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "pa_hash_batched": ([ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p], ctypes.c_int),
    "pa_prepare": ([ctypes.c_uint64], ctypes.c_int),
    "pa_workspace_bytes": ([ctypes.c_uint64], ctypes.c_uint64),
    "pa_plan_info": ([ctypes.c_uint64, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
    "pa_wrap_mode": ([ctypes.c_int], ctypes.c_int),
    "pa_digit_width": ([ctypes.c_int], ctypes.c_int),
    "pa_batch_mode": ([ctypes.c_int], ctypes.c_int),
    "pa_plan_digits": ([ctypes.c_uint64, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint32)], ctypes.c_int),
    "pa_wrap_flags": ([ctypes.POINTER(ctypes.c_uint64), ctypes.c_int], ctypes.c_int),
    "pa_shutdown": ([], ctypes.c_int),
    "pa_profile": ([ctypes.c_int], ctypes.c_int),
    "pa_init": ([ctypes.c_int, ctypes.c_void_p], ctypes.c_int),
    "pa_stream_status": ([ctypes.c_void_p, ctypes.c_int], ctypes.c_int),
    "pa_submit": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
    "pa_poll": ([ctypes.c_uint64, ctypes.c_uint32, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "pa_serve_stats": ([ctypes.c_void_p], ctypes.c_int),
    "pa_serve_stop": ([], ctypes.c_int),
    "pa_profile_collect": ([ctypes.c_void_p, ctypes.c_int], ctypes.c_int),
    "pa_device_status": ([ctypes.c_int], ctypes.c_int),
    "pa_fault_inject": ([ctypes.c_int], ctypes.c_int),
    "pa_last_error": ([], ctypes.c_char_p),
    "pa_version": ([], ctypes.c_char_p),
}


class PaBlock(ctypes.Structure):
    """Mirror of ``pa_block`` in include/pa.h."""

    _fields_ = [("key", ctypes.c_void_p), ("seed_a", ctypes.c_void_p), ("seed_b", ctypes.c_void_p),
                ("n", ctypes.c_uint64), ("m", ctypes.c_uint64), ("out", ctypes.c_void_p)]


class PaKernelStat(ctypes.Structure):
    """Mirror of ``pa_kernel_stat`` in include/pa.h."""

    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_uint32), ("total_ms", ctypes.c_double)]


class PaConfig(ctypes.Structure):
    """Mirror of ``pa_config`` in include/pa.h."""

    _fields_ = [("max_batch", ctypes.c_uint32), ("streams", ctypes.c_uint32), ("max_pending", ctypes.c_uint32),
                ("idle_poll_us", ctypes.c_uint32), ("hbm_budget_bytes", ctypes.c_uint64)]


class PaServeStats(ctypes.Structure):
    """Mirror of ``pa_serve_stats_t`` in include/pa.h."""

    _fields_ = [("completed", ctypes.c_uint64), ("pending", ctypes.c_uint64), ("batches", ctypes.c_uint64),
                ("bits", ctypes.c_uint64), ("peak_inflight_bytes", ctypes.c_uint64),
                ("peak_inflight_blocks", ctypes.c_uint64), ("hbm_budget_bytes", ctypes.c_uint64),
                ("p50_us", ctypes.c_double), ("p99_us", ctypes.c_double), ("max_us", ctypes.c_double),
                ("mbps", ctypes.c_double)]


class PaError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{msg} (status {code})")
        self.code = code


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load the CUDA library (building it from csrc/ if it is absent or stale)."""
    global _lib
    lib = _lib
    if lib is not None:  # loaded: no lock on the per-call path
        return lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if build_if_missing:
                _build.build()
            if not os.path.exists(path):
                raise PaError(PA_ECUDA, f"CUDA library {path} is missing; run build()")
            lib = ctypes.CDLL(path)
            for name, (args, res) in _SIGS.items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = res
            _lib = lib
    return _lib


def _check(rc: int, what: str):
    if rc != PA_OK:
        raise PaError(rc, f"{what}: {load().pa_last_error().decode()}")


_LIMB_DTYPES = None  # (torch.int64, torch.uint64), set on first use


def _dev_ptr(t, limbs: int, name: str):
    global _LIMB_DTYPES
    if _LIMB_DTYPES is None:
        import torch

        _LIMB_DTYPES = (torch.int64, torch.uint64)
    try:
        cuda, dtype = t.is_cuda, t.dtype
    except AttributeError:
        raise TypeError(f"{name} must be a CUDA tensor") from None
    if not cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if dtype not in _LIMB_DTYPES or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous int64/uint64 tensor")
    if t.numel() < limbs:
        raise ValueError(f"{name} has {t.numel()} limbs, needs {limbs}")
    return t.data_ptr()  # a plain int: the c_void_p argtype converts it


def _stream_ptr(stream):
    if stream is None:
        import torch

        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def limbs(bits: int) -> int:
    return (bits + 63) // 64


limbs_for = limbs


def hash(key, seed_a, seed_b, n: int, m: int, out=None, stream=None):
    """out = floor(((seed_a*key + seed_b) mod 2^n) / 2^(n-m)) on the GPU (asynchronous)."""
    import torch

    L = limbs(n)
    if out is None:
        out = torch.empty(limbs(m), dtype=torch.int64, device=key.device)
    args = [_dev_ptr(key, L, "key"), _dev_ptr(seed_a, L, "seed_a"), _dev_ptr(seed_b, L, "seed_b")]
    _check(load().pa_hash(*args, n, m, _dev_ptr(out, limbs(m), "out"), _stream_ptr(stream)), "pa_hash")
    return out


def hash_noalloc(key, seed_a, seed_b, n: int, m: int, out=None, stream=None):
    """pa_hash_noalloc: the hash using only the library's fixed device scratch
    (n <= 2^20 bits), for callers that cannot allocate device memory."""
    import torch

    L = limbs(n)
    if out is None:
        out = torch.empty(limbs(m), dtype=torch.int64, device=key.device)
    args = [_dev_ptr(key, L, "key"), _dev_ptr(seed_a, L, "seed_a"), _dev_ptr(seed_b, L, "seed_b")]
    _check(load().pa_hash_noalloc(*args, n, m, _dev_ptr(out, limbs(m), "out"), _stream_ptr(stream)),
           "pa_hash_noalloc")
    return out


class Seed:
    """A seed whose transform is computed once (pa_seed_create); hash keys of
    the same length against it with ``hash``. Free with ``close``."""

    def __init__(self, seed_a, n: int, stream=None):
        h = ctypes.c_void_p(0)
        _check(load().pa_seed_create(_dev_ptr(seed_a, limbs(n), "seed_a"), n, _stream_ptr(stream),
                                     ctypes.byref(h)), "pa_seed_create")
        self.handle, self.n = h, n

    def hash(self, key, seed_b, m: int, out=None, stream=None):
        import torch

        if out is None:
            out = torch.empty(limbs(m), dtype=torch.int64, device=key.device)
        _check(load().pa_hash_seeded(self.handle, _dev_ptr(key, limbs(self.n), "key"),
                                     _dev_ptr(seed_b, limbs(self.n), "seed_b"), m,
                                     _dev_ptr(out, limbs(m), "out"), _stream_ptr(stream)), "pa_hash_seeded")
        return out

    def close(self):
        if self.handle:
            _check(load().pa_seed_destroy(self.handle), "pa_seed_destroy")
            self.handle = None


def toeplitz(key, seed, n: int, m: int, out=None, stream=None):
    """Toeplitz hash y = T key over GF(2), T[i][j] = seed[i - j + n - 1] (m x n,
    seed of n + m - 1 bits), on the GPU (asynchronous)."""
    import torch

    if out is None:
        out = torch.empty(limbs(m), dtype=torch.int64, device=key.device)
    _check(load().pa_toeplitz(_dev_ptr(key, limbs(n), "key"), _dev_ptr(seed, limbs(n + m - 1), "seed"),
                              n, m, _dev_ptr(out, limbs(m), "out"), _stream_ptr(stream)), "pa_toeplitz")
    return out


def toeplitz_autotune(n: int, m: int, reps: int = 5) -> int:
    """Tune the plan of the transform length pa_toeplitz(n, m) uses; returns the variant."""
    v = ctypes.c_int(0)
    _check(load().pa_toeplitz_autotune(n, m, reps, ctypes.byref(v)), "pa_toeplitz_autotune")
    return int(v.value)


def toeplitz_workspace_bytes(n: int, m: int) -> int:
    return int(load().pa_toeplitz_workspace_bytes(n, m))


class ToeplitzSeed:
    """A Toeplitz seed transformed once (pa_toeplitz_seed_create); hash keys of
    n bits to m bits against it with ``hash``. Free with ``close``."""

    def __init__(self, seed, n: int, m: int, stream=None):
        h = ctypes.c_void_p(0)
        _check(load().pa_toeplitz_seed_create(_dev_ptr(seed, limbs(n + m - 1), "seed"), n, m,
                                              _stream_ptr(stream), ctypes.byref(h)), "pa_toeplitz_seed_create")
        self.handle, self.n, self.m = h, n, m

    def hash(self, key, out=None, stream=None):
        import torch

        if out is None:
            out = torch.empty(limbs(self.m), dtype=torch.int64, device=key.device)
        _check(load().pa_toeplitz_seeded(self.handle, _dev_ptr(key, limbs(self.n), "key"),
                                         _dev_ptr(out, limbs(self.m), "out"), _stream_ptr(stream)),
               "pa_toeplitz_seeded")
        return out

    def close(self):
        if self.handle:
            _check(load().pa_seed_destroy(self.handle), "pa_seed_destroy")
            self.handle = None


def _host_ptr(v, count: int, name: str):
    """Address of a host buffer: a contiguous uint64 numpy array, or a CPU
    int64/uint64 torch tensor (e.g. pinned)."""
    if isinstance(v, np.ndarray):
        if v.dtype != np.uint64 or not v.flags.c_contiguous or v.size < count:
            raise ValueError(f"{name} must be a contiguous uint64 array of >= {count} limbs")
        return ctypes.c_void_p(v.ctypes.data)
    import torch

    if not isinstance(v, torch.Tensor) or v.is_cuda or v.dtype not in (torch.int64, torch.uint64) \
            or not v.is_contiguous() or v.numel() < count:
        raise ValueError(f"{name} must be a contiguous host uint64 array or int64 tensor of >= {count} limbs")
    return ctypes.c_void_p(v.data_ptr())


def hash_host(key, seed_a, seed_b, n: int, m: int, out=None, stream=None):
    """pa_hash_host: host arrays in, host array out (synchronous)."""
    L = limbs(n)
    arrs = [_host_ptr(v, L, nm) for nm, v in (("key", key), ("seed_a", seed_a), ("seed_b", seed_b))]
    if out is None:
        out = np.zeros(limbs(m), dtype=np.uint64)
    st = ctypes.c_void_p(0) if stream is None else _stream_ptr(stream)
    _check(load().pa_hash_host(*arrs, n, m, _host_ptr(out, limbs(m), "out"), st), "pa_hash_host")
    return out


def hash_host_async(key, seed_a, seed_b, n: int, m: int, out, stream=None):
    """pa_hash_host_async: queued host-buffer hash (pinned buffers overlap with
    earlier calls); ``out`` is valid once ``stream`` has passed the call."""
    L = limbs(n)
    arrs = [_host_ptr(v, L, nm) for nm, v in (("key", key), ("seed_a", seed_a), ("seed_b", seed_b))]
    st = ctypes.c_void_p(0) if stream is None else _stream_ptr(stream)
    _check(load().pa_hash_host_async(*arrs, n, m, _host_ptr(out, limbs(m), "out"), st), "pa_hash_host_async")
    return out


def convolve16(key, seed_a, n: int, coef=None, stream=None):
    """Digit product coef[k] = sum_{i+j=k} x_i a_j, k < ceil(n/16) (no carry)."""
    import torch

    L16 = (n + 15) // 16
    if coef is None:
        coef = torch.empty(L16, dtype=torch.int64, device=key.device)
    _check(load().pa_convolve16(_dev_ptr(key, limbs(n), "key"), _dev_ptr(seed_a, limbs(n), "seed_a"),
                                n, _dev_ptr(coef, L16, "coef"), _stream_ptr(stream)), "pa_convolve16")
    return coef


def carry_extract(coef, seed_b, n: int, m: int, out=None, stream=None):
    import torch

    if out is None:
        out = torch.empty(limbs(m), dtype=torch.int64, device=seed_b.device)
    L = coef.numel()
    _check(load().pa_carry_extract(_dev_ptr(coef, L, "coef"), L, _dev_ptr(seed_b, limbs(n), "seed_b"),
                                   n, m, _dev_ptr(out, limbs(m), "out"), _stream_ptr(stream)),
           "pa_carry_extract")
    return out


def hash_batched(blocks, stream=None):
    """blocks: sequence of (key, seed_a, seed_b, n, m, out) with CUDA tensors."""
    arr = (PaBlock * len(blocks))()
    for i, (k, a, b, n, m, o) in enumerate(blocks):
        L = limbs(n)
        arr[i] = PaBlock(_dev_ptr(k, L, "key"), _dev_ptr(a, L, "seed_a"),
                         _dev_ptr(b, L, "seed_b"), n, m, _dev_ptr(o, limbs(m), "out"))
    _check(load().pa_hash_batched(arr, len(blocks), _stream_ptr(stream)), "pa_hash_batched")


def serve_init(device: int = -1, max_batch: int = 0, streams: int = 0, max_pending: int = 0,
               hbm_budget_bytes: int = 0, idle_poll_us: int = 0):
    """pa_init(device, cfg): start the serving loop (device -1: the current one)."""
    cfg = PaConfig(max_batch, streams, max_pending, idle_poll_us, hbm_budget_bytes)
    _check(load().pa_init(device, ctypes.byref(cfg)), "pa_init")


def submit(key, seed_a, seed_b, n: int, m: int, out) -> int:
    """Queue one block (CUDA tensors that must stay alive until it completes)."""
    L = limbs(n)
    blk = PaBlock(_dev_ptr(key, L, "key"), _dev_ptr(seed_a, L, "seed_a"),
                  _dev_ptr(seed_b, L, "seed_b"), n, m, _dev_ptr(out, limbs(m), "out"))
    t = ctypes.c_uint64(0)
    rc = load().pa_submit(ctypes.byref(blk), ctypes.byref(t))
    if rc != PA_OK:
        raise PaError(rc, f"pa_submit: {load().pa_last_error().decode()}")
    return int(t.value)


def poll(ticket: int, timeout_us: int = 0):
    """(rc, status): rc PA_OK when done (status = hashing status), PA_EAGAIN if not yet."""
    st = ctypes.c_int(0)
    rc = load().pa_poll(ticket, timeout_us, ctypes.byref(st))
    return rc, st.value


def serve_stats() -> dict:
    s = PaServeStats()
    _check(load().pa_serve_stats(ctypes.byref(s)), "pa_serve_stats")
    return {name: getattr(s, name) for name, _ in PaServeStats._fields_}


def serve_stop():
    _check(load().pa_serve_stop(), "pa_serve_stop")


def bits_to_limbs(bits, nbits: int, msb_string: bool, msb_bytes: bool, limbs=None, stream=None):
    """Packed bit string (CUDA uint8 tensor) -> little-endian limbs (CUDA int64 tensor)."""
    import torch

    if limbs is None:
        limbs = torch.empty(limbs_for(nbits), dtype=torch.int64, device=bits.device)
    _check(load().pa_bits_to_limbs(ctypes.c_void_p(bits.data_ptr()), nbits, int(msb_string), int(msb_bytes),
                                   _dev_ptr(limbs, limbs_for(nbits), "limbs"), _stream_ptr(stream)),
           "pa_bits_to_limbs")
    return limbs


def limbs_to_bits(limbs, nbits: int, msb_string: bool, msb_bytes: bool, bits=None, stream=None):
    """Little-endian limbs (CUDA int64 tensor) -> packed bit string (CUDA uint8 tensor)."""
    import torch

    if bits is None:
        bits = torch.empty((nbits + 7) // 8, dtype=torch.uint8, device=limbs.device)
    _check(load().pa_limbs_to_bits(_dev_ptr(limbs, limbs_for(nbits), "limbs"), nbits, int(msb_string),
                                   int(msb_bytes), ctypes.c_void_p(bits.data_ptr()), _stream_ptr(stream)),
           "pa_limbs_to_bits")
    return bits


def final_key_length(hmin_bits: float, eps: float) -> int:
    """Eq. 1: largest r <= hmin - 2 log2(1/eps)."""
    r = ctypes.c_uint64(0)
    _check(load().pa_final_key_length(hmin_bits, eps, ctypes.byref(r)), "pa_final_key_length")
    return int(r.value)


def leftover_epsilon(hmin_bits: float, r: int, eps: float) -> float:
    """Definition 2: 1/2 * 2^(-(hmin - r)/2) + eps."""
    v = ctypes.c_double(0)
    _check(load().pa_leftover_epsilon(hmin_bits, r, eps, ctypes.byref(v)), "pa_leftover_epsilon")
    return float(v.value)


class Batch:
    """A fixed set of blocks captured into a CUDA graph (pa_batch_create);
    ``run`` replays it. The tensors must stay alive until ``close``."""

    def __init__(self, blocks):
        arr = (PaBlock * len(blocks))()
        for i, (k, a, b, n, m, o) in enumerate(blocks):
            L = limbs(n)
            arr[i] = PaBlock(_dev_ptr(k, L, "key"), _dev_ptr(a, L, "seed_a"),
                             _dev_ptr(b, L, "seed_b"), n, m, _dev_ptr(o, limbs(m), "out"))
        h = ctypes.c_void_p(0)
        _check(load().pa_batch_create(arr, len(blocks), ctypes.byref(h)), "pa_batch_create")
        self.handle = h
        self._keep = blocks

    def run(self, stream=None):
        _check(load().pa_batch_run(self.handle, _stream_ptr(stream)), "pa_batch_run")

    def close(self):
        if self.handle:
            _check(load().pa_batch_destroy(self.handle), "pa_batch_destroy")
            self.handle = None


def autotune(n: int, reps: int = 5) -> int:
    """Time the plan variants for keys of n bits and keep the fastest; returns it."""
    v = ctypes.c_int(0)
    _check(load().pa_autotune(n, reps, ctypes.byref(v)), "pa_autotune")
    return int(v.value)


# plan variant bits (include/pa.h PA_PLAN_*); variants are 0 .. PLAN_VARIANTS - 1
PLAN_R0_LAST, PLAN_DIRECT_FWD, PLAN_DIRECT_INV, PLAN_NARROW, PLAN_BULK, PLAN_CLUSTER = 1, 2, 4, 8, 16, 32
PLAN_VARIANTS = 64


def plan_override(n: int, variant: int):
    """Force a plan variant for the transform length of n (-1 clears)."""
    _check(load().pa_plan_override(n, variant), "pa_plan_override")


def plan_override_length(N: int, variant: int):
    """Force a plan variant for the transform length N itself (-1 clears)."""
    _check(load().pa_plan_override_length(N, variant), "pa_plan_override_length")


def prepare(n: int):
    _check(load().pa_prepare(n), "pa_prepare")


def workspace_bytes(n: int) -> int:
    return int(load().pa_workspace_bytes(n))


def plan_info(n: int, m: int) -> dict:
    """Transform lengths of a hash of n bits with m output bits (host only):
    {"first": length run first, "full": the full-length product's, "dropped":
    low coefficients the wrapped product drops (0: not wrapped)}."""
    info = (ctypes.c_uint64 * 3)()
    _check(load().pa_plan_info(n, m, info), "pa_plan_info")
    return {"first": int(info[0]), "full": int(info[1]), "dropped": int(info[2])}


def wrap_mode(mode: int) -> int:
    """1: wrapped products where shorter (default); 0: always full length;
    2: wrapped with the check forced to fail (tests). Returns the previous mode."""
    rc = load().pa_wrap_mode(mode)
    if rc < 0:
        _check(rc, "pa_wrap_mode")
    return int(rc)


def digit_width(width: int) -> int:
    """0: each hash takes the exact digit width whose product is shortest
    (default); 16 .. 20: that width where exact. Returns the previous setting."""
    rc = load().pa_digit_width(width)
    if rc < 0:
        _check(rc, "pa_digit_width")
    return int(rc)


def batch_mode(mode: int) -> int:
    """1: batched transforms in one persistent kernel where the plan allows;
    0: by size class; 2 (default): persistent for small batches, else by size
    class. Returns the previous mode."""
    rc = load().pa_batch_mode(mode)
    if rc < 0:
        _check(rc, "pa_batch_mode")
    return int(rc)


def plan_digits(n: int, m: int) -> int:
    """The digit width a hash of n bits with m output bits uses (host only)."""
    w = ctypes.c_uint32(0)
    _check(load().pa_plan_digits(n, m, ctypes.byref(w)), "pa_plan_digits")
    return int(w.value)


def wrap_flags(clear: bool = False) -> int:
    """Failed wrapped-product checks (each ran the full-length product) since the last clear."""
    v = ctypes.c_uint64(0)
    _check(load().pa_wrap_flags(ctypes.byref(v), 1 if clear else 0), "pa_wrap_flags")
    return int(v.value)


def profile(on: bool):
    _check(load().pa_profile(1 if on else 0), "pa_profile")


def profile_collect() -> dict:
    """{kernel name: (launches, total_ms)} recorded since pa_profile(1)."""
    cap = 64
    arr = (PaKernelStat * cap)()
    n = load().pa_profile_collect(ctypes.cast(arr, ctypes.c_void_p), cap)
    if n < 0:
        _check(n, "pa_profile_collect")
    return {arr[i].name.decode(): (int(arr[i].launches), float(arr[i].total_ms)) for i in range(n)}


def device_status(clear: bool = False) -> int:
    """PA_OK, or PA_ETIMEOUT if a bounded device wait ran out since the last clear."""
    return int(load().pa_device_status(1 if clear else 0))


def stream_status(stream=None, clear: bool = False) -> int:
    """pa_stream_status: PA_OK, or PA_ETIMEOUT if a bounded wait of the library's
    kernels ran out on this stream (waits for that stream only)."""
    return int(load().pa_stream_status(_stream_ptr(stream), 1 if clear else 0))


def fault_inject(what: int = PA_FAULT_CARRY_WAIT):
    _check(load().pa_fault_inject(what), "pa_fault_inject")


def version() -> str:
    return load().pa_version().decode()


def raw():
    """The loaded ctypes library (for status-code tests)."""
    return load()
