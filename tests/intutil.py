"""Python-int helpers for the tests: limb arrays <-> arbitrary-precision ints.

Python's built-in integers are an arbitrary-precision implementation that is
independent of both the C oracle and the CUDA path.
"""
import numpy as np


def to_int(limbs) -> int:
    return int.from_bytes(np.ascontiguousarray(limbs, dtype="<u8").tobytes(), "little")


def from_int(v: int, k: int) -> np.ndarray:
    if v < 0:
        raise ValueError("negative")
    return np.frombuffer(v.to_bytes(8 * k, "little"), dtype="<u8").astype(np.uint64)


def hash_int(x: int, a: int, b: int, n: int, m: int) -> int:
    """The definition of Eq. 7 in Python ints (operands reduced into Z_{2^n})."""
    mask = (1 << n) - 1
    return (((a & mask) * (x & mask) + (b & mask)) & mask) >> (n - m)
