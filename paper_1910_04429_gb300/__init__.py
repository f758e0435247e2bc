"""GB300 (sm_103a) implementation of the G_{c,d} privacy-amplification hash of
arXiv 1910.04429: out = floor(((a*x + b) mod 2^n) / 2^(n-m)).

The compute path is the CUDA library ``libpa_gb300.so`` (C ABI in
``include/pa.h``); ``binding`` is its ctypes wrapper and ``inputs`` draws
seeded synthetic keys and seeds. Importing the package loads nothing: the
library is loaded on first use and every call fails loudly if it is missing.
"""

__all__ = ["binding", "inputs", "build"]
