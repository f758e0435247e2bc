"""Write the stored oracle digests used by the full-size GPU parity tests.

Only the oracle (``oracle/``) and the seeded input generator are called here.
The 10^9-bit block takes the oracle minutes even on many host cores, so the
GPU test compares against the SHA-256 of the oracle's output stored by this
script instead of re-running the oracle.

Usage:  python tests/golden/make_golden.py [n ...]
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1910_04429_gb300 import inputs  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def golden_path(n: int, m: int, seed: int) -> str:
    return os.path.join(HERE, f"oracle_digest_n{n}_m{m}_seed{seed}.json")


def make(n: int, m: int, seed: int = 1) -> str:
    blk = inputs.make_block(n, m, seed)
    t0 = time.time()
    out = oracle.pa_hash(blk.x, blk.a, blk.b, n, m, threads=oracle.default_threads())
    dt = time.time() - t0
    rec = {
        "what": "SHA-256 of the oracle output limbs (little-endian uint64) for the seeded block",
        "generator": "paper_1910_04429_gb300.inputs.make_block(n, m, seed)",
        "n": n, "m": m, "seed": seed,
        "out_limbs": int(out.size),
        "sha256": hashlib.sha256(out.astype("<u8").tobytes()).hexdigest(),
        "first_limbs": [f"{int(v):016x}" for v in out[:4]],
        "last_limbs": [f"{int(v):016x}" for v in out[-4:]],
        "oracle_seconds": round(dt, 1),
        "oracle_threads": oracle.default_threads(),
    }
    path = golden_path(n, m, seed)
    with open(path, "w") as f:
        json.dump(rec, f, indent=1)
        f.write("\n")
    return path


if __name__ == "__main__":
    sizes = [int(v) for v in sys.argv[1:]] or [1_000_000_000]
    for n in sizes:
        print(make(n, n // 4), flush=True)
