"""The C ABI from plain C: tests/c_client.c (only include/pa.h and the library)
is compiled with gcc, run, and its output compared with the oracle's."""
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_1910_04429_gb300 import binding, inputs

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def client(tmp_path_factory):
    lib = binding.library_path()
    assert os.path.exists(lib), "build the library first"
    exe = str(tmp_path_factory.mktemp("c_client") / "c_client")
    libdir = os.path.dirname(lib)
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-I", os.path.join(ROOT, "include"),
                           os.path.join(ROOT, "tests", "c_client.c"), "-o", exe, "-L", libdir,
                           "-lpa_gb300", f"-Wl,-rpath,{libdir}"])
    return exe


@pytest.mark.parametrize("n,m,seed", [(1, 1, 3), (1000, 333, 5), (1_000_003, 250_001, 1),
                                      (10_000_000, 2_500_000, 9)])
def test_c_client_matches_oracle(client, n, m, seed):
    res = subprocess.run([client, str(n), str(m), str(seed)], capture_output=True, text=True, timeout=300)
    assert res.returncode == 0, res.stderr
    got = np.array([int(v, 16) for v in res.stdout.split()], dtype=np.uint64)
    blk = inputs.make_block(n, m, seed=seed)  # the same SplitMix64 draw as the C client
    np.testing.assert_array_equal(got, oracle.pa_hash(blk.x, blk.a, blk.b, n, m, threads=oracle.default_threads()))
