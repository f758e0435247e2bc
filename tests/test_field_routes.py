"""The field helpers the kernels use (csrc/gl.cuh), compiled for the host with
g++ and checked against 128-bit arithmetic: every multiply-by-2^s route
(including the chains of multiplier-based routes the transforms take for
32 <= s < 64 and 96 < s < 160), sub, add and mul, on 0, 1, p - 1, p and random
values. The device variants (inline PTX) are covered by the GPU parity tests."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_field_routes_on_host(tmp_path):
    if not shutil.which("g++"):
        pytest.skip("g++ not available")
    exe = str(tmp_path / "field_routes")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_1910_04429_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "cpp", "field_routes.cpp"), "-o", exe])
    res = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert res.returncode == 0, res.stdout + res.stderr
    assert res.stdout.strip() == "ok"
