"""The benchmark's reference arm (the oracle, timed on the host cores) on CPU:
one JSON line with the contract's keys, from rank 0 only under torchrun."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SMALL = ["--n-bits", "100000", "--m-bits", "25000", "--steps", "2", "--warmup", "1"]
KEYS = {"impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
        "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
        "cpu_baseline", "e2e", "gpu_launches"}


def _env():
    env = dict(os.environ)
    env.pop("RANK", None)
    env.pop("WORLD_SIZE", None)
    env.pop("LOCAL_RANK", None)
    return env


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _check_line(line, gpus):
    assert KEYS <= set(line), KEYS - set(line)
    assert line["impl"] == "reference"
    assert line["n_gpus"] == gpus and line["steps"] == 2 and line["warmup"] == 1
    assert line["value"] > 0 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"],
                           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    # value = steps * sample bits / total seconds, in the line's unit (Mbit/s)
    assert line["value"] == pytest.approx(100_000 / line["ms_per_step"] / 1e3, rel=1e-2)
    # the same workload (config) as the device arm's line, on the bench's own block size
    import bench

    assert line["config"] == bench.bench_config(100_000, 25_000, gpus)
    assert "n=100000, m=25000" in line["cpu_baseline"]["sample"]


def test_reference_arm_single_process():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", *SMALL], cwd=ROOT,
                         env=_env(), capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    _check_line(json.loads(lines[0]), 1)


def test_reference_arm_two_ranks_prints_once():
    """torchrun with two ranks (gloo): rank 0 prints the line, rank 1 exits 0
    without work."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py", "--gpus", "2",
           "--impl", "reference", *SMALL]
    out = subprocess.run(cmd, cwd=ROOT, env=_env(), capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    _check_line(json.loads(lines[0]), 2)
