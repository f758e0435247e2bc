"""Benchmark: PA input throughput (Mbps of key bits) of the G_{c,d} hash on GB300.

Workload (default): one privacy-amplification block of n = 10^8 key bits,
m = 2.5 * 10^7 output bits, uniform key and seeds from SplitMix64 (the
10^8-bit row of the paper's Table 2, hashed as Eq. 7 defines). A step is one
full hash: digit split, three length-2^24 NTTs, pointwise product, carry
resolve, + b, mod 2^n and extraction. Inputs rotate over several seeded
blocks whose total size exceeds the 129 MB L2, so no step reads another
step's inputs from L2.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0). Under torchrun each rank hashes its own blocks
(independent problems, no data-path collective): weak scaling.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1910_04429_gb300 import inputs  # noqa: E402

METRIC = "PA input throughput (Mbps of key bits) at n=1e8, m=2.5e7"
UNIT = "Mbps"
N_BITS = 100_000_000
M_BITS = 25_000_000
ROTATE = 4                      # distinct input blocks: 4 x 37.5 MB > L2
PAPER_I9_N1E8_MBPS = 140.96     # Table 2, i9-9900k, 100M-bit block (other hardware)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=500)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--n", type=int, default=N_BITS)
    p.add_argument("--m", type=int, default=M_BITS)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-profile", action="store_true")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons while timing."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def kernel_bytes(name: str, n: int, m: int, N: int) -> float:
    """Bytes a launch of this kernel must read and write (its own inputs and
    outputs; the transform's workspace words are 8 bytes)."""
    L = (n + 15) // 16
    Ly = (n + 63) // 64
    Mo = (m + 63) // 64
    w = 8
    return {
        "ntt_fwd_strided_first": 2 * L * 2 + 2 * N * w,       # digits of x, a in; both buffers out
        "ntt_fwd_strided_r64": 2 * (2 * N * w),               # both operands, read + write
        "ntt_contig_seed": 2 * N * w,
        "ntt_contig_fused": 3 * N * w,                        # x tile, a spectrum in; product out
        "ntt_inv_strided_r64": 2 * N * w,
        "ntt_inv_strided_last": N * w + L * w,                # only digits k < L written
        "carry_tiles": L * w + Ly * w,
        "carry_scan": 0,
        "carry_out": L * w + Ly * w + Mo * w,
    }.get(name, 0.0)


def run_ours(args, rank, world, local):
    import torch

    from paper_1910_04429_gb300 import binding

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    binding.load()
    n, m = args.n, args.m
    L = (n + 63) // 64
    Mo = (m + 63) // 64
    blocks = [inputs.make_block(n, m, seed=1 + rank * ROTATE + i) for i in range(ROTATE)]

    def to_dev(a):
        return torch.from_numpy(a.view(np.int64)).to(dev)

    dblocks = [(to_dev(b.x), to_dev(b.a), to_dev(b.b)) for b in blocks]
    outs = [torch.empty(Mo, dtype=torch.int64, device=dev) for _ in blocks]
    stream = torch.cuda.current_stream(dev)
    binding.prepare(n)

    def step(i):
        x, a, b = dblocks[i % ROTATE]
        binding.hash(x, a, b, n, m, out=outs[i % ROTATE], stream=stream)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for i in range(args.steps):
        step(i)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms_total = ev0.elapsed_time(ev1)
    clk = clocks.stop()

    # per-kernel CUDA events over the same K steps (separate, identical pass)
    kstats = {}
    if not args.no_profile:
        binding.profile(True)
        for i in range(args.steps):
            step(i)
        torch.cuda.synchronize()
        binding.profile(False)
        kstats = binding.profile_collect()

    # end to end through the C ABI with pinned host buffers
    hx = [torch.from_numpy(b.x.view(np.int64)).pin_memory() for b in blocks]
    ha = [torch.from_numpy(b.a.view(np.int64)).pin_memory() for b in blocks]
    hb = [torch.from_numpy(b.b.view(np.int64)).pin_memory() for b in blocks]
    hout = [torch.empty(Mo, dtype=torch.int64).pin_memory() for _ in blocks]
    import ctypes

    lib = binding.load()

    def e2e_step(i):
        j = i % ROTATE
        rc = lib.pa_hash_host(ctypes.c_void_p(hx[j].data_ptr()), ctypes.c_void_p(ha[j].data_ptr()),
                              ctypes.c_void_p(hb[j].data_ptr()), n, m,
                              ctypes.c_void_p(hout[j].data_ptr()), ctypes.c_void_p(stream.cuda_stream))
        if rc != 0:
            raise RuntimeError(f"pa_hash_host failed: {lib.pa_last_error().decode()}")

    e2e_steps = max(3, min(args.steps, 20))
    for i in range(2):
        e2e_step(i)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(e2e_steps):
        e2e_step(i)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / e2e_steps
    # the result read back must equal the device path's result (every rotating
    # block hashed once more by both paths, outside the timed regions)
    for j in range(ROTATE):
        step(j)
        e2e_step(j)
    torch.cuda.synchronize()
    ok = all(np.array_equal(hout[j].numpy(), outs[j].cpu().numpy()) for j in range(ROTATE))
    if not ok:
        raise RuntimeError("host-buffer results differ from device-buffer results")

    t = torch.tensor([ms_total, e2e_ms], dtype=torch.float64, device=dev)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_total, e2e_ms = float(t[0]), float(t[1])
    return dict(ms_total=ms_total, e2e_ms=e2e_ms, kstats=kstats, clocks=clk,
                h2d=3 * L * 8, d2h=Mo * 8)


def cpu_oracle_rate(n_sample: int, reps: int = 1):
    import oracle

    blk = inputs.make_block(n_sample, max(1, n_sample // 4), seed=1)
    th = oracle.default_threads()
    t0 = time.perf_counter()
    for _ in range(reps):
        oracle.pa_hash(blk.x, blk.a, blk.b, blk.n, blk.m, threads=th)
    dt = (time.perf_counter() - t0) / reps
    return n_sample / dt / 1e6, th, dt


def gmp_rate(n_sample: int):
    from oracle import gmp_ref

    if not gmp_ref.available():
        return None
    blk = inputs.make_block(n_sample, max(1, n_sample // 4), seed=1)
    t0 = time.perf_counter()
    gmp_ref.pa_hash(blk.x, blk.a, blk.b, blk.n, blk.m)
    dt = time.perf_counter() - t0
    return {"value": round(n_sample / dt / 1e6, 3), "unit": UNIT, "cores": 1,
            "kind": "gmp", "version": gmp_ref.version(),
            "sample": f"one block n={n_sample}, m={n_sample // 4}, mpz_import/addmul/fdiv_r_2exp/"
                      f"fdiv_q_2exp/export, single-threaded ({dt:.2f} s)"}


def main():
    args = parse()
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")

    if args.impl == "reference":
        if rank != 0:
            return 0
        # the oracle, as it stands, on the host cores: each step hashes one
        # 10^7-bit block (a tenth of the 10^8-bit workload; the oracle's cost
        # grows faster than linearly, so this favours the oracle)
        n_s = min(args.n, 10_000_000)
        rates = []
        for i in range(args.warmup + args.steps):
            r, th, dt = cpu_oracle_rate(n_s)
            if i >= args.warmup:
                rates.append(dt)
        total = sum(rates)
        value = args.steps * n_s / total / 1e6
        line = {"impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": UNIT,
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": round(1e3 * total / args.steps, 3), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
                "config": {"workload": f"G_cd hash, key n={args.n} bits, m={args.m}",
                           "sample": f"oracle on one block of n={n_s}, m={n_s // 4} per step"},
                "cpu_baseline": {"value": round(value, 3), "unit": UNIT, "cores": th,
                                 "kind": "oracle",
                                 "sample": f"one n={n_s}-bit block per step, {th} threads"},
                "e2e": {"value": round(value, 3), "unit": UNIT, "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0},
                "gpu_launches": 0}
        print(json.dumps(line), flush=True)
        return 0

    res = run_ours(args, rank, world, local)
    n, m = args.n, args.m
    K = args.steps
    ms_step = res["ms_total"] / K
    value = world * K * n / (res["ms_total"] / 1e3) / 1e6
    e2e_value = world * n / (res["e2e_ms"] / 1e3) / 1e6
    N = 1 << max(12, math.ceil(math.log2(2 * ((n + 15) // 16) - 1)))

    roofline = None
    launches = None
    if res["kstats"]:
        launches = sum(v[0] for v in res["kstats"].values())
        top = max(res["kstats"].items(), key=lambda kv: kv[1][1])
        name, (cnt, tot_ms) = top
        per_launch_ms = tot_ms / cnt
        peak, src = load_peaks()
        achieved = kernel_bytes(name, n, m, N) / (per_launch_ms / 1e3) / 1e9
        roofline = {"kernel": name, "bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                    "peak_source": src, "unit": "GB/s", "frac": round(achieved / peak, 4),
                    "traffic": None, "launch_ms": round(per_launch_ms, 4),
                    "share": round(tot_ms / sum(v[1] for v in res["kstats"].values()), 3)}

    line = {"metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
            "steps": K, "warmup": args.warmup, "ms_per_step": round(ms_step, 4),
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": round(value / PAPER_I9_N1E8_MBPS, 1),
            "baseline_ref": "paper Table 2, i9-9900k CPU, 100M-bit block: 140.96 Mbps (context)",
            "dtype": "u64", "data": "synthetic",
            "config": {"workload": f"G_cd hash, one key of n={n} bits, m={m} output bits per step",
                       "transform": f"Goldilocks NTT length {N}", "seeds": f"{ROTATE} rotating blocks",
                       "l2": f"inputs rotate over {ROTATE} blocks ({ROTATE * 3 * ((n + 63) // 64) * 8 / 1e6:.0f}"
                             f" MB) plus {2 * N * 8 / 1e6:.0f} MB workspace per step, > 129 MB L2",
                       "parallelism": f"replicas x{world}"},
            "e2e": {"value": round(e2e_value, 1), "unit": UNIT, "h2d_bytes_per_step": res["h2d"],
                    "d2h_bytes_per_step": res["d2h"]},
            "gpu_launches": launches,
            "kernels": {k: {"launches": v[0], "ms": round(v[1], 3)} for k, v in res["kstats"].items()},
            "roofline": roofline,
            "clocks": res["clocks"]}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        n_s = min(n, 100_000_000)
        r, th, dt = cpu_oracle_rate(n_s)
        line["cpu_baseline"] = {"value": round(r, 3), "unit": UNIT, "cores": th, "kind": "oracle",
                                "sample": f"one block n={n_s}, m={n_s // 4}, {th} threads, {dt:.1f} s"}
        g = gmp_rate(n_s)
        if g:
            line["gmp_baseline"] = g
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
