"""Benchmark: Posit(32,2) Rgemm on GB300 through the C ABI.

Workload (default): C = A B, M = N = K = 8192, column-major Posit(32,2)
words drawn uniform in [-1, 1] (FP64, seeded) and rounded to posit on the
GPU; alpha = 1, beta = 0.  A step is one posit_rgemm call.  value = posit
Gflops (2 M N K posit multiplies and adds per call / time).

    python bench.py [--steps K] [--warmup W] [--gpus N] [--impl ours|reference]

Under torchrun each rank runs its own independent problem (weak scaling, no
collective); value = ops of all ranks / max time over ranks.

The line also carries:
  roofline      integer-issue roofline of the rgemm kernel: warp instructions
                issued per second (instructions per launch from ncu's
                smsp__inst_executed.sum, scaled per multiply-add) against
                SMs x 4 schedulers x max SM clock
  e2e           the same metric measured with host buffers: host->device copy
                of A and B, the call, device->host copy of C, every step
  cpu_baseline  the CPU oracle (plain C, OpenMP) on a bounded sample of the
                same workload (a few columns of C) on this host's cores
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Posit(32,2) Rgemm/Rgetrf Gflops vs INT-issue roofline; served-solve p50/p99"
UNIT = "Gflops"
ONE = 0x40000000

# Warp instructions the rgemm kernel issues per posit multiply-add:
# smsp__inst_executed.sum / (M N K) of one ncu capture of the current kernel
# (NN, 2048^3, uniform [-1,1]: 2.3357e10 / 8.590e9; profiles/rgemm_nn_ncu.md).
# The count is set by the inner loop, so it scales with M N K.
INST_PER_MAC = 2.7191
SM_COUNT = 152
SCHEDULERS_PER_SM = 4


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--size", type=int, default=8192, help="M = N = K")
    p.add_argument("--k", type=int, default=None, help="override K (e.g. 256)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=15.0)
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload_name(m, n, k):
    return f"rgemm_nn_{m}x{n}x{k}_uniform"


def config(m, n, k):
    return {"workload": workload_name(m, n, k), "m": m, "n": n, "k": k,
            "alpha": 1, "beta": 0, "layout": "column-major uint32 posit words",
            "inputs": "uniform [-1,1] fp64 (seeded) rounded to Posit(32,2)",
            "l2": "inputs larger than L2 (A, B 256 MiB each at 8192)"
            if 4 * m * k > 129e6 else "L2 flushed between steps"}


# ------------------------------------------------------------------ oracle
def oracle_sample_rate(m, n, k, seconds, seed=20240126):
    """The CPU oracle on whole columns of C (OpenMP parallelises over
    columns, so the sample is at least one column per thread), grown until
    one sample takes about `seconds`.  Returns (Gflops, threads, description)."""
    import numpy as np

    import oracle
    from paper_2401_14117_gb300 import inputs
    threads = oracle.get_threads()
    rng = np.random.default_rng(seed)
    A = oracle.from_double_array(inputs.uniform((m, k), seed))
    cols = min(n, threads)
    while True:
        B = oracle.from_double_array(rng.uniform(-1, 1, (k, cols)))
        C = np.zeros((m, cols), np.uint32)
        t0 = time.perf_counter()
        oracle.rgemm("N", "N", ONE, A, B, 0, C)
        dt = time.perf_counter() - t0
        if dt >= seconds * 0.4 or cols >= n:
            rate = 2 * m * cols * k / dt / 1e9
            return rate, threads, (
                f"{cols} whole columns of C ({m}x{cols}x{k}, {2 * m * cols * k:.3g} posit ops) "
                f"of the {m}x{n}x{k} product, {dt:.1f} s")
        grow = max(2.0, seconds * 0.6 / max(dt, 1e-3))
        cols = min(n, threads * max(1, int(round(cols * grow / threads))))


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    m = n = args.size
    k = args.k or args.size
    import numpy as np
    from paper_2401_14117_gb300 import inputs
    A = oracle.from_double_array(inputs.uniform((m, k), 1))
    cols = max(oracle.get_threads(), int(2e9 / (2 * m * k)))  # a few seconds of work per step
    B = oracle.from_double_array(inputs.uniform((k, cols), 2))
    C = np.zeros((m, cols), np.uint32)
    for _ in range(args.warmup):
        oracle.rgemm("N", "N", ONE, A, B, 0, C)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.rgemm("N", "N", ONE, A, B, 0, C)
    dt = time.perf_counter() - t0
    value = 2 * m * cols * k * args.steps / dt / 1e9
    sample = f"{cols} columns of C ({m}x{cols}x{k}) per step"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "posit32",
            "data": "synthetic", "config": config(m, n, k),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.get_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ ours
def run_ours(args):
    import numpy as np
    import torch

    from paper_2401_14117_gb300 import binding, inputs

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    m = n = args.size
    k = args.k or args.size
    seed = inputs.SEED_BASE + 1 + 1000 * rank
    stream = torch.cuda.current_stream()

    def dev_words(shape, s):
        x = torch.from_numpy(inputs.uniform(shape, s)).to(dev)
        w = torch.empty(shape, dtype=torch.int32, device=dev)
        binding.posit_from_double(x, w, x.numel(), stream)
        del x
        return w

    # column-major m x k == row-major (k, m) bytes
    dA = dev_words((k, m), seed)
    dB = dev_words((n, k), seed + 1)
    dC = torch.empty((n, m), dtype=torch.int32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.int8, device=dev)
    need_flush = 4 * m * k <= 129e6

    def step():
        if need_flush:
            flush.zero_()
        binding.posit_rgemm("N", "N", m, n, k, ONE, dA, m, dB, k, 0, dC, m, stream)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step()
    barrier()
    # kernel-only: events bracket each launch on the launching stream
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    total0 = torch.cuda.Event(enable_timing=True)
    total1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        total0.record(stream)
        for e0, e1 in evs:
            if need_flush:
                flush.zero_()
            e0.record(stream)
            binding.posit_rgemm("N", "N", m, n, k, ONE, dA, m, dB, k, 0, dC, m, stream)
            e1.record(stream)
        total1.record(stream)
        barrier()
    clocks = clk.summary()
    kernel_ms = [e0.elapsed_time(e1) for e0, e1 in evs]
    total_ms = total0.elapsed_time(total1)
    t_local = torch.tensor([total_ms], dtype=torch.float64, device=dev)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t_local, op=dist.ReduceOp.MAX)
    t_max_ms = float(t_local.item())
    ops = 2.0 * m * n * k
    value = ops * world * args.steps / (t_max_ms / 1e3) / 1e9
    launch_ms = statistics.mean(kernel_ms)

    # ---------------------------------------------------------- e2e
    e2e = None
    if not args.no_e2e:
        hA = torch.empty((k, m), dtype=torch.int32, pin_memory=True)
        hB = torch.empty((n, k), dtype=torch.int32, pin_memory=True)
        hC = torch.empty((n, m), dtype=torch.int32, pin_memory=True)
        hA.copy_(dA.cpu())
        hB.copy_(dB.cpu())
        eA = torch.empty_like(dA)
        eB = torch.empty_like(dB)
        eC = torch.empty_like(dC)

        def e2e_step():
            eA.copy_(hA, non_blocking=True)
            eB.copy_(hB, non_blocking=True)
            binding.posit_rgemm("N", "N", m, n, k, ONE, eA, m, eB, k, 0, eC, m, stream)
            hC.copy_(eC, non_blocking=True)

        e2e_step()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        barrier()
        t_e2e = torch.tensor([time.perf_counter() - t0], dtype=torch.float64, device=dev)
        if world > 1:
            import torch.distributed as dist
            dist.all_reduce(t_e2e, op=dist.ReduceOp.MAX)
        e2e = {"value": ops * world * args.steps / float(t_e2e.item()) / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": 4 * (m * k + k * n), "d2h_bytes_per_step": 4 * m * n}
        del eA, eB, eC

    # ---------------------------------------------------------- roofline
    peak_clock = clocks.get("sm_max_mhz") or 2070.0
    peak = SM_COUNT * SCHEDULERS_PER_SM * peak_clock * 1e6 / 1e9  # G warp-inst/s
    macs = m * n * k
    if INST_PER_MAC is not None:
        achieved = INST_PER_MAC * macs / (launch_ms / 1e3) / 1e9
        frac = achieved / peak
    else:
        achieved = frac = None
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gwarp-inst/s",
                "frac": frac, "traffic": None, "kernel": "rgemm_kernel<false,false,0>",
                "launch_ms": launch_ms, "inst_per_mac": INST_PER_MAC,
                "peak_basis": f"{SM_COUNT} SMs x {SCHEDULERS_PER_SM} schedulers x 1 warp-inst/clk x {peak_clock:.0f} MHz"}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "posit32", "data": "synthetic", "config": config(m, n, k),
            "e2e": e2e, "gpu_launches": args.steps, "clocks": clocks, "roofline": roofline}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, cores, sample = oracle_sample_rate(m, n, k, args.cpu_seconds)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores,
                                "kind": "oracle", "sample": sample}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
