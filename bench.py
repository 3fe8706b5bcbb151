"""Benchmark: Posit(32,2) Rgemm on GB300 through the C ABI.

Workload (default): C = A B, M = N = K = 8192, column-major Posit(32,2)
words drawn uniform in [-1, 1] (FP64, seeded) and rounded to posit on the
GPU; alpha = 1, beta = 0.  A step is one posit_rgemm call.  value = posit
Gflops (2 M N K posit multiplies and adds per call / time).

    python bench.py [--steps K] [--warmup W] [--gpus N] [--impl ours|reference]

Under torchrun each rank runs its own independent problem (weak scaling, no
collective); value = ops of all ranks / max time over ranks.

The line also carries:
  roofline      integer-ALU-pipe roofline of the rgemm kernel: ALU-pipe warp
                instructions per second (per multiply-add from ncu's
                sm__inst_executed_pipe_alu.sum, times M N K, over the launch
                time) against SMs x 4 schedulers x 0.5 x max SM clock; the
                issue-slot figures ride along; traffic = DRAM bytes of one
                8192^3 launch from an ncu capture
  e2e           the same metric measured with host buffers: host->device copy
                of A and B, the call, device->host copy of C, every step (the
                copies on a second stream, overlapping the previous step's
                product; the copy rate alone is reported beside it)
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

# Per posit multiply-add of the rgemm kernel, from one ncu capture of one
# 4096^3 launch of the current kernel (NN, uniform [-1,1]; the counts are set
# by the inner loop, so they scale with M N K): integer-ALU-pipe warp
# instructions (sm__inst_executed_pipe_alu.sum / M N K), all warp
# instructions (smsp__inst_executed.sum / M N K) and FMA-heavy-pipe ones.
ALU_INST_PER_MAC = 1.06493  # 7.31809e10 / 6.87195e10 (NN 4096^3)
INST_PER_MAC = 2.00693      # 1.37914e11 / 6.87195e10
FMA_INST_PER_MAC = 0.80698  # sm__inst_executed_pipe_fmaheavy.sum: 5.54547e10 / 6.87195e10
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one captured
# 8192^3 launch (one-pass capture of the full-size workload).
TRAFFIC_8192 = 4.972963e9 + 0.419838e9
# The counters above belong to one build of the kernel: the SHA-256 (first 16
# hex digits) of the two source files that define it when they were taken.
# If the sources differ, the line says "counters_stale": true, its traffic is
# null, and the achieved figures are estimates from the old counts.
COUNTERS_SOURCES = ("paper_2401_14117_gb300/csrc/rgemm.cu",
                    "paper_2401_14117_gb300/csrc/posit_core.cuh")
COUNTERS_SOURCE_SHA = "118032ce3e53eee9"
# The kernel is bound by the integer ALU pipe: 0.5 warp instruction per clock
# per scheduler, measured by the issue probe (python bench.py --probe under
# ncu): LOP3 chains alone, all on the ALU pipe, run at 0.4993.
ALU_WARP_INST_PER_CLK = 0.5
SM_COUNT = 152
SCHEDULERS_PER_SM = 4


def kernel_source_sha() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in COUNTERS_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--probe", action="store_true",
                   help="run the dependency-free issue probe instead of the benchmark")
    p.add_argument("--size", type=int, default=8192, help="M = N = K")
    p.add_argument("--k", type=int, default=None, help="override K (e.g. 256)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=15.0)
    p.add_argument("--no-extras", action="store_true",
                   help="skip the other workloads (LU/Cholesky/solves, batched, serving)")
    p.add_argument("--serve-seconds", type=float, default=10.0)
    p.add_argument("--serve-rate-sustained", type=float, default=60.0,
                   help="arrival rate (requests/s) of the sustainable serving run")
    p.add_argument("--batch-count", type=int, default=4096,
                   help="problems in the batched section")
    p.add_argument("--batch-plan", default="",
                   help="threads,ctas_per_sm,smem_bytes for the batched section (default: autotuned)")
    p.add_argument("--serve-pool", type=int, default=96,
                   help="seeded problems in the serving pool")
    p.add_argument("--serve-rates", default="40,80,120,160,200,240,320,480",
                   help="arrival rates of the serving_sweep section")
    p.add_argument("--serve-slo-ms", type=float, default=250.0,
                   help="p99 latency objective of the serving_sweep section")
    p.add_argument("--extras", default="all",
                   help="comma list of extra workloads: elementwise, rgemm, ksweep, sigma, "
                        "factor, power, accuracy, batched, serving; or all (serving_sweep, "
                        "the arrival-rate sweep, only when named)")
    p.add_argument("--ew-size", type=int, default=1 << 24,
                   help="elements per element-wise launch")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_seed(rank):
    """Each rank multiplies its own seeded matrices (independent problems)."""
    from paper_2401_14117_gb300 import inputs
    return inputs.SEED_BASE + 1 + 1000 * rank


def max_over_ranks(x, world, device):
    """The largest x over all ranks (x itself on one rank)."""
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_gflops(ops_per_rank_step, world, steps, t_max_ms):
    """Whole-job rate: the work of every rank over the slowest rank's time."""
    return ops_per_rank_step * world * steps / (t_max_ms / 1e3) / 1e9


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


def oracle_one_thread_rate(m, k, seed=20240127):
    """The CPU oracle on one thread: one whole column of C (m x 1 x k)."""
    import numpy as np

    import oracle
    from paper_2401_14117_gb300 import inputs
    threads = oracle.get_threads()
    A = oracle.from_double_array(inputs.uniform((m, k), seed))
    B = oracle.from_double_array(np.random.default_rng(seed).uniform(-1, 1, (k, 1)))
    C = np.zeros((m, 1), np.uint32)
    oracle.set_threads(1)
    try:
        t0 = time.perf_counter()
        oracle.rgemm("N", "N", ONE, A, B, 0, C)
        dt = time.perf_counter() - t0
    finally:
        oracle.set_threads(threads)
    return 2 * m * k / dt / 1e9


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
        sm, mx, pw, reasons = [], [], [], set()
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
            try:
                pw.append(float(f[2]))
            except ValueError:
                pass
            for nm, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0,
                    "power_w": None}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w": statistics.median(pw) if pw else None}


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
    seed = rank_seed(rank)
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
    t_max_ms = max_over_ranks(total_ms, world, dev)
    ops = 2.0 * m * n * k
    value = job_gflops(ops, world, args.steps, t_max_ms)
    launch_ms = statistics.mean(kernel_ms)

    # ---------------------------------------------------------- e2e
    e2e = None
    if not args.no_e2e:
        hA = torch.empty((k, m), dtype=torch.int32, pin_memory=True)
        hB = torch.empty((n, k), dtype=torch.int32, pin_memory=True)
        hC = torch.empty((n, m), dtype=torch.int32, pin_memory=True)
        hA.copy_(dA.cpu())
        hB.copy_(dB.cpu())
        # Two device buffer sets and a copy stream: step i+1's inputs travel
        # while step i computes, and step i's result returns meanwhile; every
        # step still copies its inputs from pinned host memory and its result
        # back, inside the timed region.
        sets = [(torch.empty_like(dA), torch.empty_like(dB), torch.empty_like(dC))
                for _ in range(2)]
        cstream = torch.cuda.Stream(device=dev)
        in_ready = [torch.cuda.Event() for _ in range(2)]
        computed = [torch.cuda.Event() for _ in range(2)]
        freed = [torch.cuda.Event() for _ in range(2)]
        for e in freed:
            e.record(cstream)

        def e2e_step(i):
            eA, eB, eC = sets[i % 2]
            with torch.cuda.stream(cstream):
                cstream.wait_event(freed[i % 2])  # step i-2 computed and read back
                eA.copy_(hA, non_blocking=True)
                eB.copy_(hB, non_blocking=True)
                in_ready[i % 2].record(cstream)
            stream.wait_event(in_ready[i % 2])
            binding.posit_rgemm("N", "N", m, n, k, ONE, eA, m, eB, k, 0, eC, m, stream)
            computed[i % 2].record(stream)
            with torch.cuda.stream(cstream):
                cstream.wait_event(computed[i % 2])
                hC.copy_(eC, non_blocking=True)
                freed[i % 2].record(cstream)

        e2e_step(0)
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        for i in range(args.steps):
            e2e_step(i)
        torch.cuda.synchronize()
        barrier()
        t_e2e_ms = max_over_ranks((time.perf_counter() - t0) * 1e3, world, dev)
        # the copies alone, for the record: one step's bytes each way
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        eA, eB, eC = sets[0]
        c0.record(stream)
        eA.copy_(hA, non_blocking=True)
        eB.copy_(hB, non_blocking=True)
        hC.copy_(eC, non_blocking=True)
        c1.record(stream)
        torch.cuda.synchronize()
        copy_ms = c0.elapsed_time(c1)
        copy_bytes = 4 * (m * k + k * n + m * n)
        e2e = {"value": job_gflops(ops, world, args.steps, t_e2e_ms), "unit": UNIT,
               "h2d_bytes_per_step": 4 * (m * k + k * n), "d2h_bytes_per_step": 4 * m * n,
               "copies": "on a second stream, overlapping the previous step's product "
                         "(two device buffer sets)",
               "copy_ms_per_step_alone": copy_ms,
               "copy_gb_per_s_alone": copy_bytes / (copy_ms / 1e3) / 1e9}
        del sets

    # ---------------------------------------------------------- roofline
    peak_clock = clocks.get("sm_max_mhz") or 2070.0
    macs = m * n * k
    launch_s = launch_ms / 1e3
    # bound: the integer ALU pipe (G warp instructions per second)
    peak = SM_COUNT * SCHEDULERS_PER_SM * ALU_WARP_INST_PER_CLK * peak_clock * 1e6 / 1e9
    achieved = ALU_INST_PER_MAC * macs / launch_s / 1e9
    # issue slots, for context: 1 warp instruction per clock per scheduler
    issue_peak = SM_COUNT * SCHEDULERS_PER_SM * peak_clock * 1e6 / 1e9
    issue = INST_PER_MAC * macs / launch_s / 1e9
    stale = kernel_source_sha() != COUNTERS_SOURCE_SHA
    traffic = TRAFFIC_8192 if (m, n, k) == (8192, 8192, 8192) and not stale else None
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak,
                "unit": "G ALU-pipe warp-inst/s", "frac": achieved / peak,
                "counters_stale": stale, "counters_source_sha": COUNTERS_SOURCE_SHA,
                # 32 threads per warp instruction, 2 posit ops per multiply-add
                "thread_inst_per_posit_op": INST_PER_MAC * 32 / 2,
                "traffic": traffic, "traffic_unit": "bytes per launch",
                "algorithmic_bytes": 4.0 * (m * k + k * n + m * n),
                "kernel": "rgemm_kernel<false,false,0,4>", "launch_ms": launch_ms,
                "alu_inst_per_mac": ALU_INST_PER_MAC, "inst_per_mac": INST_PER_MAC,
                "fma_inst_per_mac": FMA_INST_PER_MAC,
                "peak_basis": (f"{SM_COUNT} SMs x {SCHEDULERS_PER_SM} schedulers x "
                               f"{ALU_WARP_INST_PER_CLK} ALU-pipe warp-inst/clk x {peak_clock:.0f} MHz"),
                "issue": {"achieved": issue, "peak": issue_peak, "frac": issue / issue_peak,
                          "unit": "G warp-inst/s"}}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "posit32", "data": "synthetic", "config": config(m, n, k),
            "e2e": e2e, "gpu_launches": args.steps, "clocks": clocks, "roofline": roofline}
    if rank == 0 and world == 1 and not args.no_extras:
        args.square_ms = launch_ms if m == n == k == 8192 else None
        line["extras"] = extras(args, dev, stream)
        line["extras"]["headline_power_w"] = clocks.get("power_w")
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, cores, sample = oracle_sample_rate(m, n, k, args.cpu_seconds)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores,
                                "kind": "oracle", "sample": sample,
                                "one_thread_value": oracle_one_thread_rate(m, k)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ------------------------------------------------------------------ probe
# A dependency-free issue probe: eight independent chains per thread of one
# instruction kind, no memory traffic in the loop.  It measures the ceilings
# the Rgemm roofline is quoted against: LOP3 only (the integer ALU pipe),
# IMAD only (the FMA-heavy pipe, which runs integer multiply-adds), and the
# two interleaved 1:1 (the issue slot).  Run it under ncu with the pipe
# counters to see where each kind executes.
PROBE_SRC = r"""
#define CHAINS(OP) OP(a0) OP(a1) OP(a2) OP(a3) OP(a4) OP(a5) OP(a6) OP(a7)
#define LOP(a) asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a) : "r"(c1), "r"(c2));
#define MAD(a) asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(a) : "r"(c1), "r"(c2));
template <int KIND>
__global__ void probe(unsigned *out, int iters, unsigned c1, unsigned c2) {
  unsigned a0 = threadIdx.x, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3;
  unsigned a4 = a0 + 4, a5 = a0 + 5, a6 = a0 + 6, a7 = a0 + 7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      if (KIND == 0) { CHAINS(LOP) CHAINS(LOP) }
      if (KIND == 1) { CHAINS(MAD) CHAINS(MAD) }
      if (KIND == 2) { CHAINS(LOP) CHAINS(MAD) }
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = a0 ^ a1 ^ a2 ^ a3 ^ a4 ^ a5 ^ a6 ^ a7;
}
extern "C" int run_probe(int kind, int blocks, int threads, int iters, float *ms) {
  unsigned *out;
  if (cudaMalloc(&out, sizeof(unsigned) * blocks * threads) != cudaSuccess) return 1;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int rep = 0; rep < 2; ++rep) {
    cudaEventRecord(e0);
    if (kind == 0) probe<0><<<blocks, threads>>>(out, iters, 0x9E3779B9u, 0x7F4A7C15u);
    if (kind == 1) probe<1><<<blocks, threads>>>(out, iters, 0x9E3779B9u, 0x7F4A7C15u);
    if (kind == 2) probe<2><<<blocks, threads>>>(out, iters, 0x9E3779B9u, 0x7F4A7C15u);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
  }
  cudaEventElapsedTime(ms, e0, e1);
  cudaFree(out);
  return cudaGetLastError() != cudaSuccess;
}
"""


def run_probe(args):
    """Compile and run the issue probe; prints one JSON line per kind with
    the warp instructions of the unrolled body (16 per inner step) per clock
    per scheduler at the sampled SM clock."""
    import ctypes
    import tempfile

    import torch
    torch.cuda.init()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "probe.cu")
        lib = os.path.join(d, "probe.so")
        with open(src, "w") as f:
            f.write(PROBE_SRC)
        from paper_2401_14117_gb300 import build as pbuild
        subprocess.run([pbuild._nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-O3",
                        "-Xcompiler", "-fPIC", "-shared", "-o", lib, src], check=True)
        L = ctypes.CDLL(lib)
        blocks, threads, iters = sms * 4, 512, 1 << 18  # about 0.25 s per launch
        for kind, name in ((0, "lop3 (ALU pipe)"), (1, "imad (FMA-heavy pipe)"),
                           (2, "lop3 + imad 1:1")):
            ms = ctypes.c_float()
            with ClockSampler(0) as clk:
                rc = L.run_probe(kind, blocks, threads, iters, ctypes.byref(ms))
            if rc:
                raise RuntimeError("probe launch failed")
            clocks = clk.summary()
            mhz = clocks.get("sm_mhz") or 2070.0
            warp_inst = blocks * threads / 32 * iters * 8 * 16
            per_clk = warp_inst / (ms.value / 1e3 * mhz * 1e6) / (sms * 4)
            print(json.dumps({"probe": name, "ms": ms.value, "sm_mhz": mhz,
                              "warp_inst_per_clk_per_scheduler": per_clk,
                              "counted": "16 per inner step (loop overhead excluded)",
                              "clocks": clocks}), flush=True)


# ------------------------------------------------------------------ extras
def _time_ms(fn, stream, reps=2, setup=None):
    import torch
    best = float("inf")
    for _ in range(reps):
        if setup is not None:
            setup()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def extras(args, dev, stream):
    """The other workloads of the hot path, each timed with CUDA events on
    its launching stream (inputs resident on the device)."""
    import numpy as np
    import torch

    from paper_2401_14117_gb300 import accuracy, autotune, binding, inputs, serving
    from paper_2401_14117_gb300.batch import ProblemSet, plan_of
    out = {}
    sections = set(args.extras.split(","))

    def want(name):
        return "all" in sections or name in sections

    def words(shape, seed, spd=False, sigma=None):
        if spd:
            x = torch.from_numpy(inputs.spd(shape[0], seed, device=dev)).to(dev)
        elif sigma is not None:
            x = torch.from_numpy(inputs.normal(shape, seed, sigma)).to(dev)
        else:
            x = torch.from_numpy(inputs.uniform(shape, seed)).to(dev)
        w = torch.empty(x.shape, dtype=torch.int32, device=dev)
        binding.posit_from_double(x.T.contiguous() if spd else x, w, x.numel(), stream)
        return w

    # element-wise Add/Mul/Div/Sqrt over the argument ranges of Sec. 4.2
    # (Table tabrandom): ns per op, and the paper's "per CUDA core" figure
    # (time x cores / S, with 152 SMs x 128 cores)
    if want("elementwise"):
        ranges = {"I0 [1,2)": (1.0, 2.0), "I1 [1e-38,1e-30)": (1e-38, 1e-30),
                  "I2 [1e30,1e38)": (1e30, 1e38), "I3 [1e-15,1e-14)": (1e-15, 1e-14),
                  "I4 [1e14,1e15)": (1e14, 1e15)}
        S = args.ew_size
        ew = {}
        for r_i, (name, (lo, hi)) in enumerate(ranges.items()):
            p = torch.from_numpy(inputs.uniform(S, inputs.SEED_BASE + 40 + 2 * r_i, lo, hi)).to(dev)
            q = torch.from_numpy(inputs.uniform(S, inputs.SEED_BASE + 41 + 2 * r_i, lo, hi)).to(dev)
            pw = torch.empty(S, dtype=torch.int32, device=dev)
            qw = torch.empty(S, dtype=torch.int32, device=dev)
            rw = torch.empty(S, dtype=torch.int32, device=dev)
            binding.posit_from_double(p, pw, S, stream)
            binding.posit_from_double(q, qw, S, stream)
            row = {}
            for op, code in (("add", 0), ("mul", 2), ("div", 3), ("sqrt", 4)):
                ms = _time_ms(lambda: binding.posit_elementwise(code, pw, qw, rw, S, stream), stream,
                              reps=3)
                nbytes = (8 if op == "sqrt" else 12) * S
                row[op] = {"ns_per_op": ms * 1e6 / S, "ns_per_op_per_core": ms * 1e6 / S * 152 * 128,
                           "GB/s": nbytes / (ms / 1e3) / 1e9}
            ew[name] = row
            del p, q, pw, qw, rw
        ew["note"] = (f"{S} elements per launch, operands uniform in the range; "
                      "GB/s counts 4-byte words read and written once")
        out["elementwise"] = ew

    # Rgemm: the other square sizes and the trailing-update shape
    if want("rgemm"):
        gemm = {}
        for (m, n, k, name) in ((1024, 1024, 1024, "1024^3"), (4096, 4096, 4096, "4096^3"),
                                (8192, 8192, 256, "8192x8192x256 alpha=-1 beta=1")):
            A, B, C = words((k, m), 11), words((n, k), 12), words((n, m), 13)
            alpha, beta = (0xC0000000, ONE) if k == 256 else (ONE, 0)
            ms = _time_ms(lambda: binding.posit_rgemm("N", "N", m, n, k, alpha, A, m, B, k, beta,
                                                      C, m, stream), stream, reps=3)
            gemm[name] = {"ms": ms, "gflops": 2.0 * m * n * k / (ms / 1e3) / 1e9}
            del A, B, C
        # the two input sets at 4096^3, with the binary32 GEMM of the same
        # words (TF32 off) and the accuracy of both against FP64
        m = 4096
        prev_tf32 = torch.backends.cuda.matmul.allow_tf32
        torch.backends.cuda.matmul.allow_tf32 = False
        for label, gen in (("uniform", inputs.uniform), ("scaled", inputs.scaled)):
            A, B = torch.empty((m, m), dtype=torch.int32, device=dev), torch.empty(
                (m, m), dtype=torch.int32, device=dev)
            binding.posit_from_double(torch.from_numpy(gen((m, m), 17)).to(dev), A, m * m, stream)
            binding.posit_from_double(torch.from_numpy(gen((m, m), 18)).to(dev), B, m * m, stream)
            C = torch.empty_like(A)
            ms = _time_ms(lambda: binding.posit_rgemm("N", "N", m, m, m, ONE, A, m, B, m, 0, C, m,
                                                      stream), stream, reps=2)
            a64, b64, c64p = (torch.empty((m, m), dtype=torch.float64, device=dev)
                              for _ in range(3))
            binding.posit_to_double(A, a64, m * m, stream)
            binding.posit_to_double(B, b64, m * m, stream)
            binding.posit_to_double(C, c64p, m * m, stream)
            # column-major words: the row-major tensors hold A^T, B^T and C^T
            ref = b64 @ a64  # (A B)^T in FP64
            a32, b32 = a64.float(), b64.float()
            ms32 = _time_ms(lambda: torch.matmul(b32, a32), torch.cuda.current_stream(), reps=2)
            c32 = torch.matmul(b32, a32).double()
            nref = torch.linalg.vector_norm(ref)
            gemm[f"4096^3 {label}"] = {
                "ms": ms, "gflops": 2.0 * m ** 3 / (ms / 1e3) / 1e9,
                "rel_error_fro": float(torch.linalg.vector_norm(c64p - ref) / nref),
                "binary32_ms": ms32,
                "binary32_rel_error_fro": float(torch.linalg.vector_norm(c32 - ref) / nref)}
            del A, B, C, a64, b64, c64p, ref, a32, b32, c32
        torch.backends.cuda.matmul.allow_tf32 = prev_tf32
        gemm["note"] = ("scaled: uniform [-1,1] x 10^u, u ~ U[-4,4] per entry; errors are "
                        "||C - C_fp64|| / ||C_fp64|| (Frobenius) on the same posit inputs; "
                        "binary32 = torch.matmul in FP32 with TF32 off")
        out["rgemm"] = gemm

    # trailing-update K sweep (Sec. 5.3, Fig. gemm_trailing): C <- C - A B with
    # M = N = 8192, relative to the square 8192^3 rate of the headline
    if want("ksweep"):
        m = n = 8192
        sq_ms = getattr(args, "square_ms", None)
        sq = 2.0 * m * n * m / (sq_ms / 1e3) / 1e9 if sq_ms else None
        ksw = {}
        for k in (32, 64, 128, 256, 512, 1024, 2048):
            A, B, C = words((k, m), 14), words((n, k), 15), words((n, m), 16)
            ms = _time_ms(lambda: binding.posit_rgemm("N", "N", m, n, k, 0xC0000000, A, m, B, k, ONE,
                                                      C, m, stream), stream, reps=3)
            gf = 2.0 * m * n * k / (ms / 1e3) / 1e9
            ksw[str(k)] = {"ms": ms, "gflops": gf, "relative_to_square": gf / sq if sq else None}
            del A, B, C
        out["trailing_k_sweep"] = ksw

    # sigma sweep (Sec. 4.3 Fig. gemm_v100, Sec. 5.1 Fig. cho_err): normal
    # N(0, sigma^2) inputs; Rgemm 4096^3 rate and the LU / Cholesky accuracy
    # advantage over binary32 at n = 2048
    if want("sigma"):
        sig = {}
        for s_i, sigma in enumerate((1e-2, 1.0, 1e2, 1e4, 1e6)):
            m = 4096
            A, B, C = (words((m, m), 60 + 3 * s_i, sigma=sigma), words((m, m), 61 + 3 * s_i, sigma=sigma),
                       torch.empty((m, m), dtype=torch.int32, device=dev))
            ms = _time_ms(lambda: binding.posit_rgemm("N", "N", m, m, m, ONE, A, m, B, m, 0, C, m,
                                                      stream), stream, reps=2)
            del A, B, C
            A64 = torch.from_numpy(inputs.normal((2048, 2048), 70 + s_i, sigma)).to(dev)
            lu = accuracy.solve_accuracy(A64, "lu")
            S64 = torch.from_numpy(inputs.spd_sigma(2048, 80 + s_i, sigma, device=dev)).to(dev)
            ch = accuracy.solve_accuracy(S64, "cholesky")
            del A64, S64
            sig[f"{sigma:g}"] = {"rgemm_4096_gflops": 2.0 * m ** 3 / (ms / 1e3) / 1e9,
                                 "lu_log10_e32_over_eposit": lu["log10_e32_over_eposit"],
                                 "cholesky_log10_e32_over_eposit": ch["log10_e32_over_eposit"],
                                 "lu_backward_error": [lu["posit"]["backward_error_2"],
                                                       lu["binary32"]["backward_error_2"]],
                                 "cholesky_backward_error": [ch["posit"]["backward_error_2"],
                                                             ch["binary32"]["backward_error_2"]],
                                 "info": [lu["info"], ch["info"]]}
        sig["note"] = ("LU: A ~ N(0, sigma^2); Cholesky: A = sigma^2 (G G^T / n + I); "
                       "backward errors listed [posit, binary32]")
        out["sigma_sweep"] = sig

    # Rgetrf / Rpotrf / Rgetrs / Rpotrs at n = 8192, nb = 256 (1 RHS)
    if want("factor"):
        n = 8192
        fac = {}
        A0 = words((n, n), 21)
        S0 = words((n, n), 22, spd=True)
        b0 = words((1, n), 23)
        A = torch.empty_like(A0)
        S = torch.empty_like(S0)
        ipiv = torch.zeros(n, dtype=torch.int32, device=dev)
        info = torch.zeros(1, dtype=torch.int32, device=dev)
        ms = _time_ms(lambda: binding.posit_rgetrf(n, n, A, n, ipiv, info, stream), stream,
                      setup=lambda: A.copy_(A0))
        fac["rgetrf_8192"] = {"ms": ms, "gflops": 2 * n ** 3 / 3 / (ms / 1e3) / 1e9,
                              "info": int(info.item())}
        ms = _time_ms(lambda: binding.posit_rpotrf("L", n, S, n, info, stream), stream,
                      setup=lambda: S.copy_(S0))
        fac["rpotrf_8192"] = {"ms": ms, "gflops": n ** 3 / 3 / (ms / 1e3) / 1e9,
                              "info": int(info.item())}
        b = torch.empty_like(b0)
        ms = _time_ms(lambda: binding.posit_rgetrs("N", n, 1, A, n, ipiv, b, n, stream), stream,
                      setup=lambda: b.copy_(b0))
        fac["rgetrs_8192"] = {"ms": ms, "GB/s (factor read once)": 4.0 * n * n / (ms / 1e3) / 1e9,
                              "us_per_32_row_block": ms * 1e3 / (2 * n / 32)}
        SU = torch.empty_like(S0)
        SU.copy_(S0)
        binding.posit_rpotrf("U", n, SU, n, info, stream)
        ms = _time_ms(lambda: binding.posit_rpotrs("U", n, 1, SU, n, b, n, stream), stream,
                      setup=lambda: b.copy_(b0))
        fac["rpotrs_U_8192"] = {"ms": ms, "us_per_32_row_block": ms * 1e3 / (2 * n / 32)}
        del SU
        ms = _time_ms(lambda: binding.posit_rpotrs("L", n, 1, S, n, b, n, stream), stream, reps=1,
                      setup=lambda: b.copy_(b0))
        fac["rpotrs_8192"] = {"ms": ms, "note": "dot-form L^T solve: one serial chain of "
                                                "n(n-1)/2 rounded additions"}
        out["factor"] = fac
        del A0, S0, A, S

    # board power during back-to-back Rgetrf 8192 (Sec. 5.3, Table PowerE):
    # NVML board power sampled every 200 ms, read only
    if want("power"):
        n = 8192
        A0 = words((n, n), 21)
        A = torch.empty_like(A0)
        ipiv = torch.zeros(n, dtype=torch.int32, device=dev)
        info = torch.zeros(1, dtype=torch.int32, device=dev)
        ms = _time_ms(lambda: binding.posit_rgetrf(n, n, A, n, ipiv, info, stream), stream,
                      reps=1, setup=lambda: A.copy_(A0))
        reps = max(3, int(4000.0 / ms))
        with ClockSampler(torch.cuda.current_device()) as clk:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(reps):
                A.copy_(A0)
                binding.posit_rgetrf(n, n, A, n, ipiv, info, stream)
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
        pc = clk.summary()
        gf = reps * 2 * n ** 3 / 3 / wall / 1e9
        out["power"] = {"workload": f"{reps} x Rgetrf 8192 back to back (with the input copy)",
                        "gflops": gf, "board_power_w": pc["power_w"], "sm_mhz": pc["sm_mhz"],
                        "gflops_per_w": gf / pc["power_w"] if pc["power_w"] else None,
                        "reasons": pc["reasons"], "samples": pc["samples"]}
        del A0, A

    # accuracy against FP64 / FP32 (Sec. 5.1), n = 2048
    if want("accuracy"):
        acc = {}
        A64 = torch.from_numpy(inputs.uniform((2048, 2048), 31)).to(dev)
        acc["lu_2048"] = accuracy.solve_accuracy(A64, "lu")
        S64 = torch.from_numpy(inputs.spd(2048, 32, device=dev)).to(dev)
        acc["cholesky_2048"] = accuracy.solve_accuracy(S64, "cholesky")
        out["accuracy"] = acc

    # batched: 4096 problems, n log-uniform [16, 512], half LU half Cholesky
    if want("batched"):
        count = args.batch_count
        ns = inputs.batched_sizes(count, inputs.SEED_BASE + 3)
        info = torch.zeros(1, dtype=torch.int32, device=dev)
        batched = {}
        for chol, label in ((binding.POSIT_CHOLESKY, "cholesky_L"), (binding.POSIT_CHOLESKY_U, "cholesky_U")):
            kinds = np.array([binding.POSIT_LU if i % 2 == 0 else chol for i in range(count)], np.int32)
            ps = ProblemSet(kinds, ns, np.ones(count, np.int64))
            for i in range(count):
                k = int(ns[i])
                a64 = torch.from_numpy(inputs.uniform((k, k), 7000 + i) if kinds[i] == 0
                                       else inputs.spd(k, 7000 + i)).to(dev)
                b64 = torch.from_numpy(inputs.uniform((k,), 9000 + i)).to(dev)
                binding.posit_from_double(a64.T.contiguous(), ps.A[ps.a_off[i]:], k * k, stream)
                binding.posit_from_double(b64, ps.B[ps.b_off[i]:], k, stream)
            torch.cuda.synchronize()
            snap = ps.snapshot()
            if args.batch_plan:
                best = tuple(int(v) for v in args.batch_plan.split(","))
            else:
                best, timings = autotune.tune_problem_set(ps, sample=None, use_cache=True)
            plan = plan_of(*best)
            ws = torch.empty(ps.workspace_bytes(plan), dtype=torch.uint8, device=dev)
            g = torch.cuda.CUDAGraph()
            gs = torch.cuda.Stream()
            ps.restore(snap)
            with torch.cuda.graph(g, stream=gs):
                ps.run(plan, ws, stream=gs)
            ms = _time_ms(g.replay, torch.cuda.current_stream(), reps=2, setup=lambda: ps.restore(snap))
            ops = float(sum((2 * k ** 3 / 3 if kd == 0 else k ** 3 / 3) + 2 * k * k
                            for k, kd in zip(ns, kinds)))
            sample = list(range(0, count, 16))
            ps.restore(snap)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for i in sample:
                k = int(ns[i])
                Ai, Bi, Pi = ps.A[ps.a_off[i]:], ps.B[ps.b_off[i]:], ps.ipiv[ps.p_off[i]:]
                if kinds[i] == 0:
                    binding.posit_rgetrf(k, k, Ai, k, Pi, info, stream)
                    binding.posit_rgetrs("N", k, 1, Ai, k, Pi, Bi, k, stream)
                else:
                    uplo = "U" if kinds[i] == binding.POSIT_CHOLESKY_U else "L"
                    binding.posit_rpotrf(uplo, k, Ai, k, info, stream)
                    binding.posit_rpotrs(uplo, k, 1, Ai, k, Bi, k, stream)
            torch.cuda.synchronize()
            plain_s = time.perf_counter() - t0
            batched[label] = {"problems": count, "plan": list(best), "graph_ms": ms,
                              "solves_per_s": count / (ms / 1e3), "gflops": ops / (ms / 1e3) / 1e9,
                              "per_matrix_launches_solves_per_s": len(sample) / plain_s,
                              "per_matrix_sample": f"every 16th problem ({len(sample)}), one stream"}
            del ps, ws, g
        out["batched"] = batched

    # serving: Poisson 2000 req/s, n log-uniform [64, 4096], nrhs 1..8
    servers = (("continuous_batching", 512), ("per_request_plain", 1))
    if want("serving"):
        serve = {}
        for chol, label in ((binding.POSIT_CHOLESKY_U, "cholesky_U"), (binding.POSIT_CHOLESKY, "cholesky_L")):
            pool = serving.Pool(args.serve_pool, 64, 4096, 8, seed=20240129, cholesky_kind=chol)
            t, idx = serving.arrivals(2000.0, args.serve_seconds, pool.size, seed=7)
            for name, small in servers:
                cfg = serving.default_config(budget_gb=40.0, small_n_max=small)
                r = serving.run(pool, t, idx, cfg, duration=args.serve_seconds, max_outstanding=256)
                r.pop("kept")
                serve[f"{label}/{name}"] = r
            if chol == binding.POSIT_CHOLESKY_U:
                # a rate the server sustains (offered work below its capacity)
                rate = args.serve_rate_sustained
                t2, idx2 = serving.arrivals(rate, args.serve_seconds, pool.size, seed=8)
                for name, small in servers:
                    cfg = serving.default_config(budget_gb=40.0, small_n_max=small)
                    r = serving.run(pool, t2, idx2, cfg, duration=args.serve_seconds,
                                    max_outstanding=256)
                    r.pop("kept")
                    serve[f"{label}/{name}@{rate:g}per_s"] = r
            del pool
        serve["workload"] = (f"Poisson 2000/s (and {args.serve_rate_sustained:g}/s), n log-uniform "
                             f"[64, 4096], nrhs 1-8, LU/Cholesky 50/50, {args.serve_seconds:.0f} s, "
                             f"40 GB budget, pool of {args.serve_pool} seeded problems; latency "
                             "from arrival (queueing included), p50/p99 over every offered "
                             "request (unfinished ones censored at the end of the run)")
        out["serving"] = serve

    # arrival-rate sweep of both servers: the highest rate each holds with
    # p99 under the SLO (requested explicitly: --extras serving_sweep)
    if "serving_sweep" in sections:
        slo = args.serve_slo_ms
        pool = serving.Pool(args.serve_pool, 64, 4096, 8, seed=20240129,
                            cholesky_kind=binding.POSIT_CHOLESKY_U)
        sweep = {"slo_ms": slo, "seconds_per_rate": args.serve_seconds, "pool": args.serve_pool,
                 "rates": [float(x) for x in args.serve_rates.split(",")]}
        for name, small in servers:
            rows, best = [], None
            for rate in sweep["rates"]:
                t, idx = serving.arrivals(rate, args.serve_seconds, pool.size, seed=11)
                cfg = serving.default_config(budget_gb=40.0, small_n_max=small)
                r = serving.run(pool, t, idx, cfg, duration=args.serve_seconds,
                                max_outstanding=1024)
                r.pop("kept")
                r["rate"] = rate
                rows.append(r)
                # p99 over every offered request, the unfinished ones at their
                # wait so far: a run that falls behind shows it there
                if r["p99_ms"] is not None and r["p99_ms"] <= slo:
                    best = rate
            sweep[name] = {"runs": rows, "highest_rate_within_slo": best}
        del pool
        out["serving_sweep"] = sweep

    return out


def main():
    args = parse()
    if args.probe:
        run_probe(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
