"""Autotuner for the batched factor+solve launch shape.

A plan is (threads per CTA, persistent CTAs per SM, shared-memory bytes per
CTA).  Every plan computes the same bits (the per-element operation order
does not depend on it), so the tuner only measures time: it runs each
candidate on a sample of the batch, keeps the fastest, and caches the choice
per (GPU name, size bucket) in a small JSON file.
"""
from __future__ import annotations

import json
import math
import os

SMEM_PER_SM = 228 * 1024          # GB300 shared memory per SM
SMEM_PER_CTA_MAX = 227 * 1024
# threads per SM a plan may ask for; the batched kernel holds 128 registers per
# thread, so at most 512 of them are resident at once and CTAs beyond that
# wait (plans asking for more are still valid and sometimes faster)
THREADS_PER_SM = 1024

_HERE = os.path.dirname(os.path.abspath(__file__))
CACHE_PATH = os.path.join(_HERE, "_build", "autotune_cache.json")


def candidates():
    """Valid (threads, ctas_per_sm, smem_bytes) launch shapes."""
    out = []
    for threads in (128, 256, 512):
        for ctas in (1, 2, 3, 4):
            if threads * ctas > THREADS_PER_SM:
                continue
            for smem in (48 * 1024, 96 * 1024, 200 * 1024):
                if smem * ctas > SMEM_PER_SM - 1024 * ctas or smem > SMEM_PER_CTA_MAX:
                    continue
                out.append((threads, ctas, smem))
    return out


def bucket_key(gpu_name: str, ns) -> str:
    """Cache key: GPU and the log2 range of the problem sizes."""
    lo = int(math.floor(math.log2(max(1, min(ns)))))
    hi = int(math.ceil(math.log2(max(1, max(ns)))))
    return f"{gpu_name}|n2^{lo}-2^{hi}"


def load_cache(path=CACHE_PATH) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(cache: dict, path=CACHE_PATH):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def choose(timings: dict):
    """Fastest plan from {plan tuple: seconds}; ties go to fewer threads."""
    return min(timings, key=lambda p: (timings[p], p[0] * p[1], p[2]))


def tune(measure, key: str, cands=None, cache_path=CACHE_PATH, use_cache=True):
    """measure(plan tuple) -> seconds.  Returns (best plan tuple, timings)."""
    cache = load_cache(cache_path) if use_cache else {}
    if use_cache and key in cache:
        return tuple(cache[key]["plan"]), cache[key].get("timings", {})
    timings = {}
    for p in (cands or candidates()):
        timings[tuple(p)] = float(measure(tuple(p)))
    best = choose(timings)
    if use_cache:
        cache[key] = {"plan": list(best),
                      "timings": {",".join(map(str, k)): v for k, v in timings.items()}}
        save_cache(cache, cache_path)
    return best, timings


def tune_problem_set(ps, sample=None, reps=1, use_cache=True, cands=None):
    """Tune on (a sample of) a ProblemSet on the current GPU."""
    import torch

    from .batch import ProblemSet, plan_of
    if sample is not None and sample < ps.count:
        idx = sorted(set(int(i) for i in
                         torch.linspace(0, ps.count - 1, sample).round().long().tolist()))
        sub = ProblemSet(ps.kinds[idx], ps.ns[idx], ps.nrhs[idx], ps.device)
        for j, i in enumerate(idx):
            n, r = int(ps.ns[i]), int(ps.nrhs[i])
            sub.A[sub.a_off[j]: sub.a_off[j] + n * n] = ps.A[ps.a_off[i]: ps.a_off[i] + n * n]
            sub.B[sub.b_off[j]: sub.b_off[j] + n * r] = ps.B[ps.b_off[i]: ps.b_off[i] + n * r]
        target = sub
    else:
        target = ps
    snap = target.snapshot()
    name = torch.cuda.get_device_name()

    def measure(p):
        plan = plan_of(*p)
        ws = torch.empty(target.workspace_bytes(plan), dtype=torch.uint8, device=target.device)
        best = float("inf")
        for _ in range(reps + 1):
            target.restore(snap)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            target.run(plan, ws)
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1) / 1e3)
        target.restore(snap)
        return best

    return tune(measure, bucket_key(name, ps.ns.tolist()), cands=cands, use_cache=use_cache)
