"""Client side of the factor+solve server (posit_serve_* in the C ABI).

Workload: a seeded pool of problems (LU on uniform [-1,1] matrices, Cholesky
on G G^T / n + I), sizes log-uniform in [n_lo, n_hi], 1..nrhs_max right-hand
sides, and Poisson arrivals.  `run` replays the arrivals in wall-clock time:
a request is handed to the server once its arrival time has passed and fewer
than `max_outstanding` requests are inside the server; the latency of a
request is measured from its arrival time, so waiting in the client queue is
part of it (reported separately from the time spent inside the server).
p50/p99 cover every request offered in the window; one not finished when the
run ends counts with its wait so far (censored, a lower bound).
All matrix data is produced and converted on the GPU (the library's
conversion kernel); this module only moves buffers and keeps time.
"""
from __future__ import annotations

import ctypes
import math
import time

import numpy as np
import torch

from . import binding, inputs


class Pool:
    """Seeded problems in page-locked host memory (posit words)."""

    def __init__(self, size, n_lo, n_hi, nrhs_max, seed, lu_fraction=0.5, device=None,
                 cholesky_kind=binding.POSIT_CHOLESKY):
        dev = device or torch.device("cuda", torch.cuda.current_device())
        g = np.random.default_rng(seed)
        self.ns = np.rint(np.exp(g.uniform(math.log(n_lo), math.log(n_hi), size))).astype(np.int64)
        self.kinds = np.where(g.random(size) < lu_fraction, binding.POSIT_LU,
                              cholesky_kind).astype(np.int32)
        self.nrhs = g.integers(1, nrhs_max + 1, size).astype(np.int64)
        self.A, self.B = [], []
        for i in range(size):
            n, r = int(self.ns[i]), int(self.nrhs[i])
            if self.kinds[i] == binding.POSIT_LU:
                a64 = torch.from_numpy(inputs.uniform((n, n), seed * 1000 + 2 * i)).to(dev)
            else:
                a64 = torch.from_numpy(inputs.spd(n, seed * 1000 + 2 * i, device=dev)).to(dev)
            b64 = torch.from_numpy(inputs.uniform((r, n), seed * 1000 + 2 * i + 1)).to(dev)
            self.A.append(self._to_pinned_words(a64.T.contiguous()))  # column-major bytes
            self.B.append(self._to_pinned_words(b64))
        self.size = size
        torch.cuda.synchronize()

    @staticmethod
    def _to_pinned_words(x64):
        w = torch.empty(x64.shape, dtype=torch.int32, device=x64.device)
        binding.posit_from_double(x64, w, x64.numel())
        h = torch.empty(x64.shape, dtype=torch.int32, pin_memory=True)
        h.copy_(w)
        return h

    def ops(self, i):
        """Posit operations of problem i (factor + solve)."""
        n, r = float(self.ns[i]), float(self.nrhs[i])
        f = 2 * n ** 3 / 3 if self.kinds[i] == binding.POSIT_LU else n ** 3 / 3
        return f + 2 * n * n * r


def default_config(budget_gb=40.0, small_n_max=512, max_batch=1024, max_nrhs=8,
                   plan=(256, 4, 48 * 1024), large_lanes=16, batch_only_n_max=128):
    """batch_only_n_max: small requests above it take an idle large lane
    (latency first); at or above small_n_max every small request is batched."""
    return binding.posit_serve_config(int(budget_gb * 2 ** 30), small_n_max, max_batch,
                                      max_nrhs, large_lanes, binding.posit_plan(*plan, 0),
                                      batch_only_n_max, 0)


def run(pool, arrival_times, pool_index, cfg, duration, max_outstanding=256, capture=None,
        drain=False):
    """Replay arrivals; returns a dict of counters and per-request timings.

    capture: optional set of request ids whose solutions (and info) are kept.
    """
    max_n = int(pool.ns.max())
    max_r = int(pool.nrhs.max())
    slots = max_outstanding
    X = torch.empty((slots, max_n * max_r), dtype=torch.int32, pin_memory=True)
    INFO = torch.zeros(slots, dtype=torch.int32, pin_memory=True)
    free = list(range(slots))[::-1]
    server = binding.posit_serve_open(cfg)
    tags = (ctypes.c_uint64 * slots)()
    arrival = np.asarray(arrival_times)
    n_req = len(arrival)
    submit_t = np.full(n_req, np.nan)
    done_t = np.full(n_req, np.nan)
    slot_of = {}
    kept = {}
    nxt = 0
    t0 = time.perf_counter()
    try:
        while True:
            now = time.perf_counter() - t0
            while nxt < n_req and arrival[nxt] <= now and arrival[nxt] < duration and free:
                i = int(pool_index[nxt])
                s = free.pop()
                req = binding.posit_request(
                    int(pool.kinds[i]), int(pool.ns[i]), int(pool.nrhs[i]), 0,
                    pool.A[i].data_ptr(), pool.B[i].data_ptr(), X[s].data_ptr(),
                    INFO.data_ptr() + 4 * s, nxt)
                binding.posit_serve_submit(server, req)
                submit_t[nxt] = time.perf_counter() - t0
                slot_of[nxt] = s
                nxt += 1
            got = binding.posit_serve_poll(server, tags, slots)
            if got:
                t = time.perf_counter() - t0
                for k in range(got):
                    rid = int(tags[k])
                    done_t[rid] = t
                    s = slot_of.pop(rid)
                    if capture is not None and rid in capture:
                        i = int(pool_index[rid])
                        cnt = int(pool.ns[i] * pool.nrhs[i])
                        kept[rid] = (X[s, :cnt].numpy().view(np.uint32).copy(), int(INFO[s]))
                    free.append(s)
            if now >= duration and (not drain or not slot_of):
                break
            if not got:
                time.sleep(20e-6)
    finally:
        stats = binding.posit_serve_stats(server)
        binding.posit_serve_close(server)
    elapsed = time.perf_counter() - t0
    in_window = arrival < duration
    completed = ~np.isnan(done_t)
    lat = (done_t - arrival)[completed]
    svc = (done_t - submit_t)[completed]
    # every request offered in the window: one still waiting (in the client
    # queue or in the server) when the run ends counts with its wait so far,
    # a lower bound of its latency (censored)
    censored = in_window & ~completed
    lat_all = np.where(completed, done_t - arrival, elapsed - arrival)[in_window]
    ops = sum(pool.ops(int(pool_index[r])) for r in np.flatnonzero(completed))

    def pct(v, q):
        return float(np.percentile(v, q) * 1e3) if v.size else None

    p99_all = pct(lat_all, 99)
    return {
        "offered": int(in_window.sum()),
        "submitted": int(nxt),
        "completed": int(completed.sum()),
        "censored": int(censored.sum()),
        "elapsed_s": elapsed,
        "solves_per_s": float(completed.sum()) / min(elapsed, duration if not drain else elapsed),
        "goodput_gflops": ops / elapsed / 1e9,
        # over every offered request, the censored ones at their wait so far
        "p50_ms": pct(lat_all, 50),
        "p99_ms": p99_all,
        "p99_is_lower_bound": bool(censored.sum() > 0 and lat_all.size
                                   and (elapsed - arrival[censored]).max() * 1e3 >= p99_all),
        # over the completed requests only
        "completed_p50_ms": pct(lat, 50),
        "completed_p99_ms": pct(lat, 99),
        "service_p50_ms": float(np.percentile(svc, 50) * 1e3) if svc.size else None,
        "service_p99_ms": float(np.percentile(svc, 99) * 1e3) if svc.size else None,
        "launches": int(stats.launches),
        "batched_requests": int(stats.batched_requests),
        "largest_batch": int(stats.largest_batch),
        "kept": kept,
    }


def arrivals(rate, duration, pool_size, seed):
    t = inputs.arrivals(rate, duration, seed)
    idx = np.random.default_rng(seed + 1).integers(0, pool_size, t.size)
    return t, idx
