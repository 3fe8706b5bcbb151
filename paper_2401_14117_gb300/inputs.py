"""Seeded synthetic inputs, shared by the tests, the benchmark and the oracle legs.

This module holds no posit arithmetic: it only draws FP64 numbers (and problem
shapes / arrival times) from seeded generators.  Conversion to posit words is
done by whichever side consumes them (the oracle on the CPU, the library's
conversion kernel on the GPU).

Workload recipes (the paper's inputs are themselves synthetic: normal
matrices with mean 0 and a chosen sigma, Sec. 4 and Sec. 5):
  * uniform:  entries uniform in [-1, 1]
  * scaled:   uniform in [-1, 1] times 10^u, u uniform in [-4, 4] per entry
              (long regimes, |x| up to 1e4)
  * normal:   N(0, sigma^2), the paper's generator (Sec. 4.2, Sec. 5.1)
  * spd:      A = G G^T / n + I with G standard normal (rounded to a
              multiple of 2^-12, which makes G G^T exact), in FP64
  * spd_sigma: sigma^2 (G G^T / n + I), the SPD matrices of the sigma sweep
  * rhs:      b = A x_sol with x_sol = 1/sqrt(n) in every entry, in FP64
              (Sec. 5.1, error study)
"""
from __future__ import annotations

import math

import numpy as np

SEED_BASE = 20240125


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def uniform(shape, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    return rng(seed).uniform(lo, hi, size=shape)


def scaled(shape, seed: int) -> np.ndarray:
    g = rng(seed)
    return g.uniform(-1.0, 1.0, size=shape) * 10.0 ** g.uniform(-4.0, 4.0, size=shape)


def normal(shape, seed: int, sigma: float = 1.0) -> np.ndarray:
    return rng(seed).normal(0.0, sigma, size=shape)


def spd(n: int, seed: int, device=None):
    """A = G G^T / n + I in FP64.  With a torch device, G G^T runs there.

    G is standard normal rounded to a multiple of 2^-12.  Every product of two
    entries is then a multiple of 2^-24 below 2^10 in magnitude, and every
    partial sum of n <= 2^19 of them fits in 53 bits, so G G^T is exact: the
    same FP64 matrix comes out on any host or device, in any summation order.
    """
    G = np.rint(rng(seed).standard_normal((n, n)) * 4096.0) / 4096.0
    if device is None:
        return G @ G.T / n + np.eye(n)
    import torch
    Gt = torch.from_numpy(G).to(device)
    A = Gt @ Gt.T / n + torch.eye(n, dtype=torch.float64, device=device)
    return A.cpu().numpy()


def spd_sigma(n: int, seed: int, sigma: float, device=None):
    """sigma^2 (G G^T / n + I): the SPD recipe with entries of size sigma^2,
    as the paper's X^T X with X ~ N(0, sigma^2) has (Sec. 5.1), while the
    condition number stays that of G G^T / n + I."""
    return spd(n, seed, device) * (sigma * sigma)


def rhs(A64: np.ndarray) -> np.ndarray:
    n = A64.shape[0]
    return A64 @ np.full(n, 1.0 / math.sqrt(n))


def batched_sizes(count: int, seed: int, lo: int = 16, hi: int = 512) -> np.ndarray:
    """n = round(exp(U[ln lo, ln hi])) per problem (log-uniform sizes)."""
    g = rng(seed)
    return np.rint(np.exp(g.uniform(math.log(lo), math.log(hi), size=count))).astype(np.int64)


def arrivals(rate_per_s: float, duration_s: float, seed: int) -> np.ndarray:
    """Poisson arrival times (exponential gaps, mean 1/rate) in [0, duration)."""
    g = rng(seed)
    n_est = int(rate_per_s * duration_s * 1.2) + 16
    t = np.cumsum(g.exponential(1.0 / rate_per_s, size=n_est))
    while t[-1] < duration_s:
        t = np.concatenate([t, t[-1] + np.cumsum(g.exponential(1.0 / rate_per_s, size=n_est))])
    return t[t < duration_s]
