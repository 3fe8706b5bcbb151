"""Accuracy of the posit solves against FP64 and FP32 (Sec. 5.1).

For A x = b with x_sol = 1/sqrt(n) in every entry and b = A x_sol computed in
FP64, the posit path (posit_rgetrf + posit_rgetrs, or posit_rpotrf +
posit_rpotrs, on A and b rounded to Posit(32,2)) and an FP32 path (LU with
partial pivoting / Cholesky in float32 on the same GPU, the binary32
reference of the paper's Sgetrs / Spotrs) each solve their own rounding of
(A, b).  Reported per path: the relative backward error
|b - A x| / |b| in FP64 with the 2-norm (and the infinity norm), the digits
of x (-log10 of the relative error to x_sol), and log10(e_binary32 /
e_posit), which is positive when posit is more accurate.
"""
from __future__ import annotations

import math

import torch

from . import binding


def _to_posit(x64: torch.Tensor) -> torch.Tensor:
    w = torch.empty(x64.shape, dtype=torch.int32, device=x64.device)
    binding.posit_from_double(x64.contiguous(), w, x64.numel())
    return w


def _to_double(w: torch.Tensor) -> torch.Tensor:
    x = torch.empty(w.shape, dtype=torch.float64, device=w.device)
    binding.posit_to_double(w.contiguous(), x, w.numel())
    return x


def _errors(A64, b64, x, x_sol):
    r = b64 - A64 @ x
    e2 = float(torch.linalg.vector_norm(r) / torch.linalg.vector_norm(b64))
    einf = float(torch.linalg.vector_norm(r, ord=float("inf")) /
                 torch.linalg.vector_norm(b64, ord=float("inf")))
    rel = float(torch.linalg.vector_norm(x - x_sol) / torch.linalg.vector_norm(x_sol))
    digits = -math.log10(rel) if rel > 0 else float("inf")
    return {"backward_error_2": e2, "backward_error_inf": einf, "solution_digits": digits}


def solve_accuracy(A64: torch.Tensor, kind: str) -> dict:
    """A64: n x n FP64 matrix on the GPU (row-major torch tensor holding the
    matrix itself); kind 'lu' or 'cholesky'."""
    n = A64.shape[0]
    dev = A64.device
    x_sol = torch.full((n,), 1.0 / math.sqrt(n), dtype=torch.float64, device=dev)
    b64 = A64 @ x_sol
    # posit: column-major words are the row-major bytes of A^T
    Aw = _to_posit(A64.T.contiguous())
    bw = _to_posit(b64)
    info = torch.zeros(1, dtype=torch.int32, device=dev)
    if kind == "lu":
        ipiv = torch.zeros(n, dtype=torch.int32, device=dev)
        binding.posit_rgetrf(n, n, Aw, n, ipiv, info)
        binding.posit_rgetrs("N", n, 1, Aw, n, ipiv, bw, n)
    else:
        binding.posit_rpotrf("L", n, Aw, n, info)
        binding.posit_rpotrs("L", n, 1, Aw, n, bw, n)
    xp = _to_double(bw)
    # binary32 on the same GPU
    A32 = A64.float()
    b32 = b64.float()
    if kind == "lu":
        LU, piv = torch.linalg.lu_factor(A32)
        x32 = torch.linalg.lu_solve(LU, piv, b32.unsqueeze(1)).squeeze(1)
    else:
        L = torch.linalg.cholesky(A32)
        x32 = torch.cholesky_solve(b32.unsqueeze(1), L).squeeze(1)
    torch.cuda.synchronize()
    ep = _errors(A64, b64, xp, x_sol)
    e32 = _errors(A64, b64, x32.double(), x_sol)
    adv = (math.log10(e32["backward_error_2"] / ep["backward_error_2"])
           if ep["backward_error_2"] > 0 and e32["backward_error_2"] > 0 else None)
    return {"n": n, "kind": kind, "info": int(info.item()), "posit": ep, "binary32": e32,
            "log10_e32_over_eposit": adv}
