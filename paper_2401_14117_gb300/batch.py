"""Packing many independent factor+solve problems for
posit_factor_solve_batched (argument marshalling: device buffers and the
descriptor array; all arithmetic runs in the library's kernels)."""
from __future__ import annotations

import numpy as np
import torch

from . import binding

DEFAULT_PLAN = (256, 1, 200 * 1024)


def plan_of(threads: int, ctas_per_sm: int, smem_bytes: int) -> binding.posit_plan:
    return binding.posit_plan(threads, ctas_per_sm, smem_bytes, 0)


class ProblemSet:
    """Device storage for a batch of problems.

    kinds: POSIT_LU / POSIT_CHOLESKY per problem; ns: sizes; nrhs: right-hand
    sides per problem.  Matrices live in one int32 buffer (each column-major
    with ld = n), right-hand sides in another; `order` starts the problems
    largest first.
    """

    def __init__(self, kinds, ns, nrhs, device=None):
        self.device = device or torch.device("cuda", torch.cuda.current_device())
        self.kinds = np.asarray(kinds, dtype=np.int32)
        self.ns = np.asarray(ns, dtype=np.int64)
        self.nrhs = np.asarray(nrhs, dtype=np.int64)
        self.count = len(self.ns)
        a_sizes = self.ns * self.ns
        b_sizes = self.ns * self.nrhs
        self.a_off = np.concatenate([[0], np.cumsum(a_sizes)[:-1]]).astype(np.int64)
        self.b_off = np.concatenate([[0], np.cumsum(b_sizes)[:-1]]).astype(np.int64)
        self.p_off = np.concatenate([[0], np.cumsum(self.ns)[:-1]]).astype(np.int64)
        self.A = torch.zeros(int(a_sizes.sum()), dtype=torch.int32, device=self.device)
        self.B = torch.zeros(int(b_sizes.sum()), dtype=torch.int32, device=self.device)
        self.ipiv = torch.zeros(int(self.ns.sum()), dtype=torch.int32, device=self.device)
        self.info = torch.zeros(self.count, dtype=torch.int32, device=self.device)
        self.max_n = int(self.ns.max()) if self.count else 0
        self.max_nrhs = int(self.nrhs.max()) if self.count else 0
        desc = np.zeros(self.count, dtype=binding.PROBLEM_DTYPE)
        desc["kind"] = self.kinds
        desc["n"] = self.ns
        desc["nrhs"] = self.nrhs
        desc["lda"] = self.ns
        desc["ldb"] = self.ns
        desc["A"] = self.A.data_ptr() + 4 * self.a_off
        desc["B"] = self.B.data_ptr() + 4 * self.b_off
        desc["ipiv"] = self.ipiv.data_ptr() + 4 * self.p_off
        desc["info"] = self.info.data_ptr() + 4 * np.arange(self.count, dtype=np.int64)
        self.desc = torch.from_numpy(desc.view(np.uint8).copy()).to(self.device)
        order = np.argsort(-(self.ns.astype(np.float64) ** 3), kind="stable").astype(np.int32)
        self.order = torch.from_numpy(order).to(self.device)

    # ------------------------------------------------------------ data
    def set_problem(self, i, A_words: np.ndarray, B_words: np.ndarray):
        """Copy column-major posit words (n x n and n x nrhs, uint32)."""
        n, r = int(self.ns[i]), int(self.nrhs[i])
        a = np.asfortranarray(A_words, dtype=np.uint32).ravel(order="F").view(np.int32)
        b = np.asfortranarray(B_words.reshape(n, r), dtype=np.uint32).ravel(order="F").view(np.int32)
        self.A[self.a_off[i]: self.a_off[i] + n * n] = torch.from_numpy(a.copy())
        self.B[self.b_off[i]: self.b_off[i] + n * r] = torch.from_numpy(b.copy())

    def get_problem(self, i):
        """(factor words n x n, solution words n x nrhs, ipiv, info) on the host."""
        n, r = int(self.ns[i]), int(self.nrhs[i])
        a = self.A[self.a_off[i]: self.a_off[i] + n * n].cpu().numpy().view(np.uint32)
        b = self.B[self.b_off[i]: self.b_off[i] + n * r].cpu().numpy().view(np.uint32)
        p = self.ipiv[self.p_off[i]: self.p_off[i] + n].cpu().numpy()
        return (a.reshape(n, n, order="F"), b.reshape(n, r, order="F"), p,
                int(self.info[i].item()))

    def snapshot(self):
        return self.A.clone(), self.B.clone()

    def restore(self, snap):
        self.A.copy_(snap[0])
        self.B.copy_(snap[1])
        self.ipiv.zero_()
        self.info.zero_()

    # ------------------------------------------------------------ run
    def workspace_bytes(self, plan) -> int:
        return binding.posit_batched_workspace_size(self.max_n, self.max_nrhs, plan)

    def run(self, plan, workspace=None, stream=None):
        binding.posit_factor_solve_batched(self.count, self.desc, self.order, self.max_n,
                                           self.max_nrhs, plan, workspace, stream)
