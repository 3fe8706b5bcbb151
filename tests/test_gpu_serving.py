"""The continuous-batching server: every served result equals the result of
the same problem solved alone (single-problem routines) -- and, for the
smaller problems, the CPU oracle -- whatever else was in flight."""
import ctypes
import time

import numpy as np
import pytest
import torch

import oracle
from paper_2401_14117_gb300 import binding, serving

pytestmark = pytest.mark.gpu


def alone(pool, i):
    """The single-problem routines on one pool problem (device)."""
    n, r = int(pool.ns[i]), int(pool.nrhs[i])
    A = pool.A[i].cuda().clone()
    B = pool.B[i].cuda().clone()
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    if pool.kinds[i] == binding.POSIT_LU:
        ipiv = torch.zeros(n, dtype=torch.int32, device="cuda")
        binding.posit_rgetrf(n, n, A, n, ipiv, info)
        binding.posit_rgetrs("N", n, r, A, n, ipiv, B, n)
    else:
        uplo = "U" if pool.kinds[i] == binding.POSIT_CHOLESKY_U else "L"
        binding.posit_rpotrf(uplo, n, A, n, info)
        torch.cuda.synchronize()
        if int(info.item()) == 0:
            binding.posit_rpotrs(uplo, n, r, A, n, B, n)
    torch.cuda.synchronize()
    return B.cpu().numpy().view(np.uint32).reshape(-1), int(info.item())


def oracle_solution(pool, i):
    n, r = int(pool.ns[i]), int(pool.nrhs[i])
    A = pool.A[i].numpy().view(np.uint32).reshape(n, n).T
    B = pool.B[i].numpy().view(np.uint32).reshape(r, n).T
    if pool.kinds[i] == binding.POSIT_LU:
        F, ipiv, info = oracle.rgetrf(A)
        X = oracle.rgetrs(F, ipiv, B)
    else:
        uplo = "U" if pool.kinds[i] == binding.POSIT_CHOLESKY_U else "L"
        F, info = oracle.rpotrf(A, uplo=uplo)
        X = oracle.rpotrs(F, B, uplo=uplo) if info == 0 else B
    return np.asfortranarray(X).ravel(order="F"), info


@pytest.mark.parametrize("small_n_max,chol", [(96, binding.POSIT_CHOLESKY),
                                              (512, binding.POSIT_CHOLESKY),
                                              (256, binding.POSIT_CHOLESKY_U)])
def test_served_results_equal_alone_and_oracle(small_n_max, chol):
    pool = serving.Pool(20, 16, 700, 4, seed=77, cholesky_kind=chol)
    t, idx = serving.arrivals(400.0, 1.5, pool.size, seed=78)
    cfg = serving.default_config(budget_gb=2.0, small_n_max=small_n_max, max_batch=64)
    res = serving.run(pool, t, idx, cfg, duration=1.5, max_outstanding=64,
                      capture=set(range(len(t))), drain=True)
    assert res["completed"] == res["submitted"] == res["offered"] > 20
    assert res["launches"] >= 2
    alone_x = {}
    for rid, (x, info) in res["kept"].items():
        i = int(idx[rid])
        if i not in alone_x:
            alone_x[i] = alone(pool, i)
        ax, ainfo = alone_x[i]
        assert info == ainfo and np.array_equal(x, ax), (rid, i)
    # the smaller problems also against the oracle
    for i in sorted(alone_x):
        if pool.ns[i] <= 200:
            ox, oinfo = oracle_solution(pool, i)
            assert alone_x[i][1] == oinfo and np.array_equal(alone_x[i][0], ox), i


def test_continuous_batching_forms_batches():
    pool = serving.Pool(16, 16, 128, 2, seed=5)
    t, idx = serving.arrivals(4000.0, 0.5, pool.size, seed=6)
    cfg = serving.default_config(budget_gb=1.0, small_n_max=512, max_batch=256)
    res = serving.run(pool, t, idx, cfg, duration=0.5, max_outstanding=256, drain=True)
    assert res["completed"] == res["offered"]
    assert res["largest_batch"] > 1
    assert res["batched_requests"] == res["completed"]


def test_budget_too_small_for_a_request_is_rejected():
    cfg = serving.default_config(budget_gb=1e-6)
    server = binding.posit_serve_open(cfg)
    try:
        A = torch.zeros(64 * 64, dtype=torch.int32, pin_memory=True)
        req = binding.posit_request(binding.POSIT_LU, 64, 1, 0, A.data_ptr(), A.data_ptr(),
                                    A.data_ptr(), A.data_ptr(), 0)
        with pytest.raises(binding.PositError) as e:
            binding.posit_serve_submit(server, req)
        assert e.value.code == -2
    finally:
        binding.posit_serve_close(server)


def test_budget_defers_admission_and_results_stay_exact():
    """Admission by device-memory budget under load: twelve requests are
    submitted at once to a server whose budget holds two of them, so the
    others wait in `pending` (never more than the budget in use) and are
    admitted as memory frees up; every result still equals the problem solved
    alone, and the CPU oracle."""
    pool = serving.Pool(12, 200, 260, 2, seed=91, cholesky_kind=binding.POSIT_CHOLESKY_U)
    sizes = [int(pool.ns[i]) ** 2 * 4 + int(pool.ns[i]) * 16 + 1024 for i in range(pool.size)]
    budget = int(2.2 * max(sizes))
    cfg = serving.default_config(budget_gb=budget / 2 ** 30, small_n_max=512, max_batch=64)
    server = binding.posit_serve_open(cfg)
    X = [torch.zeros(int(pool.ns[i] * pool.nrhs[i]), dtype=torch.int32, pin_memory=True)
         for i in range(pool.size)]
    INFO = torch.zeros(pool.size, dtype=torch.int32, pin_memory=True)
    done, max_pending, max_used = set(), 0, 0
    tags = (ctypes.c_uint64 * pool.size)()
    try:
        for i in range(pool.size):
            binding.posit_serve_submit(server, binding.posit_request(
                int(pool.kinds[i]), int(pool.ns[i]), int(pool.nrhs[i]), 0, pool.A[i].data_ptr(),
                pool.B[i].data_ptr(), X[i].data_ptr(), INFO.data_ptr() + 4 * i, i))
        t0 = time.perf_counter()
        while len(done) < pool.size and time.perf_counter() - t0 < 60:
            got = binding.posit_serve_poll(server, tags, pool.size)
            st = binding.posit_serve_stats(server)
            max_pending = max(max_pending, int(st.pending))
            max_used = max(max_used, int(st.device_bytes_in_use))
            done.update(int(tags[k]) for k in range(got))
            time.sleep(50e-6)
    finally:
        binding.posit_serve_close(server)
    assert len(done) == pool.size
    assert max_pending >= pool.size - 3  # the budget, not a slot limit, held them back
    assert 0 < max_used <= budget
    for i in range(pool.size):
        x = X[i].numpy().view(np.uint32)
        ax, ainfo = alone(pool, i)
        assert int(INFO[i]) == ainfo and np.array_equal(x, ax), i
        ox, oinfo = oracle_solution(pool, i)
        assert oinfo == ainfo and np.array_equal(ax, ox), i
