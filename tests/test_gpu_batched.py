"""GPU parity of posit_factor_solve_batched: every problem's factor, pivots,
info and solution equal the oracle's single-problem results, for several
launch plans (the plan must not change any bit)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2401_14117_gb300 import binding, inputs
from paper_2401_14117_gb300.batch import ProblemSet, plan_of

pytestmark = pytest.mark.gpu

L, C, CU = binding.POSIT_LU, binding.POSIT_CHOLESKY, binding.POSIT_CHOLESKY_U


def make_set(kinds, ns, nrhs, seed):
    ps = ProblemSet(kinds, ns, nrhs)
    host = []
    for i, (k, n, r) in enumerate(zip(kinds, ns, nrhs)):
        if k == L:
            A = oracle.from_double_array(inputs.uniform((n, n), seed + 2 * i))
        else:
            A = oracle.from_double_array(inputs.spd(n, seed + 2 * i))
        B = oracle.from_double_array(inputs.uniform((n, r), seed + 2 * i + 1))
        ps.set_problem(i, A, B)
        host.append((A, B))
    return ps, host


def expected(kind, A, B):
    if B.shape[1] == 0:  # no right-hand side: the factorisation only
        if kind == L:
            F, ipiv, info = oracle.rgetrf(A)
            return F, B, ipiv, info
        F, info = oracle.rpotrf(A, uplo="U" if kind == CU else "L")
        return F, B, None, info
    if kind == L:
        F, ipiv, info = oracle.rgetrf(A)
        X = oracle.rgetrs(F, ipiv, B)
        return F, X, ipiv, info
    uplo = "U" if kind == CU else "L"
    F, info = oracle.rpotrf(A, uplo=uplo)
    X = oracle.rpotrs(F, B, uplo=uplo) if info == 0 else B
    return F, X, None, info


def check(ps, host, idxs=None):
    for i in (range(ps.count) if idxs is None else idxs):
        A, B = host[i]
        F, X, ipiv, info = expected(int(ps.kinds[i]), A, B)
        gF, gX, gp, ginfo = ps.get_problem(i)
        n = int(ps.ns[i])
        assert ginfo == info, (i, ginfo, info)
        if ps.kinds[i] == L:
            assert np.array_equal(gF, F), i
            assert np.array_equal(gp, ipiv), i
        elif ps.kinds[i] == C:
            assert np.array_equal(np.tril(gF), np.tril(F)), i
            assert np.array_equal(np.triu(gF, 1), np.triu(A, 1)), i  # upper untouched
        else:
            assert np.array_equal(np.triu(gF), np.triu(F)), i
            assert np.array_equal(np.tril(gF, -1), np.tril(A, -1)), i  # lower untouched
        assert np.array_equal(gX, X.reshape(n, -1)), i


PLANS = [(256, 1, 200 * 1024), (128, 2, 96 * 1024), (512, 1, 48 * 1024), (256, 4, 48 * 1024)]


@pytest.mark.parametrize("plan", PLANS)
def test_batched_matches_oracle(plan):
    rng = np.random.default_rng(3)
    count = 40
    ns = np.concatenate([[1, 2, 3, 200, 300], rng.integers(4, 140, count - 5)])
    kinds = np.array([(L, C, CU)[i % 3] for i in range(count)], np.int32)
    nrhs = rng.integers(1, 4, count)
    ps, host = make_set(kinds, ns, nrhs, 100)
    ps.run(plan_of(*plan))
    torch.cuda.synchronize()
    check(ps, host)


def test_batched_singular_and_not_positive_definite():
    kinds = np.array([L, C, L, C], np.int32)
    ns = np.array([30, 30, 150, 150])
    nrhs = np.array([2, 2, 1, 1])
    ps, host = make_set(kinds, ns, nrhs, 7)
    A0, B0 = host[0]
    A0 = A0.copy()
    A0[:, 5] = 0
    A1, B1 = host[1]
    A1 = A1.copy()
    A1[20, 20] = oracle.from_double(-3.0)
    ps.set_problem(0, A0, B0)
    ps.set_problem(1, A1, B1)
    host[0] = (A0, B0)
    host[1] = (A1, B1)
    ps.run(plan_of(*PLANS[0]))
    torch.cuda.synchronize()
    F, X, ip, info = ps.get_problem(0)
    assert info == 6
    F, X, ip, info = ps.get_problem(1)
    assert info == 21 and np.array_equal(X, B1)
    check(ps, host, [0, 2, 3])


def test_batched_nar_and_no_right_hand_side():
    """NaR inside a matrix takes the general arithmetic (NaR propagates
    exactly as in the single-problem routines); nrhs = 0 factors only."""
    kinds = np.array([L, C, CU, L, C, CU, L, C], np.int32)
    ns = np.array([20, 20, 20, 33, 40, 17, 150, 150])
    nrhs = np.array([1, 2, 1, 0, 0, 0, 0, 3])
    ps, host = make_set(kinds, ns, nrhs, 11)
    NAR = np.uint32(0x80000000)
    for i in (0, 1, 2, 7):
        A, B = host[i]
        A = A.copy()
        A[3, 5] = NAR
        A[5, 3] = NAR
        ps.set_problem(i, A, B)
        host[i] = (A, B)
    for plan in (PLANS[0], PLANS[2]):
        snap = ps.snapshot()
        ps.run(plan_of(*plan))
        torch.cuda.synchronize()
        check(ps, host)
        ps.restore(snap)


def test_batched_in_band_switches():
    """The factorisation drops the long-regime test while every value it is
    about to use has a scale in [-40, 40]: Wilkinson's growth matrix leaves
    that band mid-way (|u| doubles every column), a nearly rank-one SPD
    matrix leaves it downwards (trailing entries near 2^-45), and a matrix
    scaled by 2^45 starts outside it."""
    n = 60
    W = np.eye(n) - np.tril(np.ones((n, n)), -1)
    W[:, -1] = 1.0
    g = np.random.default_rng(9)
    v = g.standard_normal(n)
    R1 = np.outer(v, v) + 2.0 ** -45 * np.eye(n)
    S = inputs.spd(n, 13) * 2.0 ** 45
    Lbig = inputs.uniform((n, n), 14) * 2.0 ** 45
    mats = [(L, W), (C, R1), (CU, R1), (C, S), (CU, S), (L, Lbig)]
    kinds = np.array([k for k, _ in mats], np.int32)
    ns = np.full(len(mats), n)
    nrhs = np.ones(len(mats), np.int64)
    ps, host = make_set(kinds, ns, nrhs, 31)
    for i, (_, A64) in enumerate(mats):
        A = oracle.from_double_array(A64)
        B = host[i][1]
        ps.set_problem(i, A, B)
        host[i] = (A, B)
    for plan in (PLANS[0], PLANS[3]):
        snap = ps.snapshot()
        ps.run(plan_of(*plan))
        torch.cuda.synchronize()
        check(ps, host)
        ps.restore(snap)


def test_batched_workload_sampled():
    """4096 problems, n log-uniform in [16, 512], half LU (uniform [-1,1]),
    half Cholesky (G G^T / n + I), 1 RHS: 160 problems (the largest ones
    included) compared with the oracle."""
    count = 4096
    ns = inputs.batched_sizes(count, inputs.SEED_BASE + 30)
    kinds = np.array([L if i % 2 == 0 else C for i in range(count)], np.int32)
    nrhs = np.ones(count, np.int64)
    ps = ProblemSet(kinds, ns, nrhs)
    rng = np.random.default_rng(5)
    big = np.argsort(-ns)[:6]
    sample = sorted(set(big.tolist()) | set(rng.integers(0, count, 154).tolist()))
    host = {}
    for i in range(count):
        n = int(ns[i])
        if kinds[i] == L:
            A = oracle.from_double_array(inputs.uniform((n, n), 50000 + i))
        else:
            A = oracle.from_double_array(inputs.spd(n, 50000 + i))
        B = oracle.from_double_array(inputs.uniform((n, 1), 90000 + i))
        ps.set_problem(i, A, B)
        if i in sample:
            host[i] = (A, B)
    ps.run(plan_of(256, 1, 200 * 1024))
    torch.cuda.synchronize()
    for i in sample:
        A, B = host[i]
        F, X, ipiv, info = expected(int(kinds[i]), A, B)
        gF, gX, gp, ginfo = ps.get_problem(i)
        assert ginfo == info == 0
        if kinds[i] == L:
            assert np.array_equal(gF, F) and np.array_equal(gp, ipiv), i
        else:
            assert np.array_equal(np.tril(gF), np.tril(F)), i
        assert np.array_equal(gX, X), i


def test_batched_argument_errors():
    plan = plan_of(256, 1, 48 * 1024)
    with pytest.raises(binding.PositError) as e:
        binding.posit_factor_solve_batched(-1, None, None, 1, 1, plan, None)
    assert e.value.code == -1
    with pytest.raises(binding.PositError) as e:
        binding.posit_factor_solve_batched(1, None, None, 1, 1, plan, None)
    assert e.value.code == -2
    with pytest.raises(binding.PositError) as e:
        binding.posit_factor_solve_batched(0, None, None, 1, 1, plan_of(100, 1, 0), None)
    assert e.value.code == -6
    binding.posit_factor_solve_batched(0, None, None, 0, 0, plan, None)


def test_native_autotune_picks_the_fastest_and_leaves_inputs():
    """posit_autotune times every candidate on copies: the caller's arrays
    are unchanged, an invalid plan is reported as -1, the plan returned is
    the fastest one, and it gives the oracle's bits."""
    rng = np.random.default_rng(9)
    count = 24
    ns = rng.integers(8, 160, count)
    kinds = np.array([(L, C, CU)[i % 3] for i in range(count)], np.int32)
    nrhs = rng.integers(0, 3, count)
    ps, host = make_set(kinds, ns, nrhs, 300)
    A0, B0 = ps.A.clone(), ps.B.clone()
    cands = [plan_of(*p) for p in PLANS] + [plan_of(33, 1, 0)]
    best, times = binding.posit_autotune(ps.count, ps.desc, ps.order, ps.max_n, ps.max_nrhs,
                                         cands, reps=2)
    torch.cuda.synchronize()
    assert times[-1] == -1 and all(t > 0 for t in times[:-1]), times
    got = (best.threads, best.ctas_per_sm, best.smem_bytes)
    assert got in PLANS
    assert times[PLANS.index(got)] == min(times[:-1])
    assert torch.equal(ps.A, A0) and torch.equal(ps.B, B0)
    ps.run(best)
    torch.cuda.synchronize()
    check(ps, host)


def test_graph_captured_launch_replays_bit_exact():
    """The batched launch as it is timed: captured once in a CUDA graph, then
    replayed twice, each time from the restored inputs; both replays equal
    the oracle problem by problem (LU, lower and upper Cholesky, 1-3 RHS)."""
    rng = np.random.default_rng(17)
    count = 48
    ns = np.concatenate([[1, 2, 160, 257], rng.integers(3, 130, count - 4)])
    kinds = np.array([(L, C, CU)[i % 3] for i in range(count)], np.int32)
    nrhs = rng.integers(1, 4, count)
    ps, host = make_set(kinds, ns, nrhs, 700)
    plan = plan_of(256, 2, 96 * 1024)
    ws = torch.empty(ps.workspace_bytes(plan), dtype=torch.uint8, device="cuda")
    snap = ps.snapshot()
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    with torch.cuda.graph(g, stream=side):
        ps.run(plan, ws, stream=side)
    for rep in range(2):
        ps.restore(snap)
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        check(ps, host)
