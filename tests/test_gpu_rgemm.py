"""GPU parity of posit_rgemm against the CPU oracle, word for word.

Small and ragged sizes are compared in full; the full-size workloads
(M = N = K in {1024, 4096, 8192} and the 8192 x 8192 x 256 trailing update)
are compared on sampled output elements, each recomputed by the oracle from
its row of op(A) and column of op(B) -- the same per-element order."""
import itertools

import numpy as np
import pytest
import torch

import oracle
from paper_2401_14117_gb300 import binding, inputs
from tests.gpu_util import DEV, from_dev, mixed_words, to_dev

pytestmark = pytest.mark.gpu

ONE, MONE = 0x40000000, 0xC0000000


def words(shape, seed, kind="uniform"):
    x = inputs.scaled(shape, seed) if kind == "scaled" else inputs.uniform(shape, seed)
    return oracle.from_double_array(x)


def run_gpu(ta, tb, alpha, A, B, beta, C):
    m, n = C.shape
    k = A.shape[0] if ta == "T" else A.shape[1]
    dA, dB, dC = to_dev(A), to_dev(B), to_dev(C)
    binding.posit_rgemm(ta, tb, m, n, k, alpha, dA, max(1, A.shape[0]), dB, max(1, B.shape[0]),
                        beta, dC, max(1, m))
    torch.cuda.synchronize()
    return from_dev(dC)


def assert_same(got, want):
    bad = np.argwhere(got != want)
    assert bad.size == 0, f"{len(bad)} words differ, first at {bad[:3].tolist()}"


@pytest.mark.parametrize("ta,tb", list(itertools.product("NT", "NT")))
@pytest.mark.parametrize("alpha,beta", [(ONE, 0), (MONE, ONE), (0x3C000000, 0xB4000000)])
def test_ragged_all_transposes(ta, tb, alpha, beta):
    m, n, k = 300, 200, 57
    A = words((m, k) if ta == "N" else (k, m), 1)
    B = words((k, n) if tb == "N" else (n, k), 2)
    C = words((m, n), 3)
    assert_same(run_gpu(ta, tb, alpha, A, B, beta, C),
                oracle.rgemm(ta, tb, alpha, A, B, beta, C))


@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (1, 70, 3), (129, 1, 300), (128, 64, 16),
                                   (257, 130, 33), (64, 513, 17)])
def test_shapes_and_tails(m, n, k):
    A, B, C = words((m, k), m), words((k, n), n), words((m, n), k)
    assert_same(run_gpu("N", "N", ONE, A, B, ONE, C), oracle.rgemm("N", "N", ONE, A, B, ONE, C))


@pytest.mark.parametrize("ta,tb", list(itertools.product("NT", "NT")))
def test_wide_and_narrow_tiles_full(ta, tb):
    """Launches that fill a wave of 128 x 64 tiles use them; smaller ones use
    64 x 64 tiles.  Both, compared in full, with ragged edges and a C that
    is read (beta = 1) and a NaR in op(A)."""
    for m, n, k in ((2048 + 37, 1216 + 5, 33), (1000 + 7, 600 + 3, 29)):
        A = words((m, k) if ta == "N" else (k, m), m + 11)
        B = words((k, n) if tb == "N" else (n, k), m + 12)
        C = words((m, n), m + 13)
        A[(5, 3) if ta == "N" else (3, 5)] = 0x80000000
        assert_same(run_gpu(ta, tb, MONE, A, B, ONE, C), oracle.rgemm(ta, tb, MONE, A, B, ONE, C))


@pytest.mark.parametrize("ta,tb", list(itertools.product("NT", "NT")))
@pytest.mark.parametrize("m", [2048, 2500, 4223])
def test_grouped_launch_order_and_remainder(ta, tb, m):
    """More than 16 row tiles: complete groups of 16 row tiles in the grouped
    launch order, plus (for 2500 and 4223) the remaining row tiles launched
    as a matrix of their own."""
    n, k = 70, 23
    A = words((m, k) if ta == "N" else (k, m), m + 1)
    B = words((k, n) if tb == "N" else (n, k), m + 2)
    C = words((m, n), m + 3)
    assert_same(run_gpu(ta, tb, MONE, A, B, ONE, C), oracle.rgemm(ta, tb, MONE, A, B, ONE, C))


def _pow2_words(rng, shape, lo, hi):
    """Posit words of +-(1 + f) 2^e with e uniform in [lo, hi] (exact doubles)."""
    e = rng.integers(lo, hi + 1, size=shape)
    f = rng.integers(0, 1 << 20, size=shape) / float(1 << 20)
    sgn = rng.choice([-1.0, 1.0], size=shape)
    return oracle.from_double_array(sgn * (1.0 + f) * np.exp2(e.astype(np.float64)))


@pytest.mark.parametrize("case", ["edge_high", "edge_low", "switch_mid_k", "c_out_of_band"])
def test_in_band_fast_path_edges(case):
    """The kernel skips the test for the long-regime band while all operands
    have scales in [-40, 40] and C in [-80, 80]: sums pushed to 2^88 by
    scale-40 operands, products at 2^-80 that cancel, a tile in the middle of
    K with an operand outside the bounds (the rest of K is then checked), and
    a starting C outside the bounds."""
    rng = np.random.default_rng({"edge_high": 1, "edge_low": 2, "switch_mid_k": 3,
                                 "c_out_of_band": 4}[case])
    m, n, k = 150, 70, 700
    if case == "edge_high":
        A = _pow2_words(rng, (m, k), 39, 40)
        B = oracle.from_double_array(np.abs(oracle.to_double_array(_pow2_words(rng, (k, n), 39, 40))))
        A = oracle.from_double_array(np.abs(oracle.to_double_array(A)))
        C = _pow2_words(rng, (m, n), 79, 80)
    elif case == "edge_low":
        A = _pow2_words(rng, (m, k), -40, -39)
        B = _pow2_words(rng, (k, n), -40, -39)
        C = _pow2_words(rng, (m, n), -80, -79)
    elif case == "switch_mid_k":
        A = _pow2_words(rng, (m, k), -20, 20)
        B = _pow2_words(rng, (k, n), -20, 20)
        A[17, 333] = oracle.from_double(2.0 ** 70)
        C = words((m, n), 5)
    else:
        A = _pow2_words(rng, (m, k), -20, 20)
        B = _pow2_words(rng, (k, n), -20, 20)
        C = words((m, n), 6)
        C[3, 4] = oracle.from_double(2.0 ** 90)
    assert_same(run_gpu("N", "N", ONE, A, B, ONE, C), oracle.rgemm("N", "N", ONE, A, B, ONE, C))


def test_special_values_inside_matrices():
    """Zeros, NaR, huge and tiny entries: the zero/NaR sentinels and the
    exponent-truncated rounding band inside the GEMM."""
    rng = np.random.default_rng(4)
    m, n, k = 160, 96, 80
    A = mixed_words(rng, m * k).reshape(m, k)
    B = mixed_words(rng, k * n).reshape(k, n)
    A[rng.random((m, k)) < 0.05] = 0
    B[rng.random((k, n)) < 0.05] = 0
    A[3, :] = 0x80000000
    B[:, 5] = 0
    C = mixed_words(rng, m * n).reshape(m, n)
    for alpha, beta in ((ONE, ONE), (0x7FFFFFFF, 0x00000001), (0x48000000, 0),
                        (0x80000000, ONE), (ONE, 0x80000000), (0, 0x80000000)):
        assert_same(run_gpu("N", "N", alpha, A, B, beta, C), oracle.rgemm("N", "N", alpha, A, B, beta, C))


def test_cancellation_to_exact_zero():
    m, n, k = 70, 40, 30
    A = words((m, k), 5)
    B = words((k, n), 6)
    C0 = oracle.rgemm("N", "N", ONE, A, B, 0, np.zeros((m, n), np.uint32))
    # C - A B with the same order gives intermediate exact zeros for k = 1
    A1, B1 = A[:, :1], B[:1, :]
    C1 = oracle.rgemm("N", "N", ONE, A1, B1, 0, np.zeros((m, n), np.uint32))
    assert_same(run_gpu("N", "N", MONE, A1, B1, ONE, C1), np.zeros((m, n), np.uint32))
    assert_same(run_gpu("N", "N", MONE, A, B, ONE, C0), oracle.rgemm("N", "N", MONE, A, B, ONE, C0))


def test_quick_returns_and_beta_zero_ignores_C():
    m, n, k = 50, 30, 20
    A, B = words((m, k), 7), words((k, n), 8)
    C = words((m, n), 9)
    C[0, 0] = 0x80000000
    assert_same(run_gpu("N", "N", ONE, A, B, 0, C), oracle.rgemm("N", "N", ONE, A, B, 0, C))
    A[0, 0] = 0x80000000
    assert_same(run_gpu("N", "N", 0, A, B, 0x48000000, C), oracle.rgemm("N", "N", 0, A, B, 0x48000000, C))
    # k = 0: C = beta C
    assert_same(run_gpu("N", "N", ONE, A[:, :0], B[:0, :], 0x48000000, C),
                oracle.rgemm("N", "N", ONE, A[:, :0], B[:0, :], 0x48000000, C))


def test_argument_errors():
    with pytest.raises(binding.PositError) as e:
        binding.posit_rgemm("X", "N", 1, 1, 1, ONE, None, 1, None, 1, 0, None, 1)
    assert e.value.code == -1
    with pytest.raises(binding.PositError) as e:
        binding.posit_rgemm("N", "N", 4, 1, 1, ONE, None, 2, None, 1, 0, None, 4)
    assert e.value.code == -8
    with pytest.raises(binding.PositError) as e:
        binding.posit_rgemm("N", "N", 4, 2, 1, ONE, None, 4, None, 1, 0, None, 3)
    assert e.value.code == -13
    binding.posit_rgemm("N", "N", 0, 5, 5, ONE, None, 1, None, 5, 0, None, 1)


# ------------------------------------------------------------- workloads
def test_workload_256_full():
    """Rgemm 256^3, uniform [-1,1], alpha = 1, beta = 0: every word."""
    n = 256
    A = words((n, n), inputs.SEED_BASE + 0)
    B = words((n, n), inputs.SEED_BASE + 100)
    C = np.zeros((n, n), np.uint32)
    assert_same(run_gpu("N", "N", ONE, A, B, 0, C), oracle.rgemm("N", "N", ONE, A, B, 0, C))


@pytest.mark.parametrize("kind", ["uniform", "scaled"])
def test_workload_512_full(kind):
    n = 512
    A, B = words((n, n), 11, kind), words((n, n), 12, kind)
    C = np.zeros((n, n), np.uint32)
    assert_same(run_gpu("N", "N", ONE, A, B, 0, C), oracle.rgemm("N", "N", ONE, A, B, 0, C))


def _sampled_check(m, n, k, kind, seed, alpha, beta, samples=48):
    gen = inputs.scaled if kind == "scaled" else inputs.uniform
    dev_words = {}
    for name, shape, s in (("A", (m, k), seed), ("B", (k, n), seed + 1), ("C", (m, n), seed + 2)):
        w = oracle.from_double_array(gen(shape, s))
        dev_words[name] = (w, to_dev(w))
    (A, dA), (B, dB), (C, dC) = dev_words["A"], dev_words["B"], dev_words["C"]
    binding.posit_rgemm("N", "N", m, n, k, alpha, dA, m, dB, k, beta, dC, m)
    torch.cuda.synchronize()
    rng = np.random.default_rng(seed)
    rows = np.concatenate([[0, m - 1], rng.integers(0, m, samples)])
    cols = np.concatenate([[0, n - 1], rng.integers(0, n, samples)])
    for i, j in zip(rows, cols):
        want = oracle.rgemm("N", "N", alpha, A[i:i + 1, :], B[:, j:j + 1], beta, C[i:i + 1, j:j + 1])
        got = int(dC[j, i].item()) & 0xFFFFFFFF
        assert got == int(want[0, 0]), (i, j, hex(got), hex(int(want[0, 0])))
    del dA, dB, dC


@pytest.mark.parametrize("n", [1024, 4096, 8192])
@pytest.mark.parametrize("kind", ["uniform", "scaled"])
def test_workload_square_sampled(n, kind):
    _sampled_check(n, n, n, kind, inputs.SEED_BASE + 1, ONE, 0)


@pytest.mark.parametrize("kind", ["uniform", "scaled"])
def test_workload_trailing_update_sampled(kind):
    _sampled_check(8192, 8192, 256, kind, inputs.SEED_BASE + 2, MONE, ONE)
