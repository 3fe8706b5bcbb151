"""GPU parity of posit_rgetrf / posit_rpotrf / posit_rgetrs / posit_rpotrs
against the CPU oracle, word for word (factors, pivots, info, solutions).

Up to n = 2048 the whole factorisation is compared with the oracle's
unblocked algorithm.  At n = 8192 the factors are checked element by element
on a sample: every sampled output must equal what its defining recurrence
gives (in the oracle's arithmetic) from the original matrix and the other
factor entries it depends on, and sampled pivot steps must pick the largest
|a|.  If every element passed, the factors would equal the oracle's by
induction over the operation order."""
import numpy as np
import pytest
import torch

import oracle
from paper_2401_14117_gb300 import binding, inputs
from tests.gpu_util import DEV, from_dev, mixed_words, to_dev

pytestmark = pytest.mark.gpu

ONE, MONE = 0x40000000, 0xC0000000


def words(shape, seed):
    return oracle.from_double_array(inputs.uniform(shape, seed))


def spd_words(n, seed):
    return oracle.from_double_array(inputs.spd(n, seed, device=DEV if n > 512 else None))


def gpu_getrf(A):
    m, n = A.shape
    dA = to_dev(A)
    ipiv = torch.zeros(max(1, min(m, n)), dtype=torch.int32, device=DEV)
    info = torch.full((1,), -7, dtype=torch.int32, device=DEV)
    binding.posit_rgetrf(m, n, dA, m, ipiv, info)
    torch.cuda.synchronize()
    return from_dev(dA), ipiv.cpu().numpy()[: min(m, n)], int(info.item())


def gpu_potrf(A, uplo="L"):
    n = A.shape[0]
    dA = to_dev(A)
    info = torch.full((1,), -7, dtype=torch.int32, device=DEV)
    binding.posit_rpotrf(uplo, n, dA, n, info)
    torch.cuda.synchronize()
    return from_dev(dA), int(info.item())


def assert_same(got, want, what=""):
    bad = np.argwhere(np.asarray(got) != np.asarray(want))
    assert bad.size == 0, f"{what}: {len(bad)} words differ, first at {bad[:3].tolist()}"


# ----------------------------------------------------------------- Rgetrf
@pytest.mark.parametrize("m,n", [(1, 1), (5, 5), (64, 64), (300, 300), (257, 513),
                                 (600, 230), (230, 600), (700, 700)])
def test_getrf_matches_oracle(m, n):
    A = words((m, n), m * 1000 + n)
    F, ipiv, info = gpu_getrf(A)
    Fo, ipo, info_o = oracle.rgetrf(A)
    assert_same(F, Fo, "factors")
    assert np.array_equal(ipiv, ipo) and info == info_o


@pytest.mark.parametrize("case", ["wilkinson", "scaled_up", "scaled_down"])
def test_getrf_values_leaving_the_band(case):
    """The trailing Rgemm and the U12 trsm round without the long-regime test
    while their values have scales in [-40, 40]: Wilkinson's growth matrix
    (|u| doubles every column, so the values leave the band part-way and
    end saturated at maxpos), and
    matrices scaled by 2^45 and 2^-45 (outside it from the start)."""
    n = 600
    if case == "wilkinson":
        A64 = np.eye(n) - np.tril(np.ones((n, n)), -1)
        A64[:, -1] = 1.0
    else:
        A64 = inputs.uniform((n, n), 42) * 2.0 ** (45 if case == "scaled_up" else -45)
    A = oracle.from_double_array(A64)
    F, ipiv, info = gpu_getrf(A)
    Fo, ipo, info_o = oracle.rgetrf(A)
    assert_same(F, Fo, "factors")
    assert np.array_equal(ipiv, ipo) and info == info_o


def test_getrf_zero_column_and_nar():
    A = words((300, 300), 5)
    A[:, 7] = 0
    A[:, 260] = 0
    F, ipiv, info = gpu_getrf(A)
    Fo, ipo, info_o = oracle.rgetrf(A)
    assert info == info_o == 8
    assert_same(F, Fo, "zero columns")
    assert np.array_equal(ipiv, ipo)
    B = words((40, 40), 6)
    B[10, 0] = 0x80000000
    F, ipiv, info = gpu_getrf(B)
    Fo, ipo, info_o = oracle.rgetrf(B)
    assert_same(F, Fo, "NaR")
    assert np.array_equal(ipiv, ipo)


def test_getrf_integer_ties():
    """Small-integer matrix: many exactly equal |a| (the pivot tie rule) and
    exact zeros produced by cancellation."""
    rng = np.random.default_rng(7)
    A = oracle.from_double_array(rng.integers(-2, 3, size=(290, 290)).astype(float))
    F, ipiv, info = gpu_getrf(A)
    Fo, ipo, info_o = oracle.rgetrf(A)
    assert_same(F, Fo, "ties")
    assert np.array_equal(ipiv, ipo) and info == info_o


def test_getrf_workload_2048_full():
    n = 2048
    A = words((n, n), inputs.SEED_BASE + 2)
    F, ipiv, info = gpu_getrf(A)
    Fo, ipo, info_o = oracle.rgetrf(A)
    assert_same(F, Fo, "2048")
    assert np.array_equal(ipiv, ipo) and info == info_o == 0


def _perm_from_ipiv(ipiv):
    rows = np.arange(ipiv.size)
    for i, p in enumerate(ipiv):
        rows[i], rows[p - 1] = rows[p - 1], rows[i]
    return rows  # final position i holds original row rows[i]


def test_getrf_workload_8192_sampled():
    n = 8192
    A = words((n, n), inputs.SEED_BASE + 3)
    F, ipiv, info = gpu_getrf(A)
    assert info == 0
    Ap = A[_perm_from_ipiv(ipiv), :]
    rng = np.random.default_rng(8192)
    idx = np.concatenate([[0, n - 1, 4095, 4096], rng.integers(0, n, 60)])
    kdx = np.concatenate([[0, n - 1, 4096, 4095], rng.integers(0, n, 60)])
    for i, k in zip(idx, kdx):
        K = min(i, k)
        c = oracle.rgemm("N", "N", MONE, F[i:i + 1, :K], F[:K, k:k + 1], ONE, Ap[i:i + 1, k:k + 1])
        if i > k:
            r = oracle.div(ONE, int(F[k, k]))
            c = np.array([[oracle.mul(int(c[0, 0]), r)]], np.uint32)
        assert int(c[0, 0]) == int(F[i, k]), (i, k)
    # sampled pivot steps: the row that ends at position k had the largest |a|
    def absw(w):
        w = w.astype(np.uint32)
        return np.where(w >> 31 == 1, (~w + np.uint32(1)).astype(np.uint32), w)
    for k in (0, 1, 255, 256, 4000, n - 2):
        vals = oracle.rgemm("N", "N", MONE, F[k:, :k], F[:k, k:k + 1], ONE, Ap[k:, k:k + 1])[:, 0]
        assert absw(vals[:1])[0] >= absw(vals).max(), k
        assert int(vals[0]) == int(F[k, k])


def _factor_record(tag):
    """The oracle's n = 8192 factorisation record for `tag` (lu / chol):
    digests, info and per-column CRC-32s (tests/golden/factor8192.txt)."""
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "factor8192.txt")
    rec, crcs = {}, {}
    with open(path) as f:
        for ln in f:
            if ln.startswith("#") or not ln.strip():
                continue
            t, key, *rest = ln.split()
            if t != tag:
                continue
            if key == "crc32":
                c0 = int(rest[0])
                for q, h in enumerate(rest[1:]):
                    crcs[c0 + q] = int(h, 16)
            else:
                rec[key] = rest[0]
    return rec, crcs


@pytest.mark.parametrize("kind", ["lu", "chol"])
def test_factor_8192_full_against_oracle_record(kind):
    """n = 8192, every word: the GPU factors, pivots and info against the CPU
    oracle's unblocked factorisation of the same matrix (Sec. 5.2), stored as
    digests by tests/golden/make_factor8192.py; on a mismatch the first
    differing column is located through the per-column CRC-32s."""
    from tests.golden import make_factor8192 as mf
    rec, crcs = _factor_record(kind)
    A = mf.lu_input() if kind == "lu" else mf.chol_input()
    assert mf.sha(A) == rec["input_sha256"], "the regenerated input is not the recorded one"
    if kind == "lu":
        F, ipiv, info = gpu_getrf(A)
        assert mf.sha(ipiv.astype(np.int32)) == rec["ipiv_sha256"], "pivots differ"
    else:
        F, info = gpu_potrf(A, "L")
    assert info == int(rec["info"])
    if mf.sha(F) != rec["factor_sha256"]:
        got = mf.column_crcs(F)
        bad = [j for j in range(len(got)) if got[j] != crcs[j]]
        pytest.fail(f"{kind} 8192: {len(bad)} columns differ from the oracle, first {bad[:5]}")


# ----------------------------------------------------------------- Rpotrf
@pytest.mark.parametrize("n", [1, 5, 64, 255, 300, 513, 700])
@pytest.mark.parametrize("uplo", ["L", "U"])
def test_potrf_matches_oracle(n, uplo):
    A = spd_words(n, n)
    F, info = gpu_potrf(A, uplo)
    Fo, info_o = oracle.rpotrf(A, uplo=uplo)
    assert info == info_o == 0
    assert_same(F, Fo, "factor")  # the other triangle is untouched on both


@pytest.mark.parametrize("uplo", ["L", "U"])
def test_potrf_not_positive_definite(uplo):
    n = 300
    A = spd_words(n, 3)
    A[270, 270] = oracle.from_double(-1.0)  # fails in the second panel
    F, info = gpu_potrf(A, uplo)
    Fo, info_o = oracle.rpotrf(A, uplo=uplo)
    assert info == info_o == 271
    tri = np.tril if uplo == "L" else np.triu
    cols = slice(0, info - 1)
    if uplo == "L":
        assert_same(np.tril(F)[:, cols], np.tril(Fo)[:, cols], "columns before the failure")
    else:
        assert_same(np.triu(F)[cols, :], np.triu(Fo)[cols, :], "rows before the failure")
    A2 = spd_words(40, 4)
    A2[0, 0] = 0
    F, info = gpu_potrf(A2, uplo)
    assert info == 1 and F[0, 0] == 0


def test_potrf_workload_2048_full():
    n = 2048
    A = spd_words(n, inputs.SEED_BASE + 4)
    F, info = gpu_potrf(A, "L")
    Fo, info_o = oracle.rpotrf(A, uplo="L")
    assert info == info_o == 0
    assert_same(F, Fo, "2048")


def test_potrf_workload_8192_sampled():
    n = 8192
    A = spd_words(n, inputs.SEED_BASE + 5)
    F, info = gpu_potrf(A, "L")
    assert info == 0
    assert np.array_equal(np.triu(F, 1), np.triu(A, 1))  # upper triangle untouched
    rng = np.random.default_rng(88)
    js = np.concatenate([[0, 1, 255, 256, n - 1], rng.integers(0, n, 60)])
    for j in js:
        i = int(rng.integers(j, n))
        for (r, c) in ((j, j), (i, j)):
            d = oracle.rgemm("N", "T", MONE, F[r:r + 1, :c], F[c:c + 1, :c], ONE, A[r:r + 1, c:c + 1])
            d = int(d[0, 0])
            if r == c:
                want = oracle.sqrt(d)
            else:
                want = oracle.mul(d, oracle.div(ONE, int(F[c, c])))
            assert want == int(F[r, c]), (r, c)


# ----------------------------------------------------------------- solves
@pytest.mark.parametrize("trans", ["N", "T"])
@pytest.mark.parametrize("n,nrhs", [(1, 1), (7, 2), (300, 1), (300, 9), (513, 3)])
def test_getrs_matches_oracle(trans, n, nrhs):
    A = words((n, n), 10 + n)
    Fo, ipo, _ = oracle.rgetrf(A)
    B = words((n, nrhs), 20 + n)
    want = oracle.rgetrs(Fo, ipo, B, trans=trans)
    dF, dB = to_dev(Fo), to_dev(B)
    dp = torch.from_numpy(ipo.astype(np.int32)).to(DEV)
    binding.posit_rgetrs(trans, n, nrhs, dF, n, dp, dB, n)
    torch.cuda.synchronize()
    assert_same(from_dev(dB), want, "getrs")


@pytest.mark.parametrize("uplo", ["L", "U"])
@pytest.mark.parametrize("n,nrhs", [(1, 1), (7, 2), (300, 1), (300, 9), (513, 3)])
def test_potrs_matches_oracle(uplo, n, nrhs):
    A = spd_words(n, 30 + n)
    Fo, _ = oracle.rpotrf(A, uplo=uplo)
    B = words((n, nrhs), 40 + n)
    want = oracle.rpotrs(Fo, B, uplo=uplo)
    dF, dB = to_dev(Fo), to_dev(B)
    binding.posit_rpotrs(uplo, n, nrhs, dF, n, dB, n)
    torch.cuda.synchronize()
    assert_same(from_dev(dB), want, "potrs")


def _chain_factor(case, n, rng):
    """A factor whose dot-form backward solve (L^T x = y) runs its serial chain
    through every path of the chain addition: 'range' -- random words of any
    scale (long regimes, saturation), 'cancel' -- entries +-2^j with small
    right-hand sides, so that sums cancel one or many bits or vanish, 'edges'
    -- magnitudes near 2^+-106, where the result scale meets the long-regime
    band, 'high' / 'low' -- entries of size 1 with right-hand sides near 2^55 /
    2^-74, so that the running sums cross the scales 56 and -75 where runs of
    links leave the signed fast form.  Zeros are sprinkled in; U (for Rgetrs) is
    the identity."""
    if case in ("high", "low"):
        v = rng.uniform(0.25, 2.0, size=(n, n)) * rng.choice([-1.0, 1.0], size=(n, n))
        F = oracle.from_double_array(v)
    elif case == "range":
        F = mixed_words(rng, n * n).reshape(n, n)
        F[F == 0x80000000] = ONE
    elif case == "cancel":
        v = np.ldexp(rng.choice([-1.0, 1.0], size=(n, n)), rng.integers(-3, 1, size=(n, n)))
        F = oracle.from_double_array(v)
    else:
        e = rng.choice([-1, 1], size=(n, n)) * rng.integers(100, 111, size=(n, n))
        v = np.ldexp(rng.uniform(1.0, 2.0, size=(n, n)) * rng.choice([-1.0, 1.0], size=(n, n)),
                     e // 2)
        F = oracle.from_double_array(v)
    F[rng.random((n, n)) < 0.05] = 0
    d = np.abs(oracle.to_double_array(np.diag(F)))
    np.fill_diagonal(F, oracle.from_double_array(np.where(d > 0, d, 1.0)))
    return F


@pytest.mark.parametrize("case", ["range", "cancel", "edges", "high", "low"])
@pytest.mark.parametrize("kind", ["getrs_T", "potrs_L"])
def test_dot_form_chain_paths(case, kind):
    n, nrhs = 300, 3
    rng = np.random.default_rng(77 + len(case))
    F = _chain_factor(case, n, rng)
    if case == "range":
        B = mixed_words(rng, n * nrhs).reshape(n, nrhs)
        B[B == 0x80000000] = 0
    elif case == "cancel":
        B = oracle.from_double_array(rng.uniform(-0.01, 0.01, size=(n, nrhs)))
    elif case in ("high", "low"):
        B = oracle.from_double_array(
            np.ldexp(rng.uniform(-2, 2, size=(n, nrhs)), 55 if case == "high" else -74))
    else:
        B = oracle.from_double_array(np.ldexp(rng.uniform(-2, 2, size=(n, nrhs)), 106))
    B[rng.random((n, nrhs)) < 0.05] = 0
    B[n // 2, 2] = 0x80000000  # a NaR right-hand side entry
    dF, dB = to_dev(F), to_dev(B)
    if kind == "getrs_T":
        Fu = F.copy()
        Fu[np.triu_indices(n, 1)] = 0
        np.fill_diagonal(Fu, ONE)  # U = I, so U^T y = b leaves y = b
        ipiv = np.arange(1, n + 1, dtype=np.int32)
        want = oracle.rgetrs(Fu, ipiv, B, trans="T")
        dF = to_dev(Fu)
        binding.posit_rgetrs("T", n, nrhs, dF, n, torch.from_numpy(ipiv).to(DEV), dB, n)
    else:
        want = oracle.rpotrs(F, B, uplo="L")
        binding.posit_rpotrs("L", n, nrhs, dF, n, dB, n)
    torch.cuda.synchronize()
    assert_same(from_dev(dB), want, f"{kind} {case}")


def test_solve_workload_2048():
    """Rgetrs / Rpotrs with 1 RHS, b = A (1/sqrt n) in FP64 (Sec. 5.1), on the
    oracle's factors of the n = 2048 workload matrices, every word."""
    n = 2048
    A64 = inputs.uniform((n, n), inputs.SEED_BASE + 6)
    A = oracle.from_double_array(A64)
    b = oracle.from_double_array(inputs.rhs(A64)).reshape(n, 1)
    Fo, ipo, _ = oracle.rgetrf(A)
    want = oracle.rgetrs(Fo, ipo, b)
    dF, dB = to_dev(Fo), to_dev(b)
    dp = torch.from_numpy(ipo.astype(np.int32)).to(DEV)
    binding.posit_rgetrs("N", n, 1, dF, n, dp, dB, n)
    torch.cuda.synchronize()
    assert_same(from_dev(dB), want, "getrs workload")
    S64 = inputs.spd(n, inputs.SEED_BASE + 7, device=DEV)
    S = oracle.from_double_array(S64)
    bs = oracle.from_double_array(inputs.rhs(S64)).reshape(n, 1)
    Fs, _ = oracle.rpotrf(S)
    want = oracle.rpotrs(Fs, bs)
    dF, dB = to_dev(Fs), to_dev(bs)
    binding.posit_rpotrs("L", n, 1, dF, n, dB, n)
    torch.cuda.synchronize()
    assert_same(from_dev(dB), want, "potrs workload")


@pytest.mark.parametrize("kind,nrhs", [("getrs", 1), ("potrs", 1), ("getrs", 8), ("potrs_U", 8)])
def test_solve_8192_synthetic_factors(kind, nrhs):
    """n = 8192: the solve alone on seeded factor-shaped matrices (the oracle
    cannot factor n = 8192 in test time): unit-lower L and upper U (or L / U
    with positive diagonal) with uniform entries and a random valid pivot
    vector.  With 8 right-hand sides the eight pipelines share one launch,
    so some helper warps bring two blocks up to date."""
    n = 8192
    rng = np.random.default_rng(8192)
    F = words((n, n), inputs.SEED_BASE + 8)
    d = np.arange(n)
    F[d, d] = oracle.from_double_array(rng.uniform(1.0, 2.0, n))
    b = words((n, nrhs), inputs.SEED_BASE + 9)
    dF, dB = to_dev(F), to_dev(b)
    if kind == "getrs":
        ipiv = (d + rng.integers(0, 16, n)).clip(max=n - 1).astype(np.int32) + 1
        want = oracle.rgetrs(F, ipiv, b)
        binding.posit_rgetrs("N", n, nrhs, dF, n, torch.from_numpy(ipiv).to(DEV), dB, n)
    elif kind == "potrs_U":
        want = oracle.rpotrs(F, b, uplo="U")
        binding.posit_rpotrs("U", n, nrhs, dF, n, dB, n)
    else:
        want = oracle.rpotrs(F, b)
        binding.posit_rpotrs("L", n, nrhs, dF, n, dB, n)
    torch.cuda.synchronize()
    assert_same(from_dev(dB), want, kind)


def test_argument_errors():
    with pytest.raises(binding.PositError) as e:
        binding.posit_rgetrf(-1, 1, None, 1, None, None)
    assert e.value.code == -1
    with pytest.raises(binding.PositError) as e:
        binding.posit_rpotrf("X", 1, None, 1, None)
    assert e.value.code == -1
    with pytest.raises(binding.PositError) as e:
        binding.posit_rgetrs("N", 4, 1, None, 2, None, None, 4)
    assert e.value.code == -5
    info = torch.zeros(1, dtype=torch.int32, device=DEV)
    binding.posit_rgetrf(0, 5, None, 1, None, info)
    binding.posit_rpotrf("L", 0, None, 1, info)
    assert int(info.item()) == 0


@pytest.mark.parametrize("case", ["tiny_pivots", "huge_entries", "nar_entry", "in_band"])
@pytest.mark.parametrize("kind", ["getrs_N", "getrs_T", "potrs_L", "potrs_U"])
def test_solve_fast_path_switches(case, kind):
    """The wavefront solves run on in-band straight-line arithmetic while the
    tiles, the unknowns and the running sums allow it, and switch to the
    general arithmetic where they do not: a pivot of 2^-45 mid-block makes an
    unknown leave the band (the step is redone), entries of 2^50 make a tile
    leave it, a NaR entry poisons the rows below it.  Every case must give the
    oracle's words, on factor-shaped matrices of 300 rows (10 blocks, ragged
    tail) with 2 right-hand sides."""
    n, nrhs = 300, 2
    rng = np.random.default_rng(4242 + len(case) + len(kind))
    F = words((n, n), 777 + len(case))
    d = np.arange(n)
    F[d, d] = oracle.from_double_array(rng.uniform(1.0, 2.0, n))
    if case == "tiny_pivots":
        for i in (37, 70, 203, 299):
            F[i, i] = oracle.from_double(2.0 ** -45)
    elif case == "huge_entries":
        for (i, k) in ((150, 20), (20, 150), (260, 100), (100, 260)):
            F[i, k] = oracle.from_double(2.0 ** 50)
    elif case == "nar_entry":
        F[180, 60] = 0x80000000
        F[60, 180] = 0x80000000
    B = words((n, nrhs), 901 + len(kind))
    dF, dB = to_dev(F), to_dev(B)
    if kind.startswith("getrs"):
        trans = kind[-1]
        ipiv = (d + rng.integers(0, 8, n)).clip(max=n - 1).astype(np.int32) + 1
        want = oracle.rgetrs(F, ipiv, B, trans=trans)
        binding.posit_rgetrs(trans, n, nrhs, dF, n, torch.from_numpy(ipiv).to(DEV), dB, n)
    else:
        uplo = kind[-1]
        want = oracle.rpotrs(F, B, uplo=uplo)
        binding.posit_rpotrs(uplo, n, nrhs, dF, n, dB, n)
    torch.cuda.synchronize()
    assert_same(from_dev(dB), want, f"{kind} {case}")

@pytest.mark.parametrize("kind", ["getrs_N", "getrs_T", "potrs_L"])
def test_solve_global_memory_fallbacks(kind, monkeypatch):
    """Columns too long for one CTA's shared memory (past about 27k rows for the
    dot-form solve, 57k for the row swaps) are solved and swapped by one-thread
    kernels in global memory.  POSIT_SOLVE_SMEM_LIMIT caps the shared memory
    the solve kernels may take, so those kernels run here at n = 300 (ragged,
    2 right-hand sides) and must give the oracle's words."""
    monkeypatch.setenv("POSIT_SOLVE_SMEM_LIMIT", "1024")
    n, nrhs = 300, 2
    rng = np.random.default_rng(3030 + len(kind))
    if kind.startswith("getrs"):
        A = words((n, n), 3100)
        F, ipiv, _ = oracle.rgetrf(A)
        B = words((n, nrhs), 3101)
        want = oracle.rgetrs(F, ipiv, B, trans=kind[-1])
        dF, dB = to_dev(F), to_dev(B)
        dp = torch.from_numpy(ipiv.astype(np.int32)).to(DEV)
        binding.posit_rgetrs(kind[-1], n, nrhs, dF, n, dp, dB, n)
    else:
        F, _ = oracle.rpotrf(spd_words(n, 3102), uplo="L")
        B = words((n, nrhs), 3103)
        B[rng.integers(0, n), 1] = 0x80000000  # a NaR right-hand side entry
        want = oracle.rpotrs(F, B, uplo="L")
        dF, dB = to_dev(F), to_dev(B)
        binding.posit_rpotrs("L", n, nrhs, dF, n, dB, n)
    torch.cuda.synchronize()
    assert_same(from_dev(dB), want, kind)
