"""Pins for the oracle's Posit(32,2) Rgemm / Rgetrf / Rpotrf / Rgetrs / Rpotrs
(CPU only).

P7: cases whose answer is known from textbook mathematics because every
intermediate is exact (small integers, power-of-two pivots).
P8: operation-order pins -- blocked == unblocked for any block size, and a
third, Fraction-based implementation of the same loop orders at tiny sizes.
"""
import itertools
import random
from fractions import Fraction

import numpy as np
import pytest

import oracle
from tests import fraction_posit as fp

ONE, MONE = 0x40000000, 0xC0000000


def P(x):
    """Posit word of an exactly representable number (via Fractions)."""
    return fp.from_fraction(Fraction(x))


def Pm(M):
    return np.array([[P(x) for x in row] for row in M], dtype=np.uint32)


def V(W):
    return [[fp.value(int(w)) for w in row] for row in np.asarray(W)]


def rand_words(rng, shape, lo=-1.0, hi=1.0):
    return oracle.from_double_array(rng.uniform(lo, hi, size=shape))


# ------------------------------------------------------------------ P7
@pytest.mark.parametrize("ta,tb", list(itertools.product("NT", "NT")))
def test_small_integer_gemm_is_exact(ta, tb):
    rng = np.random.default_rng(7)
    m, n, k = 23, 17, 256
    A = rng.integers(-8, 9, size=(m, k) if ta == "N" else (k, m))
    B = rng.integers(-8, 9, size=(k, n) if tb == "N" else (n, k))
    C0 = rng.integers(-100, 101, size=(m, n))
    opA = A if ta == "N" else A.T
    opB = B if tb == "N" else B.T
    for alpha, beta in ((1, 0), (1, 1), (-1, 1), (2, -3)):
        want = alpha * (opA @ opB) + beta * C0  # all partial sums < 2^24
        got = oracle.rgemm(ta, tb, P(alpha), Pm(A.tolist()), Pm(B.tolist()),
                           P(beta), Pm(C0.tolist()))
        assert np.array_equal(oracle.to_double_array(got), want.astype(float))


def test_gemm_quick_returns():
    rng = np.random.default_rng(1)
    A, B, C = rand_words(rng, (5, 4)), rand_words(rng, (4, 3)), rand_words(rng, (5, 3))
    A[0, 0] = 0x80000000  # NaR in A must not be read when alpha = 0
    got = oracle.rgemm("N", "N", 0, A, B, P(2), C)
    assert np.array_equal(got, oracle.elementwise("mul", np.full(C.shape, P(2), np.uint32), C))
    C[1, 1] = 0x80000000  # beta = 0: C is not read
    got = oracle.rgemm("N", "N", ONE, A[:, 1:], B[1:, :], 0, C)
    assert got[1, 1] != 0x80000000


def _exact_lu_case(rng, n):
    """A = P L U with |l_ij| <= 1/2 and power-of-two diagonal of U, so every
    LU intermediate is exact and partial pivoting recovers P."""
    L = [[Fraction(0)] * n for _ in range(n)]
    U = [[Fraction(0)] * n for _ in range(n)]
    for i in range(n):
        L[i][i] = Fraction(1)
        for j in range(i):
            L[i][j] = Fraction(rng.choice([-2, -1, 0, 1, 2]), 4)
        U[i][i] = Fraction(rng.choice([-4, -2, -1, 1, 2, 4]))
        for j in range(i + 1, n):
            U[i][j] = Fraction(rng.randint(-3, 3))
    perm = list(range(n))
    rng.shuffle(perm)
    LU = [[sum(L[i][t] * U[t][j] for t in range(n)) for j in range(n)] for i in range(n)]
    A = [LU[perm.index(r)] for r in range(n)]  # row r of A = row perm^-1(r) of LU
    return A, L, U, perm


@pytest.mark.parametrize("n", [1, 2, 5, 16, 40])
def test_lu_of_plu_is_exact(n):
    rng = random.Random(n)
    A, L, U, perm = _exact_lu_case(rng, n)
    F, ipiv, info = oracle.rgetrf(Pm(A))
    assert info == 0
    got = V(F)
    for i in range(n):
        for j in range(n):
            want = L[i][j] if i > j else U[i][j]
            assert got[i][j] == want, (i, j)
    # applying the recorded swaps to the rows of A gives P^T A = L U
    rows = list(range(n))
    for i, p in enumerate(ipiv):
        rows[i], rows[p - 1] = rows[p - 1], rows[i]
    assert [perm.index(r) for r in rows] == list(range(n))


def test_lu_identity_permutation_singular():
    n = 6
    I = np.array([[ONE if i == j else 0 for j in range(n)] for i in range(n)], np.uint32)
    F, ipiv, info = oracle.rgetrf(I)
    assert info == 0 and np.array_equal(F, I) and list(ipiv) == list(range(1, n + 1))
    perm = [3, 0, 5, 1, 4, 2]
    Pmat = np.zeros((n, n), np.uint32)
    for i, p in enumerate(perm):
        Pmat[i, p] = ONE
    F, ipiv, info = oracle.rgetrf(Pmat)
    assert info == 0
    assert np.array_equal(np.tril(F), np.eye(n, dtype=np.uint32) * ONE)
    rows = list(range(n))
    for i, p in enumerate(ipiv):
        rows[i], rows[p - 1] = rows[p - 1], rows[i]
    assert [perm[r] for r in rows] == list(range(n))
    # a zero column 3 gives info = 4 and no swap at that step
    rng = np.random.default_rng(2)
    A = rand_words(rng, (n, n))
    A[:, 3] = 0
    F, ipiv, info = oracle.rgetrf(A)
    assert info == 4 and ipiv[3] == 4


def test_cholesky_exact_cases():
    n = 7
    D = np.zeros((n, n), np.uint32)
    for k in range(n):
        D[k, k] = P(4 ** (k - 3))
    F, info = oracle.rpotrf(D)
    assert info == 0
    assert [fp.value(int(F[k, k])) for k in range(n)] == [Fraction(2) ** (k - 3) for k in range(n)]
    # A = L L^T with power-of-two diagonal and small integer entries: exact
    rng = random.Random(3)
    for uplo in "LU":
        L = [[Fraction(0)] * n for _ in range(n)]
        for i in range(n):
            L[i][i] = Fraction(rng.choice([1, 2, 4]))
            for j in range(i):
                L[i][j] = Fraction(rng.randint(-2, 2))
        A = [[sum(L[i][t] * L[j][t] for t in range(n)) for j in range(n)] for i in range(n)]
        F, info = oracle.rpotrf(Pm(A), uplo=uplo)
        assert info == 0
        got = V(F)
        for i in range(n):
            for j in range(i + 1):
                if uplo == "L":
                    assert got[i][j] == L[i][j]
                else:
                    assert got[j][i] == L[i][j]
    # not positive definite: first bad column reported, a_jj left as is
    A = np.array(Pm([[4, 2, 0], [2, 1, 0], [0, 0, 9]]))
    F, info = oracle.rpotrf(A)
    assert info == 2 and F[1, 1] == 0  # 1 - (2/2)^2 = 0
    F, info = oracle.rpotrf(Pm([[-1, 0], [0, 1]]))
    assert info == 1 and F[0, 0] == P(-1)


def test_solves_exact():
    rng = random.Random(4)
    n = 12
    A, L, U, perm = _exact_lu_case(rng, n)
    x = [Fraction(rng.randint(-4, 4)) for _ in range(n)]
    b = [sum(A[i][j] * x[j] for j in range(n)) for i in range(n)]
    F, ipiv, info = oracle.rgetrf(Pm(A))
    sol = oracle.rgetrs(F, ipiv, np.array([[P(v)] for v in b], np.uint32))
    assert [fp.value(int(w)) for w in sol[:, 0]] == x
    At = [list(r) for r in zip(*A)]
    bt = [sum(At[i][j] * x[j] for j in range(n)) for i in range(n)]
    sol = oracle.rgetrs(F, ipiv, np.array([[P(v)] for v in bt], np.uint32), trans="T")
    assert [fp.value(int(w)) for w in sol[:, 0]] == x


# ------------------------------------------------------------------ P8
@pytest.mark.parametrize("n", [1, 2, 3, 7, 31, 64, 100])
@pytest.mark.parametrize("nb", [1, 3, 16, 64])
def test_blocked_lu_equals_unblocked(n, nb):
    rng = np.random.default_rng(100 * n + nb)
    A = rand_words(rng, (n, n))
    F0, p0, i0 = oracle.rgetrf(A)
    F1, p1, i1 = oracle.rgetrf(A, nb=nb)
    assert np.array_equal(F0, F1) and np.array_equal(p0, p1) and i0 == i1


@pytest.mark.parametrize("m,n", [(50, 20), (20, 50), (300, 300)])
def test_blocked_lu_rectangular_and_larger(m, n):
    rng = np.random.default_rng(m + n)
    A = rand_words(rng, (m, n))
    F0, p0, _ = oracle.rgetrf(A)
    for nb in (3, 64, 256):
        F1, p1, _ = oracle.rgetrf(A, nb=nb)
        assert np.array_equal(F0, F1) and np.array_equal(p0, p1)


def _spd_words(rng, n):
    G = rng.standard_normal((n, n))
    return oracle.from_double_array(G @ G.T / n + np.eye(n))


@pytest.mark.parametrize("n", [1, 2, 5, 33, 64, 130])
@pytest.mark.parametrize("uplo", "LU")
def test_blocked_cholesky_equals_unblocked(n, uplo):
    rng = np.random.default_rng(n)
    A = _spd_words(rng, n)
    F0, i0 = oracle.rpotrf(A, uplo=uplo)
    for nb in (1, 3, 64):
        F1, i1 = oracle.rpotrf(A, uplo=uplo, nb=nb)
        assert i0 == i1 == 0 and np.array_equal(F0, F1)


def test_cholesky_upper_is_transposed_lower():
    rng = np.random.default_rng(9)
    A = _spd_words(rng, 40)
    FL, _ = oracle.rpotrf(A, "L")
    FU, _ = oracle.rpotrf(A, "U")
    assert np.array_equal(np.tril(FL), np.tril(FU.T))


@pytest.mark.parametrize("ta,tb", list(itertools.product("NT", "NT")))
def test_gemm_matches_fraction_implementation(ta, tb):
    rng = np.random.default_rng(11)
    m, n, k = 4, 3, 6
    A = rand_words(rng, (m, k) if ta == "N" else (k, m), -3, 3)
    B = rand_words(rng, (k, n) if tb == "N" else (n, k), -3, 3)
    C = rand_words(rng, (m, n))
    for alpha, beta in ((ONE, 0), (MONE, ONE), (P(0.75), P(-1.5))):
        got = oracle.rgemm(ta, tb, alpha, A, B, beta, C)
        want = fp.rgemm(ta, tb, alpha, A.tolist(), B.tolist(), beta, C.tolist())
        assert got.tolist() == want


@pytest.mark.parametrize("n", [1, 4, 9])
def test_lu_and_solve_match_fraction_implementation(n):
    rng = np.random.default_rng(20 + n)
    A = rand_words(rng, (n, n))
    F, ipiv, info = oracle.rgetrf(A)
    F2, ipiv2, info2 = fp.rgetrf(A.tolist())
    assert F.tolist() == F2 and list(ipiv) == ipiv2 and info == info2
    b = rand_words(rng, (n,))
    x = oracle.rgetrs(F, ipiv, b.reshape(-1, 1))
    assert x[:, 0].tolist() == fp.rgetrs(F2, ipiv2, b.tolist())


@pytest.mark.parametrize("n", [1, 4, 9])
def test_cholesky_and_solve_match_fraction_implementation(n):
    rng = np.random.default_rng(40 + n)
    A = _spd_words(rng, n)
    F, info = oracle.rpotrf(A)
    F2, info2 = fp.rpotrf_lower(A.tolist())
    assert info == info2 == 0
    assert np.tril(F).tolist() == np.tril(np.array(F2, np.uint32)).tolist()
    b = rand_words(rng, (n,))
    x = oracle.rpotrs(F, b.reshape(-1, 1))
    assert x[:, 0].tolist() == fp.rpotrs_lower(F2, b.tolist())


def _dirty_words(rng, n):
    """Random words spread over several binades, so that sums of products
    round differently in different orders (exact-integer systems cannot see
    the order)."""
    return oracle.from_double_array(rng.uniform(-1, 1, size=n) * 2.0 ** rng.integers(-6, 7, size=n))


@pytest.mark.parametrize("n", [2, 5, 9])
def test_lu_transposed_solve_matches_fraction_implementation(n):
    """O4 with trans = T: U^T forward (k ascending, then divide), unit L^T
    backward (k ascending), swaps in reverse -- word for word on random
    words, where the summation order decides the bits."""
    rng = np.random.default_rng(60 + n)
    A = rand_words(rng, (n, n))
    F, ipiv, _ = oracle.rgetrf(A)
    for rep in range(3):
        b = _dirty_words(rng, n)
        x = oracle.rgetrs(F, ipiv, b.reshape(-1, 1), trans="T")
        assert x[:, 0].tolist() == fp.rgetrs_trans(F.tolist(), list(ipiv), b.tolist())


@pytest.mark.parametrize("n", [2, 5, 9])
def test_upper_cholesky_solve_matches_fraction_implementation(n):
    """O5 with uplo = U: U^T forward (k ascending, then divide), U backward
    (k descending, then divide) on the oracle's upper factor."""
    rng = np.random.default_rng(80 + n)
    A = _spd_words(rng, n)
    F, info = oracle.rpotrf(A, uplo="U")
    assert info == 0
    for rep in range(3):
        b = _dirty_words(rng, n)
        x = oracle.rpotrs(F, b.reshape(-1, 1), uplo="U")
        assert x[:, 0].tolist() == fp.rpotrs_upper(F.tolist(), b.tolist())


def _solve_orders_differ(seed_base, solver, wrong, make):
    """True when, on one of a few seeded systems, the loop order `wrong`
    gives other words than `solver`: the pins above can see the order."""
    for s in range(8):
        rng = np.random.default_rng(seed_base + s)
        F, extra, b = make(rng)
        if solver(F, extra, b) != wrong(F, extra, b):
            return True
    return False


def test_solve_pins_are_order_sensitive():
    """The Fraction restatements of the transposed LU solve and the upper
    Cholesky solve, with one inner loop reversed, give different words on
    these inputs -- so the word-for-word pins above would fail an oracle
    with that loop order."""
    n = 9

    def lu_case(rng):
        F, ipiv, _ = oracle.rgetrf(rand_words(rng, (n, n)))
        return F.tolist(), list(ipiv), _dirty_words(rng, n).tolist()

    def lu_wrong(LU, ipiv, b):  # L^T backward with k descending
        b = b[:]
        for i in range(n):
            for k in range(i):
                b[i] = fp.sub(b[i], fp.mul(LU[k][i], b[k]))
            b[i] = fp.div(b[i], LU[i][i])
        for i in range(n - 1, -1, -1):
            for k in range(n - 1, i, -1):
                b[i] = fp.sub(b[i], fp.mul(LU[k][i], b[k]))
        for i in range(n - 1, -1, -1):
            p = ipiv[i] - 1
            b[i], b[p] = b[p], b[i]
        return b

    assert _solve_orders_differ(500, lambda F, p, b: fp.rgetrs_trans(F, p, b), lu_wrong, lu_case)

    def chol_case(rng):
        F, _ = oracle.rpotrf(_spd_words(rng, n), uplo="U")
        return F.tolist(), None, _dirty_words(rng, n).tolist()

    def chol_wrong(U, _, b):  # U backward with k ascending
        b = b[:]
        for i in range(n):
            for k in range(i):
                b[i] = fp.sub(b[i], fp.mul(U[k][i], b[k]))
            b[i] = fp.div(b[i], U[i][i])
        for i in range(n - 1, -1, -1):
            for k in range(i + 1, n):
                b[i] = fp.sub(b[i], fp.mul(U[i][k], b[k]))
            b[i] = fp.div(b[i], U[i][i])
        return b

    assert _solve_orders_differ(600, lambda F, _, b: fp.rpotrs_upper(F, b), chol_wrong, chol_case)


def test_nar_pivot_propagates():
    """G8: NaR compares as the largest |a| and is chosen as pivot."""
    rng = np.random.default_rng(5)
    A = rand_words(rng, (4, 4))
    A[2, 0] = 0x80000000
    F, ipiv, info = oracle.rgetrf(A)
    assert ipiv[0] == 3 and F[0, 0] == 0x80000000
