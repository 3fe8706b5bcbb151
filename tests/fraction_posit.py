"""A third, deliberately naive Posit(32,2) implementation on Python Fractions.

Test helper only.  It shares nothing with the C oracle or the CUDA library:
patterns are decoded by parsing their binary string (Sec. 2, Eq. 1), and a
rounded result is found by binary search over the sorted posit patterns,
using as decision points the values of the 33-bit posits 2p+1 (the midpoints
between neighbouring 32-bit posits), ties going to the even pattern, with
saturation at minpos / maxpos.  It is slow (a few hundred microseconds per
operation) and is used for tiny problems only.

The LAPACK-style routines below restate the operation orders O1-O5 (the
reference-BLAS loop order for Rgemm, right-looking LU with partial pivoting,
right-looking Cholesky, and the substitution orders of the solves) as plain
loops.
"""
from __future__ import annotations

from fractions import Fraction
from functools import lru_cache

NAR = 0x80000000
MAXPAT = 0x7FFFFFFF


@lru_cache(maxsize=None)
def value(p: int, nbits: int = 32):
    """Exact value of an nbits posit pattern (None for NaR)."""
    p &= (1 << nbits) - 1
    if p == 0:
        return Fraction(0)
    if p == 1 << (nbits - 1):
        return None
    neg = p >> (nbits - 1)
    if neg:
        p = (-p) & ((1 << nbits) - 1)
    s = format(p, f"0{nbits}b")[1:]  # bits after the sign
    first = s[0]
    m = len(s) - len(s.lstrip(first))
    k = m - 1 if first == "1" else -m
    rest = s[m + 1:]  # skip the terminating bit
    ebits = (rest[:2] + "00")[:2]
    frac = rest[2:]
    e = int(ebits, 2)
    f = Fraction(int(frac, 2), 2 ** len(frac)) if frac else Fraction(0)
    v = Fraction(2) ** (4 * k + e) * (1 + f)
    return -v if neg else v


def _round(sign_of_x_minus) -> int:
    """Round the positive exact x described by sign_of_x_minus(m) = sign(x-m)."""
    lo, hi = 1, MAXPAT
    while lo < hi:
        mid = (lo + hi) // 2
        c = sign_of_x_minus(value(2 * mid + 1, 33))
        if c < 0 or (c == 0 and mid % 2 == 0):
            hi = mid
        else:
            lo = mid + 1
    return lo


def from_fraction(x: Fraction) -> int:
    if x == 0:
        return 0
    neg = x < 0
    ax = -x if neg else x
    p = _round(lambda m: (ax > m) - (ax < m))
    return (-p) & 0xFFFFFFFF if neg else p


def _cmp(a, b):
    return (a > b) - (a < b)


def add(a: int, b: int) -> int:
    va, vb = value(a), value(b)
    if va is None or vb is None:
        return NAR
    return from_fraction(va + vb)


def sub(a: int, b: int) -> int:
    va, vb = value(a), value(b)
    if va is None or vb is None:
        return NAR
    return from_fraction(va - vb)


def mul(a: int, b: int) -> int:
    va, vb = value(a), value(b)
    if va is None or vb is None:
        return NAR
    return from_fraction(va * vb)


def div(a: int, b: int) -> int:
    va, vb = value(a), value(b)
    if va is None or vb is None or vb == 0:
        return NAR
    return from_fraction(va / vb)


def sqrt(a: int) -> int:
    va = value(a)
    if va is None or va < 0:
        return NAR
    if va == 0:
        return 0
    return _round(lambda m: _cmp(va, m * m))


def absword(w: int) -> int:
    return (-w) & 0xFFFFFFFF if w >> 31 else w


ONE = 0x40000000
MINUS_ONE = 0xC0000000


# ----------------------------------------------------------- O1 .. O5
def rgemm(ta, tb, alpha, A, B, beta, C):
    """A, B, C: lists of lists indexed [row][col]; returns new C."""
    m, n = len(C), len(C[0]) if C else 0
    k = len(A) if ta == "T" else (len(A[0]) if A else 0)
    out = [row[:] for row in C]
    for i in range(m):
        for j in range(n):
            c = out[i][j]
            if beta == 0:
                c = 0
            elif beta != ONE:
                c = mul(beta, c)
            if alpha != 0:
                for l in range(k):
                    b = B[j][l] if tb == "T" else B[l][j]
                    a = A[l][i] if ta == "T" else A[i][l]
                    c = add(c, mul(mul(alpha, b), a))
            out[i][j] = c
    return out


def rgetrf(A):
    A = [row[:] for row in A]
    m, n = len(A), len(A[0])
    ipiv, info = [], 0
    for col in range(min(m, n)):
        p = col
        for i in range(col + 1, m):
            if absword(A[i][col]) > absword(A[p][col]):
                p = i
        ipiv.append(p + 1)
        if A[p][col] != 0:
            A[col], A[p] = A[p], A[col]
            r = div(ONE, A[col][col])
            for i in range(col + 1, m):
                A[i][col] = mul(A[i][col], r)
        elif info == 0:
            info = col + 1
        for k in range(col + 1, n):
            for i in range(col + 1, m):
                A[i][k] = sub(A[i][k], mul(A[i][col], A[col][k]))
    return A, ipiv, info


def rpotrf_lower(A):
    A = [row[:] for row in A]
    n = len(A)
    for j in range(n):
        d = A[j][j]
        if d == 0 or d >> 31:
            return A, j + 1
        A[j][j] = sqrt(d)
        r = div(ONE, A[j][j])
        for i in range(j + 1, n):
            A[i][j] = mul(A[i][j], r)
        for k in range(j + 1, n):
            for i in range(k, n):
                A[i][k] = sub(A[i][k], mul(A[i][j], A[k][j]))
    return A, 0


def rgetrs(LU, ipiv, b):
    b = b[:]
    n = len(LU)
    for i in range(n):
        p = ipiv[i] - 1
        b[i], b[p] = b[p], b[i]
    for i in range(n):
        for j in range(i):
            b[i] = sub(b[i], mul(LU[i][j], b[j]))
    for i in range(n - 1, -1, -1):
        for k in range(n - 1, i, -1):
            b[i] = sub(b[i], mul(LU[i][k], b[k]))
        b[i] = div(b[i], LU[i][i])
    return b


def rpotrs_lower(L, b):
    b = b[:]
    n = len(L)
    for i in range(n):
        for j in range(i):
            b[i] = sub(b[i], mul(L[i][j], b[j]))
        b[i] = div(b[i], L[i][i])
    for i in range(n - 1, -1, -1):
        for k in range(i + 1, n):
            b[i] = sub(b[i], mul(L[k][i], b[k]))
        b[i] = div(b[i], L[i][i])
    return b


def rgetrs_trans(LU, ipiv, b):
    """A^T x = b with A = P L U (Sec. 5.1 solves, transposed): U^T y = b with
    k ascending then a division by u_ii, the unit L^T z = y with i descending
    and k = i+1 .. n-1 ascending, then x = P z (the swaps in reverse)."""
    b = b[:]
    n = len(LU)
    for i in range(n):
        for k in range(i):
            b[i] = sub(b[i], mul(LU[k][i], b[k]))
        b[i] = div(b[i], LU[i][i])
    for i in range(n - 1, -1, -1):
        for k in range(i + 1, n):
            b[i] = sub(b[i], mul(LU[k][i], b[k]))
    for i in range(n - 1, -1, -1):
        p = ipiv[i] - 1
        b[i], b[p] = b[p], b[i]
    return b


def rpotrs_upper(U, b):
    """A x = b with A = U^T U: U^T y = b with k ascending then a division by
    u_ii, then U x = y with i descending, k = n-1 .. i+1 descending and a
    division by u_ii (reference trsm Left-Upper-T, then Left-Upper-N)."""
    b = b[:]
    n = len(U)
    for i in range(n):
        for k in range(i):
            b[i] = sub(b[i], mul(U[k][i], b[k]))
        b[i] = div(b[i], U[i][i])
    for i in range(n - 1, -1, -1):
        for k in range(n - 1, i, -1):
            b[i] = sub(b[i], mul(U[i][k], b[k]))
        b[i] = div(b[i], U[i][i])
    return b
