"""Leading dimensions larger than the row count, through the C ABI: every
routine must read and write only the rows [0, rows) of each column, leave the
padding words untouched, and give the same words as with packed storage."""
import itertools

import numpy as np
import pytest
import torch

import oracle
from paper_2401_14117_gb300 import binding, inputs
from tests.gpu_util import DEV

pytestmark = pytest.mark.gpu

ONE, MONE = 0x40000000, 0xC0000000
PAD = np.uint32(0x5A5A5A5A)


def words(shape, seed):
    return oracle.from_double_array(inputs.uniform(shape, seed))


def padded(M, ld):
    """Column-major (cols, ld) device tensor holding M in rows [0, rows) and
    the PAD word below."""
    rows, cols = M.shape
    P = np.full((cols, ld), PAD, dtype=np.uint32)
    P[:, :rows] = M.T
    return torch.from_numpy(P.view(np.int32)).to(DEV)


def unpad(T, rows):
    P = T.cpu().numpy().view(np.uint32)
    assert np.all(P[:, rows:] == PAD), "padding rows were written"
    return np.ascontiguousarray(P[:, :rows].T)


@pytest.mark.parametrize("ta,tb", list(itertools.product("NT", "NT")))
def test_rgemm_padded(ta, tb):
    m, n, k = 150, 70, 45
    A = words((m, k) if ta == "N" else (k, m), 1)
    B = words((k, n) if tb == "N" else (n, k), 2)
    C = words((m, n), 3)
    dA, dB, dC = padded(A, A.shape[0] + 5), padded(B, B.shape[0] + 3), padded(C, m + 7)
    binding.posit_rgemm(ta, tb, m, n, k, MONE, dA, A.shape[0] + 5, dB, B.shape[0] + 3, ONE,
                        dC, m + 7)
    torch.cuda.synchronize()
    assert np.array_equal(unpad(dC, m), oracle.rgemm(ta, tb, MONE, A, B, ONE, C))
    assert np.array_equal(unpad(dA, A.shape[0]), A) and np.array_equal(unpad(dB, B.shape[0]), B)


@pytest.mark.parametrize("m,n", [(300, 200), (200, 300), (257, 257)])
def test_getrf_getrs_padded(m, n):
    A = words((m, n), 4)
    lda = m + 9
    dA = padded(A, lda)
    mn = min(m, n)
    ipiv = torch.zeros(mn, dtype=torch.int32, device=DEV)
    info = torch.zeros(1, dtype=torch.int32, device=DEV)
    binding.posit_rgetrf(m, n, dA, lda, ipiv, info)
    torch.cuda.synchronize()
    F, ipo, info_o = oracle.rgetrf(A)
    assert np.array_equal(unpad(dA, m), F)
    assert np.array_equal(ipiv.cpu().numpy(), ipo) and int(info.item()) == info_o
    if m == n:
        B = words((n, 3), 5)
        dB = padded(B, n + 6)
        for trans in "NT":
            dB = padded(B, n + 6)
            binding.posit_rgetrs(trans, n, 3, dA, lda, ipiv, dB, n + 6)
            torch.cuda.synchronize()
            assert np.array_equal(unpad(dB, n), oracle.rgetrs(F, ipo, B, trans=trans)), trans


@pytest.mark.parametrize("uplo", ["L", "U"])
def test_potrf_potrs_padded(uplo):
    n = 280
    A = oracle.from_double_array(inputs.spd(n, 6))
    lda = n + 4
    dA = padded(A, lda)
    info = torch.zeros(1, dtype=torch.int32, device=DEV)
    binding.posit_rpotrf(uplo, n, dA, lda, info)
    torch.cuda.synchronize()
    F, info_o = oracle.rpotrf(A, uplo=uplo)
    got = unpad(dA, n)
    tri = np.tril if uplo == "L" else np.triu
    other = (lambda X: np.triu(X, 1)) if uplo == "L" else (lambda X: np.tril(X, -1))
    assert int(info.item()) == info_o == 0
    assert np.array_equal(tri(got), tri(F))
    assert np.array_equal(other(got), other(A))  # the other triangle is never touched
    B = words((n, 2), 7)
    dB = padded(B, n + 6)
    binding.posit_rpotrs(uplo, n, 2, dA, lda, dB, n + 6)
    torch.cuda.synchronize()
    assert np.array_equal(unpad(dB, n), oracle.rpotrs(F, B, uplo=uplo))
