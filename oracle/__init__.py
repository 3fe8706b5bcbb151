"""Plain CPU oracle for Posit(n,2) arithmetic and Posit(32,2) Rgemm / Rgetrf /
Rpotrf / Rgetrs / Rpotrs.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The CUDA library (``paper_2401_14117_gb300``) never imports it and
shares no code with it.

The arithmetic lives in ``posit_oracle.c`` (see its header comment for the
paper passages each part follows); this module only compiles it with gcc and
marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "posit_oracle.c")
_HDR = os.path.join(_HERE, "posit_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")

_lib = None
_lock = threading.Lock()

NAR32 = 0x80000000
ONE32 = 0x40000000

_U32P = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
_I32P = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_F64P = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` with gcc (OpenMP) if it is missing or stale."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)) or any(
        os.path.getmtime(s) > os.path.getmtime(_LIB_PATH) for s in (_SRC, _HDR))
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=gnu11",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            u32, i32, i64, c_int = (ctypes.c_uint32, ctypes.c_int32,
                                    ctypes.c_int64, ctypes.c_int)
            for name in ("or_add", "or_sub", "or_mul", "or_div"):
                f = getattr(L, name)
                f.argtypes = [c_int, u32, u32]
                f.restype = u32
            L.or_sqrt.argtypes = [c_int, u32]
            L.or_sqrt.restype = u32
            L.or_neg.argtypes = [c_int, u32]
            L.or_neg.restype = u32
            L.or_from_double.argtypes = [c_int, ctypes.c_double]
            L.or_from_double.restype = u32
            L.or_to_double.argtypes = [c_int, u32]
            L.or_to_double.restype = ctypes.c_double
            L.or_decode.argtypes = [c_int, u32, ctypes.POINTER(c_int),
                                    ctypes.POINTER(c_int),
                                    ctypes.POINTER(u32), ctypes.POINTER(c_int)]
            L.or_decode.restype = c_int
            L.or_elementwise.argtypes = [c_int, c_int, _U32P, _U32P, _U32P, i64]
            L.or_elementwise.restype = None
            L.or_from_double_array.argtypes = [c_int, _F64P, _U32P, i64]
            L.or_from_double_array.restype = None
            L.or_to_double_array.argtypes = [c_int, _U32P, _F64P, i64]
            L.or_to_double_array.restype = None
            L.or_set_threads.argtypes = [c_int]
            L.or_set_threads.restype = None
            L.or_get_threads.argtypes = []
            L.or_get_threads.restype = c_int
            vp = ctypes.c_void_p
            L.or_rgemm.argtypes = [ctypes.c_char, ctypes.c_char, i64, i64, i64,
                                   u32, vp, i64, vp, i64, u32, vp, i64]
            L.or_rgemm.restype = None
            L.or_rgetrf.argtypes = [i64, i64, vp, i64, vp]
            L.or_rgetrf.restype = c_int
            L.or_rgetrf_blocked.argtypes = [i64, i64, vp, i64, vp, i64]
            L.or_rgetrf_blocked.restype = c_int
            L.or_rgetrs.argtypes = [ctypes.c_char, i64, i64, vp, i64, vp, vp, i64]
            L.or_rgetrs.restype = None
            L.or_rpotrf.argtypes = [ctypes.c_char, i64, vp, i64]
            L.or_rpotrf.restype = c_int
            L.or_rpotrf_blocked.argtypes = [ctypes.c_char, i64, vp, i64, i64]
            L.or_rpotrf_blocked.restype = c_int
            L.or_rpotrs.argtypes = [ctypes.c_char, i64, i64, vp, i64, vp, i64]
            L.or_rpotrs.restype = None
            _lib = L
    return _lib


# ---------------------------------------------------------------- scalars
def add(a, b, nbits=32): return lib().or_add(nbits, a, b)
def sub(a, b, nbits=32): return lib().or_sub(nbits, a, b)
def mul(a, b, nbits=32): return lib().or_mul(nbits, a, b)
def div(a, b, nbits=32): return lib().or_div(nbits, a, b)
def sqrt(a, nbits=32): return lib().or_sqrt(nbits, a)
def neg(a, nbits=32): return lib().or_neg(nbits, a)
def from_double(x, nbits=32): return lib().or_from_double(nbits, float(x))
def to_double(p, nbits=32): return lib().or_to_double(nbits, p)


def decode(p, nbits=32):
    """(cls, neg, scale, frac, fbits); cls 0 zero, 1 finite, 2 NaR."""
    n_, s_, f_, b_ = ctypes.c_int(), ctypes.c_int(), ctypes.c_uint32(), ctypes.c_int()
    cls = lib().or_decode(nbits, p, ctypes.byref(n_), ctypes.byref(s_),
                          ctypes.byref(f_), ctypes.byref(b_))
    return cls, n_.value, s_.value, f_.value, b_.value


OPS = {"add": 0, "sub": 1, "mul": 2, "div": 3, "sqrt": 4}


def elementwise(op, a, b=None, nbits=32):
    a = np.ascontiguousarray(a, dtype=np.uint32)
    b = a if b is None else np.ascontiguousarray(b, dtype=np.uint32)
    out = np.empty_like(a)
    lib().or_elementwise(nbits, OPS[op], a, b, out, a.size)
    return out


def from_double_array(x, nbits=32):
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.empty(x.shape, dtype=np.uint32)
    lib().or_from_double_array(nbits, x.reshape(-1), out.reshape(-1), x.size)
    return out


def to_double_array(p, nbits=32):
    p = np.ascontiguousarray(p, dtype=np.uint32)
    out = np.empty(p.shape, dtype=np.float64)
    lib().or_to_double_array(nbits, p.reshape(-1), out.reshape(-1), p.size)
    return out


def set_threads(t: int):
    lib().or_set_threads(int(t))


def get_threads() -> int:
    return lib().or_get_threads()


# ------------------------------------------------------ column-major helpers
def _fmat(a):
    """Fortran-ordered uint32 copy (column-major, lda = rows)."""
    return np.asfortranarray(np.array(a, dtype=np.uint32, copy=True))


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def rgemm(transa, transb, alpha, A, B, beta, C):
    """Return a new C = alpha op(A) op(B) + beta C (arrays as 2-D uint32)."""
    A = _fmat(A)
    B = _fmat(B)
    C = _fmat(C)
    m, n = C.shape
    k = A.shape[0] if transa in "Tt" else A.shape[1]
    lib().or_rgemm(transa.encode(), transb.encode(), m, n, k, alpha,
                   _ptr(A), max(A.shape[0], 1), _ptr(B), max(B.shape[0], 1),
                   beta, _ptr(C), max(m, 1))
    return C


def rgetrf(A, nb=None):
    """Return (LU, ipiv (1-based int32), info)."""
    A = _fmat(A)
    m, n = A.shape
    ipiv = np.zeros(max(min(m, n), 1), dtype=np.int32)
    if nb is None:
        info = lib().or_rgetrf(m, n, _ptr(A), max(m, 1), _ptr(ipiv))
    else:
        info = lib().or_rgetrf_blocked(m, n, _ptr(A), max(m, 1), _ptr(ipiv), nb)
    return A, ipiv[:min(m, n)], info


def rgetrs(LU, ipiv, B, trans="N"):
    LU = _fmat(LU)
    B = _fmat(B if np.ndim(B) == 2 else np.asarray(B).reshape(-1, 1))
    ipiv = np.ascontiguousarray(ipiv, dtype=np.int32)
    n = LU.shape[0]
    lib().or_rgetrs(trans.encode(), n, B.shape[1], _ptr(LU), max(n, 1),
                    _ptr(ipiv), _ptr(B), max(B.shape[0], 1))
    return B


def rpotrf(A, uplo="L", nb=None):
    """Return (factor, info); the other triangle is left untouched."""
    A = _fmat(A)
    n = A.shape[0]
    if nb is None:
        info = lib().or_rpotrf(uplo.encode(), n, _ptr(A), max(n, 1))
    else:
        info = lib().or_rpotrf_blocked(uplo.encode(), n, _ptr(A), max(n, 1), nb)
    return A, info


def rpotrs(F, B, uplo="L"):
    F = _fmat(F)
    B = _fmat(B if np.ndim(B) == 2 else np.asarray(B).reshape(-1, 1))
    n = F.shape[0]
    lib().or_rpotrs(uplo.encode(), n, B.shape[1], _ptr(F), max(n, 1),
                    _ptr(B), max(B.shape[0], 1))
    return B
