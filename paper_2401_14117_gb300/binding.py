"""ctypes binding of libposit_gb300.so -- argument marshalling only.

Every function has the name and argument order of the C ABI declared in
include/posit_gb300.h.  Matrix / vector arguments may be torch tensors (their
data_ptr() is passed), plain integers (device addresses) or None (NULL).
`stream` may be a torch.cuda.Stream, a raw cudaStream_t integer, or None for
torch's current stream.  A nonzero return code raises PositError; the code
is kept in its `.code` attribute.

There is no fallback: if the library is not built, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import re

from .build import INCLUDE, LIB

_lib = None

c_i64 = ctypes.c_int64
c_u32 = ctypes.c_uint32
c_int = ctypes.c_int
c_vp = ctypes.c_void_p
c_char = ctypes.c_char

# argument types per exported symbol (order of the C signatures)
_SIGS = {
    "posit_from_double": [c_vp, c_vp, c_i64, c_vp],
    "posit_to_double": [c_vp, c_vp, c_i64, c_vp],
    "posit_elementwise": [c_int, c_vp, c_vp, c_vp, c_i64, c_vp],
    "posit_rgemm": [c_char, c_char, c_i64, c_i64, c_i64, c_u32, c_vp, c_i64,
                    c_vp, c_i64, c_u32, c_vp, c_i64, c_vp],
    "posit_rgetrf": [c_i64, c_i64, c_vp, c_i64, c_vp, c_vp, c_vp],
    "posit_rgetrs": [c_char, c_i64, c_i64, c_vp, c_i64, c_vp, c_vp, c_i64, c_vp],
    "posit_rpotrf": [c_char, c_i64, c_vp, c_i64, c_vp, c_vp],
    "posit_rpotrs": [c_char, c_i64, c_i64, c_vp, c_i64, c_vp, c_i64, c_vp],
    "posit_batched_workspace_size": [c_i64, c_i64, c_vp, c_vp],
    "posit_factor_solve_batched": [c_i64, c_vp, c_vp, c_i64, c_i64, c_vp, c_vp, c_vp],
    "posit_autotune": [c_i64, c_vp, c_vp, c_i64, c_i64, c_vp, ctypes.c_int32, ctypes.c_int32,
                       c_vp, c_vp, c_vp],
    "posit_serve_open": [c_vp, c_vp],
    "posit_serve_submit": [c_vp, c_vp],
    "posit_serve_poll": [c_vp, c_vp, c_i64, c_vp],
    "posit_serve_stats": [c_vp, c_vp],
    "posit_serve_close": [c_vp],
    "posit_rgetrf_static": [c_i64, c_i64, c_vp, c_i64, c_vp, c_vp, c_vp],
    "posit_selftest_wait": [c_i64, c_vp, c_vp],
}

POSIT_LU = 0
POSIT_CHOLESKY = 1     # uplo 'L'
POSIT_CHOLESKY_U = 2   # uplo 'U'


class posit_plan(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("smem_bytes", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class posit_serve_config(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_int64), ("small_n_max", ctypes.c_int32),
                ("max_batch", ctypes.c_int32), ("max_nrhs", ctypes.c_int32),
                ("large_lanes", ctypes.c_int32), ("plan", posit_plan),
                ("batch_only_n_max", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class posit_request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("n", ctypes.c_int32), ("nrhs", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("A", ctypes.c_void_p), ("B", ctypes.c_void_p),
                ("X", ctypes.c_void_p), ("info", ctypes.c_void_p), ("tag", ctypes.c_uint64)]


class posit_serve_stats_t(ctypes.Structure):
    _fields_ = [("pending", ctypes.c_int64), ("admitted", ctypes.c_int64),
                ("completed", ctypes.c_int64), ("inflight_launches", ctypes.c_int64),
                ("launches", ctypes.c_int64), ("device_bytes_in_use", ctypes.c_int64),
                ("batched_requests", ctypes.c_int64), ("largest_batch", ctypes.c_int64)]


# layout of struct posit_problem (include/posit_gb300.h), for building the
# device descriptor array from numpy
PROBLEM_DTYPE = [("kind", "<i4"), ("n", "<i4"), ("nrhs", "<i4"), ("reserved", "<i4"),
                 ("lda", "<i8"), ("ldb", "<i8"), ("A", "<u8"), ("B", "<u8"),
                 ("ipiv", "<u8"), ("info", "<u8")]


class PositError(RuntimeError):
    def __init__(self, func: str, code: int):
        super().__init__(f"{func} returned {code}")
        self.func = func
        self.code = code


def header_symbols() -> list[str]:
    """Names of the functions declared in include/posit_gb300.h."""
    names = []
    for h in sorted(os.listdir(INCLUDE)):
        if h.endswith(".h"):
            with open(os.path.join(INCLUDE, h)) as f:
                names += re.findall(r"POSIT_API\s+\w+\s+(posit_\w+)\s*\(", f.read())
    return names


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError(
                f"{LIB} is not built; run `python -c 'import __graft_entry__ as g; g.build()'` "
                "(the library has no CPU fallback)")
        L = ctypes.CDLL(LIB)
        for name, args in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = c_int
        _lib = L
    return _lib


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    raise TypeError(f"cannot pass {type(x)} as a device pointer")


def _stream(s):
    if s is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _char(c):
    return c.encode() if isinstance(c, str) else c


def _check(name, rc):
    if rc != 0:
        raise PositError(name, rc)
    return rc


def posit_from_double(x, p, count, stream=None):
    return _check("posit_from_double",
                  lib().posit_from_double(_ptr(x), _ptr(p), count, _stream(stream)))


def posit_to_double(p, x, count, stream=None):
    return _check("posit_to_double",
                  lib().posit_to_double(_ptr(p), _ptr(x), count, _stream(stream)))


def posit_elementwise(op, p, q, r, count, stream=None):
    return _check("posit_elementwise",
                  lib().posit_elementwise(op, _ptr(p), _ptr(q), _ptr(r), count, _stream(stream)))


def posit_rgemm(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, stream=None):
    return _check("posit_rgemm", lib().posit_rgemm(
        _char(transa), _char(transb), m, n, k, alpha, _ptr(A), lda, _ptr(B), ldb,
        beta, _ptr(C), ldc, _stream(stream)))


def posit_rgetrf(m, n, A, lda, ipiv, info, stream=None):
    return _check("posit_rgetrf", lib().posit_rgetrf(m, n, _ptr(A), lda, _ptr(ipiv), _ptr(info),
                                                      _stream(stream)))


def posit_rgetrs(trans, n, nrhs, A, lda, ipiv, B, ldb, stream=None):
    return _check("posit_rgetrs", lib().posit_rgetrs(_char(trans), n, nrhs, _ptr(A), lda,
                                                      _ptr(ipiv), _ptr(B), ldb, _stream(stream)))


def posit_rpotrf(uplo, n, A, lda, info, stream=None):
    return _check("posit_rpotrf", lib().posit_rpotrf(_char(uplo), n, _ptr(A), lda, _ptr(info),
                                                      _stream(stream)))


def posit_rpotrs(uplo, n, nrhs, A, lda, B, ldb, stream=None):
    return _check("posit_rpotrs", lib().posit_rpotrs(_char(uplo), n, nrhs, _ptr(A), lda,
                                                      _ptr(B), ldb, _stream(stream)))


def posit_batched_workspace_size(max_n, max_nrhs, plan):
    out = ctypes.c_size_t(0)
    _check("posit_batched_workspace_size", lib().posit_batched_workspace_size(
        max_n, max_nrhs, ctypes.byref(plan), ctypes.byref(out)))
    return out.value


def posit_factor_solve_batched(count, problems, order, max_n, max_nrhs, plan, workspace,
                               stream=None):
    return _check("posit_factor_solve_batched", lib().posit_factor_solve_batched(
        count, _ptr(problems), _ptr(order), max_n, max_nrhs, ctypes.byref(plan),
        _ptr(workspace), _stream(stream)))


def posit_autotune(count, problems, order, max_n, max_nrhs, cands, reps=1, stream=None):
    """Fastest of the candidate plans (a list of posit_plan) on the batch;
    returns (best posit_plan, list of per-candidate ms, -1 where a plan could
    not be launched).  The problems' arrays are left unchanged."""
    arr = (posit_plan * len(cands))(*cands)
    times = (ctypes.c_float * len(cands))()
    best = posit_plan()
    _check("posit_autotune", lib().posit_autotune(
        count, _ptr(problems), _ptr(order), max_n, max_nrhs, ctypes.byref(arr), len(cands), reps,
        ctypes.byref(best), ctypes.byref(times), _stream(stream)))
    return best, [float(t) for t in times]


def posit_serve_open(cfg):
    h = ctypes.c_void_p()
    _check("posit_serve_open", lib().posit_serve_open(ctypes.byref(cfg), ctypes.byref(h)))
    return h.value


def posit_serve_submit(server, req):
    return _check("posit_serve_submit", lib().posit_serve_submit(server, ctypes.byref(req)))


def posit_serve_poll(server, tags_buf, max_done):
    """tags_buf: ctypes array of c_uint64; returns the number of tags written."""
    n = ctypes.c_int64(0)
    _check("posit_serve_poll", lib().posit_serve_poll(server, tags_buf, max_done, ctypes.byref(n)))
    return n.value


def posit_serve_stats(server):
    st = posit_serve_stats_t()
    _check("posit_serve_stats", lib().posit_serve_stats(server, ctypes.byref(st)))
    return st


def posit_serve_close(server):
    return _check("posit_serve_close", lib().posit_serve_close(server))


def posit_rgetrf_static(m, n, A, lda, ipiv, info, stream=None):
    """posit_rgetrf without any device allocation (fixed scratch in the library)."""
    return _check("posit_rgetrf_static", lib().posit_rgetrf_static(
        m, n, _ptr(A), lda, _ptr(ipiv), _ptr(info), _stream(stream)))


def posit_selftest_wait(wait_ns, info, stream=None):
    """Run the factorisations' bounded grid-barrier wait where it cannot
    complete; *info becomes POSIT_ERR_TIMEOUT once the stream completes."""
    return _check("posit_selftest_wait", lib().posit_selftest_wait(wait_ns, _ptr(info),
                                                                    _stream(stream)))
