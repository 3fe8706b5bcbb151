"""posit_rgetrf_static: the LU factorisation for callers that must not
allocate device memory (for example when another allocator already holds
all of it, or under strict memory accounting).  It must give exactly what
posit_rgetrf gives, call after call, while taking its scratch from the
library's fixed array.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2401_14117_gb300 import binding, inputs

pytestmark = pytest.mark.gpu


def _words(m, n, seed):
    x = torch.from_numpy(inputs.uniform((n, m), seed)).cuda()  # column-major m x n
    w = torch.empty((n, m), dtype=torch.int32, device="cuda")
    binding.posit_from_double(x, w, x.numel())
    return w


def _factor(fn, A, m, n):
    F = A.clone()
    ipiv = torch.zeros(min(m, n), dtype=torch.int32, device="cuda")
    info = torch.full((1,), -9, dtype=torch.int32, device="cuda")
    fn(m, n, F, m, ipiv, info)
    torch.cuda.synchronize()
    return F.cpu().numpy(), ipiv.cpu().numpy(), int(info.item())


@pytest.mark.parametrize("m,n", [(700, 700), (300, 520)])
def test_static_scratch_lu_equals_allocating_lu_twice(m, n):
    for call, seed in enumerate((11, 12)):  # two calls in a row share the array
        A = _words(m, n, seed + m)
        if call == 1:
            A[:, :] = A.flip(0)  # a different matrix on the second call
        F0, p0, i0 = _factor(binding.posit_rgetrf, A, m, n)
        F1, p1, i1 = _factor(binding.posit_rgetrf_static, A, m, n)
        assert i0 == i1 == 0
        assert np.array_equal(F0, F1) and np.array_equal(p0, p1), (m, n, call)


def test_static_scratch_argument_errors():
    with pytest.raises(binding.PositError) as e:
        binding.posit_rgetrf_static(-1, 1, None, 1, None, None)
    assert e.value.code == -1
    # an empty matrix: info cleared and POSIT_OK, exactly as posit_rgetrf
    for fn in (binding.posit_rgetrf, binding.posit_rgetrf_static):
        for m, n in ((0, 4), (4, 0)):
            info = torch.full((1,), 5, dtype=torch.int32, device="cuda")
            assert fn(m, n, None, max(1, m), None, info) == 0
            torch.cuda.synchronize()
            assert int(info.item()) == 0


def _cudart():
    """The CUDA runtime the library itself is linked against."""
    binding.lib()
    with open("/proc/self/maps") as f:
        paths = {ln.split()[-1] for ln in f if "libcudart.so" in ln}
    assert paths, "libcudart not loaded"
    return ctypes.CDLL(sorted(paths)[0])


def test_static_scratch_lu_allocates_nothing():
    """The point of the entry point: no device allocation.  posit_rgetrf takes
    its scratch from the device's current memory pool (stream-ordered), so the
    pool's high-water mark of used bytes, reset just before the call, rises
    above the bytes in use before it under posit_rgetrf and never does under
    posit_rgetrf_static."""
    rt = _cudart()
    dev = torch.cuda.current_device()
    pool = ctypes.c_void_p()
    assert rt.cudaDeviceGetMemPool(ctypes.byref(pool), dev) == 0
    used_high, used_now = 0x8, 0x7  # cudaMemPoolAttrUsedMemHigh / UsedMemCurrent

    def reset_and_run(fn):
        """(pool bytes in use before the call, high-water mark during it)"""
        A = _words(300, 300, 5)
        torch.cuda.synchronize()
        before, hi = ctypes.c_uint64(), ctypes.c_uint64()
        assert rt.cudaMemPoolGetAttribute(pool, used_now, ctypes.byref(before)) == 0
        zero = ctypes.c_uint64(0)
        assert rt.cudaMemPoolSetAttribute(pool, used_high, ctypes.byref(zero)) == 0
        _factor(fn, A, 300, 300)
        assert rt.cudaMemPoolGetAttribute(pool, used_high, ctypes.byref(hi)) == 0
        return before.value, hi.value

    reset_and_run(binding.posit_rgetrf_static)  # first call: the one-time set-up
    before, hi = reset_and_run(binding.posit_rgetrf)
    assert hi > before, "posit_rgetrf should have drawn its scratch from the pool"
    for _ in range(2):
        before, hi = reset_and_run(binding.posit_rgetrf_static)
        assert hi <= before, f"posit_rgetrf_static drew {hi - before} bytes from the pool"
