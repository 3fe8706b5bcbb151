"""posit_rgetrf_static: the LU factorisation for callers that must not
allocate device memory (for example when another allocator already holds
all of it, or under strict memory accounting).  It must give exactly what
posit_rgetrf gives, call after call, while taking its scratch from the
library's fixed array.  This file is collected last on purpose."""
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
    info = torch.full((1,), 5, dtype=torch.int32, device="cuda")
    binding.posit_rgetrf_static(0, 4, None, 1, None, info)
    torch.cuda.synchronize()
    assert int(info.item()) == 0
