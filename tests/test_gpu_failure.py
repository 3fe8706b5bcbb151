"""Failure detection on the GPU without a fault or a hang: the factorisations'
grid barriers wait with a time limit, after which they set an error flag,
write POSIT_ERR_TIMEOUT into info and return.  posit_selftest_wait runs that
same barrier where it can never complete (two CTAs waiting for a third), with
a 5 ms limit, and the context must stay usable afterwards."""
import time

import numpy as np
import pytest
import torch

import oracle
from paper_2401_14117_gb300 import binding, inputs
from tests.gpu_util import DEV, from_dev, to_dev

pytestmark = pytest.mark.gpu

POSIT_ERR_TIMEOUT = -1003


def test_bounded_wait_gives_up_and_reports_timeout():
    info = torch.full((1,), 77, dtype=torch.int32, device=DEV)
    for wait_ns in (5_000_000, 20_000_000):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        assert binding.posit_selftest_wait(wait_ns, info) == 0
        torch.cuda.synchronize()
        elapsed = time.perf_counter() - t0
        assert int(info.item()) == POSIT_ERR_TIMEOUT
        # the wait ran out (not earlier than its limit, and not much later)
        assert wait_ns * 1e-9 * 0.9 <= elapsed < wait_ns * 1e-9 + 2.0, elapsed
    # the context is still usable: a small LU right after is bit-exact
    A = oracle.from_double_array(inputs.uniform((70, 70), 3))
    dA = to_dev(A)
    ipiv = torch.zeros(70, dtype=torch.int32, device=DEV)
    binding.posit_rgetrf(70, 70, dA, 70, ipiv, info)
    torch.cuda.synchronize()
    F, p, i = oracle.rgetrf(A)
    assert int(info.item()) == i == 0
    assert np.array_equal(from_dev(dA), F) and np.array_equal(ipiv.cpu().numpy(), p)


def test_selftest_argument_errors():
    info = torch.zeros(1, dtype=torch.int32, device=DEV)
    for bad in (0, 999, 10_000_000_001):
        with pytest.raises(binding.PositError) as e:
            binding.posit_selftest_wait(bad, info)
        assert e.value.code == -1
    with pytest.raises(binding.PositError) as e:
        binding.posit_selftest_wait(5_000_000, None)
    assert e.value.code == -2
