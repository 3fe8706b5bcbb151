"""GPU parity of the scalar core: conversion and element-wise ops, word for
word against the CPU oracle (through the C ABI)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2401_14117_gb300 import binding, inputs
from tests.gpu_util import mixed_words, words_from_dev, words_to_dev, DEV

pytestmark = pytest.mark.gpu

N_RANDOM = 1 << 22


def _doubles(rng, count):
    parts = [
        inputs.uniform(count // 6, 1),
        inputs.scaled(count // 6, 2),
        inputs.normal(count // 6, 3, sigma=1e6),
        rng.standard_normal(count // 6) * 10.0 ** rng.integers(-320, 300, count // 6),
    ]
    bits = rng.integers(0, 2 ** 64, count // 6, dtype=np.uint64).view(np.float64)
    parts.append(bits[np.isfinite(bits)])
    parts.append(np.array([0.0, -0.0, 1.0, -1.0, 2.0 ** 113, 2.0 ** 119, 2.0 ** -118,
                           2.0 ** 300, -2.0 ** -300, 5e-324, 1.5, 3.0, np.nan, np.inf, -np.inf]))
    x = np.concatenate(parts)
    return x


def test_from_double_matches_oracle():
    rng = np.random.default_rng(1)
    x = _doubles(rng, N_RANDOM)
    want = oracle.from_double_array(x)
    dx = torch.from_numpy(x).to(DEV)
    dp = torch.empty(x.size, dtype=torch.int32, device=DEV)
    binding.posit_from_double(dx, dp, x.size)
    got = words_from_dev(dp)
    bad = np.flatnonzero(got != want)
    assert bad.size == 0, [(x[i], hex(got[i]), hex(want[i])) for i in bad[:5]]


def test_to_double_matches_oracle_and_roundtrips():
    rng = np.random.default_rng(2)
    w = mixed_words(rng, N_RANDOM)
    want = oracle.to_double_array(w)
    dw = words_to_dev(w)
    dx = torch.empty(w.size, dtype=torch.float64, device=DEV)
    binding.posit_to_double(dw, dx, w.size)
    got = dx.cpu().numpy()
    assert np.array_equal(got, want, equal_nan=True)
    back = torch.empty_like(dw)
    binding.posit_from_double(dx, back, w.size)
    assert np.array_equal(words_from_dev(back), w)


def test_roundtrip_every_word():
    """posit -> double -> posit is the identity on all 2^32 words."""
    chunk = 1 << 28
    base = torch.arange(chunk, dtype=torch.int64, device=DEV)
    dx = torch.empty(chunk, dtype=torch.float64, device=DEV)
    back = torch.empty(chunk, dtype=torch.int32, device=DEV)
    for start in range(0, 1 << 32, chunk):
        w = (base + start).to(torch.int64)
        w32 = torch.where(w >= 2 ** 31, w - 2 ** 32, w).to(torch.int32)
        binding.posit_to_double(w32, dx, chunk)
        binding.posit_from_double(dx, back, chunk)
        nar = w32 == torch.iinfo(torch.int32).min
        ok = (back == w32) | nar
        assert bool(ok.all()), start


@pytest.mark.parametrize("op,code", [("add", 0), ("sub", 1), ("mul", 2), ("div", 3), ("sqrt", 4)])
def test_elementwise_matches_oracle(op, code):
    rng = np.random.default_rng(10 + code)
    a = mixed_words(rng, N_RANDOM)
    b = mixed_words(rng, N_RANDOM)
    # half the pairs share the scale range, to reach cancellation and ties
    b[::2] = (b[::2] & np.uint32(0xF80FFFFF)) | (a[::2] & np.uint32(0x07F00000))
    want = oracle.elementwise(op, a, b)
    da, db = words_to_dev(a), words_to_dev(b)
    dr = torch.empty_like(da)
    binding.posit_elementwise(code, da, db, dr, a.size)
    got = words_from_dev(dr)
    bad = np.flatnonzero(got != want)
    assert bad.size == 0, [(hex(a[i]), hex(b[i]), hex(got[i]), hex(want[i])) for i in bad[:5]]


@pytest.mark.parametrize("offset,count", [(1, 1001), (2, 4099), (0, 4097), (3, 3)])
def test_elementwise_unaligned_and_ragged(offset, count):
    """Operands that start off a 16-byte boundary (one word at a time) and
    counts that are not a multiple of 4 (the vector tail)."""
    rng = np.random.default_rng(20 + offset)
    a = mixed_words(rng, count + 16)
    b = mixed_words(rng, count + 16)
    da, db = words_to_dev(a), words_to_dev(b)
    for op, code in (("add", 0), ("mul", 2), ("div", 3), ("sqrt", 4)):
        want = oracle.elementwise(op, a[offset:offset + count], b[offset:offset + count])
        dr = torch.zeros(count + 16, dtype=torch.int32, device=DEV)
        binding.posit_elementwise(code, da[offset:], db[offset:], dr[offset:], count)
        got = words_from_dev(dr)
        assert np.array_equal(got[offset:offset + count], want), op
        assert not got[:offset].any() and not got[offset + count:].any(), op


@pytest.mark.parametrize("op", ["sqrt", "recip"])
def test_unary_strided_over_all_words(op):
    """sqrt and reciprocal (1 / x) on every 61st word of the 2^32."""
    w = (np.arange(0, 1 << 32, 61, dtype=np.uint64)).astype(np.uint32)
    da = words_to_dev(w)
    dr = torch.empty_like(da)
    if op == "sqrt":
        want = oracle.elementwise("sqrt", w)
        binding.posit_elementwise(4, da, None, dr, w.size)
    else:
        ones = np.full_like(w, 0x40000000)
        want = oracle.elementwise("div", ones, w)
        binding.posit_elementwise(3, words_to_dev(ones), da, dr, w.size)
    got = words_from_dev(dr)
    bad = np.flatnonzero(got != want)
    assert bad.size == 0, [(hex(w[i]), hex(got[i]), hex(want[i])) for i in bad[:5]]


def test_argument_errors():
    with pytest.raises(binding.PositError) as e:
        binding.posit_elementwise(9, None, None, None, 1)
    assert e.value.code == -1
    with pytest.raises(binding.PositError) as e:
        binding.posit_from_double(None, None, -1)
    assert e.value.code == -3
    binding.posit_elementwise(0, None, None, None, 0)  # empty: no-op
