"""Pins for the oracle's scalar Posit(n,2) arithmetic (CPU only).

Each test checks the oracle against something other than itself: values
derived by hand from the format definition (Sec. 2, Eq. 1), the f_s formula
of Sec. 2 and the per-range fraction widths quoted in Sec. 4, an independent
checker (tests/c/posit_check.c) that verifies every rounded result against the
exact value with its own decoder and 256-bit arithmetic, a third Fraction-based
implementation, and algebraic invariants.
"""
import math
import os
import random
from fractions import Fraction

import numpy as np
import pytest

import oracle
from tests import fraction_posit as fp

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            yield line.split(None, 2)


def _exact(expr):
    return eval(expr, {"Fraction": Fraction})


def _exact_of_word(w):
    cls, neg, scale, frac, fbits = oracle.decode(w)
    if cls == 0:
        return Fraction(0)
    if cls == 2:
        return None
    v = Fraction(2) ** scale * (1 + Fraction(frac, 2 ** fbits))
    return -v if neg else v


# ---------------------------------------------------------------- P1
def test_constants_decode():
    """P1: hand-derived pattern values (golden/posit32_constants.txt)."""
    n = 0
    for pat, val, _why in _rows("posit32_constants.txt"):
        assert _exact_of_word(int(pat, 16)) == _exact(val), (pat, val)
        n += 1
    assert n >= 20
    assert _exact_of_word(0x80000000) is None  # NaR


def test_constants_encode_and_negation():
    for pat, val, _why in _rows("posit32_constants.txt"):
        w = int(pat, 16)
        x = _exact(val)
        assert fp.from_fraction(Fraction(x)) == w  # third implementation agrees
        if isinstance(x, int) or x.denominator & (x.denominator - 1) == 0:
            d = float(x)
            if math.isfinite(d):
                assert oracle.from_double(d) == w, (pat, val)
        # negation is the two's complement (Sec. 2 reading of the sign)
        assert oracle.neg(w) == (-w) & 0xFFFFFFFF


# ---------------------------------------------------------------- P2
def test_fraction_width_table():
    """P2: f_s = 32 - m - 2 - 2 (Sec. 2); [1,2) has f_s = 27 (Sec. 4, I0)."""
    expect = {0: 27, 1: 26, 2: 25, 3: 24, -1: 27, -2: 26, -3: 25, -4: 24}
    for k, fs in expect.items():
        w = oracle.from_double(16.0 ** k)
        cls, neg, scale, frac, fbits = oracle.decode(w)
        assert scale == 4 * k and fbits == fs, (k, fbits)
    for x in np.linspace(1.0, 1.999, 50):
        assert oracle.decode(oracle.from_double(x))[4] == 27
    # Sec. 4: ranges I1 [1e-38,1e-30) and I2 [1e30,1e38) have f_s in 0..3
    for x in (1e-38, 3e-35, 9.9e-31, 1e30, 4e34, 9.9e37):
        fb = oracle.decode(oracle.from_double(x))[4]
        assert 0 <= fb <= 3, (x, fb)
    # exponent-truncated words: regime of 29+ bits leaves no fraction
    for w in (0x7FFFFFFC, 0x7FFFFFFD, 0x7FFFFFFE, 0x7FFFFFFF, 1, 2, 3, 4):
        assert oracle.decode(w)[4] == 0


# ---------------------------------------------------------------- P3
def test_worked_rounding_cases():
    """P3: hand-derived rounding cases (golden/posit32_rounding.txt)."""
    for val, pat, _why in _rows("posit32_rounding.txt"):
        x = Fraction(_exact(val))
        w = int(pat, 16)
        assert fp.from_fraction(x) == w, (val, pat)
        d = float(x) if abs(x) < 2 ** 1000 else None
        if d is not None and d != 0 and Fraction(d) == x:
            assert oracle.from_double(d) == w, (val, hex(oracle.from_double(d)), pat)


def test_rounding_through_arithmetic():
    """Worked cases reached through ops, not conversion."""
    one, two = 0x40000000, 0x48000000
    assert oracle.add(one, one) == two
    assert oracle.mul(0x7FFFFFFF, 0x7FFFFFFF) == 0x7FFFFFFF  # saturate, not NaR
    assert oracle.mul(1, 1) == 1                              # never to zero
    assert oracle.div(one, 0) == 0x80000000
    assert oracle.sqrt(0xC0000000) == 0x80000000
    assert oracle.sub(0x44000000, 0x44000000) == 0
    assert oracle.add(0x80000000, one) == 0x80000000
    assert oracle.mul(0, 0x80000000) == 0x80000000
    # 1 + 2^-28 -> tie -> 1 (even); reached as 1 + (2^-28 as a posit)
    assert oracle.add(one, oracle.from_double(2.0 ** -28)) == one
    assert oracle.add(one, oracle.from_double(3 * 2.0 ** -28)) == 0x40000002


# ---------------------------------------------------------------- P4
@pytest.mark.parametrize("nbits", [6, 8, 10, 12, 14])
@pytest.mark.parametrize("op", ["add", "sub", "mul", "div", "sqrt", "recip"])
def test_exhaustive_small(posit_checker, nbits, op):
    """P4 (smaller widths): every pair, independent rounding check."""
    checked, bad, out = posit_checker("exhaustive", nbits, op)
    expect = (1 << nbits) if op in ("sqrt", "recip") else (1 << (2 * nbits))
    assert checked == expect and bad == 0, out


@pytest.mark.slow
@pytest.mark.parametrize("op", ["add", "sub", "mul", "div", "sqrt", "recip"])
def test_exhaustive_posit16(posit_checker, op):
    """P4: all 2^32 pairs of Posit(16,2) (same parametric code as n = 32)."""
    checked, bad, out = posit_checker("exhaustive", 16, op)
    assert bad == 0, out


@pytest.mark.parametrize("op", ["add", "sub", "mul", "div"])
def test_posit16_slice_exhaustive(posit_checker, op):
    """P4 in the default run: Posit(16,2), every second operand against the
    first operands a = 37 (mod 64) -- 2^26 pairs per operation, a fixed 1/64
    slice of the full all-pairs run (recorded in tests/golden/
    posit16_exhaustive.txt: 0 failures in 2^32 pairs per operation)."""
    checked, bad, out = posit_checker("exhaustive", 16, op, 64, 37)
    assert checked == (1 << 26) and bad == 0, out


def test_posit16_full_run_record():
    """The recorded full Posit(16,2) run covers every operation with every
    pair and reports no failure."""
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                        "posit16_exhaustive.txt")
    rows = {}
    with open(path) as f:
        for ln in f:
            if ln.startswith("#") or not ln.strip():
                continue
            op, *kv = ln.split()
            rows[op] = dict(p.split("=") for p in kv)
    for op in ("add", "sub", "mul", "div"):
        assert int(rows[op]["checked"]) == 1 << 32 and int(rows[op]["bad"]) == 0
    for op in ("sqrt", "recip"):
        assert int(rows[op]["checked"]) == 1 << 16 and int(rows[op]["bad"]) == 0


@pytest.mark.parametrize("op", ["add", "mul", "div"])
def test_posit16_sampled(op):
    """P4 in the default run: Posit(16,2) all a against a stride of b, checked
    by the Fraction implementation re-targeted to 16 bits (rounding by the
    17-bit midpoints)."""
    rng = random.Random(16)
    idx = list(range(0, 1 << 16, 257))
    bs = [rng.randrange(1 << 16) for _ in range(24)] + [0, 1, 0x7FFF, 0x8000, 0x4000]
    A = np.array([a for a in idx for _ in bs], dtype=np.uint32)
    B = np.array([b for _ in idx for b in bs], dtype=np.uint32)
    got = oracle.elementwise(op, A, B, nbits=16)

    def rnd16(x):
        if x == 0:
            return 0
        neg = x < 0
        ax = -x if neg else x
        lo, hi = 1, 0x7FFF
        while lo < hi:
            mid = (lo + hi) // 2
            m = fp.value(2 * mid + 1, 17)
            if ax < m or (ax == m and mid % 2 == 0):
                hi = mid
            else:
                lo = mid + 1
        return (-lo) & 0xFFFF if neg else lo

    for a, b, r in zip(A.tolist(), B.tolist(), got.tolist()):
        va, vb = fp.value(a, 16), fp.value(b, 16)
        if va is None or vb is None or (op == "div" and vb == 0):
            assert r == 0x8000
            continue
        x = va + vb if op == "add" else va * vb if op == "mul" else va / vb
        assert r == rnd16(x), (op, hex(a), hex(b), hex(r))


# ---------------------------------------------------------------- P5
@pytest.mark.parametrize("op", ["add", "sub", "mul", "div", "sqrt", "recip"])
def test_random_posit32(posit_checker, op):
    """P5: 4*10^6 random Posit(32,2) cases per op (uniform words, golden zone,
    long regimes, few-bit fractions), verified with exact arithmetic."""
    checked, bad, out = posit_checker("random", op, 4_000_000, 20240125)
    assert checked == 4_000_000 and bad == 0, out


def test_random_posit32_fraction():
    """P5 second route: Python Fractions (exact rational) on 3000 pairs."""
    rng = random.Random(5)
    words = [rng.getrandbits(32) for _ in range(1500)]
    words += [oracle.from_double(rng.uniform(-4, 4)) for _ in range(1500)]
    for i in range(0, len(words) - 1):
        a, b = words[i], words[i + 1]
        assert oracle.add(a, b) == fp.add(a, b)
        assert oracle.mul(a, b) == fp.mul(a, b)
        if i % 5 == 0:
            assert oracle.div(a, b) == fp.div(a, b)
            assert oracle.sqrt(a) == fp.sqrt(a)


def test_from_double(posit_checker):
    checked, bad, out = posit_checker("double", 2_000_000, 11)
    assert checked > 1_900_000 and bad == 0, out
    assert oracle.from_double(float("nan")) == 0x80000000
    assert oracle.from_double(float("inf")) == 0x80000000
    assert oracle.from_double(0.0) == 0 and oracle.from_double(-0.0) == 0


# ---------------------------------------------------------------- P6
def test_invariants_random():
    """P6: sign symmetry, commutativity, identities, monotonicity, order."""
    rng = np.random.default_rng(6)
    a = rng.integers(0, 2 ** 32, 200_000, dtype=np.uint64).astype(np.uint32)
    b = rng.integers(0, 2 ** 32, 200_000, dtype=np.uint64).astype(np.uint32)
    neg = lambda x: ((~x.astype(np.uint64) + 1) & 0xFFFFFFFF).astype(np.uint32)
    nar = np.uint32(0x80000000)
    ok = (a != nar) & (b != nar)
    a, b = a[ok], b[ok]
    for op in ("add", "mul"):
        ab = oracle.elementwise(op, a, b)
        assert np.array_equal(ab, oracle.elementwise(op, b, a)), op
        # round(-x) = -round(x)
        assert np.array_equal(oracle.elementwise(op, neg(a), neg(b)) if op == "add"
                              else oracle.elementwise(op, neg(a), b), neg(ab)), op
    assert np.array_equal(oracle.elementwise("sub", a, b),
                          oracle.elementwise("add", a, neg(b)))
    one = np.full_like(a, 0x40000000)
    assert np.array_equal(oracle.elementwise("mul", a, one), a)
    assert np.array_equal(oracle.elementwise("div", a, one), a)
    zero = np.zeros_like(a)
    assert np.array_equal(oracle.elementwise("add", a, zero), a)
    # monotone: a1 <= a2 (as int32) => a1 + b <= a2 + b
    s = np.sort(a.view(np.int32))
    s1, s2 = s[:-1].view(np.uint32), s[1:].view(np.uint32)
    bb = b[: s1.size]
    r1 = oracle.elementwise("add", s1, bb).view(np.int32)
    r2 = oracle.elementwise("add", s2, bb).view(np.int32)
    assert np.all(r1 <= r2)
    # posit order equals int32 order
    d = oracle.to_double_array(np.unique(s).view(np.uint32))
    assert np.all(np.diff(d) > 0)


def test_roundtrip_double_strided(posit_checker):
    """P6: posit -> double -> posit is the identity (every 97th word)."""
    checked, bad, out = posit_checker("roundtrip32", 97)
    assert checked > 44_000_000 and bad == 0, out


@pytest.mark.slow
@pytest.mark.parametrize("op", ["sqrt", "recip"])
def test_exhaustive_unary32(posit_checker, op):
    """P6: sqrt and reciprocal over all 2^32 words."""
    checked, bad, out = posit_checker("unary32", op, 1)
    assert bad == 0, out


@pytest.mark.parametrize("op", ["sqrt", "recip"])
def test_strided_unary32(posit_checker, op):
    checked, bad, out = posit_checker("unary32", op, 211)
    assert checked > 20_000_000 and bad == 0, out
