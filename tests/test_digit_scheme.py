"""The arithmetic of the digit-sliced tensor-core line operators, on the CPU in exact integers.

The GPU kernels (FP64 form: seven digits; mixed form's tensor option: four)
compute a dense line product y = B x from balanced base-256 digits of
fixed-point images of each line and operator row, with the digit levels
accumulated exactly.  These tests restate that scheme in exact integer and
rational arithmetic and check the claims the kernels rely on:

* the balanced digits reproduce the fixed-point integer and stay within
  [-128, 128], so every digit is exact in BF16;
* every level sum of digit products stays below 2^24 for lines of up to 80
  entries, so an FP32 accumulator holds it exactly;
* the result, rounded once, is within a few units of 2^-53 of
  max|x| sum|B| + max|B| sum|x| (seven digits), or of 2^-24 (four digits,
  FP32 output), also for lines whose entries span many orders of magnitude;
* the kernels' integer rounding of the final accumulator to FP64 or FP32 is
  exact round-to-nearest-even.

The GPU parity tests (tests/test_gpu_digit.py, tests/test_gpu_mixed.py)
check the kernels themselves against the oracle.
"""
import math
import random
import struct
from fractions import Fraction

import numpy as np
import pytest

C_OFFSET = {7: 0x80808080808080, 4: 0x80808080}


def _bits(v):
    return struct.unpack("<Q", struct.pack("<d", float(v)))[0]


def _exponent(v):
    return (_bits(v) >> 52) & 0x7FF


def fixed_point(v, E, nd):
    """Round v to the integer X = round(v / 2^(E - 1023 - 52 - kTop)), kTop = 8 nd - 1 - 53."""
    b = _bits(v)
    e = (b >> 52) & 0x7FF
    M = (b & ((1 << 52) - 1)) | ((1 << 52) if e else 0)
    sh = E - max(e, 1) - (8 * nd - 1 - 53)
    if sh <= 0:
        mag = M << (-sh)
    else:
        mag = 0 if sh >= 60 else (M + (1 << (sh - 1))) >> sh
    return -mag if b >> 63 else mag


def digits(X, nd):
    """Balanced base-256 digits of X, most significant first, from the bytes of X + C."""
    u = X + C_OFFSET[nd]
    assert 0 < u < 2 ** (8 * nd + 1)
    low = [((u >> (8 * j)) & 255) - 128 for j in range(nd - 1)][::-1]
    return [((u >> (8 * (nd - 1))) & 511) - 128] + low


def scale(E, nd):
    """log2 of the fixed-point unit of a line whose largest exponent field is E."""
    return E - 1023 - 52 - (8 * nd - 1 - 53)


def digit_product(B, x, nd):
    """y_i = sum_k B_ik x_k by the scheme: levels 0..nd-1 of the digit products, Horner, one rounding."""
    n = len(x)
    E = max([1] + [_exponent(v) for v in x])
    dx = [digits(fixed_point(v, E, nd), nd) for v in x]
    y = []
    for i in range(B.shape[0]):
        F = max([1] + [_exponent(v) for v in B[i]])
        db = [digits(fixed_point(v, F, nd), nd) for v in B[i]]
        levels = []
        for lv in range(nd):
            P = sum(db[k][lv - t] * dx[k][t] for t in range(lv + 1) for k in range(n))
            assert abs(P) < 2 ** 24, "a level sum must be exact in FP32"
            levels.append(P)
        acc = levels[0]
        for lv in range(1, nd - 1):
            acc = acc * 256 + levels[lv]
        acc += levels[nd - 1] >> 8  # floor
        y.append(Fraction(acc) * Fraction(2) ** (8 * nd + scale(E, nd) + scale(F, nd)))
    return y


@pytest.mark.parametrize("nd", [7, 4])
def test_digits_reconstruct_and_fit_bf16(nd):
    rng = np.random.default_rng(11)
    vals = np.concatenate([rng.standard_normal(300) * np.exp(rng.uniform(-30, 30, 300)),
                           [np.nextafter(2.0, 0.0), -np.nextafter(1.0, 0.0), 1e-310, -0.0, 0.0]])
    E = max(_exponent(v) for v in vals)
    for v in vals:
        X = fixed_point(v, E, nd)
        d = digits(X, nd)
        assert sum(dd * 256 ** (nd - 1 - t) for t, dd in enumerate(d)) == X
        assert all(-128 <= dd <= 128 for dd in d)
        assert abs(X) < 2 ** (8 * nd - 1)


def _bound(B, x, i):
    ax, ab = np.abs(x), np.abs(B[i])
    return Fraction(float(ax.max() * ab.sum() + ab.max() * ax.sum()))


@pytest.mark.parametrize("n,spread", [(66, 1.0), (80, 8.0), (9, 20.0)])
def test_seven_digits_reach_fp64_accuracy(n, spread):
    """Error of the seven-digit product, before the final rounding to FP64, within 2^-53 of the bound
    (the final rounding adds at most half an ulp of |y|)."""
    rng = np.random.default_rng(n)
    B = rng.standard_normal((n, n)) * np.exp(rng.uniform(-3, 3, (n, n)))
    X = rng.standard_normal((3, n)) * np.exp(rng.uniform(-spread, spread, (3, n)))
    X[1, 0] = np.nextafter(2.0, 0.0) * np.max(np.abs(X[1]))  # a mantissa next to a power of two
    for x in X:
        y = digit_product(B, x, 7)
        for i in range(n):
            exact = sum(Fraction(float(B[i, k])) * Fraction(float(x[k])) for k in range(n))
            assert abs(y[i] - exact) <= Fraction(2) ** -53 * _bound(B, x, i)


def test_four_digits_reach_fp32_accuracy():
    """The mixed form's four digits: error within 2^-29 of the bound, below the final FP32 rounding."""
    rng = np.random.default_rng(4)
    n = 66
    B = rng.standard_normal((n, n))
    x = rng.standard_normal(n) * np.exp(rng.uniform(-2, 2, n))
    y = digit_product(B, x, 4)
    for i in range(n):
        exact = sum(Fraction(float(B[i, k])) * Fraction(float(x[k])) for k in range(n))
        assert abs(y[i] - exact) <= Fraction(2) ** -29 * _bound(B, x, i)


def test_worst_case_level_sums_fit_fp32():
    """All-extreme digits (every digit -128 or 128) over 80 entries: the largest level sum is
    7 * 80 * 128^2 < 2^24."""
    worst = 7 * 80 * 128 * 128
    assert worst < 2 ** 24
    # the top digit reaches 128 only for |X| close to 2^55; the bound above already assumes it
    assert digits(2 ** 55 - 1, 7)[0] == 128


def _clz64(a):
    return 64 - a.bit_length()


def _kernel_round(acc, e2, mant):
    """The digit kernels' integer rounding of acc * 2^e2 to a normal FP64 (mant = 52) or FP32
    (mant = 23) number, restated: leading bit to position mant by a left shift, or a right shift
    that adds half - 1 plus the kept part's lowest bit (half to even); the significand keeps its
    leading bit, so adding it to (biased exponent - 1) << mant carries a rounding overflow into
    the exponent.  None where the kernels take their slow path (outside the normal range)."""
    if acc == 0:
        return 0.0
    bias, emax = (1023, 2046) if mant == 52 else (127, 254)
    a = -acc if acc < 0 else acc
    lz = _clz64(a)
    top = 63 - mant
    if lz >= top:
        m = a << (lz - top)
    else:
        sh = top - lz
        m = (a + ((1 << (sh - 1)) - 1) + ((a >> sh) & 1)) >> sh
    be = 63 - lz + e2 + bias
    if be < 1 or be + (m >> (mant + 1)) > emax:
        return None
    bits = ((be - 1) << mant) + m
    if mant == 52:
        return struct.unpack("<d", struct.pack("<Q", bits | ((1 << 63) if acc < 0 else 0)))[0]
    return float(struct.unpack("<f", struct.pack("<I", bits | ((1 << 31) if acc < 0 else 0)))[0])


def _exact_round(acc, e2, mant):
    """acc * 2^e2 rounded to mant + 1 significant bits, ties to even, with exact integers."""
    a = abs(acc)
    pb = a.bit_length() - 1
    if pb > mant:
        sh = pb - mant
        q, r, half = a >> sh, a & ((1 << sh) - 1), 1 << (sh - 1)
        if r > half or (r == half and q & 1):
            q += 1
        v = math.ldexp(q, sh + e2)
    else:
        v = math.ldexp(a, e2)
    return -v if acc < 0 else v


@pytest.mark.parametrize("mant", [52, 23])
def test_integer_rounding_of_the_accumulators(mant):
    """The final rounding of the digit kernels (FP64 and FP32 outputs) equals exact
    round-to-nearest-even of acc * 2^e2 on random accumulators below 2^62, on exact ties and on
    carries into the next power of two."""
    rng = random.Random(7 + mant)
    cases = []
    for _ in range(20000):
        cases.append(rng.getrandbits(rng.randint(1, 62)) * rng.choice([1, -1]))
    for k in range(1, 12):  # exact ties at every dropped-bit count
        for _ in range(200):
            cases.append((((rng.getrandbits(50) | 1) << k) | (1 << (k - 1))) * rng.choice([1, -1]))
    for n in range(mant + 1, 62):  # all ones: rounding carries into the next power of two
        cases.append((1 << n) - 1)
    checked = 0
    for acc in cases:
        e2 = rng.randint(-900, 900) if mant == 52 else rng.randint(-120, 60)
        got = _kernel_round(acc, e2, mant)
        if got is None:
            continue
        assert got == _exact_round(acc, e2, mant), (acc, e2)
        checked += 1
    assert checked > 15000
