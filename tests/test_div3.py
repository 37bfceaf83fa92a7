"""The division by 3 of the RK4 combination (w + y4)/3 runs as a product with
RN(1/3) and one fused multiply-add correction (Markstein's theorem).  The
same three correctly rounded operations are replayed here in exact rational
arithmetic, in float32 and float64: the result must be the correctly rounded
quotient, for random values over the exponent range and for edge cases.
"""
import math
from fractions import Fraction

import numpy as np
import pytest


def round_to(v: Fraction, mant_bits: int) -> Fraction:
    """v rounded to nearest, ties to even, with a mant_bits-bit significand
    (no exponent limits: the tested values stay in the normal range)."""
    if v == 0:
        return Fraction(0)
    s = -1 if v < 0 else 1
    a = abs(v)
    e = math.floor(math.log2(a.numerator) - math.log2(a.denominator))
    # adjust e so that 2^(mant_bits-1) <= a / 2^(e - mant_bits + 1) < 2^mant_bits
    while a >= Fraction(2) ** (e + 1):
        e += 1
    while a < Fraction(2) ** e:
        e -= 1
    scale = Fraction(2) ** (e - mant_bits + 1)
    m = a / scale
    fl = m.numerator // m.denominator
    rem = m - fl
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and fl % 2 == 1):
        fl += 1
    return s * fl * scale


def div3_emulated(x: Fraction, mant_bits: int) -> Fraction:
    t = round_to(Fraction(1, 3), mant_bits)
    q = round_to(x * t, mant_bits)
    r = round_to(Fraction(-3) * q + x, mant_bits)     # fma(-3, q, x)
    return round_to(r * t + q, mant_bits)             # fma(r, t, q)


def samples(dtype, n, seed):
    rng = np.random.default_rng(seed)
    finfo = np.finfo(dtype)
    lo, hi = (-120, 120) if dtype == np.float32 else (-1000, 1000)
    m = rng.uniform(1.0, 2.0, n).astype(dtype)
    e = rng.integers(lo, hi, n)
    x = (m * np.exp2(e.astype(np.float64))).astype(dtype) * rng.choice([-1, 1], n).astype(dtype)
    edge = [1.0, 3.0, 1.5, 2.0 ** -10, 3.0 * 2 ** 20, float(finfo.max) / 4, float(finfo.tiny) * 8,
            1.0 + float(finfo.eps), 2.0 - float(finfo.eps), 6.0, 0.75]
    return [Fraction(float(v)) for v in x] + [Fraction(v) for v in edge] + [Fraction(-v) for v in edge]


@pytest.mark.parametrize("dtype,mant_bits", [(np.float32, 24), (np.float64, 53)])
def test_div3_is_correctly_rounded(dtype, mant_bits):
    for x in samples(dtype, 4000, 5):
        x = round_to(x, mant_bits)
        assert div3_emulated(x, mant_bits) == round_to(x / 3, mant_bits), float(x)


def test_product_with_rounded_third_alone_is_biased():
    """Why the correction step is there: x * RN(1/3) alone is not the
    correctly rounded quotient, and RN(1/3) > 1/3 in float32 biases it up."""
    t = round_to(Fraction(1, 3), 24)
    assert t > Fraction(1, 3)
    bad = 0
    for x in samples(np.float32, 2000, 6):
        x = round_to(x, 24)
        bad += round_to(x * t, 24) != round_to(x / 3, 24)
    assert bad > 0
