"""Pins of the oracle's final rounding step.

Every exact weighted sum (3pCF, 4pCF, pairs) is an integer times a power of
two that the oracle holds in a 256-bit accumulator and rounds to FP64 once.
The expected values here come from Python's ``Fraction.__float__``
(integer true division, correctly rounded to nearest with ties to even by
CPython), an implementation that shares nothing with the oracle's C++.
Cases: built ties and near-ties at the 53-bit boundary (including the sum
2^64 + 2^11 + 1, which a truncate-then-round conversion gets wrong), every
sign, results below the smallest normal number, overflow to infinity, and
random integers of every width up to 255 bits.
"""
import math
import random
import struct
from fractions import Fraction

import pytest

import oracle


def bits(x: float) -> int:
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def expected(v: int, scale: int) -> float:
    q = Fraction(v) / Fraction(2) ** scale if scale >= 0 else Fraction(v * (1 << -scale))
    try:
        return float(q)
    except OverflowError:
        return math.copysign(math.inf, v)


BUILT = [
    (2 ** 64 + 2 ** 11 + 1, 0),        # just above a tie: rounds up to 2^64 + 2^12
    (2 ** 64 + 2 ** 11, 0),            # exact tie, even neighbour below
    (2 ** 64 + 3 * 2 ** 11, 0),        # exact tie, even neighbour above
    (2 ** 53 + 1, 0),                  # first integer that is not a double
    (2 ** 53 + 3, 0),
    ((2 ** 53 + 1) * 2 ** 150, 0),     # tie far above 64 bits
    ((2 ** 53 + 1) * 2 ** 150 + 1, 0),  # sticky bit 150 places below
    ((2 ** 53 - 1) * 2 ** 100 + 2 ** 99, 100),  # tie that carries into a new binade
    (2 ** 254 - 1, 0),                 # largest positive accumulator value class
    (1, 0), (3, 1), (7, 75), (123456789, 72),
    (1, 1074), (1, 1075), (3, 1075), (2 ** 60 + 1, 1130), (5, 1076),  # subnormal results
    (2 ** 200 + 2 ** 147, 300), (0, 0), (0, 500),
]


@pytest.mark.parametrize("v,scale", BUILT)
@pytest.mark.parametrize("sign", [1, -1])
def test_built_cases(v, scale, sign):
    got = oracle.exact_to_double(sign * v, scale)
    exp = expected(sign * v, scale)
    if v == 0:
        assert got == 0.0
    else:
        assert bits(got) == bits(exp), (hex(v), scale, got, exp)


def test_truncation_case_differs_from_top_64_bits():
    """The sum 2^64 + 2^11 + 1 rounds to 2^64 + 2^12; a conversion that keeps
    the top 64 significant bits and then rounds gives 2^64 instead."""
    assert oracle.exact_to_double(2 ** 64 + 2 ** 11 + 1, 0) == float(2 ** 64 + 2 ** 12)
    assert oracle.exact_to_double(-(2 ** 65 + 2 ** 12 + 1), 1) == -float(2 ** 64 + 2 ** 12)


def test_overflow_to_infinity():
    assert oracle.exact_to_double(2 ** 200, -900) == math.inf
    assert oracle.exact_to_double(-(2 ** 200), -900) == -math.inf
    # the largest finite double stays finite; the tie half an ulp above it
    # rounds to the even neighbour 2^1024, i.e. overflows
    dmax = 1.7976931348623157e308
    assert oracle.exact_to_double((2 ** 53 - 1) * 2 ** 150, 150 - 971) == dmax
    assert oracle.exact_to_double(2 ** 54 - 1, -970) == math.inf
    assert oracle.exact_to_double((2 ** 54 - 1) * 2 ** 10 - 1, -960) == dmax


def test_random_widths():
    rng = random.Random(20261204)
    for _ in range(4000):
        width = rng.randint(1, 254)
        v = rng.getrandbits(width) | (1 << (width - 1))
        if rng.random() < 0.3:  # plant a tie pattern below the 53-bit window
            if width > 60:
                cut = width - 53
                v = (v >> cut << cut) | (1 << (cut - 1))
                if rng.random() < 0.5:
                    v |= 1
        v = v if rng.random() < 0.5 else -v
        scale = rng.randint(-200, 900)
        exp = expected(v, scale)
        got = oracle.exact_to_double(v, scale)
        assert bits(got) == bits(exp), (hex(v), scale)
