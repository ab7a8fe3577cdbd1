"""Exactness of two device-side decision rules, checked on the host with the
device's arithmetic emulated bit for bit (IEEE binary64 with round-to-nearest is
Python's float; binary32 rounding is numpy's float32; fused multiply-adds are
formed exactly with rationals and rounded once).

1. The changeover band side in FP32 (the small-group Bulirsch-Stoer and KickS
   kernels): from r truncated to float and 1/rc rounded towards zero, the float
   product p decides K = 0 (p < 0.09999) or K = 1 (p > 1.0001) only where the FP64
   evaluation of changeover_fast takes the same branch: y = fma(r, 1/rc, -0.1) *
   RN(1/0.9) <= 0, resp. >= 1 (the changeover function K of Sec. 6.3, reading R4:
   K = 0 below 0.1 rc, K = 1 above rc).
2. The kick's fold (the compensated sum of the partial sums): Fast2Sum on the
   two operands ordered by the high 32 bits of their magnitudes returns the same
   sum and the same exact error term as TwoSum, for finite operands.
"""
import struct
from fractions import Fraction

import numpy as np

RNG = np.random.default_rng(20220125)


def _bits(x: float) -> int:
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def _from_bits(b: int) -> float:
    return struct.unpack("<d", struct.pack("<Q", b))[0]


def _trunc_to_f32(x: float) -> float:
    """A positive normal double in the float range truncated to 24 significant
    bits (the device's f32_of_f64_trunc and, for positive values, RZ)."""
    return _from_bits(_bits(x) & ~((1 << 29) - 1))


def _side_f32(r: float, irc: float) -> int:
    p = np.float32(_trunc_to_f32(r) * _trunc_to_f32(irc))    # exact product, one float rounding
    if p < np.float32(0.09999):
        return -1
    if p > np.float32(1.0001):
        return 1
    return 0


INV09 = 1.0 / 0.9                                             # RN(1/0.9), as the device constant


def _y_fp64(r: float, irc: float) -> float:
    fma = float(Fraction(r) * Fraction(irc) - Fraction(0.1))  # fma(r, irc, -0.1): one rounding
    return fma * INV09


def _check_side(r: float, irc: float) -> int:
    side = _side_f32(r, irc)
    y = _y_fp64(r, irc)
    if side < 0:
        assert y <= 0.0, (r, irc, y)
    elif side > 0:
        assert y >= 1.0, (r, irc, y)
    return side


def test_changeover_side_decisions_are_exact():
    sides = {-1: 0, 0: 0, 1: 0}
    # log-uniform r and 1/rc over the ranges of the disks (AU; rc from ~1e-5 to 1 AU)
    r = np.exp(RNG.uniform(np.log(1e-7), np.log(1e2), 4000))
    irc = np.exp(RNG.uniform(np.log(1e-1), np.log(1e6), 4000))
    for a, b in zip(r, irc):
        sides[_check_side(float(a), float(b))] += 1
    # adversarial: r/rc within 2e-4 of the two thresholds, where the margins bite
    for target in (0.1, 1.0):
        irc = np.exp(RNG.uniform(np.log(1e-1), np.log(1e6), 4000))
        rel = RNG.uniform(-2e-4, 2e-4, 4000)
        for b, e in zip(irc, rel):
            a = target * (1.0 + e) / float(b)
            sides[_check_side(a, float(b))] += 1
    assert sides[-1] > 1000 and sides[1] > 1000 and sides[0] > 1000


def _two_sum(a: float, b: float):
    s = a + b
    bb = s - a
    return s, (a - (s - bb)) + (b - bb)


def _two_sum_ordered(a: float, b: float):
    ha = (_bits(a) >> 32) & 0x7FFFFFFF
    hb = (_bits(b) >> 32) & 0x7FFFFFFF
    big, small = (a, b) if ha >= hb else (b, a)
    s = big + small
    return s, small - (s - big)


def test_fast2sum_ordered_by_high_word_is_exact():
    n = 20000
    # magnitudes over 60 binades, both signs; pairs with equal exponents and
    # near-cancelling pairs included
    a = RNG.standard_normal(n) * np.exp2(RNG.integers(-30, 30, n))
    b = RNG.standard_normal(n) * np.exp2(RNG.integers(-30, 30, n))
    b[: n // 4] = a[: n // 4] * (1.0 + RNG.uniform(-1e-9, 1e-9, n // 4)) * -1.0
    b[n // 4: n // 2] = a[n // 4: n // 2] * RNG.uniform(0.5, 2.0, n // 4)
    b[-10:] = 0.0
    for x, y in zip(a, b):
        x, y = float(x), float(y)
        s1, e1 = _two_sum(x, y)
        s2, e2 = _two_sum_ordered(x, y)
        assert s1 == s2 and e1 == e2, (x, y, s1, e1, s2, e2)
        # and the error term is the exact rounding error of the sum
        assert Fraction(s2) + Fraction(e2) == Fraction(x) + Fraction(y)
