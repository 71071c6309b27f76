"""Exact-rational restatements used to pin the oracle (tests only).

Everything here is written directly from the definitions with Python's
``fractions.Fraction``; it shares nothing with ``oracle/lcp_oracle.c``.
"""
from __future__ import annotations

import math
import struct
from fractions import Fraction

import numpy as np


def F(x) -> Fraction:
    return Fraction(float(np.float32(x)))


def q1(x, m, e) -> int:
    """Eq. quantization: floor((x - min) / (2 eb))."""
    return math.floor((F(x) - F(m)) / (2 * F(e)))


def rn32(v: Fraction) -> np.float32:
    """Nearest binary32 to v, ties to even (no overflow handling needed)."""
    if v == 0:
        return np.float32(0.0)
    neg = v < 0
    a = -v if neg else v
    # exponent E with 2^E <= a < 2^(E+1)
    E = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** E > a:
        E -= 1
    elif Fraction(2) ** (E + 1) <= a:
        E += 1
    quantum = Fraction(2) ** (max(E, -126) - 23)
    k = a / quantum
    fl = math.floor(k)
    rem = k - fl
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and fl % 2 == 1):
        fl += 1
    r = np.float32(float(fl * quantum))
    assert Fraction(float(r)) == fl * quantum
    return np.float32(-r) if neg else r


def q2(q: int, m, e) -> np.float32:
    """Eq. quantization (reverse): (2q + 1) eb + min, rounded once."""
    return rn32(F(m) + (2 * q + 1) * F(e))


def q3(x, xr, e) -> bool:
    """|x - x'| > eb."""
    return abs(F(x) - F(xr)) > F(e)


def round_down_f32(d: float) -> np.float32:
    f = np.float32(d)
    if Fraction(float(f)) > Fraction(d):
        f = np.nextafter(f, np.float32(-np.inf), dtype=np.float32)
    return f


def f32_bits(x) -> int:
    return struct.unpack("<I", struct.pack("<f", float(np.float32(x))))[0]


def total_order_key(x) -> int:
    b = f32_bits(x)
    return (~b & 0xFFFFFFFF) if b & 0x80000000 else (b | 0x80000000)
