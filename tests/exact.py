"""Exact rational arithmetic for pinning the oracle (test infrastructure).

Nothing here calls the oracle or the CUDA library.  Values are computed from
the fields of a code with the IEEE-754 value formula (Sec. 2 of the paper:
v = (-1)^s (1 + sum m_i 2^-i) 2^(e - bias), subnormals 0.m 2^(1 - bias)),
using Python's exact ``Fraction``; rounding is decided by comparing exact
distances to neighbouring codes.
"""
from __future__ import annotations

import math
from fractions import Fraction

INF = "inf"
NAN = "nan"


def params(base: int) -> tuple[int, int, int]:
    """(W, E, bias) of the native type a flyte widens to (Table 1)."""
    return (32, 8, 127) if base == 0 else (64, 11, 1023)


def code_value(base: int, k: int, q: int):
    """Exact value of a k-byte code from its own fields: Fraction, ('inf', s) or 'nan'."""
    W, E, bias = params(base)
    bits = 8 * k
    s = q >> (bits - 1)
    rest = q & ((1 << (bits - 1)) - 1)
    if k == 1:
        # only the top 7 exponent bits are kept; the dropped ones read as zero
        e = rest << (E - 7)
        mbits, m = 0, 0
    else:
        mbits = bits - 1 - E
        e = rest >> mbits
        m = rest & ((1 << mbits) - 1)
        if e == (1 << E) - 1:
            return NAN if m else (INF, s)
    if e == 0:
        v = Fraction(m, 1 << mbits) * Fraction(2) ** (1 - bias)
    else:
        v = (1 + Fraction(m, 1 << mbits)) * Fraction(2) ** (e - bias)
    return -v if s else v


def native_value(base: int, u: int):
    """Exact value of a native bit pattern (binary32 or binary64)."""
    W, _, _ = params(base)
    return code_value(base, W // 8, u)


def max_code(base: int, k: int) -> int:
    """Largest magnitude code that is finite (all-ones exponent excluded for k >= 2)."""
    W, E, _ = params(base)
    bits = 8 * k
    if k == 1:
        return 0x7F
    mbits = bits - 1 - E
    return (((1 << E) - 2) << mbits) | ((1 << mbits) - 1)


def _floor_code(base: int, k: int, a: Fraction) -> int:
    """Largest magnitude code t (sign 0) with value(t) <= a, for 0 <= a."""
    lo, hi = 0, max_code(base, k)
    if code_value(base, k, hi) <= a:
        return hi
    while hi - lo > 1:
        mid = (lo + hi) // 2
        if code_value(base, k, mid) <= a:
            lo = mid
        else:
            hi = mid
    return lo


def round_to_code(base: int, k: int, x: Fraction, negative: bool, mode: str) -> int:
    """Code of the k-byte format nearest to the finite value x, by exact search.

    mode: 'rne' (nearest, ties to the even code), 'rtz' (toward zero),
    'rto' (round to odd).  IEEE overflow: rne gives Inf at or beyond max +
    half an ULP; rtz and rto stay at the largest finite code.  k >= 2 only.
    """
    assert k >= 2
    W, E, _ = params(base)
    bits = 8 * k
    sign = (1 << (bits - 1)) if negative else 0
    a = abs(x)
    t = _floor_code(base, k, a)
    top = max_code(base, k)
    vt = code_value(base, k, t)
    if mode == "rtz":
        return sign | t
    if mode == "rto":
        return sign | (t if vt == a else (t | 1))
    # rne
    if vt == a:
        return sign | t
    if t == top:
        ulp = vt - code_value(base, k, t - 1)
        return sign | (t + 1 if a >= vt + ulp / 2 else t)   # t + 1 is the Inf code
    vn = code_value(base, k, t + 1)
    if a - vt < vn - a:
        return sign | t
    if a - vt > vn - a:
        return sign | (t + 1)
    return sign | (t if t % 2 == 0 else t + 1)


def round_to_native(base: int, x: Fraction) -> int:
    """Bit pattern of x rounded to nearest-even in binary32/binary64 (for fma pins)."""
    W, _, _ = params(base)
    return round_to_code(base, W // 8, x, x < 0, "rne")


def f64_fraction(v: float) -> Fraction:
    assert math.isfinite(v)
    return Fraction(v)
