"""Pins of the CPU oracle against what the paper and mathematics fix.

No test here compares the oracle with itself: each checks it against a
closed form read off the format definition (Sec. 3.1, Table 1, Sec. 2's value
formula), exact rational arithmetic (tests/exact.py), a library routine
(PyTorch's binary32 -> bfloat16 rounding, NumPy's float64 products), brute
force over every code of the small widths, or hand-derived worked examples
(tests/golden/pack_examples.txt).
"""
from __future__ import annotations

import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1601_07789_gb300 import inputs
from tests import exact

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "pack_examples.txt")
MODES = {"rne": oracle.RNE, "rtz": oracle.RTZ, "half": oracle.HALF_UP, "rto": oracle.RTO}
FORMATS = [(0, k) for k in range(1, 5)] + [(1, k) for k in range(1, 9)]


def _bits_of(values, base):
    return np.asarray(values, dtype=np.float32 if base == 0 else np.float64).view(
        np.uint32 if base == 0 else np.uint64)


def _codes_from_stream(stream: np.ndarray, k: int) -> np.ndarray:
    b = stream.reshape(-1, k).astype(np.uint64)
    q = np.zeros(b.shape[0], dtype=np.uint64)
    for i in range(k):
        q |= b[:, i] << np.uint64(8 * i)
    return q


def _stream_from_codes(q: np.ndarray, k: int) -> np.ndarray:
    q = q.astype(np.uint64)
    out = np.empty((q.size, k), dtype=np.uint8)
    for i in range(k):
        out[:, i] = ((q >> np.uint64(8 * i)) & np.uint64(0xFF)).astype(np.uint8)
    return out.reshape(-1)


def _is_nan_bits(u: np.ndarray, base: int) -> np.ndarray:
    if base == 0:
        return ((u & 0x7F800000) == 0x7F800000) & ((u & 0x007FFFFF) != 0)
    return ((u & np.uint64(0x7FF0000000000000)) == np.uint64(0x7FF0000000000000)) & (
        (u & np.uint64(0x000FFFFFFFFFFFFF)) != 0)


# ---- golden worked examples ------------------------------------------------

def _golden_rows():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split(None, 5)
            rows.append((parts[0], int(parts[1]), parts[2], int(parts[3], 16), int(parts[4], 16)))
    return rows


@pytest.mark.parametrize("row", _golden_rows(), ids=lambda r: f"{r[0]}k{r[1]}{r[2]}_{r[3]:x}")
def test_golden_pack_examples(row):
    base_s, k, mode, u, expect = row
    base = 0 if base_s == "f32" else 1
    assert oracle.pack_bits(base, k, MODES[mode], u) == expect


def test_golden_stream_byte_order():
    # 1.0 at k = 5: the stream holds the top five bytes least significant first (Fig. 1)
    s = oracle.pack(np.array([1.0]), 1, 5)
    assert list(s) == [0x00, 0x00, 0x00, 0xF0, 0x3F]


# ---- unpack ------------------------------------------------------------------

@pytest.mark.parametrize("base,k", FORMATS)
def test_unpack_value_formula(base, k):
    """unpack(q) has the value Sec. 2's formula gives for q's own fields."""
    n = 3000
    codes = inputs.random_codes(n, k, seed=100 + 10 * base + k)
    bits = oracle.unpack(codes, base, k)
    q = _codes_from_stream(codes, k)
    for i in range(n):
        want = exact.code_value(base, k, int(q[i]))
        got = exact.native_value(base, int(bits[i]))
        if want == exact.NAN:
            assert got == exact.NAN
        else:
            assert got == want


def test_unpack_flyte24_fig1():
    """Fig. 1: a 24-bit flyte widens to binary32 as num << 8."""
    q = np.arange(0, 1 << 24, 4099, dtype=np.uint64)
    bits = oracle.unpack(_stream_from_codes(q, 3), 0, 3)
    assert np.array_equal(bits.astype(np.uint64), (q << np.uint64(8)) & np.uint64(0xFFFFFFFF))


def test_unpack_bf16_library_exhaustive():
    torch = pytest.importorskip("torch")
    q = np.arange(1 << 16, dtype=np.uint64)
    bits = oracle.unpack(_stream_from_codes(q, 2), 0, 2)
    lib = torch.from_numpy(q.astype(np.uint16).view(np.int16)).view(torch.bfloat16).float()
    assert np.array_equal(bits, lib.numpy().view(np.uint32))


@pytest.mark.parametrize("base", [0, 1])
def test_full_width_identity(base):
    k = 4 if base == 0 else 8
    codes = inputs.random_codes(20000, k, seed=7 + base)
    bits = oracle.unpack(codes, base, k)
    assert np.array_equal(_codes_from_stream(codes, k), bits.astype(np.uint64))
    for mode in MODES.values():
        assert np.array_equal(oracle.pack(bits, base, k, mode), codes)


# ---- pack against the library's bfloat16 rounding -----------------------------

def test_pack_f32_k2_equals_bfloat16_library():
    torch = pytest.importorskip("torch")
    hi = np.arange(1 << 16, dtype=np.uint32) << 16
    lows = np.array([0, 1, 0x7FFF, 0x8000, 0x8001, 0xFFFF], dtype=np.uint32)
    u = (hi[:, None] | lows[None, :]).reshape(-1)
    u = np.concatenate([u, np.random.default_rng(11).integers(0, 1 << 32, size=1 << 20,
                                                              dtype=np.uint64).astype(np.uint32)])
    u = u[~_is_nan_bits(u, 0)]
    got = _codes_from_stream(oracle.pack(u, 0, 2, oracle.RNE), 2)
    lib = torch.from_numpy(u.view(np.float32)).to(torch.bfloat16).view(torch.int16).numpy()
    assert np.array_equal(got.astype(np.uint16), lib.view(np.uint16))


# ---- pack against exact nearest / toward-zero / odd -----------------------------

def _finite_samples(base, n, seed):
    if base == 0:
        u = inputs.mixture_f32(n, seed=seed)
    else:
        u = inputs.mixture_f64(n, seed=seed)
    u = u[~_is_nan_bits(u, base)]
    W = 32 if base == 0 else 64
    inf = (0x7F800000 if base == 0 else 0x7FF0000000000000)
    mag = u & ((1 << (W - 1)) - 1) if base == 0 else u & np.uint64((1 << 63) - 1)
    return u[mag != inf]


@pytest.mark.parametrize("base,k", [f for f in FORMATS if f[1] >= 2 and f[1] < (4 if f[0] == 0 else 8)])
@pytest.mark.parametrize("mode", ["rne", "rtz", "rto"])
def test_pack_matches_exact_rounding(base, k, mode):
    u = _finite_samples(base, 1500, seed=500 + 17 * k + base)
    codes = _codes_from_stream(oracle.pack(u, base, k, MODES[mode]), k)
    W = 32 if base == 0 else 64
    for i in range(u.size):
        ui = int(u[i])
        x = exact.native_value(base, ui)
        want = exact.round_to_code(base, k, x, bool(ui >> (W - 1)), mode)
        assert int(codes[i]) == want, (hex(ui), mode)


@pytest.mark.parametrize("base,k", [f for f in FORMATS if 2 <= f[1] < (4 if f[0] == 0 else 8)])
def test_pack_half_up_is_fig6(base, k):
    """Fig. 6 on the whole pattern: (u + half ULP) >> dropped bits, for non-NaN input."""
    u = _finite_samples(base, 4000, seed=900 + k + base)
    W = 32 if base == 0 else 64
    d = W - 8 * k
    got = _codes_from_stream(oracle.pack(u, base, k, oracle.HALF_UP), k)
    fig6 = [(int(v) + (1 << (d - 1))) >> d for v in u]
    assert [int(c) for c in got] == fig6


# ---- k = 1: rounding in bit-pattern order, found by search ----------------------
# A one-byte code keeps the sign and the top 7 exponent bits only (the "top k
# bytes" reading of Sec. 3.1 / Table 1), so its 128 magnitudes are the patterns
# c << d (d = W - 8).  Nearest, ties, Fig. 6 and round to odd are taken in that
# pattern order, and the magnitude saturates at 0x7F: there is no Inf or NaN
# code.  The search below looks the neighbours up in the list of all 128
# patterns; it shares nothing with the oracle's shift-and-compare.

def _k1_by_search(base: int, u: int, mode: str) -> int:
    import bisect
    W = 32 if base == 0 else 64
    d = W - 8
    sign = u >> (W - 1)
    mag = u & ((1 << (W - 1)) - 1)
    exp_all_ones = (0xFF << 23) if base == 0 else (0x7FF << 52)
    if mag & exp_all_ones == exp_all_ones:           # Inf or NaN: no such code at k = 1
        return (sign << 7) | 0x7F
    patterns = [c << d for c in range(128)]          # every magnitude a code can hold
    lo = bisect.bisect_right(patterns, mag) - 1      # largest pattern <= mag
    if patterns[lo] == mag:
        c = lo
    elif mode == "rtz":
        c = lo
    elif mode == "rto":
        c = lo if lo % 2 == 1 else lo + 1           # the odd one of the two neighbours
    elif lo == 127:
        c = 127                                      # beyond the largest code: saturate
    else:
        below, above = mag - patterns[lo], patterns[lo + 1] - mag
        if below < above:
            c = lo
        elif below > above:
            c = lo + 1
        elif mode == "half":
            c = lo + 1
        else:
            c = lo if lo % 2 == 0 else lo + 1
    return (sign << 7) | c


def _k1_samples(base: int) -> list[int]:
    W = 32 if base == 0 else 64
    d = W - 8
    h = 1 << (d - 1)
    drops = [0, 1, h - 1, h, h + 1, 2 * h - 1, h // 3, h + h // 5]
    out = [(top << d) | r for top in range(256) for r in drops]
    g = np.random.default_rng(1234 + base)
    out += [int(v) for v in g.integers(0, 1 << (W - 1), size=3000, dtype=np.uint64)]
    out += [int(v) | (1 << (W - 1)) for v in g.integers(0, 1 << (W - 1), size=1000, dtype=np.uint64)]
    return out


@pytest.mark.parametrize("base", [0, 1])
@pytest.mark.parametrize("mode", ["rne", "rtz", "rto", "half"])
def test_pack_k1_matches_pattern_order_search(base, mode):
    """Every top byte with ties at even and odd kept parts, near-ties, Inf/NaN and random patterns."""
    u = np.array(_k1_samples(base), dtype=np.uint32 if base == 0 else np.uint64)
    got = _codes_from_stream(oracle.pack(u, base, 1, MODES[mode]), 1)
    for ui, c in zip(u, got):
        assert int(c) == _k1_by_search(base, int(ui), mode), (hex(int(ui)), mode)


# ---- round trip, exhaustive over small widths ----------------------------------

@pytest.mark.parametrize("base,k", [(0, 1), (0, 2), (0, 3), (1, 1), (1, 2)])
def test_round_trip_exhaustive(base, k):
    q = np.arange(1 << (8 * k), dtype=np.uint64)
    stream = _stream_from_codes(q, k)
    bits = oracle.unpack(stream, base, k)
    nan = _is_nan_bits(bits, base)
    E = 8 if base == 0 else 11
    quiet = np.uint64(1 << (8 * k - 2 - E)) if k >= 2 else np.uint64(0)
    expect = np.where(nan, q | quiet, q)   # a signalling NaN comes back quiet
    for mode in MODES.values():
        back = _codes_from_stream(oracle.pack(bits, base, k, mode), k)
        assert np.array_equal(back, expect)


# ---- monotonicity of pack ---------------------------------------------------

@pytest.mark.parametrize("base,k", FORMATS)
@pytest.mark.parametrize("mode", ["rne", "rtz", "rto", "half"])
def test_pack_monotone(base, k, mode):
    g = np.random.default_rng(31 + k)
    if base == 0:
        v = np.sort(np.concatenate([g.standard_normal(20000), g.uniform(-3e38, 3e38, 2000),
                                    g.uniform(-1e-38, 1e-38, 2000)]).astype(np.float32))
    else:
        v = np.sort(np.concatenate([g.standard_normal(20000), g.uniform(-1.0, 1.0, 2000) * 1e308,
                                    g.uniform(-1e-306, 1e-306, 2000)]))
    v = v[np.isfinite(v)]
    back = oracle.unpack(oracle.pack(v, base, k, MODES[mode]), base, k)
    w = back.view(np.float32 if base == 0 else np.float64).astype(np.float64)
    assert np.all(np.diff(w) >= 0)


# ---- special values (Sec. 5.3) ------------------------------------------------

@pytest.mark.parametrize("base,k", [f for f in FORMATS if f[1] >= 2])
@pytest.mark.parametrize("mode", ["rne", "rtz", "rto", "half"])
def test_specials_stay_special(base, k, mode):
    W = 32 if base == 0 else 64
    E = 8 if base == 0 else 11
    full = W // 8
    u = inputs.special_f32(np.random.default_rng(5), 4000) if base == 0 else \
        inputs.special_f64(np.random.default_rng(5), 4000)
    codes = _codes_from_stream(oracle.pack(u, base, k, MODES[mode]), k)
    for ui, c in zip(u, codes):
        ui, c = int(ui), int(c)
        x = exact.native_value(base, ui)
        v = exact.code_value(base, k, c)
        if x == exact.NAN:
            assert v == exact.NAN or k == full
        elif isinstance(x, tuple):
            assert v == x                     # signed infinity preserved
        else:
            assert c >> (8 * k - 1) == ui >> (W - 1)   # sign preserved, zeros included


# ---- dot / axpy / gemv / gemm against exact sums and libraries -------------------

def _dot2_bound(n, exact_sum, absum):
    eps = 2.0 ** -53
    gam = n * eps / (1 - n * eps)
    return eps * abs(exact_sum) + gam * gam * absum


@pytest.mark.parametrize("n", [1, 2, 7, 33, 64])
@pytest.mark.parametrize("kind", ["random", "cancel", "positive"])
def test_dot_exact_small(n, kind):
    g = np.random.default_rng(1000 + n)
    fx, fy = (1, 7), (1, 8)      # products need more than 53 bits: the error term matters
    xv = g.standard_normal(n) * np.exp2(g.integers(-30, 30, n))
    yv = g.standard_normal(n)
    if kind == "cancel" and n > 1:
        yv[n // 2:] = -yv[: n - n // 2] if n % 2 == 0 else yv[n // 2:]
        xv[n // 2:] = xv[: n - n // 2] if n % 2 == 0 else xv[n // 2:]
    if kind == "positive":
        xv, yv = np.abs(xv), np.abs(yv)
    xs = oracle.pack(xv, *fx)
    ys = oracle.pack(yv, *fy)
    d2, naive, absum = oracle.dot(n, xs, fx, 1, ys, fy, 1)
    xq = [exact.native_value(1, int(b)) for b in oracle.unpack(xs, *fx)]
    yq = [exact.native_value(1, int(b)) for b in oracle.unpack(ys, *fy)]
    s = sum((a * b for a, b in zip(xq, yq)), Fraction(0))
    ab = float(sum((abs(a * b) for a, b in zip(xq, yq)), Fraction(0)))
    assert abs(Fraction(d2) - s) <= Fraction(_dot2_bound(n, float(s), ab)) * 1.000001
    eps = 2.0 ** -53
    assert abs(Fraction(naive) - s) <= Fraction(n * eps / (1 - n * eps) * ab) * 1.000001
    assert abs(absum - ab) <= n * eps * ab


@pytest.mark.parametrize("incx,incy", [(1, 1), (2, 3), (3, 1)])
def test_dot_strides_vs_numpy(incx, incy):
    n = 5000
    g = np.random.default_rng(77)
    fx, fy = (1, 4), (1, 6)
    xs = oracle.pack(g.standard_normal(n * incx), *fx)
    ys = oracle.pack(g.standard_normal(n * incy), *fy)
    xv = oracle.values(xs, *fx)[::incx][:n]
    yv = oracle.values(ys, *fy)[::incy][:n]
    d2, _, absum = oracle.dot(n, xs, fx, incx, ys, fy, incy)
    ref = float(np.dot(xv, yv))
    assert abs(d2 - ref) <= 2 * n * 2.0 ** -53 * float(np.abs(xv * yv).sum())


@pytest.mark.parametrize("base,kx,ky", [(1, 4, 4), (1, 5, 3), (1, 8, 2), (1, 8, 8), (0, 3, 2),
                                        (0, 4, 3), (0, 4, 4)])
@pytest.mark.parametrize("mode", ["rne", "rtz"])
def test_axpy_exact(base, kx, ky, mode):
    n = 400
    g = np.random.default_rng(300 + kx * 10 + ky)
    alpha = 0.1234567890123 if base == 1 else -0.37   # many bits: alpha*x is inexact
    dt = np.float32 if base == 0 else np.float64
    xs = oracle.pack(g.standard_normal(n).astype(dt), base, kx)
    ys = oracle.pack(g.standard_normal(n).astype(dt), base, ky)
    out = _codes_from_stream(oracle.axpy(n, alpha, xs, (base, kx), 1, ys, (base, ky), 1, MODES[mode]), ky)
    xq = [exact.native_value(base, int(b)) for b in oracle.unpack(xs, base, kx)]
    yq = [exact.native_value(base, int(b)) for b in oracle.unpack(ys, base, ky)]
    a = Fraction(alpha) if base == 1 else Fraction(float(np.float32(alpha)))
    for i in range(n):
        r = a * xq[i] + yq[i]                                # exact
        ub = exact.round_to_native(base, r)                  # fma: one rounding
        ri = exact.native_value(base, ub)
        if ri == 0:
            continue
        want = exact.round_to_code(base, ky, ri, ri < 0, mode) if ky < (4 if base == 0 else 8) else ub
        assert int(out[i]) == want


@pytest.mark.parametrize("base,k", [(1, 3), (1, 5), (1, 7), (1, 8), (0, 2), (0, 3), (0, 4)])
@pytest.mark.parametrize("mode", ["rne", "rtz", "rto"])
def test_scal_exact(base, k, mode):
    """scal against the exact rational product rounded once to the native type, then packed."""
    n = 300
    g = np.random.default_rng(500 + 10 * k + base)
    alpha = -0.1234567890123 if base == 1 else 0.37
    dt = np.float32 if base == 0 else np.float64
    xs = oracle.pack(g.standard_normal(n).astype(dt), base, k)
    out = _codes_from_stream(oracle.scal(n, alpha, xs, (base, k), 1, MODES[mode]), k)
    xq = [exact.native_value(base, int(b)) for b in oracle.unpack(xs, base, k)]
    a = Fraction(alpha) if base == 1 else Fraction(float(np.float32(alpha)))
    for i in range(n):
        ub = exact.round_to_native(base, a * xq[i])
        ri = exact.native_value(base, ub)
        if ri == 0:
            continue
        want = exact.round_to_code(base, k, ri, ri < 0, mode) if k < (4 if base == 0 else 8) else ub
        assert int(out[i]) == want


def test_scal_special_factors():
    """alpha = 1 leaves codes unchanged, -1 flips the sign bit, 2 raises the exponent by one."""
    k, base = 5, 1
    v = np.random.default_rng(9).standard_normal(257)
    xs = oracle.pack(v, base, k)
    q = _codes_from_stream(xs, k).astype(np.uint64)
    assert np.array_equal(oracle.scal(257, 1.0, xs, (base, k)), xs)
    q_neg = _codes_from_stream(oracle.scal(257, -1.0, xs, (base, k)), k).astype(np.uint64)
    assert np.array_equal(q_neg, q ^ np.uint64(1 << (8 * k - 1)))
    q_two = _codes_from_stream(oracle.scal(257, 2.0, xs, (base, k)), k).astype(np.uint64)
    assert np.array_equal(q_two, q + np.uint64(1 << (8 * k - 12)))   # exponent field starts at bit 8k - 12
    # strided: untouched elements keep their bytes
    out = oracle.scal(100, 2.0, xs, (base, k), incx=2)
    qs = _codes_from_stream(out, k).astype(np.uint64)
    assert np.array_equal(qs[1:200:2], q[1:200:2]) and np.array_equal(qs[0:200:2], q[0:200:2] + np.uint64(1 << (8 * k - 12)))


def test_gemv_exact_small():
    g = np.random.default_rng(41)
    for (m, n) in [(1, 1), (3, 5), (9, 4), (17, 23)]:
        fa = (1, 5)
        A = oracle.pack(g.standard_normal(m * n), *fa)
        Aq = [exact.native_value(1, int(b)) for b in oracle.unpack(A, *fa)]
        x = g.standard_normal(max(m, n))
        y = g.standard_normal(max(m, n))
        for trans in "NT":
            alpha, beta = 1.5, -0.5
            out, absum = oracle.gemv(trans, m, n, alpha, A, fa, n, x, 1, beta, y, 1)
            leny, lenx = (m, n) if trans == "N" else (n, m)
            for i in range(leny):
                t = sum((Aq[(i * n + j) if trans == "N" else (j * n + i)] * Fraction(x[j])
                         for j in range(lenx)), Fraction(0))
                ref = Fraction(alpha) * t + Fraction(beta) * Fraction(y[i])
                bound = 4 * (lenx + 2) * 2.0 ** -53 * (abs(alpha) * float(absum[i]) + abs(beta * y[i]))
                assert abs(Fraction(out[i]) - ref) <= Fraction(bound)


@pytest.mark.parametrize("trans", ["N", "T"])
def test_gemv_vs_numpy(trans):
    m, n, lda = 130, 211, 215
    g = np.random.default_rng(52)
    fa = (1, 4)
    Afull = g.standard_normal((m, lda))
    A = oracle.pack(Afull.reshape(-1), *fa)
    Av = oracle.values(A, *fa).reshape(m, lda)[:, :n]
    x = g.standard_normal(3 * max(m, n))
    y = g.standard_normal(2 * max(m, n))
    incx, incy = 3, 2
    out, absum = oracle.gemv(trans, m, n, 1.5, A, fa, lda, x, incx, -0.5, y, incy)
    if trans == "N":
        ref = 1.5 * (Av @ x[::incx][:n]) - 0.5 * y[::incy][:m]
        got = out[::incy][:m]
    else:
        ref = 1.5 * (Av.T @ x[::incx][:m]) - 0.5 * y[::incy][:n]
        got = out[::incy][:n]
    assert np.allclose(got, ref, rtol=1e-13, atol=1e-12)
    # entries of y between the strided ones are untouched
    mask = np.ones(out.size, bool)
    mask[::incy] = False
    assert np.array_equal(out[mask], y[mask])


def test_gemv_quick_returns():
    fa = (1, 4)
    A = oracle.pack(np.array([np.nan, 1.0, 2.0, 3.0]), *fa)
    x = np.array([1.0, 1.0])
    y = np.array([np.nan, 5.0])
    out, _ = oracle.gemv("N", 2, 2, 1.0, A, fa, 2, x, 1, 0.0, y, 1)   # beta = 0: y not read
    assert np.isnan(out[0]) and out[1] == 5.0
    out, _ = oracle.gemv("N", 2, 2, 0.0, A, fa, 2, x, 1, 2.0, np.array([1.0, 5.0]), 1)  # alpha = 0: A not read
    assert list(out) == [2.0, 10.0]


@pytest.mark.parametrize("fa,fb", [((0, 2), (0, 2)), ((0, 3), (0, 3)), ((0, 4), (0, 4)), ((1, 5), (1, 5))])
def test_gemm_entries_vs_numpy(fa, fb):
    M, N, K = 37, 29, 61
    g = np.random.default_rng(61)
    dt = np.float32 if fa[0] == 0 else np.float64
    A = oracle.pack(g.uniform(-1, 1, M * K).astype(dt), *fa)
    B = oracle.pack(g.uniform(-1, 1, K * N).astype(dt), *fb)
    Av = oracle.values(A, *fa).reshape(M, K)
    Bv = oracle.values(B, *fb).reshape(K, N)
    ref = Av @ Bv
    rows, cols = np.meshgrid(np.arange(M), np.arange(N), indexing="ij")
    out, absum = oracle.gemm_entries(rows.reshape(-1), cols.reshape(-1), K, 1.0, A, fa, K, B, fb, N)
    assert np.allclose(out.reshape(M, N), ref, rtol=0, atol=4 * K * 2.0 ** -53 * float(absum.max()))
    assert np.allclose(absum.reshape(M, N), np.abs(Av) @ np.abs(Bv), rtol=1e-13)


def test_dot_and_gemv_special_value_classes():
    """Sec. 5.3: an infinite term gives a signed infinity, infinities of both
    signs or a NaN term give NaN (the error-free transforms are not applied)."""
    f = (1, 8)
    def d(vals_x, vals_y):
        xs = oracle.pack(np.array(vals_x, dtype=np.float64), *f)
        ys = oracle.pack(np.array(vals_y, dtype=np.float64), *f)
        return oracle.dot(len(vals_x), xs, f, 1, ys, f, 1)[0]
    assert d([1.0, np.inf, 2.0], [1.0, 1.0, 1.0]) == np.inf
    assert d([1.0, np.inf, 2.0], [1.0, -1.0, 1.0]) == -np.inf
    assert np.isnan(d([1.0, np.inf, np.inf], [1.0, 1.0, -1.0]))
    assert np.isnan(d([1.0, np.nan, 2.0], [1.0, 1.0, 1.0]))
    assert np.isnan(d([0.0, np.inf], [np.inf, 0.0]))           # 0 * Inf
    A = oracle.pack(np.array([1.0, np.inf, 3.0, 4.0]), *f)
    y, _ = oracle.gemv("N", 2, 2, 1.0, A, f, 2, np.array([1.0, 1.0]), 1, 0.0, np.zeros(2), 1)
    assert y[0] == np.inf and y[1] == 7.0


# ---- mixed-precision iterative refinement ------------------------------------------

def _dd_system(n, seed):
    g = np.random.default_rng(seed)
    A = g.standard_normal((n, n)) / np.sqrt(n) + n * np.eye(n)
    return A, g.standard_normal(n)


@pytest.mark.parametrize("k", [3, 4, 5])
def test_refine_converges_to_the_solution(k):
    """The refinement reaches the requested residual, and its x agrees with LAPACK's solve."""
    n = 256
    A, b = _dd_system(n, 70 + k)
    Ak = oracle.pack(A.reshape(-1), 1, k)
    x, it, rel = oracle.refine_jacobi(n, A, Ak, (1, k), b, np.zeros(n), 1e-12, 30, 2)
    assert rel <= 1e-12 and 1 <= it <= 30
    true_rel = np.linalg.norm(b - A @ x) / np.linalg.norm(b)     # residual recomputed by NumPy
    assert true_rel <= 2e-12
    xs = np.linalg.solve(A, b)
    smin = np.linalg.svd(A, compute_uv=False)[-1]                # ||x - xs|| <= ||A^-1|| ||r||
    assert np.linalg.norm(x - xs) <= 1.01 * np.linalg.norm(b - A @ x) / smin + 1e-15 * np.linalg.norm(xs)


@pytest.mark.parametrize("k", [3, 4, 5])
def test_refine_harder_system_converges(k):
    """With diagonal 10 (Jacobi contraction about 1/10 per sweep) and 8 sweeps per correction the
    refinement still reaches 1e-12; its x agrees with LAPACK's solve; k = 3, whose stored entries err
    by up to 2^-13 relative, needs at least as many corrections as k = 5."""
    n = 256
    g = np.random.default_rng(40 + k)
    A = g.standard_normal((n, n)) / np.sqrt(n) + 10.0 * np.eye(n)
    b = g.standard_normal(n)
    Ak = oracle.pack(A.reshape(-1), 1, k)
    x, it, rel = oracle.refine_jacobi(n, A, Ak, (1, k), b, np.zeros(n), 1e-12, 40, 8)
    assert rel <= 1e-12 and 1 <= it <= 40
    xs = np.linalg.solve(A, b)
    smin = np.linalg.svd(A, compute_uv=False)[-1]
    assert np.linalg.norm(x - xs) <= 1.01 * np.linalg.norm(b - A @ x) / smin + 1e-15 * np.linalg.norm(xs)
    it5 = oracle.refine_jacobi(n, A, oracle.pack(A.reshape(-1), 1, 5), (1, 5), b, np.zeros(n), 1e-12, 40, 8)[1]
    assert it >= it5 if k == 3 else True


def test_refine_one_step_semantics():
    """max_outer = 1 with one sweep is exactly x1 = x0 + D^-1 (b - A x0), written out in NumPy; with
    tol = inf nothing is corrected; the contraction per correction follows the stored precision."""
    n = 64
    A, b = _dd_system(n, 7)
    x0 = np.random.default_rng(8).standard_normal(n)
    Ak = oracle.pack(A.reshape(-1), 1, 4)
    x1, it, _ = oracle.refine_jacobi(n, A, Ak, (1, 4), b, x0, 0.0, 1, 1)
    want = x0 + (b - A @ x0) / np.diag(A)
    assert it == 1 and np.max(np.abs(x1 - want)) <= 1e-12 * np.max(np.abs(want))
    x2, it2, rel2 = oracle.refine_jacobi(n, A, Ak, (1, 4), b, x0, np.inf, 10, 2)
    assert it2 == 0 and np.array_equal(x2, x0)
    assert abs(rel2 - np.linalg.norm(b - A @ x0) / np.linalg.norm(b)) <= 1e-12
    # fewer stored bytes converge more slowly: k = 3 needs at least as many corrections as k = 5
    its = [oracle.refine_jacobi(n, A, oracle.pack(A.reshape(-1), 1, k), (1, k), b, np.zeros(n), 1e-14, 30, 4)[1]
           for k in (3, 5)]
    assert its[0] >= its[1]
