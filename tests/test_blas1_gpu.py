"""GPU parity of flyte_dot, flyte_axpy and flyte_scal against the CPU oracle.

dot: |s_gpu - s_ref| <= 4 n 2^-53 sum|x_i y_i| + 2^-52 |s_ref| (s_ref is the
oracle's Dot2); Inf/NaN results must match in class.  axpy and scal: bit-exact codes,
except that a NaN result only has to be a NaN code (the GPU's fma returns a
canonical NaN while the CPU propagates the payload).
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
from paper_1601_07789_gb300 import flyte, inputs
from tests.gpu_util import Guarded, span_bytes, sync

pytestmark = pytest.mark.gpu
EPS = 2.0 ** -53
FORMATS = [(k, 1) for k in range(1, 9)] + [(k, 0) for k in range(1, 5)]
MODES = ["rne", "rtz", "half_up", "rto"]
ORC_MODE = {"rne": oracle.RNE, "rtz": oracle.RTZ, "half_up": oracle.HALF_UP, "rto": oracle.RTO}


def _stream(values, f):
    k, base = f
    if base == 0:
        values = np.asarray(values, dtype=np.float64).astype(np.float32)
    return oracle.pack(values, base, k)


def gpu_dot(n, xs, fx, incx, ys, fy, incy, x_off=0, y_off=0):
    X = Guarded(xs.size, x_off, fill=xs)
    Y = Guarded(ys.size, y_off, fill=ys)
    out = torch.full((1,), 12345.0, dtype=torch.float64, device="cuda")
    wsb = flyte.workspace_bytes("dot", 0, n, 0, fx)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    flyte.dot_raw(out, n, X.ptr, fx, incx, Y.ptr, fy, incy, ws, wsb)
    sync()
    return float(out.item())


def check_dot(got, n, xs, fx, incx, ys, fy, incy):
    ref, _, absum = oracle.dot(n, xs, fx[::-1], incx, ys, fy[::-1], incy)
    if np.isnan(ref):
        assert np.isnan(got)
    elif np.isinf(ref):
        assert got == ref
    else:
        assert abs(got - ref) <= 4 * n * EPS * absum + 2 * EPS * abs(ref), (got, ref, absum)


@pytest.mark.parametrize("f", FORMATS, ids=lambda f: f"k{f[0]}{'d' if f[1] else 'f'}")
def test_dot_sizes(f):
    g = np.random.default_rng(f[0] * 7 + f[1])
    for n in [0, 1, 3, 4, 5, 127, 255, 256, 1000, 4099, 65537, 1 << 20]:
        xs = _stream(g.standard_normal(n), f)
        ys = _stream(g.standard_normal(n), f)
        check_dot(gpu_dot(n, xs, f, 1, ys, f, 1), n, xs, f, 1, ys, f, 1)


@pytest.mark.parametrize("kind", ["positive", "cancel", "wide"])
@pytest.mark.parametrize("f", [(3, 1), (4, 1), (7, 1), (2, 0)])
def test_dot_adversarial(kind, f):
    n = 300001
    g = np.random.default_rng(5)
    x = g.standard_normal(n)
    y = g.standard_normal(n)
    if kind == "positive":
        x, y = np.abs(x) + 0.1, np.abs(y) + 0.1
    elif kind == "cancel":
        y[n // 2: 2 * (n // 2)] = -y[: n // 2]
        x[n // 2: 2 * (n // 2)] = x[: n // 2]
    else:
        x *= np.exp2(g.integers(-45, 45, n))
    xs, ys = _stream(x, f), _stream(y, f)
    check_dot(gpu_dot(n, xs, f, 1, ys, f, 1), n, xs, f, 1, ys, f, 1)


def test_dot_config_mixture_k4():
    """The 1,048,576-value binary64 mixtures (seeds 1601, 1602) at double-based k = 4."""
    n = 1 << 20
    f = (4, 1)
    for finite in (False, True):
        xs = oracle.pack(inputs.mixture_f64(n, 1601, finite), 1, 4)
        ys = oracle.pack(inputs.mixture_f64(n, 1602, finite), 1, 4)
        check_dot(gpu_dot(n, xs, f, 1, ys, f, 1), n, xs, f, 1, ys, f, 1)


@pytest.mark.parametrize("fx,fy,incx,incy,xo,yo", [
    ((4, 1), (4, 1), 1, 1, 3, 0), ((4, 1), (5, 1), 1, 1, 0, 0), ((3, 0), (7, 1), 2, 3, 1, 2),
    ((8, 1), (2, 0), 1, 2, 0, 5), ((6, 1), (6, 1), 3, 1, 0, 0)])
def test_dot_generic_paths(fx, fy, incx, incy, xo, yo):
    n = 20011
    g = np.random.default_rng(9)
    xs = _stream(g.standard_normal(n * incx), fx)
    ys = _stream(g.standard_normal(n * incy), fy)
    check_dot(gpu_dot(n, xs, fx, incx, ys, fy, incy, xo, yo), n, xs, fx, incx, ys, fy, incy)


def test_dot_specials_and_determinism():
    n = 100003
    f = (5, 1)
    g = np.random.default_rng(10)
    x = g.standard_normal(n)
    y = g.standard_normal(n)
    x[77] = np.inf
    xs, ys = _stream(x, f), _stream(y, f)
    got = gpu_dot(n, xs, f, 1, ys, f, 1)
    check_dot(got, n, xs, f, 1, ys, f, 1)
    y2 = y.copy()
    y2[5000] = np.nan
    ys2 = _stream(y2, f)
    assert np.isnan(gpu_dot(n, xs, f, 1, ys2, f, 1))
    xs3 = _stream(g.standard_normal(n), f)
    a = gpu_dot(n, xs3, f, 1, ys, f, 1)
    b = gpu_dot(n, xs3, f, 1, ys, f, 1)
    assert np.float64(a).tobytes() == np.float64(b).tobytes()


# ---- axpy --------------------------------------------------------------------------

def run_axpy(n, alpha, xs, fx, incx, ys, fy, incy, mode, x_off=0, y_off=0):
    X = Guarded(xs.size, x_off, fill=xs)
    Y = Guarded(ys.size, y_off, fill=ys)
    flyte.lib()
    flyte._check(flyte.lib().flyte_axpy(n, float(alpha), X.ptr, flyte.fmt(fx), incx, Y.ptr, flyte.fmt(fy),
                                        incy, flyte._mode(mode), flyte._stream(None)))
    sync()
    Y.check_guards()
    return Y.inner()


def check_axpy(got, n, alpha, xs, fx, incx, ys, fy, incy, mode):
    want = oracle.axpy(n, alpha, xs, fx[::-1], incx, ys, fy[::-1], incy, ORC_MODE[mode])
    k, base = fy
    if np.array_equal(got, want):
        return
    # only NaN results may differ, and then both must be NaN codes
    nat = (np.uint32, 4) if base == 0 else (np.uint64, 8)
    gb = oracle.unpack(got, base, k, n=n, inc_src=incy)
    wb = oracle.unpack(want, base, k, n=n, inc_src=incy)
    gv = gb.view(np.float32 if base == 0 else np.float64)
    wv = wb.view(np.float32 if base == 0 else np.float64)
    diff = gb != wb
    assert np.all(np.isnan(gv[diff]) & np.isnan(wv[diff])), f"{diff.sum()} codes differ"
    # bytes outside the strided elements are untouched
    mask = np.ones(got.size, bool)
    for i in range(n):
        mask[i * incy * k: i * incy * k + k] = False
    assert np.array_equal(got[mask], ys[mask])


@pytest.mark.parametrize("f", FORMATS, ids=lambda f: f"k{f[0]}{'d' if f[1] else 'f'}")
@pytest.mark.parametrize("mode", MODES)
def test_axpy_sizes(f, mode):
    g = np.random.default_rng(f[0] + 31 * f[1])
    for n in [1, 3, 4, 5, 130, 4099, 65539]:
        xs = _stream(g.standard_normal(n), f)
        ys = _stream(g.standard_normal(n), f)
        got = run_axpy(n, 0.1234567890123, xs, f, 1, ys, f, 1, mode)
        check_axpy(got, n, 0.1234567890123, xs, f, 1, ys, f, 1, mode)


def test_axpy_config_mixture_k4():
    """Config 1: alpha = 1.5 on the 1M mixtures (specials included) at double-based k = 4."""
    n = 1 << 20
    f = (4, 1)
    xs = oracle.pack(inputs.mixture_f64(n, 1601), 1, 4)
    ys = oracle.pack(inputs.mixture_f64(n, 1602), 1, 4)
    for mode in MODES:
        got = run_axpy(n, 1.5, xs, f, 1, ys, f, 1, mode)
        check_axpy(got, n, 1.5, xs, f, 1, ys, f, 1, mode)


@pytest.mark.parametrize("fx,fy,incx,incy,xo,yo", [
    ((4, 1), (4, 1), 1, 1, 1, 0), ((4, 1), (4, 1), 1, 1, 0, 6), ((3, 1), (6, 1), 1, 1, 0, 0),
    ((8, 1), (2, 1), 2, 1, 0, 0), ((2, 0), (3, 0), 1, 3, 5, 1), ((4, 0), (1, 0), 3, 2, 0, 0)])
def test_axpy_generic_paths(fx, fy, incx, incy, xo, yo):
    n = 10007
    g = np.random.default_rng(12)
    xs = _stream(g.standard_normal(n * incx), fx)
    ys = _stream(g.standard_normal(n * incy), fy)
    got = run_axpy(n, -2.5, xs, fx, incx, ys, fy, incy, "rne", xo, yo)
    check_axpy(got, n, -2.5, xs, fx, incx, ys, fy, incy, "rne")


def test_axpy_rejects_mixed_bases():
    buf = torch.zeros(64, dtype=torch.uint8, device="cuda")
    with pytest.raises(flyte.FlyteError) as e:
        flyte.axpy(1.0, buf, (4, 1), buf, (2, 0), n=4)
    assert e.value.status == 2


# ---- scal (in place) --------------------------------------------------------------

def run_scal(n, alpha, xs, fx, incx, mode, x_off=0):
    X = Guarded(xs.size, x_off, fill=xs)
    flyte._check(flyte.lib().flyte_scal(n, float(alpha), X.ptr, flyte.fmt(fx), incx, flyte._mode(mode),
                                        flyte._stream(None)))
    sync()
    X.check_guards()
    return X.inner()


def check_scal(got, n, alpha, xs, fx, incx, mode):
    want = oracle.scal(n, alpha, xs, fx[::-1], incx, ORC_MODE[mode])
    if np.array_equal(got, want):
        return
    k, base = fx
    gb = oracle.unpack(got, base, k, n=n, inc_src=incx)
    wb = oracle.unpack(want, base, k, n=n, inc_src=incx)
    gv = gb.view(np.float32 if base == 0 else np.float64)
    wv = wb.view(np.float32 if base == 0 else np.float64)
    diff = gb != wb
    assert np.all(np.isnan(gv[diff]) & np.isnan(wv[diff])), f"{diff.sum()} codes differ"
    mask = np.ones(got.size, bool)
    for i in range(n):
        mask[i * incx * k: i * incx * k + k] = False
    assert np.array_equal(got[mask], xs[mask])


@pytest.mark.parametrize("f", FORMATS, ids=lambda f: f"k{f[0]}{'d' if f[1] else 'f'}")
@pytest.mark.parametrize("mode", MODES)
def test_scal_sizes(f, mode):
    g = np.random.default_rng(f[0] + 37 * f[1])
    for n in [1, 3, 4, 5, 130, 4099, 65539]:
        xs = _stream(g.standard_normal(n), f)
        got = run_scal(n, -0.1234567890123, xs, f, 1, mode)
        check_scal(got, n, -0.1234567890123, xs, f, 1, mode)


@pytest.mark.parametrize("k", [2, 3, 4, 5, 6, 7])
@pytest.mark.parametrize("mode", MODES)
def test_scal_binary32_alpha_exact_path(k, mode):
    """A binary32 alpha takes the binary32 decision for double-based k = 2..7 (alpha x = p + e exactly,
    and for k >= 5 the pairs of the wide axpy without y): bit-exact against the oracle on N(0,1), short
    integers (exact products and ties) and out-of-window values (binary64 fallback)."""
    f = (k, 1)
    g = np.random.default_rng(70 + k)
    n = 1 << 15
    xv = g.standard_normal(n)
    xv[3::17] *= 2.0 ** g.integers(-60, 60, xv[3::17].size)
    xv[5::19] = 0.0
    xs = _stream(xv, f)
    xi = _stream(g.integers(-4096, 4096, n).astype(np.float64) / 8.0, f)
    for alpha in (1.5, -2.0, float(np.float32(0.1)), float(np.float32(1 / 3)), float(np.float32(12345.678)),
                  2.0 ** -30):
        for data in (xs, xi):
            got = run_scal(n, alpha, data, f, 1, mode)
            check_scal(got, n, alpha, data, f, 1, mode)


def test_scal_config_mixture_and_paths():
    """The 1M double mixture (specials included) at k = 3, 4, 5, and strided / offset streams."""
    n = 1 << 20
    for k in (3, 4, 5):
        xs = oracle.pack(inputs.mixture_f64(n, 1601), 1, k)
        for mode in MODES:
            got = run_scal(n, 1.5, xs, (k, 1), 1, mode)
            check_scal(got, n, 1.5, xs, (k, 1), 1, mode)
    g = np.random.default_rng(21)
    for f, inc, off in [((5, 1), 3, 0), ((4, 1), 1, 1), ((3, 0), 2, 7), ((2, 0), 1, 2)]:
        m = 10007
        xs = _stream(g.standard_normal(m * inc), f)
        got = run_scal(m, 2.75, xs, f, inc, "rne", off)
        check_scal(got, m, 2.75, xs, f, inc, "rne")
    with pytest.raises(flyte.FlyteError):
        flyte.scal(1.0, torch.zeros(16, dtype=torch.uint8, device="cuda"), (9, 1), n=2)


@pytest.mark.parametrize("k", [2, 3, 4, 5, 6, 7])
@pytest.mark.parametrize("mode", MODES)
def test_axpy_binary32_alpha_exact_path(k, mode):
    """alpha exactly representable in binary32 takes the binary32 error-free path for double-based
    k <= 7 (k = 5..7 through the exact hi/lo pairs of x and y): bit-exact against the oracle on data
    that make exact results, ties, cancellations, near-cancellations and out-of-window values (which
    fall back to binary64) frequent."""
    f = (k, 1)
    g = np.random.default_rng(40 + k)
    n = 1 << 16
    xv = g.standard_normal(n)
    yv = g.standard_normal(n)
    yv[::7] = -1.5 * xv[::7]                                   # cancellation (exact zero for alpha = 1.5)
    yv[1::11] = 0.0
    xv[2::13] *= 2.0 ** g.integers(-60, 60, xv[2::13].size)   # outside the window for some
    xs = _stream(xv, f)
    ys = _stream(yv, f)
    for alpha in (1.5, -2.0, 0.75, 3.0, -0.3125, 1.0, 2.0 ** -30):
        got = run_axpy(n, alpha, xs, f, 1, ys, f, 1, mode)
        check_axpy(got, n, alpha, xs, f, 1, ys, f, 1, mode)
    # small integers: many exactly representable sums and exact midpoints
    xi = _stream(g.integers(-64, 64, n).astype(np.float64), f)
    yi = _stream(g.integers(-4096, 4096, n).astype(np.float64) * 0.5, f)
    for alpha in (1.5, 0.5, 3.0):
        got = run_axpy(n, alpha, xi, f, 1, yi, f, 1, mode)
        check_axpy(got, n, alpha, xi, f, 1, yi, f, 1, mode)
    # binary32 alphas with long expansions, and y within 2^-30 relative of -alpha x (near-cancellation:
    # the exact sum is far below the terms, so the decision has to see the small error terms)
    for alpha in (float(np.float32(0.1)), float(np.float32(1 / 3)), float(np.float32(12345.678))):
        yc = -alpha * xv * (1 + np.ldexp(g.integers(-500, 500, n).astype(np.float64), -30))
        ycs = _stream(yc, f)
        got = run_axpy(n, alpha, xs, f, 1, ycs, f, 1, mode)
        check_axpy(got, n, alpha, xs, f, 1, ycs, f, 1, mode)
        got = run_axpy(n, alpha, xs, f, 1, ys, f, 1, mode)
        check_axpy(got, n, alpha, xs, f, 1, ys, f, 1, mode)


@pytest.mark.parametrize("k", [2, 3, 4])
@pytest.mark.parametrize("mode", MODES)
def test_axpy_split_alpha_exact_path(k, mode):
    """Any other alpha inside the window takes the two-part binary32 path for double-based k <= 4:
    bit-exact against the oracle, with near-cancellations (y close to -alpha x), zeros, small
    integers and out-of-window values mixed in."""
    f = (k, 1)
    g = np.random.default_rng(60 + k)
    n = 1 << 16
    xv = g.standard_normal(n)
    yv = g.standard_normal(n)
    yv[1::11] = 0.0
    xv[2::13] *= 2.0 ** g.integers(-60, 60, xv[2::13].size)
    alphas = (0.1, -1e-9 - 1e-25, np.pi, 1.0 / 3.0, 1.5 + 2.0 ** -30, -1.1 * 2.0 ** -39, 123456.789,
              float(g.uniform(-4, 4)), float(g.uniform(-4, 4)) * 2.0 ** 30)
    xs = _stream(xv, f)
    for alpha in alphas:
        assert float(np.float32(alpha)) != alpha
        yc = yv.copy()
        yc[::7] = -alpha * xv[::7]          # near-cancellation: y is alpha x rounded to the format
        ys = _stream(yc, f)
        got = run_axpy(n, alpha, xs, f, 1, ys, f, 1, mode)
        check_axpy(got, n, alpha, xs, f, 1, ys, f, 1, mode)
    xi = _stream(g.integers(-64, 64, n).astype(np.float64), f)
    yi = _stream(g.integers(-4096, 4096, n).astype(np.float64) * 0.5, f)
    for alpha in (0.1, 1.0 / 3.0, 0.5 + 2.0 ** -40):
        got = run_axpy(n, alpha, xi, f, 1, yi, f, 1, mode)
        check_axpy(got, n, alpha, xi, f, 1, yi, f, 1, mode)
