"""GPU parity of flyte_gemv (N and T) against the CPU oracle.

Bound (header and spec tolerance, plus the oracle's own rounding):
  |y_gpu - y_ref| <= 4 (len + 2) 2^-53 (|alpha| sum_j |A_ij x_j| + |beta y_i|) + 2^-52 |y_ref|
where len is the length of each dot product (n for 'N', m for 'T') and y_ref
is the oracle's Dot2-based result.  NaN/Inf results must match in class.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
from paper_1601_07789_gb300 import flyte, inputs
from tests.gpu_util import sync

pytestmark = pytest.mark.gpu
EPS = 2.0 ** -53


def _dev(a: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def check_bound(got, ref, absum, alpha, beta, y0, length):
    got = np.asarray(got, dtype=np.float64)
    fin = np.isfinite(ref)
    assert np.array_equal(np.isnan(got), np.isnan(ref)), "NaN class differs"
    inf = np.isinf(ref)
    assert np.array_equal(got[inf], ref[inf]), "Inf differs"
    bound = 4 * (length + 2) * EPS * (abs(alpha) * absum + abs(beta) * np.abs(y0)) + 2 * EPS * np.abs(ref)
    err = np.abs(got - ref)
    bad = fin & ~(err <= bound)
    assert not bad.any(), (f"{bad.sum()} entries out of bound; worst ratio "
                           f"{np.max(err[fin] / np.maximum(bound[fin], 1e-300)):.3g}")
    return float(np.max(err[fin] / np.maximum(bound[fin], 1e-300))) if fin.any() else 0.0


def run_gemv(trans, m, n, fa, Acodes, lda, x, y0, alpha, beta, incx=1, incy=1, a_off=0):
    k = fa[0]
    buf = torch.zeros(Acodes.size + 16 + a_off, dtype=torch.uint8, device="cuda")
    buf[a_off:a_off + Acodes.size] = _dev(Acodes)
    A_ptr = buf.data_ptr() + a_off
    xd = _dev(x)
    yd = _dev(y0.copy())
    wsb = flyte.workspace_bytes("gemv_n" if trans == "N" else "gemv_t", m, n, 0, fa)
    ws = torch.full((max(wsb, 16),), 0x55, dtype=torch.uint8, device="cuda")
    flyte.gemv_raw(trans, m, n, alpha, A_ptr, fa, lda, xd, incx, beta, yd, incy, ws, ws.numel())
    sync()
    if alpha != 0.0:
        # the first word of the workspace is the pipelines' error word: no timeout happened
        status = int(ws[:4].cpu().numpy().view(np.int32)[0])
        assert status in (0, 0x55555555), f"pipeline status {status:#x}"
    return yd.cpu().numpy()


def reference(trans, m, n, fa, Acodes, lda, x, y0, alpha, beta, incx=1, incy=1):
    return oracle.gemv(trans, m, n, alpha, Acodes, fa[::-1], lda, x, incx, beta, y0, incy)


def make_A(m, lda, fa, seed, kind="normal"):
    k, base = fa
    g = np.random.default_rng(seed)
    if kind == "normal":
        v = g.standard_normal(m * lda)
    elif kind == "positive":
        v = np.abs(g.standard_normal(m * lda)) + 0.5
    elif kind == "wide":
        v = g.standard_normal(m * lda) * np.exp2(g.integers(-60, 60, m * lda))
    else:
        raise ValueError(kind)
    if base == 0:
        v = v.astype(np.float32)
    return oracle.pack(v, base, k)


DFORMATS = [(k, 1) for k in range(1, 9)] + [(k, 0) for k in range(1, 5)]


@pytest.mark.parametrize("fa", DFORMATS, ids=lambda f: f"k{f[0]}{'d' if f[1] else 'f'}")
@pytest.mark.parametrize("trans", ["N", "T"])
@pytest.mark.parametrize("shape", [(777, 1283, 1288), (2100, 613, 618), (777, 1283, 1296),
                                   (2100, 1024, 1024), (1500, 5000, 5008)])
def test_gemv_parity_moderate(fa, trans, shape):
    m, n, lda = shape
    A = make_A(m, lda, fa, seed=3 + fa[0])
    g = np.random.default_rng(17)
    x = g.standard_normal(max(m, n))
    y0 = g.standard_normal(max(m, n))
    for alpha, beta in [(1.5, -0.5), (-0.75, 0.0), (1.0, 1.0)]:
        got = run_gemv(trans, m, n, fa, A, lda, x, y0, alpha, beta)
        ref, absum = reference(trans, m, n, fa, A, lda, x, y0, alpha, beta)
        L = n if trans == "N" else m
        check_bound(got[: (m if trans == "N" else n)], ref[: (m if trans == "N" else n)], absum,
                    alpha, beta, y0[: (m if trans == "N" else n)], L)
        assert np.array_equal(got[(m if trans == "N" else n):], y0[(m if trans == "N" else n):])


@pytest.mark.parametrize("trans", ["N", "T"])
@pytest.mark.parametrize("shape", [(1, 1), (3, 7), (5, 300), (300, 5), (257, 1029), (64, 4099),
                                   (1030, 64), (4099, 37), (2500, 2500), (2500, 2560), (3000, 9000),
                                   (16, 12288), (1027, 2048), (131, 1040)])
def test_gemv_shapes_and_tails(trans, shape):
    m, n = shape
    fa = (5, 1)
    lda = n
    A = make_A(m, lda, fa, seed=m + n)
    g = np.random.default_rng(m * n)
    x = g.standard_normal(max(m, n))
    y0 = g.standard_normal(max(m, n))
    got = run_gemv(trans, m, n, fa, A, lda, x, y0, 1.5, -0.5)
    ref, absum = reference(trans, m, n, fa, A, lda, x, y0, 1.5, -0.5)
    ly = m if trans == "N" else n
    check_bound(got[:ly], ref[:ly], absum, 1.5, -0.5, y0[:ly], n if trans == "N" else m)


@pytest.mark.parametrize("trans", ["N", "T"])
@pytest.mark.parametrize("kind", ["positive", "wide"])
@pytest.mark.parametrize("n", [2051, 2048])
def test_gemv_adversarial(trans, kind, n):
    """All-positive terms (errors cannot cancel) and a 2^+-60 spread of magnitudes."""
    m = 2600
    fa = (4, 1)
    A = make_A(m, n, fa, seed=5, kind=kind)
    x = np.abs(np.random.default_rng(6).standard_normal(max(m, n))) + 0.25
    y0 = np.random.default_rng(7).standard_normal(max(m, n))
    got = run_gemv(trans, m, n, fa, A, n, x, y0, 1.5, -0.5)
    ref, absum = reference(trans, m, n, fa, A, n, x, y0, 1.5, -0.5)
    ly = m if trans == "N" else n
    check_bound(got[:ly], ref[:ly], absum, 1.5, -0.5, y0[:ly], n if trans == "N" else m)


@pytest.mark.parametrize("trans", ["N", "T"])
@pytest.mark.parametrize("n", [1030, 1040])
def test_gemv_specials_and_zeros(trans, n):
    """Zeros, subnormals, Inf and NaN in A, and Inf in x, take the binary64 path."""
    m = 2101
    fa = (6, 1)
    g = np.random.default_rng(8)
    v = g.standard_normal(m * n)
    v[g.integers(0, m * n, 200)] = 0.0
    v[g.integers(0, m * n, 5)] = np.inf
    v[g.integers(0, m * n, 5)] = -np.inf
    v[g.integers(0, m * n, 5)] = np.nan
    v[g.integers(0, m * n, 20)] = 1e-310
    A = oracle.pack(v, 1, 6)
    x = g.standard_normal(max(m, n))
    y0 = g.standard_normal(max(m, n))
    got = run_gemv(trans, m, n, fa, A, n, x, y0, 1.5, -0.5)
    ref, absum = reference(trans, m, n, fa, A, n, x, y0, 1.5, -0.5)
    ly = m if trans == "N" else n
    check_bound(got[:ly], ref[:ly], absum, 1.5, -0.5, y0[:ly], n if trans == "N" else m)
    x2 = x.copy()
    x2[3] = np.inf
    got = run_gemv(trans, m, n, fa, A, n, x2, y0, 1.5, -0.5)
    ref, absum = reference(trans, m, n, fa, A, n, x2, y0, 1.5, -0.5)
    check_bound(got[:ly], ref[:ly], absum, 1.5, -0.5, y0[:ly], n if trans == "N" else m)


@pytest.mark.parametrize("trans", ["N", "T"])
def test_gemv_strides_offsets_quick_returns(trans):
    m, n = 130, 517
    fa = (3, 1)
    lda = 530
    A = make_A(m, lda, fa, seed=9)
    g = np.random.default_rng(10)
    incx, incy = 3, 2
    x = g.standard_normal(3 * max(m, n))
    y0 = g.standard_normal(2 * max(m, n))
    for a_off in (0, 1, 5):
        got = run_gemv(trans, m, n, fa, A, lda, x, y0, 1.5, -0.5, incx, incy, a_off=a_off)
        ref, absum = reference(trans, m, n, fa, A, lda, x, y0, 1.5, -0.5, incx, incy)
        ly = m if trans == "N" else n
        check_bound(got[::incy][:ly], ref[::incy][:ly], absum, 1.5, -0.5, y0[::incy][:ly],
                    n if trans == "N" else m)
        mask = np.ones(y0.size, bool)
        mask[: ly * incy: incy] = False
        assert np.array_equal(got[mask], y0[mask])
    # beta = 0: y is not read (NaN in y is ignored)
    yn = np.full(max(m, n), np.nan)
    got = run_gemv(trans, m, n, fa, A, lda, x, yn, 2.0, 0.0, incx, 1)
    assert np.isfinite(got[: (m if trans == "N" else n)]).all()
    # alpha = 0: y <- beta y; A and x are not read
    yd = torch.from_numpy(y0.copy()).cuda()
    flyte.gemv_raw(trans, m, n, 0.0, 0, fa, lda, 0, 1, 3.0, yd, 1, 0, 0)
    sync()
    ly = m if trans == "N" else n
    assert np.array_equal(yd.cpu().numpy()[:ly], 3.0 * y0[:ly])
    # m = 0 or n = 0: nothing happens
    flyte.gemv_raw(trans, 0, n, 1.0, 0, fa, lda, 0, 1, 3.0, yd, 1, 0, 0)
    flyte.gemv_raw(trans, m, 0, 1.0, 0, fa, 1, 0, 1, 3.0, yd, 1, 0, 0)
    sync()


def test_gemv_rejects_bad_args():
    fa = (4, 1)
    y = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(flyte.FlyteError):
        flyte.gemv_raw("X", 2, 2, 1.0, y, fa, 2, y, 1, 0.0, y, 1, y, 64)
    with pytest.raises(flyte.FlyteError):
        flyte.gemv_raw("N", 2, 4, 1.0, y, fa, 3, y, 1, 0.0, y, 1, y, 64)   # lda < n
    with pytest.raises(flyte.FlyteError) as e:
        flyte.gemv_raw("N", 2, 4, 1.0, y, fa, 4, y, 1, 0.0, y, 1, y, 8)    # workspace too small
    assert e.value.status == 5


def test_gemv_k8_matches_library_fp64():
    """k = 8 is plain binary64: compare with torch's float64 mv (cuBLAS) within the bound."""
    m, n = 2048, 3001
    A = torch.randn(m, n, dtype=torch.float64, device="cuda")
    x = torch.randn(n, dtype=torch.float64, device="cuda")
    y = torch.zeros(m, dtype=torch.float64, device="cuda")
    codes = A.contiguous().view(torch.uint8).reshape(-1)
    flyte.gemv("N", m, n, 1.0, codes, (8, 1), n, x, 0.0, y)
    ref = A @ x
    absum = A.abs() @ x.abs()
    assert torch.all((y - ref).abs() <= 8 * (n + 2) * EPS * absum)


# ---- full size (16384 x 16384), sampled rows/columns --------------------------------

@pytest.fixture(scope="module")
def big_A():
    m = n = 16384
    A, x, y = inputs.gemv_operands(m, n)
    return A.reshape(-1), x, y


@pytest.mark.parametrize("k", [3, 4, 5, 6])
def test_gemv_full_size_sampled(big_A, k):
    Af, x, y0 = big_A
    m = n = 16384
    fa = (k, 1)
    codes = oracle.pack(Af, 1, k)
    g = np.random.default_rng(100 + k)
    rows = np.sort(g.choice(m, 48, replace=False))
    cols = np.sort(g.choice(n, 48, replace=False))
    A3 = codes.reshape(m, n, k)
    for trans in "NT":
        got = run_gemv(trans, m, n, fa, codes, n, x, y0, 1.5, -0.5)
        if trans == "N":
            sub = np.ascontiguousarray(A3[rows]).reshape(-1)
            ref, absum = oracle.gemv("N", rows.size, n, 1.5, sub, (1, k), n, x, 1, -0.5, y0[rows], 1)
            check_bound(got[rows], ref, absum, 1.5, -0.5, y0[rows], n)
        else:
            sub = np.ascontiguousarray(A3[:, cols]).reshape(-1)
            ref, absum = oracle.gemv("T", m, cols.size, 1.5, sub, (1, k), cols.size, x, 1, -0.5,
                                     y0[cols], 1)
            check_bound(got[cols], ref, absum, 1.5, -0.5, y0[cols], m)
    del codes


# ---- y stored as double-based flytes (the pack fused into the epilogue) -------------------

def run_gemv_packed(trans, m, n, fa, Acodes, lda, x, ycodes, fy, alpha, beta, mode, incy=1):
    buf = _dev(Acodes)
    xd = _dev(x)
    yd = _dev(ycodes.copy())
    wsb = flyte.workspace_bytes("gemv_n" if trans == "N" else "gemv_t", m, n, 0, fa)
    ws = torch.full((max(wsb, 16),), 0x55, dtype=torch.uint8, device="cuda")
    flyte.gemv_packed_y_raw(trans, m, n, alpha, buf, fa, lda, xd, 1, beta, yd, fy, incy, mode, ws, ws.numel())
    sync()
    return yd.cpu().numpy()


@pytest.mark.parametrize("trans", ["N", "T"])
@pytest.mark.parametrize("ky", [2, 3, 5, 7, 8])
@pytest.mark.parametrize("shape", [(777, 1283), (2100, 1024), (64, 9000)])
def test_gemv_packed_y(trans, ky, shape):
    """y as a ky-byte stream: equals the GPU's own pack of the binary64 gemv result bit for bit,
    and meets the gemv bound plus one rounding to ky bytes against the oracle."""
    m, n = shape
    fa = (4, 1)
    fy = (ky, 1)
    A = make_A(m, n, fa, seed=11 + ky)
    g = np.random.default_rng(23 + ky)
    ly = m if trans == "N" else n
    x = g.standard_normal(max(m, n))
    ycodes = oracle.pack(g.standard_normal(ly), 1, ky)
    yq = oracle.values(ycodes, 1, ky)                      # the values the codes stand for
    for alpha, beta, mode in [(1.5, -0.5, "rne"), (-0.75, 0.0, "rtz"), (1.0, 1.0, "rto"),
                              (0.0, 2.0, "rne"), (0.0, 0.0, "half_up")]:
        got = run_gemv_packed(trans, m, n, fa, A, n, x, ycodes, fy, alpha, beta, mode)
        # self-consistency on the GPU: pack(flyte_gemv(.., unpack(y), ..)) with the library's own pack
        y64 = run_gemv(trans, m, n, fa, A, n, x, yq, alpha, beta)[:ly]
        same = flyte.pack(torch.from_numpy(y64).cuda(), ky, mode).cpu().numpy()
        assert np.array_equal(got, same), f"{np.sum(got != same)} bytes differ from pack(gemv)"
        # against the oracle: the binary64 bound plus one rounding to ky bytes
        ref, absum = reference(trans, m, n, fa, A, n, x, yq, alpha, beta)
        v = oracle.values(got, 1, ky)
        mag = abs(alpha) * absum + abs(beta) * np.abs(yq)
        L = n if trans == "N" else m
        bound = 4 * (L + 2) * EPS * mag + 2 * EPS * np.abs(ref) + np.abs(ref) * 2.0 ** -(8 * ky - 12)
        assert np.all(np.abs(v - ref[:ly]) <= bound), "packed y out of bound"


def test_gemv_packed_y_rejects_float_base():
    A = torch.zeros(64, dtype=torch.uint8, device="cuda")
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    y = torch.zeros(64, dtype=torch.uint8, device="cuda")
    with pytest.raises(flyte.FlyteError) as e:
        flyte.gemv_packed_y_raw("N", 4, 4, 1.0, A, (4, 1), 4, x, 1, 0.0, y, (3, 0), 1, "rne", A, 64)
    assert e.value.status == 2
