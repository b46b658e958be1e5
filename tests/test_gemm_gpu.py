"""GPU parity of flyte_gemm against the CPU oracle (Dot2 entries).

Bounds (header tolerances):
  float-based:  |C - C_ref| <= 2^-22 (|alpha| sum_l |A_il B_lj| + |beta C0_ij|), mixed-sign and
                same-sign data alike (test_gemm_same_sign_long_k)
  double-based: |C - C_ref| <= 4 k 2^-53 (|alpha| sum_l |A_il B_lj| + |beta C0_ij|) + 2^-52 |C_ref|
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
from paper_1601_07789_gb300 import flyte

pytestmark = pytest.mark.gpu


def _codes(values, f):
    k, base = f
    v = np.asarray(values, dtype=np.float32 if base == 0 else np.float64)
    return oracle.pack(v.reshape(-1), base, k)


def run_gemm(m, n, kk, f, A, lda, B, ldb, alpha=1.0, beta=0.0, C0=None, ldc=None, a_off=0):
    k, base = f
    ldc = n if ldc is None else ldc
    dt = torch.float32 if base == 0 else torch.float64
    bufA = torch.zeros(A.size + 16 + a_off, dtype=torch.uint8, device="cuda")
    bufA[a_off:a_off + A.size] = torch.from_numpy(A).cuda()
    Bd = torch.from_numpy(B).cuda()
    if C0 is None:
        C = torch.full((m * ldc,), 7.0, dtype=dt, device="cuda")
    else:
        C = torch.from_numpy(np.ascontiguousarray(C0).astype(np.float32 if base == 0 else np.float64)).cuda()
    wsb = flyte.workspace_bytes("gemm", m, n, kk, f)
    ws = torch.empty(max(wsb, 256), dtype=torch.uint8, device="cuda")
    flyte.gemm_raw(m, n, kk, alpha, bufA.data_ptr() + a_off, f, lda, Bd, f, ldb, beta, C, ldc, ws, ws.numel())
    torch.cuda.synchronize()
    return C.cpu().numpy().reshape(m, ldc)


def check(got, m, n, kk, f, A, lda, B, ldb, alpha, beta, C0, rows=None, cols=None):
    k, base = f
    if rows is None:
        rr, cc = np.meshgrid(np.arange(m), np.arange(n), indexing="ij")
        rows, cols = rr.reshape(-1), cc.reshape(-1)
    cin = None if C0 is None else C0[rows, cols].astype(np.float64)
    ref, absum = oracle.gemm_entries(rows, cols, kk, alpha, A, (base, k), lda, B, (base, k), ldb, beta, cin)
    g = got[rows, cols].astype(np.float64)
    mag = abs(alpha) * absum + (0 if cin is None else abs(beta) * np.abs(cin))
    if base == 0:
        bound = 2.0 ** -22 * mag
    else:
        bound = 4 * kk * 2.0 ** -53 * mag + 2.0 ** -52 * np.abs(ref)
    err = np.abs(g - ref)
    bad = ~(err <= bound)
    assert not bad.any(), (f"{bad.sum()} of {bad.size} out of bound; worst err/bound "
                           f"{np.max(err / np.maximum(bound, 1e-300)):.3g}")
    return float(np.max(err / np.maximum(bound, 1e-300)))


FORMATS = [(k, 0) for k in (1, 2, 3, 4)] + [(k, 1) for k in (1, 2, 3, 4, 5, 6, 7, 8)]


@pytest.mark.parametrize("f", FORMATS, ids=lambda f: f"k{f[0]}{'d' if f[1] else 'f'}")
@pytest.mark.parametrize("shape", [(257, 263, 259), (128, 256, 64), (300, 520, 1000), (1, 1, 1), (5, 700, 3)])
def test_gemm_parity(f, shape):
    m, n, kk = shape
    g = np.random.default_rng(m * 7 + n + kk)
    A = _codes(g.uniform(-1, 1, m * kk), f)
    B = _codes(g.uniform(-1, 1, kk * n), f)
    got = run_gemm(m, n, kk, f, A, kk, B, n)
    check(got, m, n, kk, f, A, kk, B, n, 1.0, 0.0, None)


@pytest.mark.parametrize("f", [(2, 0), (3, 0), (4, 0), (5, 1)], ids=["k2f", "k3f", "k4f", "k5d"])
def test_gemm_alpha_beta_strides(f):
    m, n, kk = 200, 300, 333
    lda, ldb, ldc = kk + 3, n + 5, n + 7
    g = np.random.default_rng(3)
    A = _codes(g.uniform(-1, 1, m * lda), f)
    B = _codes(g.uniform(-1, 1, kk * ldb), f)
    C0 = g.uniform(-1, 1, (m, ldc))
    for a_off in (0, 2):
        got = run_gemm(m, n, kk, f, A, lda, B, ldb, alpha=-1.5, beta=0.25, C0=C0, ldc=ldc, a_off=a_off)
        check(got, m, n, kk, f, A, lda, B, ldb, -1.5, 0.25, C0)
        # columns beyond n are untouched
        dt = np.float32 if f[1] == 0 else np.float64
        assert np.array_equal(got[:, n:], C0[:, n:].astype(dt))


def test_gemm_quick_returns():
    f = (3, 0)
    m, n = 40, 50
    C0 = np.random.default_rng(4).uniform(-1, 1, (m, n)).astype(np.float32)
    C = torch.from_numpy(C0.copy()).cuda()
    flyte.gemm_raw(m, n, 10, 0.0, 0, f, 10, 0, f, n, 2.0, C, n, 0, 0)     # alpha = 0: C <- beta C
    torch.cuda.synchronize()
    assert np.array_equal(C.cpu().numpy(), 2.0 * C0)
    flyte.gemm_raw(m, n, 0, 1.0, 0, f, 1, 0, f, n, 0.0, C, n, 0, 0)       # k = 0, beta = 0: C <- 0
    torch.cuda.synchronize()
    assert not C.cpu().numpy().any()
    with pytest.raises(flyte.FlyteError):
        flyte.gemm_raw(m, n, 10, 1.0, C, f, 10, C, (2, 0), n, 0.0, C, n, C, 1 << 20)   # mixed formats


@pytest.mark.parametrize("k", [2, 3, 4])
def test_gemm_8192_sampled(k):
    """The 8192^3 float-based workload, U(-1,1) (seeds 5, 6), 4096 sampled entries."""
    M = N = K = 8192
    f = (k, 0)
    gA = np.random.default_rng(5)
    gB = np.random.default_rng(6)
    A = _codes(gA.uniform(-1, 1, M * K).astype(np.float32), f)
    B = _codes(gB.uniform(-1, 1, K * N).astype(np.float32), f)
    got = run_gemm(M, N, K, f, A, K, B, N)
    s = np.random.default_rng(100 + k)
    rows = s.integers(0, M, 4096)
    cols = s.integers(0, N, 4096)
    worst = check(got, M, N, K, f, A, K, B, N, 1.0, 0.0, None, rows, cols)
    print(f"k={k}: worst error / bound = {worst:.3g}")


def test_gemm_4096_double_k5_sampled():
    M = N = K = 4096
    f = (5, 1)
    A = _codes(np.random.default_rng(5).uniform(-1, 1, M * K), f)
    B = _codes(np.random.default_rng(6).uniform(-1, 1, K * N), f)
    got = run_gemm(M, N, K, f, A, K, B, N)
    s = np.random.default_rng(7)
    rows = s.integers(0, M, 2048)
    cols = s.integers(0, N, 2048)
    check(got, M, N, K, f, A, K, B, N, 1.0, 0.0, None, rows, cols)


# ---- C stored as flytes (the pack fused into the epilogue) ---------------------------------

@pytest.mark.parametrize("f,kc", [((2, 0), 2), ((3, 0), 3), ((4, 0), 2), ((3, 0), 4), ((5, 1), 3), ((5, 1), 6),
                                  ((4, 1), 8)])
def test_gemm_packed_c(f, kc):
    """C as a kc-byte stream: the pack of the native-C gemm (same C0 = unpack(C)) bit for bit,
    and within the gemm bound plus one rounding to kc bytes against the oracle."""
    m, n, kk = 200, 300, 333
    k, base = f
    fc = (kc, base)
    g = np.random.default_rng(40 + kc)
    A = _codes(g.uniform(-1, 1, m * kk), f)
    B = _codes(g.uniform(-1, 1, kk * n), f)
    ct = np.float32 if base == 0 else np.float64
    Cq = oracle.pack(g.uniform(-1, 1, m * n).astype(ct), base, kc)
    C0 = oracle.values(Cq, base, kc).reshape(m, n)
    wsb = flyte.workspace_bytes("gemm", m, n, kk, f)
    ws = torch.empty(max(wsb, 256), dtype=torch.uint8, device="cuda")
    Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    for alpha, beta, mode in [(1.0, 0.0, "rne"), (-1.5, 0.25, "rtz"), (0.75, 1.0, "rto"), (0.0, -2.0, "rne"),
                              (0.0, 0.0, "half_up")]:
        Cd = torch.from_numpy(Cq.copy()).cuda()
        flyte.gemm_packed_c_raw(m, n, kk, alpha, Ad, f, kk, Bd, f, n, beta, Cd, fc, n, mode, ws, ws.numel())
        torch.cuda.synchronize()
        got = Cd.cpu().numpy()
        native = run_gemm(m, n, kk, f, A, kk, B, n, alpha=alpha, beta=beta, C0=C0)
        same = flyte.pack(torch.from_numpy(np.ascontiguousarray(native).reshape(-1).astype(ct)).cuda(), kc,
                          mode).cpu().numpy()
        assert np.array_equal(got, same), f"{np.sum(got != same)} bytes differ from pack(gemm)"
        if alpha != 0.0:
            v = oracle.values(got, base, kc).reshape(m, n)
            mbits = (8 * kc - 9) if base == 0 else (8 * kc - 12)
            rr, cc = np.meshgrid(np.arange(m), np.arange(n), indexing="ij")
            rows, cols = rr.reshape(-1), cc.reshape(-1)
            ref, absum = oracle.gemm_entries(rows, cols, kk, alpha, A, (base, k), kk, B, (base, k), n, beta,
                                             C0[rows, cols])
            mag = abs(alpha) * absum + abs(beta) * np.abs(C0[rows, cols])
            bound = (2.0 ** -22 if base == 0 else 4 * kk * 2.0 ** -53) * mag + np.abs(ref) * 2.0 ** -min(mbits, 52)
            assert np.all(np.abs(v[rows, cols] - ref) <= bound + 2.0 ** -52 * np.abs(ref))


@pytest.mark.parametrize("k", [2, 3, 4])
@pytest.mark.parametrize("dist,K", [("u01", 8192), ("absn", 2048), ("neg", 8192)])
def test_gemm_same_sign_long_k(k, dist, K):
    """Operands of one sign (no cancellation: the partial sums grow to sum|ab| and the tensor core's
    truncation errors all point one way) with a long K, held to the same 2^-22 sum|ab| as mixed signs."""
    M, N = 384, 640
    f = (k, 0)
    g1, g2 = np.random.default_rng(21), np.random.default_rng(22)
    if dist == "absn":
        a, b = np.abs(g1.standard_normal(M * K)), np.abs(g2.standard_normal(K * N))
    else:
        a, b = g1.uniform(0, 1, M * K), g2.uniform(0, 1, K * N)
        if dist == "neg":
            a = -a
    A = _codes(a.astype(np.float32), f)
    B = _codes(b.astype(np.float32), f)
    got = run_gemm(M, N, K, f, A, K, B, N)
    s = np.random.default_rng(23)
    rows = s.integers(0, M, 2048)
    cols = s.integers(0, N, 2048)
    worst = check(got, M, N, K, f, A, K, B, N, 1.0, 0.0, None, rows, cols)
    print(f"k={k} {dist} K={K}: worst error = {worst:.3g} x 2^-22 sum|ab|")


@pytest.mark.parametrize("k", [3, 4])
def test_gemm_near_float_max(k):
    """Entries up to the largest binary32 values times small partners: finite products, so the
    split into bf16 parts must stay finite (no rounding of the top part up to infinity)."""
    m, n, kk = 130, 140, 96
    f = (k, 0)
    g = np.random.default_rng(31)
    a = g.uniform(-1, 1, m * kk).astype(np.float32)
    a[::7] = np.float32(3.4e38) * np.sign(g.uniform(-1, 1, a[::7].size)).astype(np.float32)
    a[3::11] = np.float32(-3.3962e38)                       # just above the bf16 rounding threshold 0x7F7F8000
    b = (g.uniform(-1, 1, kk * n) * 1e-30).astype(np.float32)
    A, B = _codes(a, f), _codes(b, f)
    got = run_gemm(m, n, kk, f, A, kk, B, n)
    assert np.all(np.isfinite(got[:, :n]))
    check(got, m, n, kk, f, A, kk, B, n, 1.0, 0.0, None)


@pytest.mark.parametrize("k", [2, 3, 4])
def test_gemm_special_values_ieee_class(k):
    """Inf and NaN inputs (Sec. 5.3): an entry whose sum meets one is NaN when a term is NaN (a NaN
    input or Inf * 0) or infinities of both signs meet, else the signed infinity; the oracle gives the
    plain IEEE sum there.  All other entries keep the 2^-22 bound; alpha and beta apply as elsewhere."""
    m, n, kk = 150, 170, 200
    f = (k, 0)
    g = np.random.default_rng(41 + k)
    a = g.uniform(-1, 1, (m, kk)).astype(np.float32)
    b = g.uniform(-1, 1, (kk, n)).astype(np.float32)
    a[3, 10] = np.inf                       # row 3: +Inf times column entries (some made 0 below)
    a[7, 20] = -np.inf
    a[7, 21] = np.inf                       # row 7: both signs -> NaN
    a[11, 30] = np.nan                      # row 11: NaN
    b[10, 5] = 0.0                          # (3, 5): Inf * 0 -> NaN
    b[40, 100] = -np.inf                    # column 100: -Inf
    b[50, 140] = np.nan                     # column 140: NaN
    A, B = _codes(a.reshape(-1), f), _codes(b.reshape(-1), f)
    C0 = g.uniform(-1, 1, (m, n))
    got = run_gemm(m, n, kk, f, A, kk, B, n, alpha=-1.5, beta=0.5, C0=C0)
    rr, cc = np.meshgrid(np.arange(m), np.arange(n), indexing="ij")
    rows, cols = rr.reshape(-1), cc.reshape(-1)
    ref, absum = oracle.gemm_entries(rows, cols, kk, -1.5, A, (0, k), kk, B, (0, k), n, 0.5,
                                     C0[rows, cols].astype(np.float64))
    g_ = got[rows, cols].astype(np.float64)
    special = ~np.isfinite(ref)
    assert special.sum() > 300
    assert np.array_equal(np.isnan(g_[special]), np.isnan(ref[special]))
    inf = special & ~np.isnan(ref)
    assert np.array_equal(g_[inf], ref[inf])
    assert np.isnan(g_[special & np.isnan(ref)]).all()
    fin = ~special
    bound = 2.0 ** -22 * (1.5 * absum[fin] + 0.5 * np.abs(C0[rows, cols][fin]))
    assert np.all(np.abs(g_[fin] - ref[fin]) <= bound)
