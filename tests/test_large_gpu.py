"""GPU parity beyond 32-bit element and byte counts.

Streams of 2^31 + 13 elements and a gemv matrix of 2.4e9 elements (7.2 GB of
codes) go through the same entry points as the smaller tests; the outputs are
checked on samples that cover the start, the region around element 2^31 (and
byte 2^32), the ragged tail and random positions, against the oracle applied
to the same sampled inputs.  The dot product keeps its bound sharp at this
length by giving every element outside a sampled set the tiny value 2^-30
(its contribution, count * 2^-60, is exact and known), so that a dropped or
repeated element of the sampled set exceeds the bound.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
from paper_1601_07789_gb300 import flyte
from tests.gpu_util import sync

pytestmark = pytest.mark.gpu
EPS = 2.0 ** -53
N_BIG = (1 << 31) + 13


def _sample_indices(n: int, seed: int, around=(1 << 31,)) -> np.ndarray:
    g = np.random.default_rng(seed)
    parts = [np.arange(0, 2048), np.arange(n - 2048, n), g.integers(0, n, size=8192)]
    for c in around:
        parts.append(np.arange(max(0, c - 1024), min(n, c + 1024)))
    return np.unique(np.concatenate(parts)).astype(np.int64)


def _gather_codes(codes: torch.Tensor, idx: np.ndarray, k: int) -> np.ndarray:
    rows = codes.view(-1, k).index_select(0, torch.from_numpy(idx).to(codes.device))
    return rows.cpu().numpy().reshape(-1)


def _free():
    sync()
    torch.cuda.empty_cache()


def test_pack_unpack_beyond_2pow31_elements():
    k = 3
    gen = torch.Generator(device="cuda")
    gen.manual_seed(31)
    x = torch.randn(N_BIG, dtype=torch.float64, device="cuda", generator=gen)
    idx = _sample_indices(N_BIG, 1)
    xs = x.index_select(0, torch.from_numpy(idx).cuda()).cpu().numpy()
    codes = flyte.pack(x, k)
    del x
    _free()
    want = oracle.pack(xs, oracle.F64, k, oracle.RNE)
    assert np.array_equal(_gather_codes(codes, idx, k), want)
    back = flyte.unpack(codes, k, flyte.F64)
    sync()
    got = back.index_select(0, torch.from_numpy(idx).cuda()).cpu().numpy()
    assert np.array_equal(got.view(np.uint64), oracle.unpack(want, oracle.F64, k))
    del back, codes
    _free()


def test_dot_axpy_beyond_2pow31_elements():
    k, n = 4, N_BIG
    g = np.random.default_rng(7)
    special = _sample_indices(n, 2)
    xv = oracle.pack(g.standard_normal(special.size), oracle.F64, k)
    yv = oracle.pack(g.standard_normal(special.size), oracle.F64, k)
    tiny = oracle.pack(np.array([2.0 ** -30]), oracle.F64, k)
    sp = torch.from_numpy(special).cuda()

    def stream(vals):
        s = torch.from_numpy(tiny).cuda().repeat(n)
        s.view(n, k).index_put_((sp,), torch.from_numpy(vals.reshape(-1, k)).cuda())
        return s

    X, Y = stream(xv), stream(yv)
    got = float(flyte.dot(X, (k, flyte.F64), Y, (k, flyte.F64)).item())
    ref_s, _, abs_s = oracle.dot(special.size, xv, (oracle.F64, k), 1, yv, (oracle.F64, k), 1)
    nbg = n - special.size
    ref = ref_s + nbg * 2.0 ** -60
    absum = abs_s + nbg * 2.0 ** -60
    assert abs(got - ref) <= 4 * n * EPS * absum + 2 * EPS * abs(ref), (got, ref)
    assert 4 * n * EPS * absum < 0.01     # the bound is sharp enough to see one dropped element

    # axpy in place over the same streams, alpha a binary32 number (exact binary32 path) and not;
    # a background element is checked too (2^-30 (alpha + 1), rounded to the code)
    sset = set(special.tolist())
    bgi = next(i for i in range(2048, n) if i not in sset)
    ybg = tiny.copy()
    for alpha, mode in ((1.5, oracle.RNE), (0.1, oracle.RTZ)):
        flyte.axpy(alpha, X, (k, flyte.F64), Y, (k, flyte.F64), mode=mode)
        sync()
        yv = oracle.axpy(special.size, alpha, xv, (oracle.F64, k), 1, yv, (oracle.F64, k), 1, mode)
        assert np.array_equal(_gather_codes(Y, special, k), yv), alpha
        ybg = oracle.axpy(1, alpha, tiny, (oracle.F64, k), 1, ybg, (oracle.F64, k), 1, mode)
        assert np.array_equal(_gather_codes(Y, np.array([bgi]), k), ybg), alpha
    del X, Y
    _free()


@pytest.mark.parametrize("trans", ["N", "T"])
def test_gemv_beyond_2pow32_bytes(trans):
    k, m, n = 3, 40000, 60000          # 2.4e9 elements, 7.2 GB of codes
    gen = torch.Generator(device="cuda")
    gen.manual_seed(32)
    A = torch.empty(m * n * k, dtype=torch.uint8, device="cuda")
    step = 4000                          # pack in row blocks to bound the binary64 temporary
    for r0 in range(0, m, step):
        blk = torch.randn(step * n, dtype=torch.float64, device="cuda", generator=gen)
        flyte.pack(blk, k, out=A[r0 * n * k:(r0 + step) * n * k])
    del blk
    _free()
    g = np.random.default_rng(3)
    lx, ly = (n, m) if trans == "N" else (m, n)
    xh = g.standard_normal(lx)
    yh = g.standard_normal(ly)
    y = torch.from_numpy(yh.copy()).cuda()
    flyte.gemv(trans, m, n, 1.5, A, (k, flyte.F64), n, torch.from_numpy(xh).cuda(), -0.5, y)
    sync()
    yg = y.cpu().numpy()
    A3 = A.view(m, n, k)
    if trans == "N":
        rows = np.unique(np.concatenate([np.arange(8), np.arange(m - 8, m), g.integers(0, m, 48)]))
        sub = A3.index_select(0, torch.from_numpy(rows).cuda()).cpu().numpy().reshape(-1)
        ref, absum = oracle.gemv("N", rows.size, n, 1.5, sub, (oracle.F64, k), n, xh, 1, -0.5, yh[rows], 1)
        got, y0 = yg[rows], yh[rows]
    else:
        cols = np.unique(np.concatenate([np.arange(8), np.arange(n - 8, n), g.integers(0, n, 48)]))
        sub = A3.index_select(1, torch.from_numpy(cols).cuda()).cpu().numpy().reshape(-1)
        ref, absum = oracle.gemv("T", m, cols.size, 1.5, sub, (oracle.F64, k), cols.size, xh, 1, -0.5,
                                 yh[cols], 1)
        got, y0 = yg[cols], yh[cols]
    L = n if trans == "N" else m
    bound = 4 * (L + 2) * EPS * (1.5 * absum + 0.5 * np.abs(y0)) + 2 * EPS * np.abs(ref)
    assert np.all(np.abs(got - ref) <= bound)
    del A, A3
    _free()
