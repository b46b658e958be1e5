"""flyte_gemv_static: gemv whose scratch is built into the library.

Callers that cannot allocate device memory (a plug-in whose host framework
owns every allocation, or a serving loop that must not call cudaMalloc once
running) use this entry point instead of flyte_gemv.  The test calls it
through the C ABI on two calls in a row (the second call must not depend on
what the first left in the shared scratch) and checks each result two ways:
against the CPU oracle within the gemv bound of tests/test_gemv_gpu.py, and
bit for bit against flyte_gemv with a caller workspace (the same kernels on
the same inputs, whose sums run in a fixed order).  This file is collected
last so that a failure here does not stop the rest of the suite in a run
that stops at the first failure.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
from paper_1601_07789_gb300 import flyte

pytestmark = pytest.mark.gpu
EPS = 2.0 ** -53


def _case(m, n, k, seed):
    g = np.random.default_rng(seed)
    A = oracle.pack(g.standard_normal(m * n), 1, k)
    x = g.standard_normal(max(m, n))
    y = g.standard_normal(max(m, n))
    return A, x, y


def _with_workspace(trans, m, n, k, Ad, xd, y0):
    yd = torch.from_numpy(y0.copy()).cuda()
    flyte.gemv(trans, m, n, 1.5, Ad, (k, 1), n, xd, -0.5, yd)
    return yd


def _static(trans, m, n, k, Ad, xd, y0):
    yd = torch.from_numpy(y0.copy()).cuda()
    flyte.gemv_static_raw(trans, m, n, 1.5, Ad, (k, 1), n, xd, 1, -0.5, yd, 1)
    return yd


@pytest.mark.parametrize("trans,m,n,k", [("N", 3000, 20000, 4), ("T", 4096, 1000, 3)])
def test_gemv_static_matches_oracle_and_workspace_path_twice(trans, m, n, k):
    for call, seed in enumerate((1, 2)):          # two calls in a row share the scratch
        A, x, y0 = _case(m, n, k, seed + 10 * k)
        Ad = torch.from_numpy(A).cuda()
        xd = torch.from_numpy(x).cuda()
        got = _static(trans, m, n, k, Ad, xd, y0).cpu().numpy()
        want = _with_workspace(trans, m, n, k, Ad, xd, y0).cpu().numpy()
        ly = m if trans == "N" else n
        lx = n if trans == "N" else m
        assert np.array_equal(got.view(np.uint64), want.view(np.uint64)), f"call {call}: differs from flyte_gemv"
        ref, absum = oracle.gemv(trans, m, n, 1.5, A, (1, k), n, x[:lx], 1, -0.5, y0[:ly], 1)
        # the stated gemv bound, plus the oracle's own binary64 rounding of its reference
        bound = 4 * (lx + 2) * EPS * (1.5 * absum + 0.5 * np.abs(y0[:ly])) + 2 * EPS * np.abs(ref)
        err = np.abs(got[:ly] - ref)
        assert np.all(err <= bound), f"call {call}: max err/bound {np.max(err / bound):.3g}"
        assert np.array_equal(got[ly:], y0[ly:])


def test_gemv_static_rejects_calls_beyond_its_scratch():
    m = n = 16384                                   # 'T' needs ~22 MB of scratch
    assert flyte.workspace_bytes("gemv_t", m, n, 0, (4, 1)) > 4 << 20
    y = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(flyte.FlyteError) as e:
        flyte.gemv_static_raw("T", m, n, 1.0, y, (4, 1), n, y, 1, 0.0, y, 1)
    assert e.value.status == 5
    assert "scratch" in str(e.value)


def test_gemv_static_reports_bad_arguments_before_the_scratch_size():
    """A bad argument on a call too large for the built-in scratch is reported as a bad argument,
    as flyte_gemv reports it."""
    m = n = 16384
    y = torch.zeros(8, dtype=torch.float64, device="cuda")
    for args in [dict(lda=n - 1), dict(incx=0), dict(fa=(9, 1))]:
        kw = dict(lda=n, incx=1, fa=(4, 1))
        kw.update(args)
        with pytest.raises(flyte.FlyteError) as e:
            flyte.gemv_static_raw("T", m, n, 1.0, y, kw["fa"], kw["lda"], y, kw["incx"], 0.0, y, 1)
        assert e.value.status == 1, args
