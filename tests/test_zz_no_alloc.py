"""flyte_gemv_static: gemv whose scratch is built into the library.

Callers that cannot allocate device memory (a plug-in whose host framework
owns every allocation, or a serving loop that must not call cudaMalloc once
running) use this entry point instead of flyte_gemv.  The test calls it
through the C ABI and checks it against flyte_gemv with a caller workspace,
within the gemv tolerance of tests/test_gemv_gpu.py, on two calls in a row
(the second call must not depend on what the first left in the shared
scratch).  This file is collected last so that a failure here does not stop
the rest of the suite in a run that stops at the first failure.
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


def _absum(trans, m, n, k, A, x):
    Av = np.abs(oracle.values(A, 1, k).reshape(m, n))
    return Av @ np.abs(x[:n]) if trans == "N" else Av.T @ np.abs(x[:m])


def _with_workspace(trans, m, n, k, Ad, xd, y0):
    yd = torch.from_numpy(y0.copy()).cuda()
    flyte.gemv(trans, m, n, 1.5, Ad, (k, 1), n, xd, -0.5, yd)
    return yd


def _static(trans, m, n, k, Ad, xd, y0):
    yd = torch.from_numpy(y0.copy()).cuda()
    flyte.gemv_static_raw(trans, m, n, 1.5, Ad, (k, 1), n, xd, 1, -0.5, yd, 1)
    return yd


@pytest.mark.parametrize("trans,m,n,k", [("N", 3000, 20000, 4), ("T", 4096, 1000, 3)])
def test_gemv_static_matches_workspace_path_twice(trans, m, n, k):
    for call, seed in enumerate((1, 2)):          # two calls in a row share the scratch
        A, x, y0 = _case(m, n, k, seed + 10 * k)
        Ad = torch.from_numpy(A).cuda()
        xd = torch.from_numpy(x).cuda()
        got = _static(trans, m, n, k, Ad, xd, y0)
        want = _with_workspace(trans, m, n, k, Ad, xd, y0)
        torch.cuda.synchronize()
        ly = m if trans == "N" else n
        length = n if trans == "N" else m
        bound = 4 * (length + 2) * EPS * (1.5 * _absum(trans, m, n, k, A, x) + 0.5 * np.abs(y0[:ly]))
        err = np.abs(got.cpu().numpy()[:ly] - want.cpu().numpy()[:ly])
        assert np.all(err <= bound), f"call {call}: max err/bound {np.max(err / bound):.3g}"
        assert np.array_equal(got.cpu().numpy()[ly:], y0[ly:])


def test_gemv_static_rejects_calls_beyond_its_scratch():
    m = n = 16384                                   # 'T' needs ~22 MB of scratch
    assert flyte.workspace_bytes("gemv_t", m, n, 0, (4, 1)) > 4 << 20
    y = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(flyte.FlyteError) as e:
        flyte.gemv_static_raw("T", m, n, 1.0, y, (4, 1), n, y, 1, 0.0, y, 1)
    assert e.value.status == 5
    assert "scratch" in str(e.value)
