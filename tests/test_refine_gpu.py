"""GPU parity of flyte_refine_jacobi (mixed-precision iterative refinement) against the oracle.

Both run the same sequence of steps: binary64 residual on A64, Jacobi-Richardson
correction sweeps on the k-byte copy.  Their products differ only by the
rounding of the dot products (both far inside the gemv bound), so on a well
conditioned system they take the same number of corrections and their
solutions differ by at most ||A^-1|| (||r_gpu|| + ||r_ref||).
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
from paper_1601_07789_gb300 import flyte, inputs
from tests.gpu_util import sync

pytestmark = pytest.mark.gpu


def gpu_refine(A, Ak, fa, b, x0, tol, max_outer, inner):
    A64 = torch.from_numpy(np.ascontiguousarray(A).reshape(-1)).cuda()
    Akd = torch.from_numpy(Ak).cuda()
    bd = torch.from_numpy(b).cuda()
    xd = torch.from_numpy(x0.copy()).cuda()
    it, rel = flyte.refine_jacobi(A64, Akd, fa, bd, xd, tol, max_outer, inner)
    sync()
    return xd.cpu().numpy(), it, rel


@pytest.mark.parametrize("k", [3, 4, 5])
@pytest.mark.parametrize("n", [1000, 1024])
def test_refine_matches_oracle(k, n):
    A, b = inputs.refine_system(n)
    Ak = oracle.pack(A.reshape(-1), 1, k)
    x0 = np.zeros(n)
    xg, itg, relg = gpu_refine(A, Ak, (k, 1), b, x0, 1e-12, 30, 2)
    xo, ito, relo = oracle.refine_jacobi(n, A, Ak, (1, k), b, x0, 1e-12, 30, 2)
    assert relg <= 1e-12 and relo <= 1e-12
    assert itg == ito
    smin = np.linalg.svd(A, compute_uv=False)[-1]
    rg = np.linalg.norm(b - A @ xg)
    ro = np.linalg.norm(b - A @ xo)
    assert rg <= 2e-12 * np.linalg.norm(b)                      # the GPU's own residual, recomputed here
    assert np.linalg.norm(xg - xo) <= 1.01 * (rg + ro) / smin + 1e-15 * np.linalg.norm(xo)


@pytest.mark.parametrize("k", [3, 4, 5])
def test_refine_harder_system_matches_oracle(k):
    """A = G/sqrt(n) + 10 I with 8 sweeps per correction: the stored precision limits each correction
    (k = 3 needs more of them); GPU and oracle take the same steps and reach the same solution."""
    n = 1024
    A, b = inputs.refine_system(n, 31, 32, diag=10.0)
    Ak = oracle.pack(A.reshape(-1), 1, k)
    x0 = np.zeros(n)
    xg, itg, relg = gpu_refine(A, Ak, (k, 1), b, x0, 1e-12, 40, 8)
    xo, ito, relo = oracle.refine_jacobi(n, A, Ak, (1, k), b, x0, 1e-12, 40, 8)
    assert relg <= 1e-12 and relo <= 1e-12
    assert itg == ito
    smin = np.linalg.svd(A, compute_uv=False)[-1]
    rg = np.linalg.norm(b - A @ xg)
    ro = np.linalg.norm(b - A @ xo)
    assert rg <= 2e-12 * np.linalg.norm(b)
    assert np.linalg.norm(xg - xo) <= 1.01 * (rg + ro) / smin + 1e-15 * np.linalg.norm(xo)


def test_refine_fixed_steps_and_edges():
    """A fixed number of steps (tol = 0) from a nonzero guess, inner = 1 and 3; tol = inf does nothing."""
    n = 777
    A, b = inputs.refine_system(n, 10, 11)
    x0 = np.random.default_rng(12).standard_normal(n)
    Ak = oracle.pack(A.reshape(-1), 1, 4)
    for inner in (1, 3):
        xg, itg, _ = gpu_refine(A, Ak, (4, 1), b, x0, 0.0, 2, inner)
        xo, ito, _ = oracle.refine_jacobi(n, A, Ak, (1, 4), b, x0, 0.0, 2, inner)
        assert itg == ito == 2
        assert np.max(np.abs(xg - xo)) <= 1e-13 * np.max(np.abs(xo))
    xg, itg, relg = gpu_refine(A, Ak, (4, 1), b, x0, np.inf, 5, 2)
    assert itg == 0 and np.array_equal(xg, x0)
    # the reported residual r = b - A64 x0 comes from a flyte gemv: within 4(n+2) 2^-53 (|A||x0| + |b|)
    # per entry of the oracle's r (Dot2), plus the rounding of the norms
    r_ref, absum = oracle.gemv("N", n, n, -1.0, oracle.pack(A.reshape(-1), 1, 8), (1, 8), n, x0, 1, 1.0, b, 1)
    e = 4 * (n + 2) * 2.0 ** -53 * (absum + np.abs(b))
    nb = np.linalg.norm(b)
    assert abs(relg - np.linalg.norm(r_ref) / nb) <= np.linalg.norm(e) / nb + 1e-13 * relg
    with pytest.raises(flyte.FlyteError):
        gpu_refine(A, Ak, (4, 1), b, x0, 1e-12, 5, 0)              # inner < 1


def test_refine_full_size_k4():
    """The n = 8192 workload at k = 4: converges to 1e-12, residual recomputed on the host."""
    n = 8192
    A, b = inputs.refine_system(n)
    Ak = oracle.pack(A.reshape(-1), 1, 4)
    xg, itg, relg = gpu_refine(A, Ak, (4, 1), b, np.zeros(n), 1e-12, 30, 2)
    assert relg <= 1e-12 and 1 <= itg <= 10
    assert np.linalg.norm(b - A @ xg) <= 2e-12 * np.linalg.norm(b)
