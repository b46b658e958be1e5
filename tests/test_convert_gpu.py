"""GPU parity of flyte_pack / flyte_unpack against the CPU oracle: bit-exact.

Inputs are the seeded mixtures (specials, halfway and carry patterns) and
uniformly random codes; sizes span several thread groups and ragged tails;
base pointers are misaligned by every offset 0..15 on a subset; strides
1..3 on both sides.  Output buffers carry guard bytes, and for strided
outputs the skipped elements must keep their previous contents.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
from paper_1601_07789_gb300 import flyte, inputs
from tests.gpu_util import Guarded, span_bytes, sync

pytestmark = pytest.mark.gpu

FORMATS = [(0, k) for k in range(1, 5)] + [(1, k) for k in range(1, 9)]
MODES = ["rne", "rtz", "half_up", "rto"]
ORC_MODE = {"rne": oracle.RNE, "rtz": oracle.RTZ, "half_up": oracle.HALF_UP, "rto": oracle.RTO}


def _nat(base):
    return (np.uint32, 4) if base == 0 else (np.uint64, 8)


def _mixture(base, n, seed):
    return inputs.mixture_f32(n, seed) if base == 0 else inputs.mixture_f64(n, seed)


def run_pack(bits, base, k, mode, n, inc_src=1, inc_dst=1, src_off=0, dst_off=0, prefill_seed=9):
    dt, W = _nat(base)
    src_bytes = span_bytes(n, inc_src, W)
    src = np.zeros(src_bytes // W if src_bytes else 0, dtype=dt)
    src[::inc_src] = bits[:n]
    dst_bytes = span_bytes(n, inc_dst, k)
    prefill = np.random.default_rng(prefill_seed).integers(0, 256, dst_bytes, dtype=np.uint8)
    s = Guarded(src_bytes, src_off, fill=src)
    d = Guarded(dst_bytes, dst_off, fill=prefill)
    flyte.pack_raw(d.ptr, s.ptr, n, (k, base), inc_dst, inc_src, mode)
    sync()
    d.check_guards()
    want = prefill.copy()
    if n:
        oracle.pack(src, base, k, ORC_MODE[mode], n=n, inc_src=inc_src, inc_dst=inc_dst, dst=want)
    return d.inner(), want


def run_unpack(codes, base, k, n, inc_src=1, inc_dst=1, src_off=0, dst_off=0, prefill_seed=8):
    dt, W = _nat(base)
    src_bytes = span_bytes(n, inc_src, k)
    src = codes[:src_bytes]
    dst_bytes = span_bytes(n, inc_dst, W)
    prefill = np.random.default_rng(prefill_seed).integers(0, 256, dst_bytes, dtype=np.uint8)
    s = Guarded(src_bytes, src_off, fill=src)
    d = Guarded(dst_bytes, dst_off, fill=prefill)
    flyte.unpack_raw(d.ptr, s.ptr, n, (k, base), inc_dst, inc_src)
    sync()
    d.check_guards()
    want = prefill.view(dt).copy() if dst_bytes else np.zeros(0, dt)
    if n:
        oracle.unpack(src, base, k, n=n, inc_src=inc_src, inc_dst=inc_dst, dst=want)
    return d.inner(), want.view(np.uint8)


SIZES = [0, 1, 3, 4, 5, 7, 31, 128, 1023, 4099, 65537, 262147]


@pytest.mark.parametrize("base,k", FORMATS)
@pytest.mark.parametrize("mode", MODES)
def test_pack_sizes(base, k, mode):
    bits = _mixture(base, max(SIZES), seed=11 + k)
    for n in SIZES:
        got, want = run_pack(bits, base, k, mode, n)
        assert np.array_equal(got, want), f"n={n}"


@pytest.mark.parametrize("base,k", FORMATS)
def test_unpack_sizes(base, k):
    codes = inputs.random_codes(max(SIZES), k, seed=21 + k)
    for n in SIZES:
        got, want = run_unpack(codes, base, k, n)
        assert np.array_equal(got, want), f"n={n}"


@pytest.mark.parametrize("base,k", FORMATS)
def test_misaligned_pointers(base, k):
    bits = _mixture(base, 3000, seed=31 + k)
    codes = inputs.random_codes(3000, k, seed=41 + k)
    for off in range(16):
        for n in (37, 2050):
            got, want = run_pack(bits, base, k, "rne", n, src_off=off, dst_off=(off * 7) % 16)
            assert np.array_equal(got, want), f"pack off={off} n={n}"
            got, want = run_unpack(codes, base, k, n, src_off=off, dst_off=(off * 5) % 16)
            assert np.array_equal(got, want), f"unpack off={off} n={n}"


@pytest.mark.parametrize("base,k", FORMATS)
@pytest.mark.parametrize("inc_src,inc_dst", [(2, 1), (1, 3), (3, 2)])
def test_strides(base, k, inc_src, inc_dst):
    n = 5001
    bits = _mixture(base, n, seed=51 + k)
    codes = inputs.random_codes(n * 3, k, seed=61 + k)
    got, want = run_pack(bits, base, k, "rne", n, inc_src, inc_dst)
    assert np.array_equal(got, want)
    got, want = run_unpack(codes, base, k, n, inc_src, inc_dst)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("base,k", [(0, 1), (0, 2), (1, 1), (1, 2), (0, 3)])
def test_exhaustive_codes(base, k):
    """Every code: unpack bit-exact, and pack(unpack) bit-exact in every mode."""
    n = 1 << (8 * k)
    q = np.arange(n, dtype=np.uint64)
    codes = np.stack([((q >> np.uint64(8 * i)) & np.uint64(0xFF)).astype(np.uint8)
                      for i in range(k)], axis=1).reshape(-1)
    got, want = run_unpack(codes, base, k, n)
    assert np.array_equal(got, want)
    dt, _ = _nat(base)
    bits = want.view(dt)
    for mode in MODES:
        got, want2 = run_pack(bits, base, k, mode, n)
        assert np.array_equal(got, want2), mode


@pytest.mark.parametrize("base,k", FORMATS)
def test_config_mixture_1m(base, k):
    """The 1,048,576-value mixtures (specials, halfway and carry patterns), all modes."""
    n = 1 << 20
    bits = _mixture(base, n, seed=1601 if base == 1 else 7789)
    for mode in MODES:
        got, want = run_pack(bits, base, k, mode, n)
        assert np.array_equal(got, want), mode
    got, want = run_unpack(got, base, k, n)
    assert np.array_equal(got, want)


def test_tensor_helpers_roundtrip():
    x = torch.randn(10001, dtype=torch.float64, device="cuda")
    s = flyte.pack(x, 8)
    assert torch.equal(flyte.unpack(s, 8, flyte.F64), x)
    y = torch.randn(10001, dtype=torch.float32, device="cuda")
    s = flyte.pack(y, 2)
    ref = y.to(torch.bfloat16).float()
    assert torch.equal(flyte.unpack(s, 2, flyte.F32), ref)


def test_error_statuses_launch_nothing():
    buf = torch.zeros(64, dtype=torch.uint8, device="cuda")
    with pytest.raises(flyte.FlyteError) as e:
        flyte.pack_raw(buf, buf, 4, (5, flyte.F32))
    assert e.value.status == 1
    with pytest.raises(flyte.FlyteError):
        flyte.pack_raw(buf, buf, -1, (2, flyte.F32))
    with pytest.raises(flyte.FlyteError):
        flyte.unpack_raw(buf, buf, 4, (2, flyte.F32), 0, 1)
    with pytest.raises(flyte.FlyteError):
        flyte.pack_raw(buf, buf, 4, (2, flyte.F32), 1, 1, 7)
    sync()
    assert torch.count_nonzero(buf).item() == 0
