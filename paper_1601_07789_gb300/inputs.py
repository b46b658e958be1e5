"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module only draws random numbers and lays out IEEE-754 bit patterns; it
holds none of the flyte arithmetic (no rounding, no packing, no BLAS).  Both
the CUDA path and the CPU oracle consume what it returns.

Recipes (the paper measured no public dataset; Sec. 6 only says problem size
is elements per vector or per matrix side):

* ``mixture_f64``: 70 % N(0,1), 25 % sign * 10**U(-300, 300), 5 % special bit
  patterns (signed zeros, subnormals, +-max finite, +-Inf, quiet/signalling
  NaN, NaN with a low-bit-only payload, and for every width the halfway and
  carry patterns of the rounding step), positions shuffled.
* ``mixture_f32``: the binary32 analogue with 10**U(-38, 38).
* ``finite`` variants replace the specials by N(0,1) and narrow the wide
  part to 10**U(-150, 150) (binary64) / 10**U(-18, 18) (binary32).
* gemv: A N(0,1), x and y N(0,1).  gemm: A and B U(-1, 1).
"""
from __future__ import annotations

import numpy as np

F32, F64 = 0, 1

_SPECIAL_FRACTION = 0.05
_WIDE_FRACTION = 0.25


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def _halfway_and_carry(g: np.random.Generator, count: int, W: int, E: int,
                       widths: range) -> list[int]:
    """Patterns u = sign | kept << d | dropped for a random width k (d = W - 8k).

    Kinds: dropped bits exactly 100..0 with the kept part even, the same with
    it odd, and a kept mantissa of all ones with dropped >= half (rounding up
    carries into the exponent).  The exponent stays below all-ones.
    """
    out = []
    for _ in range(count):
        k = int(g.integers(widths.start, widths.stop))
        d = W - 8 * k
        kept_bits = 8 * k - 1                       # kept magnitude bits
        mant_bits = kept_bits - E                   # kept mantissa bits (< 0 for k = 1)
        sign = int(g.integers(0, 2)) << (W - 1)
        kind = int(g.integers(0, 3))
        if kind < 2 or mant_bits <= 0:
            t = int(g.integers(0, 1 << kept_bits))
            if mant_bits > 0:                       # keep the exponent finite
                t = (t & ((1 << mant_bits) - 1)) | (int(g.integers(1, (1 << E) - 1)) << mant_bits)
            t = (t & ~1) | (kind & 1)
            dropped = 1 << (d - 1)
        else:
            exp = int(g.integers(1, (1 << E) - 1))
            t = (exp << mant_bits) | ((1 << mant_bits) - 1)
            dropped = (1 << (d - 1)) | int(g.integers(0, 1 << (d - 1)))
        out.append(sign | (t << d) | dropped)
    return out


def _halfway_and_carry_f64(g: np.random.Generator, count: int) -> np.ndarray:
    return np.array(_halfway_and_carry(g, count, 64, 11, range(1, 8)), dtype=np.uint64)


def _halfway_and_carry_f32(g: np.random.Generator, count: int) -> np.ndarray:
    return np.array(_halfway_and_carry(g, count, 32, 8, range(1, 4)), dtype=np.uint32)


def special_f64(g: np.random.Generator, count: int) -> np.ndarray:
    """``count`` binary64 special bit patterns drawn from the fixed list."""
    fixed = np.array([
        0x0000000000000000, 0x8000000000000000,          # +-0
        0x0000000000000001, 0x800FFFFFFFFFFFFF,          # min subnormal, -max subnormal
        0x000FFFFFFFFFFFFF, 0x0008000000000000,          # max subnormal, a mid subnormal
        0x7FEFFFFFFFFFFFFF, 0xFFEFFFFFFFFFFFFF,          # +-max finite
        0x7FF0000000000000, 0xFFF0000000000000,          # +-Inf
        0x7FF8000000000000, 0xFFF8000000000001,          # quiet NaNs
        0x7FF0000000000001, 0x7FF4000000000000,          # signalling NaNs
        0x7FF000000000FFFF, 0xFFF0000000000100,          # NaN with a low-bit-only payload
        0x0010000000000000, 0x7FE0000000000000,          # min normal, 2**1023
    ], dtype=np.uint64)
    n_fixed = count // 2
    pick = fixed[g.integers(0, fixed.size, size=n_fixed)]
    sub = g.integers(1, 1 << 52, size=max(count - n_fixed, 0) // 4, dtype=np.uint64)
    sub |= np.uint64(1 << 63) * g.integers(0, 2, size=sub.size, dtype=np.uint64)
    rest = count - n_fixed - sub.size
    return np.concatenate([pick, sub, _halfway_and_carry_f64(g, rest)])


def special_f32(g: np.random.Generator, count: int) -> np.ndarray:
    fixed = np.array([
        0x00000000, 0x80000000, 0x00000001, 0x807FFFFF, 0x007FFFFF, 0x00400000,
        0x7F7FFFFF, 0xFF7FFFFF, 0x7F800000, 0xFF800000, 0x7FC00000, 0xFFC00001,
        0x7F800001, 0x7FA00000, 0x7F8000FF, 0xFF800100, 0x00800000, 0x7F000000,
    ], dtype=np.uint32)
    n_fixed = count // 2
    pick = fixed[g.integers(0, fixed.size, size=n_fixed)]
    sub = g.integers(1, 1 << 23, size=max(count - n_fixed, 0) // 4, dtype=np.uint32)
    sub |= np.uint32(1 << 31) * g.integers(0, 2, size=sub.size, dtype=np.uint32)
    rest = count - n_fixed - sub.size
    return np.concatenate([pick, sub, _halfway_and_carry_f32(g, rest)])


def mixture_f64(n: int, seed: int = 1601, finite: bool = False) -> np.ndarray:
    """Bit patterns (uint64) of the binary64 mixture; see the module docstring."""
    g = rng(seed)
    n_spec = int(round(n * _SPECIAL_FRACTION))
    n_wide = int(round(n * _WIDE_FRACTION))
    n_norm = n - n_spec - n_wide
    lo, hi = (-150.0, 150.0) if finite else (-300.0, 300.0)
    normal = g.standard_normal(n_norm)
    sign = np.where(g.integers(0, 2, size=n_wide) == 1, -1.0, 1.0)
    wide = sign * np.power(10.0, g.uniform(lo, hi, size=n_wide))
    if finite:
        spec = g.standard_normal(n_spec).view(np.uint64)
    else:
        spec = special_f64(g, n_spec)
    bits = np.concatenate([normal.view(np.uint64), wide.view(np.uint64), spec])
    return bits[g.permutation(n)].copy()


def mixture_f32(n: int, seed: int = 7789, finite: bool = False) -> np.ndarray:
    """Bit patterns (uint32) of the binary32 mixture."""
    g = rng(seed)
    n_spec = int(round(n * _SPECIAL_FRACTION))
    n_wide = int(round(n * _WIDE_FRACTION))
    n_norm = n - n_spec - n_wide
    lo, hi = (-18.0, 18.0) if finite else (-38.0, 38.0)
    normal = g.standard_normal(n_norm).astype(np.float32)
    sign = np.where(g.integers(0, 2, size=n_wide) == 1, -1.0, 1.0)
    wide = (sign * np.power(10.0, g.uniform(lo, hi, size=n_wide))).astype(np.float32)
    if finite:
        spec = g.standard_normal(n_spec).astype(np.float32).view(np.uint32)
    else:
        spec = special_f32(g, n_spec)
    bits = np.concatenate([normal.view(np.uint32), wide.view(np.uint32), spec])
    return bits[g.permutation(n)].copy()


def normal_f64(n: int, seed: int) -> np.ndarray:
    return rng(seed).standard_normal(n)


def uniform_f64(n: int, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    return rng(seed).uniform(lo, hi, size=n)


def uniform_f32(n: int, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    return rng(seed).uniform(lo, hi, size=n).astype(np.float32)


def random_codes(n: int, k: int, seed: int) -> np.ndarray:
    """n uniformly random k-byte codes as a contiguous byte stream."""
    return rng(seed).integers(0, 256, size=n * k, dtype=np.uint8)


def gemv_operands(m: int, n: int, seed_a: int = 2, seed_x: int = 3, seed_y: int = 4):
    """FP64 A (m x n, row-major, N(0,1)), x (n), y (m) for y <- alpha A x + beta y."""
    A = rng(seed_a).standard_normal((m, n))
    x = rng(seed_x).standard_normal(max(m, n))
    y = rng(seed_y).standard_normal(max(m, n))
    return A, x, y


def gemm_operands_f32(M: int, N: int, K: int, seed_a: int = 5, seed_b: int = 6):
    A = rng(seed_a).uniform(-1.0, 1.0, size=(M, K)).astype(np.float32)
    B = rng(seed_b).uniform(-1.0, 1.0, size=(K, N)).astype(np.float32)
    return A, B


def gemm_operands_f64(M: int, N: int, K: int, seed_a: int = 5, seed_b: int = 6):
    A = rng(seed_a).uniform(-1.0, 1.0, size=(M, K))
    B = rng(seed_b).uniform(-1.0, 1.0, size=(K, N))
    return A, B


def refine_system(n: int, seed_g: int = 8, seed_b: int = 9, diag: float | None = None):
    """Diagonally dominant system of the refinement workload: A = G / sqrt(n) + d I with G N(0,1)
    (row-major float64), d = n unless given (d = 10: a Jacobi contraction of about 1/10 per sweep),
    and b N(0,1)."""
    A = rng(seed_g).standard_normal((n, n)) / np.sqrt(n)
    A[np.arange(n), np.arange(n)] += n if diag is None else diag
    b = rng(seed_b).standard_normal(n)
    return A, b


BATCH_FORMATS = [(k, 1) for k in range(2, 8)] + [(2, 0), (3, 0)]   # (k, base): double 2..7, float 2..3


def batch_specs(njobs: int, seed: int = 5, len_range=(1e3, 1e6), side_range=(64, 4096)):
    """Uneven jobs of the batched workload: op uniformly among unpack/dot/axpy/gemv N/gemv T, a
    format from BATCH_FORMATS, vector lengths log-uniform in len_range and gemv sides log-uniform in
    side_range.  Returns dicts {op, k, base, n, m} (op: 0 unpack, 1 dot, 2 axpy, 3 gemv N, 4 gemv T)."""
    g = rng(seed)
    out = []
    for _ in range(njobs):
        op = int(g.integers(0, 5))
        k, base = BATCH_FORMATS[int(g.integers(0, len(BATCH_FORMATS)))]
        if op <= 2:
            n = int(np.exp(g.uniform(np.log(len_range[0]), np.log(len_range[1]))))
            m = 0
        else:
            n = int(np.exp(g.uniform(np.log(side_range[0]), np.log(side_range[1]))))
            m = int(np.exp(g.uniform(np.log(side_range[0]), np.log(side_range[1]))))
        out.append({"op": op, "k": k, "base": base, "n": n, "m": m})
    return out
