"""CPU oracle for the flyte multibyte floating-point scheme (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  The product path (the CUDA library and its
Python binding) never does.  The arithmetic lives in ``flyte_oracle.c``, a
plain scalar C file that shares nothing with the CUDA sources; this module
compiles it with gcc and marshals numpy arrays into it.

Integer conventions (the oracle's own; they happen to match the C ABI's
numbering, which is fixed by the paper's notions, not shared code):
  base: 0 = binary32-based, 1 = binary64-based
  mode: 0 = nearest-even (Sec. 5.2), 1 = toward zero (Sec. 5.1),
        2 = add half an ULP and truncate (Fig. 6), 3 = round to odd (Sec. 7)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "flyte_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

F32, F64 = 0, 1
RNE, RTZ, HALF_UP, RTO = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile flyte_oracle.c into a shared library (gcc, -O2, no contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-Wall", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            i64, i32, u64 = ctypes.c_int64, ctypes.c_int, ctypes.c_uint64
            vp, dbl = ctypes.c_void_p, ctypes.c_double
            L.orc_read_code.argtypes = [vp, i32]
            L.orc_read_code.restype = u64
            L.orc_unpack_code.argtypes = [i32, i32, u64]
            L.orc_unpack_code.restype = u64
            L.orc_pack_bits.argtypes = [i32, i32, i32, u64]
            L.orc_pack_bits.restype = u64
            L.orc_unpack.argtypes = [i32, i32, vp, i64, i64, vp, i64]
            L.orc_unpack.restype = i32
            L.orc_pack.argtypes = [i32, i32, i32, vp, i64, i64, vp, i64]
            L.orc_pack.restype = i32
            L.orc_code_value.argtypes = [i32, i32, vp]
            L.orc_code_value.restype = dbl
            L.orc_dot.argtypes = [i64, vp, i32, i32, i64, vp, i32, i32, i64, vp]
            L.orc_dot.restype = i32
            L.orc_axpy.argtypes = [i64, dbl, vp, i32, i32, i64, vp, i32, i32, i64, i32]
            L.orc_axpy.restype = i32
            L.orc_scal.argtypes = [i64, dbl, vp, i32, i32, i64, i32]
            L.orc_scal.restype = i32
            L.orc_refine_jacobi.argtypes = [i64, vp, i64, vp, i32, i32, i64, vp, vp, dbl, i32, i32,
                                            ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]
            L.orc_refine_jacobi.restype = i32
            L.orc_gemv.argtypes = [ctypes.c_char, i64, i64, dbl, vp, i32, i32, i64, vp, i64, dbl,
                                   vp, i64, vp]
            L.orc_gemv.restype = i32
            L.orc_gemm_entries.argtypes = [i64, vp, vp, i64, dbl, vp, i32, i32, i64, vp, i32, i32,
                                           i64, dbl, vp, vp, vp]
            L.orc_gemm_entries.restype = i32
            _lib = L
    return _lib


def _ptr(a: np.ndarray | None):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"], "oracle arrays must be C-contiguous"
    return a.ctypes.data


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise ValueError(f"oracle {what}: invalid argument")


def native_dtype(base: int):
    return np.uint32 if base == F32 else np.uint64


def float_dtype(base: int):
    return np.float32 if base == F32 else np.float64


# ---- scalar helpers -------------------------------------------------------

def pack_bits(base: int, k: int, mode: int, u: int) -> int:
    return int(lib().orc_pack_bits(base, k, mode, u))


def unpack_code(base: int, k: int, q: int) -> int:
    return int(lib().orc_unpack_code(base, k, q))


# ---- array operations -------------------------------------------------------

def pack(src: np.ndarray, base: int, k: int, mode: int = RNE, n: int | None = None,
         inc_src: int = 1, inc_dst: int = 1, dst: np.ndarray | None = None) -> np.ndarray:
    """Pack native values (float32/float64 or their bit patterns) to a k-byte stream."""
    src = np.ascontiguousarray(src).view(native_dtype(base))
    if n is None:
        n = (src.size + inc_src - 1) // inc_src
    if dst is None:
        dst = np.zeros(max(n - 1, 0) * inc_dst * k + (k if n > 0 else 0), dtype=np.uint8)
    _check(lib().orc_pack(base, k, mode, _ptr(src), n, inc_src, _ptr(dst), inc_dst), "pack")
    return dst


def unpack(src: np.ndarray, base: int, k: int, n: int | None = None, inc_src: int = 1,
           inc_dst: int = 1, dst: np.ndarray | None = None) -> np.ndarray:
    """Unpack a k-byte stream to native bit patterns (uint32/uint64)."""
    src = np.ascontiguousarray(src, dtype=np.uint8)
    if n is None:
        n = src.size // (k * inc_src) + (1 if src.size % (k * inc_src) >= k else 0)
    if dst is None:
        dst = np.zeros(max(n - 1, 0) * inc_dst + (1 if n > 0 else 0), dtype=native_dtype(base))
    _check(lib().orc_unpack(base, k, _ptr(src), n, inc_src, _ptr(dst), inc_dst), "unpack")
    return dst


def values(src: np.ndarray, base: int, k: int) -> np.ndarray:
    """Unpacked values of a contiguous k-byte stream, widened exactly to float64."""
    return unpack(src, base, k).view(float_dtype(base)).astype(np.float64)


def dot(n: int, x: np.ndarray, fx: tuple[int, int], incx: int, y: np.ndarray,
        fy: tuple[int, int], incy: int) -> tuple[float, float, float]:
    """(Dot2 reference, naive FP64 sum, sum |x_i y_i|) of two flyte streams."""
    out = np.zeros(3, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.uint8)
    y = np.ascontiguousarray(y, dtype=np.uint8)
    _check(lib().orc_dot(n, _ptr(x), fx[0], fx[1], incx, _ptr(y), fy[0], fy[1], incy, _ptr(out)),
           "dot")
    return float(out[0]), float(out[1]), float(out[2])


def axpy(n: int, alpha: float, x: np.ndarray, fx: tuple[int, int], incx: int, y: np.ndarray,
         fy: tuple[int, int], incy: int, mode: int = RNE) -> np.ndarray:
    """Return a copy of stream y after y <- pack(fma(alpha, x, y))."""
    x = np.ascontiguousarray(x, dtype=np.uint8)
    y = np.array(y, dtype=np.uint8, copy=True)
    _check(lib().orc_axpy(n, alpha, _ptr(x), fx[0], fx[1], incx, _ptr(y), fy[0], fy[1], incy,
                          mode), "axpy")
    return y


def scal(n: int, alpha: float, x: np.ndarray, fx: tuple[int, int], incx: int = 1,
         mode: int = RNE) -> np.ndarray:
    """Return a copy of stream x after x <- pack(alpha * x)."""
    x = np.array(x, dtype=np.uint8, copy=True)
    _check(lib().orc_scal(n, alpha, _ptr(x), fx[0], fx[1], incx, mode), "scal")
    return x


def gemv(trans: str, m: int, n: int, alpha: float, A: np.ndarray, fa: tuple[int, int], lda: int,
         x: np.ndarray, incx: int, beta: float, y: np.ndarray, incy: int):
    """Return (y_out, absum): reference y and per-entry sum |A_ij x_j|."""
    A = np.ascontiguousarray(A, dtype=np.uint8)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.array(y, dtype=np.float64, copy=True)
    leny = m if trans == "N" else n
    absum = np.zeros(max(leny, 1), dtype=np.float64)
    _check(lib().orc_gemv(trans.encode(), m, n, alpha, _ptr(A), fa[0], fa[1], lda, _ptr(x), incx,
                          beta, _ptr(y), incy, _ptr(absum)), "gemv")
    return y, absum[:leny]


def refine_jacobi(n: int, A64: np.ndarray, Ak: np.ndarray, fa: tuple[int, int], b: np.ndarray, x0: np.ndarray,
                  tol: float, max_outer: int, inner: int):
    """Return (x, corrections, relres) of the refinement solve (A64: binary64 values, Ak: k-byte codes)."""
    A64 = np.ascontiguousarray(A64, dtype=np.float64).view(np.uint8)
    Ak = np.ascontiguousarray(Ak, dtype=np.uint8)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.array(x0, dtype=np.float64, copy=True)
    it = ctypes.c_int(0)
    rel = ctypes.c_double(0.0)
    _check(lib().orc_refine_jacobi(n, _ptr(A64), n, _ptr(Ak), fa[0], fa[1], n, _ptr(b), _ptr(x), tol,
                                   max_outer, inner, ctypes.byref(it), ctypes.byref(rel)), "refine_jacobi")
    return x, it.value, rel.value


def gemm_entries(rows: np.ndarray, cols: np.ndarray, kk: int, alpha: float, A: np.ndarray,
                 fa: tuple[int, int], lda: int, B: np.ndarray, fb: tuple[int, int], ldb: int,
                 beta: float = 0.0, cin: np.ndarray | None = None):
    """Reference entries C[rows[p], cols[p]] and their sum |A_il B_lj|."""
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    cols = np.ascontiguousarray(cols, dtype=np.int64)
    A = np.ascontiguousarray(A, dtype=np.uint8)
    B = np.ascontiguousarray(B, dtype=np.uint8)
    npairs = rows.size
    out = np.zeros(max(npairs, 1), dtype=np.float64)
    absum = np.zeros(max(npairs, 1), dtype=np.float64)
    cin_arr = None if cin is None else np.ascontiguousarray(cin, dtype=np.float64)
    _check(lib().orc_gemm_entries(npairs, _ptr(rows), _ptr(cols), kk, alpha, _ptr(A), fa[0], fa[1],
                                  lda, _ptr(B), fb[0], fb[1], ldb, beta, _ptr(cin_arr), _ptr(out),
                                  _ptr(absum)), "gemm")
    return out[:npairs], absum[:npairs]
