"""Python binding of libflyte.so (ctypes).

Argument marshalling only: every step of the computation runs in the CUDA
kernels behind the C ABI declared in ``include/flyte.h``.  PyTorch supplies
device memory and the current stream.  There is no CPU fallback: if the
library is missing or a call fails, an exception is raised.

Formats are ``(k, base)`` pairs or ``Fmt`` values; base ``F32`` (0) or
``F64`` (1).  Rounding modes: ``"rne"``, ``"rtz"``, ``"half_up"``, ``"rto"``.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

F32, F64 = 0, 1
RNE, RTZ, HALF_UP, RTO = 0, 1, 2, 3
_MODES = {"rne": RNE, "rtz": RTZ, "half_up": HALF_UP, "half": HALF_UP, "rto": RTO}

STATUS = {0: "FLYTE_OK", 1: "FLYTE_ERR_INVALID_ARG", 2: "FLYTE_ERR_UNSUPPORTED",
          3: "FLYTE_ERR_ALIGNMENT", 4: "FLYTE_ERR_CUDA", 5: "FLYTE_ERR_WORKSPACE"}

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "libflyte.so")

# every entry point declared in include/flyte.h
EXPORTS = ("flyte_pack", "flyte_unpack", "flyte_dot", "flyte_axpy", "flyte_scal", "flyte_gemv",
           "flyte_gemv_packed_y", "flyte_gemv_static", "flyte_gemm", "flyte_gemm_packed_c",
           "flyte_refine_jacobi", "flyte_batch_prepare", "flyte_batch_workspace_bytes", "flyte_batch_launch",
           "flyte_batch_autotune", "flyte_batch_autotune_bytes", "flyte_batch_autotune_jobs",
           "flyte_batch_tile_size", "flyte_batch_resident_blocks", "flyte_workspace_bytes",
           "flyte_last_error_string", "flyte_version")


class FlyteError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class Fmt(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("base", ctypes.c_int32)]

    def __repr__(self):
        return f"Fmt(k={self.k}, base={'F32' if self.base == F32 else 'F64'})"


class Job(ctypes.Structure):
    """flyte_job: one job of a batch (see include/flyte.h)."""
    _fields_ = [("op", ctypes.c_int32), ("mode", ctypes.c_int32), ("fx", Fmt), ("fy", Fmt),
                ("m", ctypes.c_int64), ("n", ctypes.c_int64), ("a", ctypes.c_void_p), ("xv", ctypes.c_void_p),
                ("y", ctypes.c_void_p), ("result", ctypes.c_void_p), ("alpha", ctypes.c_double),
                ("beta", ctypes.c_double)]


JOB_UNPACK, JOB_DOT, JOB_AXPY, JOB_GEMV_N, JOB_GEMV_T = 0, 1, 2, 3, 4


def fmt(f) -> Fmt:
    if isinstance(f, Fmt):
        return f
    k, base = f
    return Fmt(int(k), int(base))


_lock = threading.Lock()
_lib = None


def lib() -> ctypes.CDLL:
    """Load libflyte.so (built by ``paper_1601_07789_gb300.build``); raise if absent."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libflyte.so is not built ({LIB_PATH}); run "
                                   "`python -m paper_1601_07789_gb300.build` first")
            L = ctypes.CDLL(LIB_PATH)
            i64, i32, vp, dbl, sz = (ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p,
                                     ctypes.c_double, ctypes.c_size_t)
            L.flyte_pack.argtypes = [vp, vp, i64, Fmt, i64, i64, i32, vp]
            L.flyte_unpack.argtypes = [vp, vp, i64, Fmt, i64, i64, vp]
            L.flyte_dot.argtypes = [vp, i64, vp, Fmt, i64, vp, Fmt, i64, vp, sz, vp]
            L.flyte_axpy.argtypes = [i64, dbl, vp, Fmt, i64, vp, Fmt, i64, i32, vp]
            L.flyte_scal.argtypes = [i64, dbl, vp, Fmt, i64, i32, vp]
            L.flyte_gemv_packed_y.argtypes = [ctypes.c_char, i64, i64, dbl, vp, Fmt, i64, vp, i64, dbl,
                                              vp, Fmt, i64, i32, vp, sz, vp]
            L.flyte_gemv.argtypes = [ctypes.c_char, i64, i64, dbl, vp, Fmt, i64, vp, i64, dbl, vp,
                                     i64, vp, sz, vp]
            L.flyte_gemv_static.argtypes = [ctypes.c_char, i64, i64, dbl, vp, Fmt, i64, vp, i64, dbl,
                                            vp, i64, vp]
            L.flyte_gemm.argtypes = [i64, i64, i64, dbl, vp, Fmt, i64, vp, Fmt, i64, dbl, vp, i64,
                                     vp, sz, vp]
            L.flyte_gemm_packed_c.argtypes = [i64, i64, i64, dbl, vp, Fmt, i64, vp, Fmt, i64, dbl, vp, Fmt,
                                              i64, i32, vp, sz, vp]
            L.flyte_refine_jacobi.argtypes = [i64, vp, i64, vp, Fmt, i64, vp, vp, dbl, i32, i32, vp, sz, vp,
                                              ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]
            L.flyte_batch_prepare.argtypes = [ctypes.POINTER(Job), i32, vp, sz, vp]
            L.flyte_batch_workspace_bytes.argtypes = [ctypes.POINTER(Job), i32]
            L.flyte_batch_workspace_bytes.restype = sz
            L.flyte_batch_launch.argtypes = [vp, vp]
            L.flyte_batch_autotune.argtypes = [vp, sz, vp]
            L.flyte_batch_autotune_bytes.argtypes = []
            L.flyte_batch_autotune_bytes.restype = sz
            L.flyte_batch_autotune_jobs.argtypes = [ctypes.POINTER(Job), i32, vp, sz, vp]
            L.flyte_batch_tile_size.argtypes = [i32, Fmt]
            L.flyte_batch_tile_size.restype = i64
            L.flyte_batch_resident_blocks.argtypes = []
            L.flyte_batch_resident_blocks.restype = i32
            for name in ("flyte_pack", "flyte_unpack", "flyte_dot", "flyte_axpy", "flyte_scal",
                         "flyte_gemv", "flyte_gemv_packed_y", "flyte_gemv_static", "flyte_gemm",
                         "flyte_gemm_packed_c", "flyte_refine_jacobi", "flyte_batch_prepare",
                         "flyte_batch_launch", "flyte_batch_autotune", "flyte_batch_autotune_jobs"):
                getattr(L, name).restype = i32
            L.flyte_workspace_bytes.argtypes = [ctypes.c_char_p, i64, i64, i64, Fmt]
            L.flyte_workspace_bytes.restype = sz
            L.flyte_last_error_string.argtypes = []
            L.flyte_last_error_string.restype = ctypes.c_char_p
            L.flyte_version.restype = ctypes.c_int
            _lib = L
    return _lib


def _check(status: int) -> None:
    if status != 0:
        msg = lib().flyte_last_error_string().decode(errors="replace")
        raise FlyteError(status, msg)


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _mode(mode) -> int:
    return _MODES[mode] if isinstance(mode, str) else int(mode)


def native_dtype(base: int) -> torch.dtype:
    return torch.float32 if base == F32 else torch.float64


# ---- raw entry points (pointers in, status checked) ---------------------------

def pack_raw(dst, src, n: int, f, inc_dst: int = 1, inc_src: int = 1, mode="rne", stream=None):
    _check(lib().flyte_pack(_ptr(dst), _ptr(src), n, fmt(f), inc_dst, inc_src, _mode(mode),
                            _stream(stream)))


def unpack_raw(dst, src, n: int, f, inc_dst: int = 1, inc_src: int = 1, stream=None):
    _check(lib().flyte_unpack(_ptr(dst), _ptr(src), n, fmt(f), inc_dst, inc_src, _stream(stream)))


def workspace_bytes(op: str, m: int, n: int, k: int, f) -> int:
    return int(lib().flyte_workspace_bytes(op.encode(), m, n, k, fmt(f)))


# ---- tensor conveniences ------------------------------------------------------

def pack(src: torch.Tensor, k: int, mode="rne", out: torch.Tensor | None = None,
         stream=None) -> torch.Tensor:
    """Pack a contiguous float32/float64 CUDA tensor to a uint8 stream of k bytes per element."""
    base = F32 if src.dtype == torch.float32 else F64
    assert src.dtype in (torch.float32, torch.float64) and src.is_cuda and src.is_contiguous()
    n = src.numel()
    if out is None:
        out = torch.empty(n * k, dtype=torch.uint8, device=src.device)
    pack_raw(out, src, n, (k, base), 1, 1, mode, stream)
    return out


def unpack(src: torch.Tensor, k: int, base: int, out: torch.Tensor | None = None,
           stream=None) -> torch.Tensor:
    """Unpack a contiguous uint8 CUDA stream of k-byte flytes to float32/float64."""
    assert src.dtype == torch.uint8 and src.is_cuda and src.is_contiguous()
    n = src.numel() // k
    if out is None:
        out = torch.empty(n, dtype=native_dtype(base), device=src.device)
    unpack_raw(out, src, n, (k, base), 1, 1, stream)
    return out


def dot_raw(result, n: int, x, fx, incx: int, y, fy, incy: int, ws, ws_bytes: int, stream=None):
    _check(lib().flyte_dot(_ptr(result), n, _ptr(x), fmt(fx), incx, _ptr(y), fmt(fy), incy,
                           _ptr(ws), ws_bytes, _stream(stream)))


def dot(x: torch.Tensor, fx, y: torch.Tensor, fy, n: int | None = None, incx: int = 1,
        incy: int = 1, out: torch.Tensor | None = None, ws: torch.Tensor | None = None,
        stream=None) -> torch.Tensor:
    """Device scalar (float64) sum_i x_i y_i of two flyte streams."""
    fx, fy = fmt(fx), fmt(fy)
    if n is None:
        n = (x.numel() // fx.k + incx - 1) // incx
    if out is None:
        out = torch.empty((), dtype=torch.float64, device=x.device)
    wsb = workspace_bytes("dot", 0, n, 0, fx)
    if ws is None:
        ws = torch.empty(max(wsb, 16), dtype=torch.uint8, device=x.device)
    dot_raw(out, n, x, fx, incx, y, fy, incy, ws, ws.numel(), stream)
    return out


def axpy(alpha: float, x: torch.Tensor, fx, y: torch.Tensor, fy, n: int | None = None,
         incx: int = 1, incy: int = 1, mode="rne", stream=None) -> torch.Tensor:
    """In place: y <- pack(fma(alpha, x, y)) on flyte streams; returns y."""
    fx, fy = fmt(fx), fmt(fy)
    if n is None:
        n = (y.numel() // fy.k + incy - 1) // incy
    _check(lib().flyte_axpy(n, float(alpha), _ptr(x), fx, incx, _ptr(y), fy, incy, _mode(mode),
                            _stream(stream)))
    return y


def scal(alpha: float, x: torch.Tensor, fx, n: int | None = None, incx: int = 1, mode="rne",
         stream=None) -> torch.Tensor:
    """In place: x <- pack(alpha * x) on a flyte stream; returns x."""
    fx = fmt(fx)
    if n is None:
        n = (x.numel() // fx.k + incx - 1) // incx
    _check(lib().flyte_scal(n, float(alpha), _ptr(x), fx, incx, _mode(mode), _stream(stream)))
    return x


def gemv_raw(trans: str, m: int, n: int, alpha: float, A, fa, lda: int, x, incx: int,
             beta: float, y, incy: int, ws, ws_bytes: int, stream=None):
    _check(lib().flyte_gemv(trans.encode(), m, n, float(alpha), _ptr(A), fmt(fa), lda, _ptr(x),
                            incx, float(beta), _ptr(y), incy, _ptr(ws), ws_bytes, _stream(stream)))


def gemv(trans: str, m: int, n: int, alpha: float, A: torch.Tensor, fa, lda: int,
         x: torch.Tensor, beta: float, y: torch.Tensor, incx: int = 1, incy: int = 1,
         ws: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """y <- alpha op(A) x + beta y with A a row-major k-byte matrix; returns y."""
    fa = fmt(fa)
    op = "gemv_n" if trans in ("N", "n") else "gemv_t"
    wsb = workspace_bytes(op, m, n, 0, fa)
    if ws is None:
        ws = torch.empty(max(wsb, 16), dtype=torch.uint8, device=A.device)
    gemv_raw(trans.upper(), m, n, alpha, A, fa, lda, x, incx, beta, y, incy, ws, ws.numel(), stream)
    return y


def gemv_packed_y_raw(trans: str, m: int, n: int, alpha: float, A, fa, lda: int, x, incx: int,
                      beta: float, y, fy, incy: int, mode, ws, ws_bytes: int, stream=None):
    """gemv whose y is a stream of double-based flytes of format fy (packed in the epilogue)."""
    _check(lib().flyte_gemv_packed_y(trans.encode(), m, n, float(alpha), _ptr(A), fmt(fa), lda, _ptr(x),
                                     incx, float(beta), _ptr(y), fmt(fy), incy, _mode(mode), _ptr(ws),
                                     ws_bytes, _stream(stream)))


def gemv_static_raw(trans: str, m: int, n: int, alpha: float, A, fa, lda: int, x, incx: int,
                    beta: float, y, incy: int, stream=None):
    """gemv with the library's built-in scratch (no workspace; see flyte_gemv_static)."""
    _check(lib().flyte_gemv_static(trans.encode(), m, n, float(alpha), _ptr(A), fmt(fa), lda, _ptr(x),
                                   incx, float(beta), _ptr(y), incy, _stream(stream)))


def gemm_raw(m: int, n: int, k: int, alpha: float, A, fa, lda: int, B, fb, ldb: int, beta: float,
             C, ldc: int, ws, ws_bytes: int, stream=None):
    _check(lib().flyte_gemm(m, n, k, float(alpha), _ptr(A), fmt(fa), lda, _ptr(B), fmt(fb), ldb,
                            float(beta), _ptr(C), ldc, _ptr(ws), ws_bytes, _stream(stream)))


def gemm_packed_c_raw(m: int, n: int, k: int, alpha: float, A, fa, lda: int, B, fb, ldb: int, beta: float,
                      C, fc, ldc: int, mode, ws, ws_bytes: int, stream=None):
    """gemm whose C is a stream of flytes of format fc (packed in the epilogue)."""
    _check(lib().flyte_gemm_packed_c(m, n, k, float(alpha), _ptr(A), fmt(fa), lda, _ptr(B), fmt(fb), ldb,
                                     float(beta), _ptr(C), fmt(fc), ldc, _mode(mode), _ptr(ws), ws_bytes,
                                     _stream(stream)))


def gemm(m: int, n: int, k: int, A: torch.Tensor, fa, B: torch.Tensor, fb,
         C: torch.Tensor | None = None, alpha: float = 1.0, beta: float = 0.0,
         lda: int | None = None, ldb: int | None = None, ldc: int | None = None,
         ws: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """C <- alpha A B + beta C on row-major k-byte A (m x k) and B (k x n); returns C."""
    fa, fb = fmt(fa), fmt(fb)
    lda = k if lda is None else lda
    ldb = n if ldb is None else ldb
    ldc = n if ldc is None else ldc
    if C is None:
        C = torch.zeros(m * ldc, dtype=native_dtype(fa.base), device=A.device)
    wsb = workspace_bytes("gemm", m, n, k, fa)
    if ws is None:
        ws = torch.empty(max(wsb, 16), dtype=torch.uint8, device=A.device)
    gemm_raw(m, n, k, alpha, A, fa, lda, B, fb, ldb, beta, C, ldc, ws, ws.numel(), stream)
    return C


def refine_jacobi(A64: torch.Tensor, Ak: torch.Tensor, fa, b: torch.Tensor, x: torch.Tensor, tol: float = 1e-12,
                  max_outer: int = 50, inner: int = 2, lda64: int | None = None, lda: int | None = None,
                  ws: torch.Tensor | None = None, stream=None) -> tuple[int, float]:
    """Iterative refinement of A x = b in place on x (binary64 residual on A64, Jacobi sweeps on the
    k-byte copy Ak); returns (corrections applied, final relative residual).  Synchronous."""
    n = b.numel()
    fa = fmt(fa)
    lda64 = n if lda64 is None else lda64
    lda = n if lda is None else lda
    if ws is None:
        ws = torch.empty(workspace_bytes("refine", n, n, 0, fa), dtype=torch.uint8, device=b.device)
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    _check(lib().flyte_refine_jacobi(n, _ptr(A64), lda64, _ptr(Ak), fa, lda, _ptr(b), _ptr(x), float(tol),
                                     int(max_outer), int(inner), _ptr(ws), ws.numel(), _stream(stream),
                                     ctypes.byref(it), ctypes.byref(rr)))
    return it.value, rr.value


def job(op: int, fx, n: int, a, y, *, fy=None, m: int = 0, xv=None, result=None, alpha: float = 0.0,
        beta: float = 0.0, mode="rne") -> Job:
    """A flyte_job from tensors or pointers."""
    return Job(op, _mode(mode), fmt(fx), fmt(fy if fy is not None else fx), m, n, _ptr(a), _ptr(xv), _ptr(y),
               _ptr(result), float(alpha), float(beta))


def batch_prepare(jobs, ws: torch.Tensor | None = None, device=None, stream=None) -> torch.Tensor:
    """Plan a batch and upload its tables; returns the workspace to pass to batch_launch."""
    arr = (Job * len(jobs))(*jobs)
    nbytes = lib().flyte_batch_workspace_bytes(arr, len(jobs))
    if nbytes == ctypes.c_size_t(-1).value:
        _check(lib().flyte_batch_prepare(arr, len(jobs), None, 0, _stream(stream)))
    if ws is None or ws.numel() < nbytes:
        ws = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device or "cuda")
    _check(lib().flyte_batch_prepare(arr, len(jobs), _ptr(ws), ws.numel(), _stream(stream)))
    return ws


def batch_launch(ws: torch.Tensor, stream=None) -> None:
    """Run a prepared batch (one persistent kernel; capturable in a CUDA graph)."""
    _check(lib().flyte_batch_launch(_ptr(ws), _stream(stream)))


def batch_autotune_jobs(jobs, ws: torch.Tensor | None = None, device=None, stream=None) -> None:
    """Tune the tile table and the resident blocks per SM on this batch of jobs (see
    flyte_batch_autotune_jobs: in-place outputs such as axpy y are changed)."""
    arr = (Job * len(jobs))(*jobs)
    nbytes = 0
    # the tables of the smallest tiles tried take at most about 4x the current ones; candidates
    # that do not fit are skipped
    cur = lib().flyte_batch_workspace_bytes(arr, len(jobs))
    if cur != ctypes.c_size_t(-1).value:
        nbytes = 16 * cur + (1 << 20)
    if ws is None or ws.numel() < nbytes:
        ws = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device or "cuda")
    _check(lib().flyte_batch_autotune_jobs(arr, len(jobs), _ptr(ws), ws.numel(), _stream(stream)))


def batch_tile_size(op: int, f) -> int:
    return int(lib().flyte_batch_tile_size(op, fmt(f)))


def batch_resident_blocks() -> int:
    return int(lib().flyte_batch_resident_blocks())


def batch_autotune(device=None, stream=None) -> None:
    """Measure the tile-size candidates of every (operation, k, base) and keep the fastest."""
    nbytes = lib().flyte_batch_autotune_bytes()
    ws = torch.empty(nbytes, dtype=torch.uint8, device=device or "cuda")
    _check(lib().flyte_batch_autotune(_ptr(ws), nbytes, _stream(stream)))
