// api.cu -- the extern "C" entry points of libflyte.so: argument checks,
// quick returns, error strings and dispatch to the kernel launchers.
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "flyte_internal.cuh"

namespace flyte {

namespace {
thread_local char g_error[512] = "";

flyte_status invalid(const char* what) {
  set_error("invalid argument: %s", what);
  return FLYTE_ERR_INVALID_ARG;
}
}  // namespace

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_error, sizeof(g_error), fmt, ap);
  va_end(ap);
}

flyte_status cuda_status(cudaError_t e, const char* what) {
  set_error("%s: CUDA error %d (%s)", what, int(e), cudaGetErrorString(e));
  return FLYTE_ERR_CUDA;
}

flyte_status check_gemv_args(char trans, int64_t m, int64_t n, double alpha, const void* A, flyte_fmt fa,
                             int64_t lda, const double* x, int64_t incx, const void* y, int64_t incy) {
  if (trans != 'N' && trans != 'T' && trans != 'n' && trans != 't') return invalid("trans must be 'N' or 'T'");
  if (!valid_fmt(fa)) return invalid("format (k, base)");
  if (m < 0 || n < 0) return invalid("m < 0 or n < 0");
  if (lda < (n > 1 ? n : 1)) return invalid("lda < max(1, n)");
  if (incx < 1 || incy < 1) return invalid("stride < 1");
  if (m == 0 || n == 0) return FLYTE_OK;
  if (!y) return invalid("null y");
  if (alpha != 0.0 && (!A || !x)) return invalid("null A or x");
  return FLYTE_OK;
}

int sm_count() {
  static thread_local int cached_dev = -1, cached = 0;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (dev != cached_dev) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 1;
    cached = v;
    cached_dev = dev;
  }
  return cached;
}

}  // namespace flyte

using namespace flyte;

extern "C" {

int flyte_version(void) { return 100; }

const char* flyte_last_error_string(void) { return g_error; }

flyte_status flyte_pack(void* dst, const void* src, int64_t n, flyte_fmt f, int64_t inc_dst,
                        int64_t inc_src, flyte_round mode, cudaStream_t stream) {
  g_error[0] = 0;
  if (!valid_fmt(f)) return invalid("format (k, base)");
  if (int(mode) < FLYTE_RNE || int(mode) > FLYTE_RTO) return invalid("rounding mode");
  if (n < 0) return invalid("n < 0");
  if (inc_dst < 1 || inc_src < 1) return invalid("stride < 1");
  if (n == 0) return FLYTE_OK;
  if (!dst || !src) return invalid("null pointer");
  return launch_pack(dst, src, n, f, inc_dst, inc_src, int(mode), stream);
}

flyte_status flyte_unpack(void* dst, const void* src, int64_t n, flyte_fmt f, int64_t inc_dst,
                          int64_t inc_src, cudaStream_t stream) {
  g_error[0] = 0;
  if (!valid_fmt(f)) return invalid("format (k, base)");
  if (n < 0) return invalid("n < 0");
  if (inc_dst < 1 || inc_src < 1) return invalid("stride < 1");
  if (n == 0) return FLYTE_OK;
  if (!dst || !src) return invalid("null pointer");
  return launch_unpack(dst, src, n, f, inc_dst, inc_src, stream);
}

flyte_status flyte_dot(double* result_dev, int64_t n, const void* x, flyte_fmt fx, int64_t incx,
                       const void* y, flyte_fmt fy, int64_t incy, void* ws, size_t ws_bytes,
                       cudaStream_t stream) {
  g_error[0] = 0;
  if (!valid_fmt(fx) || !valid_fmt(fy)) return invalid("format (k, base)");
  if (n < 0) return invalid("n < 0");
  if (incx < 1 || incy < 1) return invalid("stride < 1");
  if (!result_dev) return invalid("null result");
  if (n > 0 && (!x || !y)) return invalid("null x or y");
  return launch_dot(result_dev, n, x, fx, incx, y, fy, incy, ws, ws_bytes, stream);
}

flyte_status flyte_axpy(int64_t n, double alpha, const void* x, flyte_fmt fx, int64_t incx, void* y,
                        flyte_fmt fy, int64_t incy, flyte_round mode, cudaStream_t stream) {
  g_error[0] = 0;
  if (!valid_fmt(fx) || !valid_fmt(fy)) return invalid("format (k, base)");
  if (fx.base != fy.base) {
    set_error("axpy: x and y must share the base type");
    return FLYTE_ERR_UNSUPPORTED;
  }
  if (int(mode) < FLYTE_RNE || int(mode) > FLYTE_RTO) return invalid("rounding mode");
  if (n < 0) return invalid("n < 0");
  if (incx < 1 || incy < 1) return invalid("stride < 1");
  if (n == 0) return FLYTE_OK;
  if (!x || !y) return invalid("null pointer");
  return launch_axpy(n, alpha, x, fx, incx, y, fy, incy, int(mode), stream);
}

flyte_status flyte_scal(int64_t n, double alpha, void* x, flyte_fmt fx, int64_t incx, flyte_round mode,
                        cudaStream_t stream) {
  g_error[0] = 0;
  if (!valid_fmt(fx)) return invalid("format (k, base)");
  if (int(mode) < FLYTE_RNE || int(mode) > FLYTE_RTO) return invalid("rounding mode");
  if (n < 0) return invalid("n < 0");
  if (incx < 1) return invalid("stride < 1");
  if (n == 0) return FLYTE_OK;
  if (!x) return invalid("null pointer");
  return launch_scal(n, alpha, x, fx, incx, int(mode), stream);
}

flyte_status flyte_gemv(char trans, int64_t m, int64_t n, double alpha, const void* A, flyte_fmt fa,
                        int64_t lda, const double* x, int64_t incx, double beta, double* y,
                        int64_t incy, void* ws, size_t ws_bytes, cudaStream_t stream) {
  g_error[0] = 0;
  const flyte_status st = check_gemv_args(trans, m, n, alpha, A, fa, lda, x, incx, y, incy);
  if (st != FLYTE_OK || m == 0 || n == 0) return st;
  trans = (trans == 'n' || trans == 'N') ? 'N' : 'T';
  return launch_gemv(trans, m, n, alpha, A, fa, lda, x, incx, beta, y, 0, incy, 0, ws, ws_bytes, stream);
}

flyte_status flyte_gemv_packed_y(char trans, int64_t m, int64_t n, double alpha, const void* A, flyte_fmt fa,
                                 int64_t lda, const double* x, int64_t incx, double beta, void* y, flyte_fmt fy,
                                 int64_t incy, flyte_round mode, void* ws, size_t ws_bytes, cudaStream_t stream) {
  g_error[0] = 0;
  if (trans == 'n') trans = 'N';
  if (trans == 't') trans = 'T';
  if (trans != 'N' && trans != 'T') return invalid("trans must be 'N' or 'T'");
  if (!valid_fmt(fa) || !valid_fmt(fy)) return invalid("format (k, base)");
  if (fy.base != FLYTE_F64) {
    set_error("gemv_packed_y: y must be double-based (the sums are binary64)");
    return FLYTE_ERR_UNSUPPORTED;
  }
  if (int(mode) < FLYTE_RNE || int(mode) > FLYTE_RTO) return invalid("rounding mode");
  if (m < 0 || n < 0) return invalid("m < 0 or n < 0");
  if (lda < (n > 1 ? n : 1)) return invalid("lda < max(1, n)");
  if (incx < 1 || incy < 1) return invalid("stride < 1");
  if (m == 0 || n == 0) return FLYTE_OK;
  if (!y) return invalid("null y");
  if (alpha != 0.0 && (!A || !x)) return invalid("null A or x");
  if (fy.k == 8 && reinterpret_cast<uintptr_t>(y) % 8 == 0)   // an aligned binary64 y
    return launch_gemv(trans, m, n, alpha, A, fa, lda, x, incx, beta, y, 0, incy, 0, ws, ws_bytes, stream);
  return launch_gemv(trans, m, n, alpha, A, fa, lda, x, incx, beta, y, fy.k, incy, int(mode), ws, ws_bytes,
                     stream);
}

flyte_status flyte_gemm(int64_t m, int64_t n, int64_t k_, double alpha, const void* A, flyte_fmt fa,
                        int64_t lda, const void* B, flyte_fmt fb, int64_t ldb, double beta, void* C,
                        int64_t ldc, void* ws, size_t ws_bytes, cudaStream_t stream) {
  g_error[0] = 0;
  if (!valid_fmt(fa) || !valid_fmt(fb)) return invalid("format (k, base)");
  if (fa.k != fb.k || fa.base != fb.base) {
    set_error("gemm: A and B must have the same format");
    return FLYTE_ERR_UNSUPPORTED;
  }
  if (m < 0 || n < 0 || k_ < 0) return invalid("m, n or k < 0");
  if (lda < (k_ > 1 ? k_ : 1) || ldb < (n > 1 ? n : 1) || ldc < (n > 1 ? n : 1)) return invalid("leading dimension");
  if (m == 0 || n == 0) return FLYTE_OK;
  if (!C) return invalid("null C");
  if (alpha != 0.0 && k_ > 0 && (!A || !B)) return invalid("null A or B");
  if (m > INT32_MAX / 2 || n > INT32_MAX / 2 || k_ > INT32_MAX / 2) {
    set_error("gemm: dimensions beyond 2^30 are not supported");
    return FLYTE_ERR_UNSUPPORTED;
  }
  return launch_gemm(m, n, k_, alpha, A, fa, lda, B, ldb, beta, C, 0, ldc, 0, ws, ws_bytes, stream);
}

flyte_status flyte_gemm_packed_c(int64_t m, int64_t n, int64_t k_, double alpha, const void* A, flyte_fmt fa,
                                 int64_t lda, const void* B, flyte_fmt fb, int64_t ldb, double beta, void* C,
                                 flyte_fmt fc, int64_t ldc, flyte_round mode, void* ws, size_t ws_bytes,
                                 cudaStream_t stream) {
  g_error[0] = 0;
  if (!valid_fmt(fa) || !valid_fmt(fb) || !valid_fmt(fc)) return invalid("format (k, base)");
  if (fa.k != fb.k || fa.base != fb.base) {
    set_error("gemm: A and B must have the same format");
    return FLYTE_ERR_UNSUPPORTED;
  }
  if (fc.base != fa.base) {
    set_error("gemm_packed_c: C must have the base of A and B");
    return FLYTE_ERR_UNSUPPORTED;
  }
  if (int(mode) < FLYTE_RNE || int(mode) > FLYTE_RTO) return invalid("rounding mode");
  if (m < 0 || n < 0 || k_ < 0) return invalid("m, n or k < 0");
  if (lda < (k_ > 1 ? k_ : 1) || ldb < (n > 1 ? n : 1) || ldc < (n > 1 ? n : 1)) return invalid("leading dimension");
  if (m == 0 || n == 0) return FLYTE_OK;
  if (!C) return invalid("null C");
  if (alpha != 0.0 && k_ > 0 && (!A || !B)) return invalid("null A or B");
  if (m > INT32_MAX / 2 || n > INT32_MAX / 2 || k_ > INT32_MAX / 2) {
    set_error("gemm: dimensions beyond 2^30 are not supported");
    return FLYTE_ERR_UNSUPPORTED;
  }
  const int native = fc.base == FLYTE_F64 ? 8 : 4;
  const int align = fc.base == FLYTE_F64 ? 8 : 4;
  const int kc = (fc.k == native && reinterpret_cast<uintptr_t>(C) % align == 0) ? 0 : fc.k;   // 0: the native C
  return launch_gemm(m, n, k_, alpha, A, fa, lda, B, ldb, beta, C, kc, ldc, int(mode), ws, ws_bytes, stream);
}

flyte_status flyte_refine_jacobi(int64_t n, const double* A64, int64_t lda64, const void* Ak, flyte_fmt fa,
                                 int64_t lda, const double* b, double* x, double tol, int max_outer, int inner,
                                 void* ws, size_t ws_bytes, cudaStream_t stream, int* iters, double* relres) {
  g_error[0] = 0;
  if (!valid_fmt(fa)) return invalid("format (k, base)");
  if (n < 0) return invalid("n < 0");
  if (lda64 < (n > 1 ? n : 1) || lda < (n > 1 ? n : 1)) return invalid("leading dimension");
  if (max_outer < 0 || inner < 1) return invalid("max_outer < 0 or inner < 1");
  if (!(tol >= 0.0)) return invalid("tol");
  if (n == 0) {
    if (iters) *iters = 0;
    if (relres) *relres = 0.0;
    return FLYTE_OK;
  }
  if (!A64 || !Ak || !b || !x) return invalid("null pointer");
  return launch_refine(n, A64, lda64, Ak, fa, lda, b, x, tol, max_outer, inner, ws, ws_bytes, stream, iters,
                       relres);
}

flyte_status flyte_batch_prepare(const flyte_job* jobs, int32_t njobs, void* ws, size_t ws_bytes,
                                 cudaStream_t stream) {
  g_error[0] = 0;
  return batch_prepare(jobs, njobs, ws, ws_bytes, stream);
}

size_t flyte_batch_workspace_bytes(const flyte_job* jobs, int32_t njobs) {
  g_error[0] = 0;
  return batch_workspace_bytes(jobs, njobs);
}

flyte_status flyte_batch_launch(void* ws, cudaStream_t stream) {
  g_error[0] = 0;
  return batch_launch(ws, stream);
}

flyte_status flyte_batch_autotune(void* ws, size_t ws_bytes, cudaStream_t stream) {
  g_error[0] = 0;
  return batch_autotune(ws, ws_bytes, stream);
}

size_t flyte_batch_autotune_bytes(void) { return batch_autotune_bytes(); }

flyte_status flyte_batch_autotune_jobs(const flyte_job* jobs, int32_t njobs, void* ws, size_t ws_bytes,
                                       cudaStream_t stream) {
  g_error[0] = 0;
  if (njobs < 0 || (njobs > 0 && jobs == nullptr)) return invalid("jobs");
  if (ws == nullptr || reinterpret_cast<uintptr_t>(ws) % 256 != 0) {
    set_error("batch autotune: a 256-byte aligned workspace is required");
    return FLYTE_ERR_WORKSPACE;
  }
  return batch_autotune_jobs(jobs, njobs, ws, ws_bytes, stream);
}

int64_t flyte_batch_tile_size(int32_t op, flyte_fmt f) { return batch_tile_size(op, f); }

int32_t flyte_batch_resident_blocks(void) { return batch_resident_blocks(); }

size_t flyte_workspace_bytes(const char* op, int64_t m, int64_t n, int64_t k_, flyte_fmt f) {
  (void)k_;
  if (!op || m < 0 || n < 0 || k_ < 0) return size_t(-1);
  if (std::strcmp(op, "dot") == 0) return dot_workspace_bytes(n);
  if (std::strcmp(op, "gemm") == 0) return gemm_workspace_bytes(m, n, k_, f);
  if (std::strcmp(op, "gemv_n") == 0) return gemv_workspace_bytes('N', m, n, f);
  if (std::strcmp(op, "gemv_t") == 0) return gemv_workspace_bytes('T', m, n, f);
  if (std::strcmp(op, "refine") == 0) return refine_workspace_bytes(n);
  return size_t(-1);
}

}  // extern "C"
