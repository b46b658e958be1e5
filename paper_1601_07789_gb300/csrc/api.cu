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
  (void)result_dev; (void)n; (void)x; (void)fx; (void)incx; (void)y; (void)fy; (void)incy;
  (void)ws; (void)ws_bytes; (void)stream;
  set_error("dot: not implemented yet");
  return FLYTE_ERR_UNSUPPORTED;
}

flyte_status flyte_axpy(int64_t n, double alpha, const void* x, flyte_fmt fx, int64_t incx, void* y,
                        flyte_fmt fy, int64_t incy, flyte_round mode, cudaStream_t stream) {
  g_error[0] = 0;
  (void)n; (void)alpha; (void)x; (void)fx; (void)incx; (void)y; (void)fy; (void)incy; (void)mode;
  (void)stream;
  set_error("axpy: not implemented yet");
  return FLYTE_ERR_UNSUPPORTED;
}

flyte_status flyte_gemv(char trans, int64_t m, int64_t n, double alpha, const void* A, flyte_fmt fa,
                        int64_t lda, const double* x, int64_t incx, double beta, double* y,
                        int64_t incy, void* ws, size_t ws_bytes, cudaStream_t stream) {
  g_error[0] = 0;
  (void)trans; (void)m; (void)n; (void)alpha; (void)A; (void)fa; (void)lda; (void)x; (void)incx;
  (void)beta; (void)y; (void)incy; (void)ws; (void)ws_bytes; (void)stream;
  set_error("gemv: not implemented yet");
  return FLYTE_ERR_UNSUPPORTED;
}

flyte_status flyte_gemm(int64_t m, int64_t n, int64_t k_, double alpha, const void* A, flyte_fmt fa,
                        int64_t lda, const void* B, flyte_fmt fb, int64_t ldb, double beta, void* C,
                        int64_t ldc, void* ws, size_t ws_bytes, cudaStream_t stream) {
  g_error[0] = 0;
  (void)m; (void)n; (void)k_; (void)alpha; (void)A; (void)fa; (void)lda; (void)B; (void)fb; (void)ldb;
  (void)beta; (void)C; (void)ldc; (void)ws; (void)ws_bytes; (void)stream;
  set_error("gemm: not implemented yet");
  return FLYTE_ERR_UNSUPPORTED;
}

size_t flyte_workspace_bytes(const char* op, int64_t m, int64_t n, int64_t k_, flyte_fmt f) {
  (void)m; (void)n; (void)k_; (void)f;
  if (!op) return size_t(-1);
  return size_t(-1);
}

}  // extern "C"
