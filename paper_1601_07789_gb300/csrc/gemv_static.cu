// gemv_static.cu -- flyte_gemv_static: gemv without a caller-provided workspace.
//
// flyte_gemv needs a few hundred KiB of device scratch (the binary32 split of
// x and, for 'T', the per-tile column sums) and expects the caller to
// allocate it.  Some callers cannot: a plug-in or callback running inside a
// framework that owns every device allocation and hands out no raw memory,
// or a serving loop that must not call cudaMalloc after start-up (cudaMalloc
// can synchronise the device and stall other streams).  This entry point
// takes its scratch from a fixed array compiled into the library instead, so
// it allocates nothing: every GPU that loads the library holds the array
// until the process exits.
//
// Contract (also stated in include/flyte.h):
//  * the scratch is kFlyteStaticScratchBytes (4 MiB); a call whose
//    flyte_workspace_bytes("gemv_n"/"gemv_t", m, n, 0, fa) exceeds it is
//    rejected with FLYTE_ERR_WORKSPACE before anything is launched;
//  * the first call on a device looks up the array's device address with
//    cudaGetSymbolAddress while that device is current; make that first call
//    before capturing a stream into a CUDA graph;
//  * all calls share the one array and it keeps the last call's contents;
//    nothing in it has to start at zero (every byte a call reads, that call
//    wrote first), but two calls whose kernels overlap on the GPU (different
//    streams, or different host threads) race on it and give wrong results.
#include <mutex>

#include "flyte_internal.cuh"

namespace {

constexpr size_t kFlyteStaticScratchBytes = size_t(4) << 20;
constexpr int kMaxDevices = 64;

// Host code may only use this symbol's name as a handle for
// cudaGetSymbolAddress; its device address comes from that call.
static __device__ __align__(256) unsigned char g_gemv_scratch[kFlyteStaticScratchBytes];

std::mutex g_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

flyte_status scratch_for_current_device(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return flyte::cuda_status(e, "gemv_static: cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) {
    flyte::set_error("gemv_static: device index %d out of range", dev);
    return FLYTE_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_mutex);
  if (g_scratch_ptr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_gemv_scratch);
    if (e != cudaSuccess || p == nullptr) {
      return flyte::cuda_status(e != cudaSuccess ? e : cudaErrorInvalidSymbol,
                                "gemv_static: cudaGetSymbolAddress");
    }
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return FLYTE_OK;
}

}  // namespace

extern "C" flyte_status flyte_gemv_static(char trans, int64_t m, int64_t n, double alpha, const void* A,
                                          flyte_fmt fa, int64_t lda, const double* x, int64_t incx,
                                          double beta, double* y, int64_t incy, cudaStream_t stream) {
  // the checks of flyte_gemv come first, so that a bad argument is reported
  // as such whatever the size of the call
  flyte::set_error("%s", "");
  const flyte_status valid = flyte::check_gemv_args(trans, m, n, alpha, A, fa, lda, x, incx, y, incy);
  if (valid != FLYTE_OK) return valid;
  if (m == 0 || n == 0 || alpha == 0.0) {
    // quick returns need no scratch: flyte_gemv handles them
    return flyte_gemv(trans, m, n, alpha, A, fa, lda, x, incx, beta, y, incy, nullptr, 0, stream);
  }
  const char* op = (trans == 'N' || trans == 'n') ? "gemv_n" : "gemv_t";
  const size_t need = flyte_workspace_bytes(op, m, n, 0, fa);
  if (need > kFlyteStaticScratchBytes) {
    flyte::set_error("gemv_static: this call needs %zu bytes of scratch but the built-in scratch holds %zu; "
                     "use flyte_gemv with a caller workspace", need, kFlyteStaticScratchBytes);
    return FLYTE_ERR_WORKSPACE;
  }
  void* ws = nullptr;
  const flyte_status st = scratch_for_current_device(&ws);
  if (st != FLYTE_OK) return st;
  return flyte_gemv(trans, m, n, alpha, A, fa, lda, x, incx, beta, y, incy, ws, kFlyteStaticScratchBytes, stream);
}
