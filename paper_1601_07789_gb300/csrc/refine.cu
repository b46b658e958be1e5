// refine.cu -- mixed-precision iterative refinement with k-byte matrix storage.
//
// The paper's case for flytes is storing values with only the precision an
// algorithm needs (Sec. 1-2).  Iterative refinement is the classic such
// algorithm: the correction equations may be solved with a less precise copy
// of A as long as the residual is formed in full precision.  Here
//
//   repeat:  r = b - A64 x                         binary64 A (k = 8 flyte gemv)
//            stop when ||r||_2 <= tol ||b||_2
//            d = 0;  repeat `inner` times:
//                d <- d + D^-1 (r - Ak d)           Jacobi-Richardson sweep on the
//                                                  k-byte copy Ak (flyte_gemv)
//            x <- x + d
//
// with D = diag(A64).  Every product is flyte_gemv, the norms are flyte_dot
// on the binary64 vectors (as k = 8 streams), and the updates are the small
// kernels below; the host only sequences the launches and reads one norm per
// outer iteration (the only synchronisation).  Jacobi needs a diagonally
// dominant A; the solver does not check that, it reports the residual it
// reached.
#include <cmath>
#include <cstring>

#include "flyte_internal.cuh"

namespace flyte {
namespace {

constexpr int kThreads = 256;

__global__ void get_diag_inv(const double* __restrict__ A, int64_t lda, int64_t n, double* __restrict__ dinv) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) dinv[i] = 1.0 / A[i * lda + i];
}

// d <- d + dinv .* t
__global__ void jacobi_step(double* __restrict__ d, const double* __restrict__ t, const double* __restrict__ dinv,
                            int64_t n) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride)
    d[i] = fma(dinv[i], t[i], d[i]);
}

// x <- x + d
__global__ void add_to(double* __restrict__ x, const double* __restrict__ d, int64_t n) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) x[i] += d[i];
}

struct RefinePlan {
  int64_t off_r, off_t, off_d, off_dinv, off_norm, off_dot, off_gemv, bytes;
};

int64_t up256(int64_t b) { return (b + 255) & ~int64_t(255); }

RefinePlan plan_refine(int64_t n) {
  RefinePlan p{};
  const int64_t v = up256(8 * n);
  p.off_r = 0;
  p.off_t = p.off_r + v;
  p.off_d = p.off_t + v;
  p.off_dinv = p.off_d + v;
  p.off_norm = p.off_dinv + v;                          // two doubles: ||b||^2, ||r||^2
  p.off_dot = p.off_norm + 256;
  p.off_gemv = p.off_dot + up256(int64_t(dot_workspace_bytes(n)));
  p.bytes = p.off_gemv + up256(int64_t(gemv_workspace_bytes('N', n, n, flyte_fmt{8, FLYTE_F64})));
  return p;
}

}  // namespace

size_t refine_workspace_bytes(int64_t n) { return size_t(plan_refine(n).bytes); }

flyte_status launch_refine(int64_t n, const double* A64, int64_t lda64, const void* Ak, flyte_fmt fa, int64_t lda,
                           const double* b, double* x, double tol, int max_outer, int inner, void* ws,
                           size_t ws_bytes, cudaStream_t s, int* iters_out, double* relres_out) {
  const RefinePlan p = plan_refine(n);
  if (ws == nullptr || ws_bytes < size_t(p.bytes) || reinterpret_cast<uintptr_t>(ws) % 256 != 0) {
    set_error("refine: workspace of %lld bytes (256-byte aligned) required", (long long)p.bytes);
    return FLYTE_ERR_WORKSPACE;
  }
  uint8_t* w8 = static_cast<uint8_t*>(ws);
  double* r = reinterpret_cast<double*>(w8 + p.off_r);
  double* t = reinterpret_cast<double*>(w8 + p.off_t);
  double* d = reinterpret_cast<double*>(w8 + p.off_d);
  double* dinv = reinterpret_cast<double*>(w8 + p.off_dinv);
  double* norm = reinterpret_cast<double*>(w8 + p.off_norm);
  void* wdot = w8 + p.off_dot;
  void* wgemv = w8 + p.off_gemv;
  const size_t dot_bytes = dot_workspace_bytes(n);
  const size_t gemv_bytes = gemv_workspace_bytes('N', n, n, flyte_fmt{8, FLYTE_F64});
  const flyte_fmt f64{8, FLYTE_F64};
  const unsigned grid = grid_for(n, kThreads);
  flyte_status st;

  get_diag_inv<<<grid, kThreads, 0, s>>>(A64, lda64, n, dinv);
  FLYTE_TRY_LAUNCH("refine");
  if ((st = launch_dot(norm, n, b, f64, 1, b, f64, 1, wdot, dot_bytes, s)) != FLYTE_OK) return st;
  double bb = 0.0;
  if (cudaMemcpyAsync(&bb, norm, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return cuda_status(cudaGetLastError(), "refine");
  const double bnorm = std::sqrt(bb);

  int it = 0;
  double relres = INFINITY;
  for (;; ++it) {
    // r = b - A64 x
    if (cudaMemcpyAsync(r, b, size_t(8 * n), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return cuda_status(cudaGetLastError(), "refine");
    if ((st = launch_gemv('N', n, n, -1.0, A64, f64, lda64, x, 1, 1.0, r, 0, 1, 0, wgemv, gemv_bytes, s)) != FLYTE_OK)
      return st;
    if ((st = launch_dot(norm + 1, n, r, f64, 1, r, f64, 1, wdot, dot_bytes, s)) != FLYTE_OK) return st;
    double rr = 0.0;
    if (cudaMemcpyAsync(&rr, norm + 1, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return cuda_status(cudaGetLastError(), "refine");
    relres = bnorm > 0.0 ? std::sqrt(rr) / bnorm : std::sqrt(rr);
    if (!(relres > tol) || it >= max_outer) break;
    // d ~ A^-1 r by Jacobi-Richardson sweeps on the k-byte copy
    if (cudaMemsetAsync(d, 0, size_t(8 * n), s) != cudaSuccess) return cuda_status(cudaGetLastError(), "refine");
    for (int j = 0; j < inner; ++j) {
      if (cudaMemcpyAsync(t, r, size_t(8 * n), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return cuda_status(cudaGetLastError(), "refine");
      if (j > 0 && (st = launch_gemv('N', n, n, -1.0, Ak, fa, lda, d, 1, 1.0, t, 0, 1, 0, wgemv, gemv_bytes, s)) !=
                       FLYTE_OK)
        return st;
      jacobi_step<<<grid, kThreads, 0, s>>>(d, t, dinv, n);
      FLYTE_TRY_LAUNCH("refine");
    }
    add_to<<<grid, kThreads, 0, s>>>(x, d, n);
    FLYTE_TRY_LAUNCH("refine");
  }
  if (iters_out) *iters_out = it;
  if (relres_out) *relres_out = relres;
  return FLYTE_OK;
}

}  // namespace flyte
