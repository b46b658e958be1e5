// gemv.cu -- y <- alpha op(A) x + beta y on a row-major k-byte matrix (Sec. 6, BLAS level 2).
//
// The matrix is the only large operand, so the kernels are HBM-bound when
// each element costs few instructions: A is streamed once with aligned
// vector loads of whole 4-element groups (4k bytes), widened in registers
// (Sec. 4.1) and folded into double-word accumulators on the binary32 pipe
// (dwacc.cuh).  x is prepared once per call as x' = x 2^-sx = x1 + x2 (two
// binary32 arrays in the workspace, sx chosen so that max |x'| is in [1, 2)).
//
//   'N': a block of 8 warps owns R rows; its 256 threads stride over the
//        row in 4-element groups, 4 accumulators per row and thread (chains
//        of n/1024 terms); warp and block reductions in binary64.
//   'T': a block of 4 warps owns 512 columns and a tile of RB rows; each
//        thread keeps 2 x 4 accumulators for its 4 columns; the per-tile
//        column sums go to the workspace and a second kernel adds the tiles
//        in a fixed order and applies the epilogue.
//
// Whenever an element is outside the binary32 window, or x is, or the
// pointers are not aligned for group loads, the affected row (N) or column
// group (T) is recomputed with binary64 FMAs over the raw bytes.
#include "dwacc.cuh"

namespace flyte {
namespace {

constexpr int kHdrBytes = 256;

// Fold element bits (widened native pattern) times x1 + x2 into acc.
template <int BASE, int K>
__device__ __forceinline__ void fold(typename Native<BASE>::bits u, float x1, float x2, DW& acc, bool& ok) {
  float p, e;
  if constexpr (BASE == FLYTE_F64) {
    float hi, lo;
    ok &= dbl_to_pair<K>(uint32_t(u >> 32), uint32_t(u), hi, lo);
    if constexpr (K <= 4) {
      single_times_x(hi, x1, x2, p, e);
    } else {
      pair_times_x(hi, lo, x1, x2, p, e);
    }
  } else {
    ok &= flt_in_window(u);
    single_times_x(__uint_as_float(u), x1, x2, p, e);
  }
  dw_add(acc, p, e);
}

__device__ __forceinline__ double epilogue(double t, double alpha, double beta, const double* yp) {
  return beta == 0.0 ? alpha * t : fma(alpha, t, beta * *yp);
}

// ---- x preparation: x' = x 2^-sx = x1 + x2 -------------------------------------

__global__ void __launch_bounds__(1024) prep_x(const double* __restrict__ x, int64_t len, int64_t incx,
                                               int* __restrict__ hdr, float* __restrict__ x1,
                                               float* __restrict__ x2) {
  __shared__ int s_emax, s_bad;
  if (threadIdx.x == 0) { s_emax = -1; s_bad = 0; }
  __syncthreads();
  int emax = -1, bad = 0;
  for (int64_t j = threadIdx.x; j < len; j += blockDim.x) {
    const uint64_t b = uint64_t(__double_as_longlong(x[j * incx]));
    const int e = int((b >> 52) & 0x7FF);
    if (e == 0x7FF) bad = 1;
    else if ((b << 1) != 0) emax = max(emax, e);
  }
  emax = __reduce_max_sync(0xFFFFFFFFu, emax);
  bad = __reduce_or_sync(0xFFFFFFFFu, bad);
  if ((threadIdx.x & 31) == 0) { atomicMax(&s_emax, emax); atomicOr(&s_bad, bad); }
  __syncthreads();
  // scale so that the largest nonzero |x| lands in [1, 2)
  const int sx = s_emax < 0 ? 0 : s_emax - 1023;
  bad = s_bad || sx > 1000 || sx < -1000;
  const double scale = __longlong_as_double((long long)(uint64_t(1023 - (bad ? 0 : sx)) << 52));
  for (int64_t j = threadIdx.x; j < len; j += blockDim.x) {
    const double v = x[j * incx] * scale;
    const float a = __double2float_rn(v);
    const float c = __double2float_rn(v - double(a));
    if (v != 0.0 && fabs(v) < 0x1p-40) bad = 1;
    x1[j] = a;
    x2[j] = c;
  }
  bad = __reduce_or_sync(0xFFFFFFFFu, bad);
  __syncthreads();
  if ((threadIdx.x & 31) == 0 && bad) atomicOr(&s_bad, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    hdr[0] = sx;
    hdr[1] = s_bad ? 0 : 1;
  }
}

// ---- gemv N ---------------------------------------------------------------------

constexpr int kNThreads = 256;

template <int BASE, int K, int R>
__global__ void __launch_bounds__(kNThreads) gemv_n_kernel(
    const uint8_t* __restrict__ A, int64_t lda, int64_t m, int64_t n, const float* __restrict__ x1,
    const float* __restrict__ x2, const int* __restrict__ hdr, const double* __restrict__ x, int64_t incx,
    double alpha, double beta, double* __restrict__ y, int64_t incy, int fast) {
  using Bits = typename Native<BASE>::bits;
  __shared__ double red[kNThreads / 32][R];
  __shared__ double bsum[kNThreads / 32];
  __shared__ int bad[R];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t r0 = int64_t(blockIdx.x) * R;
  const bool use_fast = fast && hdr[1] != 0;
  if (threadIdx.x < R) bad[threadIdx.x] = use_fast ? 0 : 1;
  __syncthreads();
  if (use_fast) {
    DW acc[R][4];
    bool ok[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      ok[r] = true;
#pragma unroll
      for (int e = 0; e < 4; ++e) dw_zero(acc[r][e]);
    }
    const int64_t ngrp = n >> 2;
    for (int64_t g = threadIdx.x; g < ngrp; g += kNThreads) {
      const float4 xa = __ldg(reinterpret_cast<const float4*>(x1) + g);
      const float4 xb = __ldg(reinterpret_cast<const float4*>(x2) + g);
      const float xs1[4] = {xa.x, xa.y, xa.z, xa.w};
      const float xs2[4] = {xb.x, xb.y, xb.z, xb.w};
      uint32_t w[R][K];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (r0 + r < m) load_group<K>(A + ((r0 + r) * lda + 4 * g) * K, w[r]);
      }
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (r0 + r < m) {
#pragma unroll
          for (int e = 0; e < 4; ++e)
            fold<BASE, K>(extract_widened<BASE, K>(w[r], e), xs1[e], xs2[e], acc[r][e], ok[r]);
        }
      }
    }
    const int64_t j = (ngrp << 2) + threadIdx.x;   // the n % 4 trailing elements
    if (j < n) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (r0 + r < m) {
          const uint64_t q = load_code_bytes<K>(A + ((r0 + r) * lda + j) * K);
          fold<BASE, K>(widen<BASE, K>(q), x1[j], x2[j], acc[r][0], ok[r]);
        }
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const bool any_bad = __any_sync(0xFFFFFFFFu, !ok[r]);
      double v = 0.0;
#pragma unroll
      for (int e = 0; e < 4; ++e) v += dw_value(acc[r][e]);
      v = warp_sum(v);
      if (lane == 0) {
        red[warp][r] = v;
        if (any_bad) bad[r] = 1;
      }
    }
  }
  __syncthreads();
  const int sx = use_fast ? hdr[0] : 0;
  for (int r = 0; r < R; ++r) {
    const int64_t row = r0 + r;
    if (row >= m) break;
    double t = 0.0;
    if (bad[r]) {
      // binary64 FMAs over the raw bytes of the row
      const uint8_t* Ar = A + row * lda * K;
      double v = 0.0;
      for (int64_t c = threadIdx.x; c < n; c += kNThreads)
        v = fma(code_to_double<BASE, K>(load_code_bytes<K>(Ar + c * K)), x[c * incx], v);
      t = block_sum(v, bsum);
    } else if (threadIdx.x == 0) {
      for (int w = 0; w < kNThreads / 32; ++w) t += red[w][r];
      t = ldexp(t, sx);
    }
    if (threadIdx.x == 0) y[row * incy] = epilogue(t, alpha, beta, y + row * incy);
  }
  (void)sizeof(Bits);
}

// ---- gemv T ---------------------------------------------------------------------

constexpr int kTThreads = 128;

template <int BASE, int K>
__global__ void __launch_bounds__(kTThreads) gemv_t_kernel(
    const uint8_t* __restrict__ A, int64_t lda, int64_t m, int64_t n, const float* __restrict__ x1,
    const float* __restrict__ x2, const int* __restrict__ hdr, const double* __restrict__ x, int64_t incx,
    int64_t rb, double* __restrict__ partial, int fast) {
  const int64_t cg = int64_t(blockIdx.x) * kTThreads + threadIdx.x;
  const int64_t c0 = cg * 4;
  if (c0 >= n) return;
  const int64_t i0 = int64_t(blockIdx.y) * rb;
  const int64_t i1 = min(m, i0 + rb);
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  bool ok = fast && hdr[1] != 0 && c0 + 4 <= n;
  if (ok) {
    DW acc[2][4];
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int e = 0; e < 4; ++e) dw_zero(acc[h][e]);
    constexpr int U = 4;
    int64_t i = i0;
    for (; i + U <= i1; i += U) {
      uint32_t w[U][K];
      float a1[U], a2[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        load_group<K>(A + ((i + u) * lda + c0) * K, w[u]);
        a1[u] = __ldg(x1 + i + u);
        a2[u] = __ldg(x2 + i + u);
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int e = 0; e < 4; ++e)
          fold<BASE, K>(extract_widened<BASE, K>(w[u], e), a1[u], a2[u], acc[u & 1][e], ok);
    }
    for (; i < i1; ++i) {
      uint32_t w[K];
      load_group<K>(A + (i * lda + c0) * K, w);
      const float a1 = __ldg(x1 + i), a2 = __ldg(x2 + i);
#pragma unroll
      for (int e = 0; e < 4; ++e) fold<BASE, K>(extract_widened<BASE, K>(w, e), a1, a2, acc[i & 1][e], ok);
    }
    const int sx = hdr[0];
#pragma unroll
    for (int e = 0; e < 4; ++e) v[e] = ldexp(dw_value(acc[0][e]) + dw_value(acc[1][e]), sx);
  }
  if (!ok) {
    // binary64 FMAs over the raw bytes of this thread's columns
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      double s = 0.0;
      if (c0 + e < n) {
        for (int64_t i = i0; i < i1; ++i)
          s = fma(code_to_double<BASE, K>(load_code_bytes<K>(A + (i * lda + c0 + e) * K)), x[i * incx], s);
      }
      v[e] = s;
    }
  }
  double* out = partial + int64_t(blockIdx.y) * n + c0;
#pragma unroll
  for (int e = 0; e < 4; ++e)
    if (c0 + e < n) out[e] = v[e];
}

__global__ void gemv_t_finish(const double* __restrict__ partial, int64_t ntiles, int64_t n, double alpha,
                              double beta, double* __restrict__ y, int64_t incy) {
  const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double t = 0.0;
  for (int64_t s = 0; s < ntiles; ++s) t += partial[s * n + j];
  y[j * incy] = epilogue(t, alpha, beta, y + j * incy);
}

__global__ void scale_y(double* __restrict__ y, int64_t len, int64_t incy, double beta) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < len; j += stride)
    y[j * incy] = beta == 0.0 ? 0.0 : beta * y[j * incy];
}

constexpr int kNRows = 4;          // rows per block in gemv N
constexpr int64_t kTMaxRB = 256;   // row tile of gemv T

int64_t align16(int64_t b) { return (b + 15) & ~int64_t(15); }

struct Plan {
  bool fast;
  int64_t rb, ntiles;
  int64_t off_x1, off_x2, off_part, bytes;
};

Plan plan_gemv(char trans, int64_t m, int64_t n, flyte_fmt f) {
  Plan p{};
  const int64_t lenx = trans == 'N' ? n : m;
  p.off_x1 = kHdrBytes;
  p.off_x2 = p.off_x1 + align16(4 * lenx);
  p.off_part = p.off_x2 + align16(4 * lenx);
  p.bytes = p.off_part;
  if (trans == 'N') {
    const int64_t L = (n / 4 + kNThreads - 1) / kNThreads + 1;
    p.fast = dw_bound_ok(n, L, 16);
    p.rb = 0;
    p.ntiles = 0;
  } else {
    int64_t rb = kTMaxRB;
    while (rb >= 16 && !dw_bound_ok(m, rb / 2, (m + rb - 1) / rb + 2)) rb /= 2;
    p.fast = rb >= 16;
    p.rb = p.fast ? rb : kTMaxRB;
    p.ntiles = (m + p.rb - 1) / p.rb;
    p.bytes = p.off_part + 8 * p.ntiles * n;
  }
  (void)f;
  return p;
}

}  // namespace

size_t gemv_workspace_bytes(char trans, int64_t m, int64_t n, flyte_fmt f) {
  return size_t(plan_gemv(trans, m, n, f).bytes);
}

flyte_status launch_gemv(char trans, int64_t m, int64_t n, double alpha, const void* A, flyte_fmt fa,
                         int64_t lda, const double* x, int64_t incx, double beta, double* y, int64_t incy,
                         void* ws, size_t ws_bytes, cudaStream_t s) {
  const int64_t leny = trans == 'N' ? m : n;
  if (alpha == 0.0) {
    if (beta == 1.0) return FLYTE_OK;
    scale_y<<<grid_for(leny, 256), 256, 0, s>>>(y, leny, incy, beta);
    FLYTE_TRY_LAUNCH("gemv");
    return FLYTE_OK;
  }
  const Plan p = plan_gemv(trans, m, n, fa);
  if (ws == nullptr || ws_bytes < size_t(p.bytes)) {
    set_error("gemv: workspace of %lld bytes required", (long long)p.bytes);
    return FLYTE_ERR_WORKSPACE;
  }
  if (reinterpret_cast<uintptr_t>(ws) % 16 != 0) {
    set_error("gemv: workspace must be 16-byte aligned");
    return FLYTE_ERR_WORKSPACE;
  }
  uint8_t* w8 = static_cast<uint8_t*>(ws);
  int* hdr = reinterpret_cast<int*>(w8);
  float* x1 = reinterpret_cast<float*>(w8 + p.off_x1);
  float* x2 = reinterpret_cast<float*>(w8 + p.off_x2);
  const int64_t lenx = trans == 'N' ? n : m;
  return dispatch_fmt(fa, [&]<int BASE, int K>() -> flyte_status {
    constexpr int S = group_bytes(K);
    const bool aligned = reinterpret_cast<uintptr_t>(A) % S == 0 && (lda * K) % S == 0;
    const int fast = (p.fast && aligned) ? 1 : 0;
    if (fast) {
      prep_x<<<1, 1024, 0, s>>>(x, lenx, incx, hdr, x1, x2);
      FLYTE_TRY_LAUNCH("gemv");
    }
    const uint8_t* A8 = static_cast<const uint8_t*>(A);
    if (trans == 'N') {
      const unsigned blocks = unsigned((m + kNRows - 1) / kNRows);
      gemv_n_kernel<BASE, K, kNRows><<<blocks, kNThreads, 0, s>>>(A8, lda, m, n, x1, x2, hdr, x, incx, alpha,
                                                                 beta, y, incy, fast);
      FLYTE_TRY_LAUNCH("gemv");
    } else {
      double* part = reinterpret_cast<double*>(w8 + p.off_part);
      dim3 grid(unsigned((n + 4 * kTThreads - 1) / (4 * kTThreads)), unsigned(p.ntiles));
      gemv_t_kernel<BASE, K><<<grid, kTThreads, 0, s>>>(A8, lda, m, n, x1, x2, hdr, x, incx, p.rb, part, fast);
      FLYTE_TRY_LAUNCH("gemv");
      gemv_t_finish<<<unsigned((n + 255) / 256), 256, 0, s>>>(part, p.ntiles, n, alpha, beta, y, incy);
      FLYTE_TRY_LAUNCH("gemv");
    }
    return FLYTE_OK;
  });
}

}  // namespace flyte
