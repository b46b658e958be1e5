// blas1.cu -- dot and axpy on k-byte streams (Sec. 6, BLAS level 1).
//
// dot: both operands are flytes.  Each thread walks 4-element groups of the
// two streams (grid-stride), widens them in registers and, when all eight
// values are inside the binary32 window, folds the exact double-word
// products into 4 double-word accumulators (dwacc.cuh); a group with any
// other value (zero, subnormal, huge, Inf, NaN) goes into a binary64 FMA
// accumulator instead, which keeps IEEE Inf/NaN semantics.  Per-block sums go
// to the workspace and a one-block kernel adds them in a fixed order, so the
// result is the same on every call.
//
// axpy: y <- pack(fma(alpha, x, y)) in place, group by group.  The fma runs in
// the native type (binary64 or binary32) so it is correctly rounded, and the
// narrowing is the integer rounding of flyte_pack: the result is bit-exact.
// Each thread reads and rewrites its own aligned 4k-byte group of y, so the
// in-place update never has two threads touch the same bytes.
//
// scal: x <- pack(alpha * x) in place (the paper's in-place "scale"
// benchmark, Sec. 6), with the product rounded once in the native type.
#include <cmath>

#include "axpy_exact.cuh"
#include "load_unaligned.cuh"
#include "dwacc.cuh"

namespace flyte {
namespace {

constexpr int kThreads = 256;
#ifndef FLYTE_AXPY_WIDE_DIV
#define FLYTE_AXPY_WIDE_DIV 3          // k = 5..7 axpy: one warp in this many runs the binary64 fma
#endif
// k = 5..7 scal: one warp in this many multiplies in binary64.  The binary32 side of scal has no y
// to carry, so fewer warps on the fp64 pipe balance it (measured at 2^28 elements, k = 5 / 6 / 7:
// one in four 3.32 / 4.19 / 4.44 TB/s, one in three 3.18 / 3.84 / 4.29, one in five 3.35 / 4.09 / 4.44)
#ifndef FLYTE_SCAL_WIDE_DIV
#define FLYTE_SCAL_WIDE_DIV 4
#endif
constexpr int kDotMaxBlocks = 2048;   // fixed, so the workspace size does not depend on the device
constexpr int kHdrBytes = 256;

template <int BASE, int K>
__device__ __forceinline__ bool to_pair(typename Native<BASE>::bits u, float& hi, float& lo) {
  if constexpr (BASE == FLYTE_F64) {
    return dbl_to_pair<K>(uint32_t(u >> 32), uint32_t(u), hi, lo);
  } else {
    hi = __uint_as_float(u);
    lo = 0.f;
    return flt_in_window(u);
  }
}

template <int BASE, int K>
__device__ __forceinline__ double bits_to_double(typename Native<BASE>::bits u) {
  if constexpr (BASE == FLYTE_F64) {
    return __longlong_as_double((long long)u);
  } else {
    return double(__uint_as_float(u));
  }
}

// UA: x or y not 4k-byte aligned (groups read with load_group_unaligned).
template <int BASE, int K, bool UA>
__global__ void __launch_bounds__(kThreads) dot_groups(const uint8_t* __restrict__ X, const uint8_t* __restrict__ Y,
                                                       int64_t ngrp, int64_t n, int fast,
                                                       double* __restrict__ partial) {
  __shared__ double smem[kThreads / 32];
  DW acc[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) dw_zero(acc[e]);
  double acc64 = 0.0;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  for (int64_t g = tid; g < ngrp; g += stride) {
    uint32_t wx[K], wy[K];
    if constexpr (UA) {
      load_group_unaligned<K>(X + g * (4 * K), wx);
      load_group_unaligned<K>(Y + g * (4 * K), wy);
    } else {
      load_group<K>(X + g * (4 * K), wx);
      load_group<K>(Y + g * (4 * K), wy);
    }
    typename Native<BASE>::bits ux[4], uy[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      ux[e] = extract_widened<BASE, K>(wx, e);
      uy[e] = extract_widened<BASE, K>(wy, e);
    }
    bool ok = fast != 0;
    float p[4], q[4];
    if (ok) {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        float xh, xl, yh, yl;
        ok &= to_pair<BASE, K>(ux[e], xh, xl);
        ok &= to_pair<BASE, K>(uy[e], yh, yl);
        if constexpr (BASE == FLYTE_F64 && K > 4) {
          pair_times_pair(xh, xl, yh, yl, p[e], q[e]);
        } else {
          p[e] = __fmul_rn(xh, yh);
          q[e] = __fmaf_rn(xh, yh, -p[e]);
        }
      }
    }
    if (ok) {
#pragma unroll
      for (int e = 0; e < 4; ++e) dw_add(acc[e], p[e], q[e]);
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e) acc64 = fma(bits_to_double<BASE, K>(ux[e]), bits_to_double<BASE, K>(uy[e]), acc64);
    }
  }
  // the n % 4 trailing elements, binary64
  const int64_t j = (ngrp << 2) + tid;
  if (j < n) {
    acc64 = fma(code_to_double<BASE, K>(load_code_bytes<K>(X + j * K)),
                code_to_double<BASE, K>(load_code_bytes<K>(Y + j * K)), acc64);
  }
  double v = acc64;
#pragma unroll
  for (int e = 0; e < 4; ++e) v += dw_value(acc[e]);
  v = block_sum(v, smem);
  if (threadIdx.x == 0) partial[blockIdx.x] = v;
}

// Any formats, strides and alignments: binary64 FMAs over the raw bytes.
__global__ void __launch_bounds__(kThreads) dot_generic(const uint8_t* __restrict__ X, int kx, int bx, int64_t incx,
                                                        const uint8_t* __restrict__ Y, int ky, int by, int64_t incy,
                                                        int64_t n, double* __restrict__ partial) {
  __shared__ double smem[kThreads / 32];
  double acc = 0.0;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double a = code_to_double_rt(load_code_bytes_rt(X + i * incx * kx, kx), kx, bx);
    const double b = code_to_double_rt(load_code_bytes_rt(Y + i * incy * ky, ky), ky, by);
    acc = fma(a, b, acc);
  }
  acc = block_sum(acc, smem);
  if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

// Fixed-order sum of the per-block partials (pairwise over the block).
__global__ void __launch_bounds__(kThreads) dot_finish(const double* __restrict__ partial, int nblocks,
                                                       double* __restrict__ result) {
  __shared__ double smem[kThreads / 32];
  double v = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += kThreads) v += partial[b];
  v = block_sum(v, smem);
  if (threadIdx.x == 0) *result = v;
}

// ---- axpy -----------------------------------------------------------------------

template <int BASE, int K>
__device__ __forceinline__ uint64_t axpy_one(typename Native<BASE>::bits ux, typename Native<BASE>::bits uy,
                                             double alpha, float alpha_f, int mode) {
  if constexpr (BASE == FLYTE_F64) {
    const double r = fma(alpha, __longlong_as_double((long long)ux), __longlong_as_double((long long)uy));
    return narrow<BASE, K>(uint64_t(__double_as_longlong(r)), mode);
  } else {
    const float r = __fmaf_rn(alpha_f, __uint_as_float(ux), __uint_as_float(uy));
    return narrow<BASE, K>(__float_as_uint(r), mode);
  }
}

template <int BASE, int K>
__global__ void __launch_bounds__(kThreads) axpy_groups(const uint8_t* __restrict__ X, uint8_t* __restrict__ Y,
                                                        int64_t ngrp, double alpha, int mode) {
  const float alpha_f = __double2float_rn(alpha);
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; g < ngrp; g += stride) {
    uint32_t wx[K], wy[K], wo[K];
    load_group<K>(X + g * (4 * K), wx);
    load_group_rw<K>(Y + g * (4 * K), wy);
#pragma unroll
    for (int j = 0; j < K; ++j) wo[j] = 0;
#pragma unroll
    for (int e = 0; e < 4; ++e)
      deposit_code<K>(wo, e, axpy_one<BASE, K>(extract_widened<BASE, K>(wx, e), extract_widened<BASE, K>(wy, e),
                                               alpha, alpha_f, mode));
    store_group<K>(Y + g * (4 * K), wo);
  }
}

// ---- axpy without binary64 arithmetic: axpy_exact.cuh ------------------------------------

// SPLIT = false: alpha is a binary32 number; true: any alpha in the window, as two binary32 parts.
template <int K, int MODE, bool SPLIT>
__global__ void __launch_bounds__(kThreads) axpy_groups_f32exact(const uint8_t* __restrict__ X,
                                                                 uint8_t* __restrict__ Y, int64_t ngrp,
                                                                 double alpha) {
  const float af = float(alpha);
  const float a2 = float(alpha - double(af));
  const float a3 = float(alpha - double(af) - double(a2));
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  // k = 5..7: one warp in FLYTE_AXPY_WIDE_DIV takes the binary64 fma for all its groups, the others
  // the binary32 decision, so that the fp64 pipe and the binary32/integer pipes work side by side:
  // either path alone is bound by its own pipe at about the same rate (k = 5 at 2^28 elements:
  // binary64 1.06 ms, binary32 decision 1.01 ms; one warp in 2, 3, 4 on binary64: 0.87, 0.85, 0.93 ms)
  const bool wide64 = K >= 5 && ((threadIdx.x >> 5) % FLYTE_AXPY_WIDE_DIV) == 0;
  for (int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; g < ngrp; g += stride) {
    uint32_t wx[K], wy[K], wo[K];
    load_group<K>(X + g * (4 * K), wx);
    load_group_rw<K>(Y + g * (4 * K), wy);
#pragma unroll
    for (int j = 0; j < K; ++j) wo[j] = 0;
    uint64_t c[4];
    bool ok = !wide64;
#pragma unroll
    for (int q = 0; q < 4 && !wide64; ++q) {
      const uint64_t ux = extract_widened<FLYTE_F64, K>(wx, q), uy = extract_widened<FLYTE_F64, K>(wy, q);
      if constexpr (K >= 5) {
        ok &= axpy_exact_wide<K, MODE>(ux, uy, af, c[q]);
      } else if constexpr (SPLIT) {
        ok &= axpy_exact_f32x2<K, MODE>(ux, uy, af, a2, a3, c[q]);
      } else {
        ok &= axpy_exact_f32<K, MODE>(ux, uy, af, c[q]);
      }
    }
    if (!ok) {
#pragma unroll
      for (int q = 0; q < 4; ++q)
        c[q] = axpy_one<FLYTE_F64, K>(extract_widened<FLYTE_F64, K>(wx, q), extract_widened<FLYTE_F64, K>(wy, q),
                                      alpha, af, MODE);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) deposit_code<K>(wo, q, c[q]);
    store_group<K>(Y + g * (4 * K), wo);
  }
}

template <int K, bool SPLIT>
void launch_axpy_f32exact(const uint8_t* X, uint8_t* Y, int64_t ngrp, double alpha, int mode, cudaStream_t s) {
  const unsigned grid = grid_for(ngrp, kThreads);
  switch (mode) {
    case FLYTE_RNE: axpy_groups_f32exact<K, FLYTE_RNE, SPLIT><<<grid, kThreads, 0, s>>>(X, Y, ngrp, alpha); break;
    case FLYTE_RTZ: axpy_groups_f32exact<K, FLYTE_RTZ, SPLIT><<<grid, kThreads, 0, s>>>(X, Y, ngrp, alpha); break;
    case FLYTE_HALF_UP:
      axpy_groups_f32exact<K, FLYTE_HALF_UP, SPLIT><<<grid, kThreads, 0, s>>>(X, Y, ngrp, alpha);
      break;
    default: axpy_groups_f32exact<K, FLYTE_RTO, SPLIT><<<grid, kThreads, 0, s>>>(X, Y, ngrp, alpha); break;
  }
}

// Any widths of one base, strides and alignments: one element per thread.
template <int BASE, int KY>
__global__ void __launch_bounds__(kThreads) axpy_generic(const uint8_t* __restrict__ X, int kx, int64_t incx,
                                                         uint8_t* __restrict__ Y, int64_t incy, int64_t first,
                                                         int64_t n, double alpha, int mode) {
  using Bits = typename Native<BASE>::bits;
  constexpr int W = Native<BASE>::W;
  const float alpha_f = __double2float_rn(alpha);
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t i = first + int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint64_t qx = load_code_bytes_rt(X + i * incx * kx, kx);
    const Bits ux = kx * 8 == W ? Bits(qx) : Bits(qx << (W - 8 * kx));
    uint8_t* py = Y + i * incy * KY;
    const Bits uy = widen<BASE, KY>(load_code_bytes<KY>(py));
    store_code_bytes<KY>(py, axpy_one<BASE, KY>(ux, uy, alpha, alpha_f, mode));
  }
}

// ---- scal ------------------------------------------------------------------------

template <int BASE, int K>
__device__ __forceinline__ uint64_t scal_one(typename Native<BASE>::bits ux, double alpha, float alpha_f,
                                             int mode) {
  if constexpr (BASE == FLYTE_F64) {
    const double r = __dmul_rn(alpha, __longlong_as_double((long long)ux));
    return narrow<BASE, K>(uint64_t(__double_as_longlong(r)), mode);
  } else {
    const float r = __fmul_rn(alpha_f, __uint_as_float(ux));
    return narrow<BASE, K>(__float_as_uint(r), mode);
  }
}

template <int BASE, int K>
__global__ void __launch_bounds__(kThreads) scal_groups(uint8_t* __restrict__ X, int64_t ngrp, double alpha,
                                                        int mode) {
  const float alpha_f = __double2float_rn(alpha);
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; g < ngrp; g += stride) {
    uint32_t wx[K], wo[K];
    load_group_rw<K>(X + g * (4 * K), wx);
#pragma unroll
    for (int j = 0; j < K; ++j) wo[j] = 0;
#pragma unroll
    for (int e = 0; e < 4; ++e)
      deposit_code<K>(wo, e, scal_one<BASE, K>(extract_widened<BASE, K>(wx, e), alpha, alpha_f, mode));
    store_group<K>(X + g * (4 * K), wo);
  }
}

// Double-based k = 2..7 with a binary32 alpha: the code of pack(RN64(alpha x)) decided in binary32
// (scal_exact_f32, and axpy_exact_wide without y for k = 5..7), binary64 for a group that needs it;
// for k = 5..7 one warp in FLYTE_SCAL_WIDE_DIV multiplies in binary64, as axpy does.
template <int K, int MODE>
__global__ void __launch_bounds__(kThreads) scal_groups_f32exact(uint8_t* __restrict__ X, int64_t ngrp,
                                                                 double alpha) {
  const float af = float(alpha);
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  const bool wide64 = K >= 5 && ((threadIdx.x >> 5) % FLYTE_SCAL_WIDE_DIV) == 0;
  for (int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; g < ngrp; g += stride) {
    uint32_t wx[K], wo[K];
    load_group_rw<K>(X + g * (4 * K), wx);
#pragma unroll
    for (int j = 0; j < K; ++j) wo[j] = 0;
    uint64_t c[4];
    bool ok = !wide64;
#pragma unroll
    for (int q = 0; q < 4 && !wide64; ++q) {
      const uint64_t ux = extract_widened<FLYTE_F64, K>(wx, q);
      if constexpr (K >= 5) {
        ok &= axpy_exact_wide<K, MODE, false>(ux, 0, af, c[q]);
      } else {
        ok &= scal_exact_f32<K, MODE>(ux, af, c[q]);
      }
    }
    if (!ok) {
#pragma unroll
      for (int q = 0; q < 4; ++q)
        c[q] = scal_one<FLYTE_F64, K>(extract_widened<FLYTE_F64, K>(wx, q), alpha, af, MODE);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) deposit_code<K>(wo, q, c[q]);
    store_group<K>(X + g * (4 * K), wo);
  }
}

template <int BASE, int K>
__global__ void __launch_bounds__(kThreads) scal_generic(uint8_t* __restrict__ X, int64_t incx, int64_t first,
                                                         int64_t n, double alpha, int mode) {
  const float alpha_f = __double2float_rn(alpha);
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t i = first + int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
    uint8_t* p = X + i * incx * K;
    store_code_bytes<K>(p, scal_one<BASE, K>(widen<BASE, K>(load_code_bytes<K>(p)), alpha, alpha_f, mode));
  }
}

bool aligned(const void* p, int bytes) { return reinterpret_cast<uintptr_t>(p) % bytes == 0; }

int dot_blocks(int64_t work) {
  int64_t b = (work + kThreads - 1) / kThreads;
  if (b > kDotMaxBlocks) b = kDotMaxBlocks;
  if (b < 1) b = 1;
  return int(b);
}

}  // namespace

size_t dot_workspace_bytes(int64_t n) {
  (void)n;
  return size_t(kHdrBytes + 8 * kDotMaxBlocks);
}

flyte_status launch_dot(double* result, int64_t n, const void* x, flyte_fmt fx, int64_t incx, const void* y,
                        flyte_fmt fy, int64_t incy, void* ws, size_t ws_bytes, cudaStream_t s) {
  if (ws == nullptr || ws_bytes < dot_workspace_bytes(n) || reinterpret_cast<uintptr_t>(ws) % 16 != 0) {
    set_error("dot: workspace of %zu bytes (16-byte aligned) required", dot_workspace_bytes(n));
    return FLYTE_ERR_WORKSPACE;
  }
  double* partial = reinterpret_cast<double*>(static_cast<uint8_t*>(ws) + kHdrBytes);
  const uint8_t* X = static_cast<const uint8_t*>(x);
  const uint8_t* Y = static_cast<const uint8_t*>(y);
  const bool same = fx.k == fy.k && fx.base == fy.base;
  const int S = group_bytes(fx.k);
  // unit strides and one format: 4-element groups (funnel-shift loads when a stream is not 4k-byte aligned)
  const bool groups = same && incx == 1 && incy == 1 && n >= 4;
  const bool ua = !(aligned(x, S) && aligned(y, S));
  int nblocks;
  if (groups) {
    const int64_t ngrp = n / 4;
    nblocks = dot_blocks(ngrp);
    const int64_t L = (ngrp + int64_t(nblocks) * kThreads - 1) / (int64_t(nblocks) * kThreads);
    const int fast = dw_bound_ok(n, L, 4 + 5 + 7 + (nblocks + kThreads - 1) / kThreads + 12, 20) ? 1 : 0;
    flyte_status st = dispatch_fmt(fx, [&]<int BASE, int K>() -> flyte_status {
      if (ua) {
        dot_groups<BASE, K, true><<<nblocks, kThreads, 0, s>>>(X, Y, ngrp, n, fast, partial);
      } else {
        dot_groups<BASE, K, false><<<nblocks, kThreads, 0, s>>>(X, Y, ngrp, n, fast, partial);
      }
      FLYTE_TRY_LAUNCH("dot");
      return FLYTE_OK;
    });
    if (st != FLYTE_OK) return st;
  } else {
    nblocks = dot_blocks(n);
    dot_generic<<<nblocks, kThreads, 0, s>>>(X, fx.k, fx.base, incx, Y, fy.k, fy.base, incy, n, partial);
    FLYTE_TRY_LAUNCH("dot");
  }
  dot_finish<<<1, kThreads, 0, s>>>(partial, nblocks, result);
  FLYTE_TRY_LAUNCH("dot");
  return FLYTE_OK;
}

flyte_status launch_axpy(int64_t n, double alpha, const void* x, flyte_fmt fx, int64_t incx, void* y,
                         flyte_fmt fy, int64_t incy, int mode, cudaStream_t s) {
  const uint8_t* X = static_cast<const uint8_t*>(x);
  uint8_t* Y = static_cast<uint8_t*>(y);
  return dispatch_fmt(fy, [&]<int BASE, int KY>() -> flyte_status {
    int64_t first = 0;
    const int S = group_bytes(KY);
    if (fx.k == KY && incx == 1 && incy == 1 && aligned(x, S) && aligned(y, S) && n >= 4) {
      const int64_t ngrp = n / 4;
      bool done = false;
      if constexpr (BASE == FLYTE_F64 && KY >= 2 && KY <= 7) {
        // alpha inside the window: the exact binary32 paths (one part when alpha is a binary32
        // number; k = 5..7 take a binary32 alpha only)
        if (std::fabs(alpha) >= 0x1p-40 && std::fabs(alpha) < 0x1p40) {
          if (double(float(alpha)) == alpha) {
            launch_axpy_f32exact<KY, false>(X, Y, ngrp, alpha, mode, s);
            done = true;
          } else if constexpr (KY <= 4) {
            launch_axpy_f32exact<KY, true>(X, Y, ngrp, alpha, mode, s);
            done = true;
          }
        }
      }
      if (!done) axpy_groups<BASE, KY><<<grid_for(ngrp, kThreads), kThreads, 0, s>>>(X, Y, ngrp, alpha, mode);
      FLYTE_TRY_LAUNCH("axpy");
      first = ngrp * 4;
    }
    if (first < n) {
      axpy_generic<BASE, KY><<<grid_for(n - first, kThreads), kThreads, 0, s>>>(X, fx.k, incx, Y, incy, first, n,
                                                                               alpha, mode);
      FLYTE_TRY_LAUNCH("axpy");
    }
    return FLYTE_OK;
  });
}

flyte_status launch_scal(int64_t n, double alpha, void* x, flyte_fmt fx, int64_t incx, int mode, cudaStream_t s) {
  uint8_t* X = static_cast<uint8_t*>(x);
  return dispatch_fmt(fx, [&]<int BASE, int K>() -> flyte_status {
    int64_t first = 0;
    if (incx == 1 && aligned(x, group_bytes(K)) && n >= 4) {
      const int64_t ngrp = n / 4;
      bool done = false;
      if constexpr (BASE == FLYTE_F64 && K >= 2 && K <= 7) {
        if (std::fabs(alpha) >= 0x1p-40 && std::fabs(alpha) < 0x1p40 && double(float(alpha)) == alpha) {
          const unsigned grid = grid_for(ngrp, kThreads);
          switch (mode) {
            case FLYTE_RNE: scal_groups_f32exact<K, FLYTE_RNE><<<grid, kThreads, 0, s>>>(X, ngrp, alpha); break;
            case FLYTE_RTZ: scal_groups_f32exact<K, FLYTE_RTZ><<<grid, kThreads, 0, s>>>(X, ngrp, alpha); break;
            case FLYTE_HALF_UP:
              scal_groups_f32exact<K, FLYTE_HALF_UP><<<grid, kThreads, 0, s>>>(X, ngrp, alpha);
              break;
            default: scal_groups_f32exact<K, FLYTE_RTO><<<grid, kThreads, 0, s>>>(X, ngrp, alpha); break;
          }
          done = true;
        }
      }
      if (!done) scal_groups<BASE, K><<<grid_for(ngrp, kThreads), kThreads, 0, s>>>(X, ngrp, alpha, mode);
      FLYTE_TRY_LAUNCH("scal");
      first = ngrp * 4;
    }
    if (first < n) {
      scal_generic<BASE, K><<<grid_for(n - first, kThreads), kThreads, 0, s>>>(X, incx, first, n, alpha, mode);
      FLYTE_TRY_LAUNCH("scal");
    }
    return FLYTE_OK;
  });
}

}  // namespace flyte
