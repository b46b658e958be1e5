// gemv.cu -- y <- alpha op(A) x + beta y on a row-major k-byte matrix (Sec. 6, BLAS level 2).
//
// The matrix is the only large operand, so the kernels are HBM-bound when
// each element costs few instructions: A is streamed once with aligned
// vector loads of whole 4-element groups (4k bytes), widened in registers
// (Sec. 4.1) and folded into double-word accumulators on the binary32 pipe
// (dwacc.cuh).  x is split once per call into x = x1 + x2 (two binary32
// arrays in the workspace); an x value outside the window gets x1 = NaN, so
// every double-word sum that uses it comes out NaN and is redone in binary64.
//
//   'N': a block of 8 warps owns 16 rows (2 per warp) and one chunk of at
//        most 4096 columns; all warps walk the same columns, so x1/x2 are
//        fetched into L1 once per block.  Each lane keeps 4 accumulators per
//        row (chains of chunk/128 terms); chunk sums go to the workspace and
//        a second kernel adds them in a fixed order and applies the epilogue.
//   'T': a block of 4 warps owns 512 columns and a tile of RB rows; each
//        thread keeps 2 x 4 accumulators for its 4 columns (rows alternate
//        between them); the per-tile column sums go to the workspace and a
//        second kernel adds the tiles in a fixed order.
//
// Whenever an element is outside the binary32 window, or the pointers are
// not aligned for group loads, the affected (row, chunk) of 'N' or (column
// group, tile) of 'T' is recomputed with binary64 FMAs over the raw bytes.
#include "bulkpipe.cuh"
#include "dwacc.cuh"
#include "load_unaligned.cuh"

namespace flyte {
namespace {


// Fold element bits (widened native pattern) times x1 + x2 into acc.
template <int BASE, int K, bool LAZY = false>
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
  if constexpr (LAZY) {
    dw_add_lazy(acc, p, e);
  } else {
    dw_add(acc, p, e);
  }
}

// ---- the fold: element times x1 + x2 into a double-word accumulator -----------------
//
// Elements are widened to binary32 (dbl_to_pair) and folded two at a time on
// the f32x2 pipe (dwacc.cuh): TwoProd of the element with x1, the x2 and low
// part products into the error word, and the (lazy or renormalising)
// double-word addition.
//
// Window test value of an element: in window iff below window_limit<BASE>().
// The kernels keep the running unsigned maximum of these values, so a whole
// row chunk or tile is tested with one compare.
template <int BASE>
__host__ __device__ constexpr uint32_t window_limit() {
  return BASE == FLYTE_F64 ? uint32_t(2 * kWinLog2) << 21 : uint32_t(2 * kWinLog2) << 24;
}

// Element bits -> binary32 value hi (+ lo for double-based k >= 5, else 0); returns the window value.
template <int BASE, int K>
__device__ __forceinline__ uint32_t widen_pair_v(typename Native<BASE>::bits u, float& hi, float& lo) {
  if constexpr (BASE == FLYTE_F64) {
    const uint32_t h = uint32_t(u >> 32);
    (void)dbl_to_pair<K>(h, uint32_t(u), hi, lo);
    return (h << 1) - ((1023u - kWinLog2) << 21);
  } else {
    hi = __uint_as_float(u);
    lo = 0.f;
    return (u << 1) - ((127u - kWinLog2) << 24);
  }
}

// acc <- acc + (a0, a1) * x for the pair of elements (a0 = h0 + l0, a1 = h1 + l1) and
// x = X1 + X2 per value (N1 = -X1): pair_times_x and dw_add(_lazy) of dwacc.cuh on both values.
template <int BASE, int K, bool LAZY>
__device__ __forceinline__ void fold_pair2(float h0, float l0, float h1, float l1, f2 X1, f2 N1, f2 X2, DW2& acc) {
  const f2 A = f2_pack(h0, h1);
  const f2 pn = f2_mul(A, N1);          // -p exactly
  f2 t = f2_fma(A, X1, pn);             // a x1 - p exactly
  if constexpr (BASE == FLYTE_F64 && K >= 5) t = f2_fma(f2_pack(l0, l1), X1, t);
  const f2 e = f2_fma(A, X2, t);
  if constexpr (LAZY) {
    dw2_add_lazy_neg(acc, pn, e);
  } else {
    dw2_add_neg(acc, pn, e);
  }
}

// A 4-element group of one row: elements 0, 1 into acc[0], elements 2, 3 into acc[1].
template <int BASE, int K, bool LAZY, int NW>
__device__ __forceinline__ void fold_group2(const uint32_t (&w)[NW], const f2 (&X1)[2], const f2 (&N1)[2],
                                            const f2 (&X2)[2], DW2 (&acc)[2], uint32_t& vmax) {
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    float h0, l0, h1, l1;
    const uint32_t v0 = widen_pair_v<BASE, K>(extract_widened<BASE, K>(w, 2 * q), h0, l0);
    const uint32_t v1 = widen_pair_v<BASE, K>(extract_widened<BASE, K>(w, 2 * q + 1), h1, l1);
    vmax = max(vmax, max(v0, v1));
    fold_pair2<BASE, K, LAZY>(h0, l0, h1, l1, X1[q], N1[q], X2[q], acc[q]);
  }
}

// One element (the ragged end of a row): into value 0 of acc; value 1 adds 0 * 0.
template <int BASE, int K, bool LAZY>
__device__ __forceinline__ void fold_one2(typename Native<BASE>::bits u, float x1, float x2, DW2& acc,
                                          uint32_t& vmax) {
  float h, l;
  vmax = max(vmax, widen_pair_v<BASE, K>(u, h, l));
  fold_pair2<BASE, K, LAZY>(h, l, 0.f, 0.f, f2_pack(x1, 0.f), f2_pack(-x1, 0.f), f2_pack(x2, 0.f), acc);
}

// The four scalar slots (elements 0..3 of the groups) of a row's two pair accumulators.
__device__ __forceinline__ void dw2_slots(const DW2 (&acc)[2], DW (&d)[4]) {
  dw2_split(acc[0], d[0], d[1]);
  dw2_split(acc[1], d[2], d[3]);
}

// Sum of a row's four slot accumulators over the warp, in double-word
// arithmetic (depth 2 + 5), as the binary64 value of lane 0 (exact
// conversion), broadcast to the warp.
__device__ __forceinline__ double row_total(const DW (&acc)[4]) {
  const DW a = dw_warp_sum(dw_sum4(acc[0], acc[1], acc[2], acc[3]));
  return __shfl_sync(0xFFFFFFFFu, dw_value(a), 0);
}

__device__ __forceinline__ double epilogue(double t, double alpha, double beta, const double* yp) {
  return beta == 0.0 ? alpha * t : fma(alpha, t, beta * *yp);
}

// ---- x preparation: x = x1 + x2 --------------------------------------------------

// x1 = RN32(x) and x2 = RN32(x - x1) (|x - x1 - x2| <= 2^-48 |x|) for x = 0 or
// 2^-40 <= |x| < 2^40; any other x (tiny, huge, Inf, NaN) gets x1 = NaN.
__global__ void __launch_bounds__(256) prep_x(const double* __restrict__ x, int64_t len, int64_t incx,
                                              float* __restrict__ x1, float* __restrict__ x2,
                                              int* __restrict__ status) {
  if (blockIdx.x == 0 && threadIdx.x == 0) *status = 0;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < len; j += stride) {
    const double v = x[j * incx];
    const double av = fabs(v);
    const bool ok = v == 0.0 || (av >= 0x1p-40 && av < 0x1p40);
    float a = __double2float_rn(v);
    float c = __double2float_rn(v - double(a));
    if (!ok) {
      a = __uint_as_float(0x7FC00000u);
      c = 0.f;
    }
    x1[j] = a;
    x2[j] = c;
  }
}

// ---- gemv N ---------------------------------------------------------------------

// Compile-time tuning knobs.  Defaults are the best of sweeps on GB300 at
// 16384 x 16384, double-based k = 3..6:
//  - 'N' runs the persistent producer/consumer ring below for every k when A
//    is 16-byte aligned (k = 4: 0.298 -> 0.233 ms, k = 5: 0.377 -> 0.338 ms),
//    8 consumer warps of 2 rows, 512 columns per stage and three blocks per
//    SM for k <= 4 (two stages each; two blocks of up to 113 KiB were 2 %
//    slower); one block per SM for k > 4, with 16 warps of one row and
//    1024 columns per stage for k = 5, 6 (k = 5: 0.338 -> 0.302 ms); 12
//    warps of one row, 512 columns and two blocks per SM for k = 7, 8 (k = 8:
//    0.355 -> 0.335 ms against one block); tiles of up to 4096
//    columns (8 warps of 4 rows, 16 warps of 2 rows, 24 warps of one row,
//    256-column stages were slower); a full stage's group loop is unrolled
//    (k = 3: 0.253 -> 0.229 ms, k = 5: 0.302 -> 0.289 ms); the direct kernel
//    (2 or 4 groups per lane and step) serves the rest;
//  - 'T' loads 8 rows per step without a software prefetch, with registers
//    capped so that 5 blocks (4 for k = 4) reside per SM (k = 6: 0.312 ->
//    0.282 ms, k = 4: 0.222 -> 0.202 ms against 4 rows with the next 4
//    prefetched; 12 or 16 rows, 4 or 6 blocks for other k were slower; with
//    no cap the compiler used more registers and the kernel ran ~15 % slower).
//    A producer/consumer ring for 'T' (8 rows per stage)
//    was not reliably faster (0.208-0.249 ms at k = 4 against 0.222 ms) and
//    was dropped, as was a warp-private bulk-copy pipeline for both.
#ifndef FLYTE_N_UNROLL_SMALL_K
#define FLYTE_N_UNROLL_SMALL_K 2
#endif
#ifndef FLYTE_N_UNROLL_LARGE_K
#define FLYTE_N_UNROLL_LARGE_K 4
#endif
#ifndef FLYTE_T_ROWS
#define FLYTE_T_ROWS 8
#endif
#ifndef FLYTE_GEMV_PC
#define FLYTE_GEMV_PC 1
#endif
#ifndef FLYTE_T_FOLD_MAX
#define FLYTE_T_FOLD_MAX 64            // longest fold period of 'T' (rows, a power of two)
#endif
#ifndef FLYTE_GEMV_PC_KMAX
#define FLYTE_GEMV_PC_KMAX 8
#endif
#ifndef FLYTE_PC_COLS_SMALL_K
#define FLYTE_PC_COLS_SMALL_K 512      // columns per ring stage, k <= 4
#endif
#ifndef FLYTE_PC_COLS_LARGE_K
#define FLYTE_PC_COLS_LARGE_K 1024     // columns per ring stage, k = 5, 6
#endif
#ifndef FLYTE_PC_CHUNK
#define FLYTE_PC_CHUNK 4096            // columns per 'N' tile (at most)
#endif
#ifndef FLYTE_GEMV_PREFETCH_T
#define FLYTE_GEMV_PREFETCH_T 0
#endif

constexpr int kNWarps = 8;
constexpr int kNRowsPerWarp = 2;
constexpr int kNRowsPerBlock = kNWarps * kNRowsPerWarp;
constexpr int64_t kNChunkCols = FLYTE_PC_CHUNK;   // columns per chunk, a multiple of 128
template <int K>
__host__ __device__ constexpr int n_unroll() { return K <= 4 ? FLYTE_N_UNROLL_SMALL_K : FLYTE_N_UNROLL_LARGE_K; }

// A group of A: vector loads, or (UA: rows not 4k-byte aligned) funnel-shift loads.
template <int K, bool UA>
__device__ __forceinline__ void load_grp(const uint8_t* p, uint32_t (&w)[K]) {
  if constexpr (UA) {
    load_group_unaligned<K>(p, w);
  } else {
    load_group<K>(p, w);
  }
}

template <int BASE, int K, bool LAZY, bool UA>
__global__ void __launch_bounds__(kNWarps * 32) gemv_n_kernel(
    const uint8_t* __restrict__ A, int64_t lda, int64_t m, int64_t n, const float* __restrict__ x1,
    const float* __restrict__ x2, const double* __restrict__ x, int64_t incx, int64_t chunk_cols,
    int64_t nchunks, double* __restrict__ partial, double alpha, double beta, double* __restrict__ y,
    int64_t incy, int fast, int direct) {
  constexpr int kNUnroll = n_unroll<K>();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t row0 = int64_t(blockIdx.x) * kNRowsPerBlock + warp * kNRowsPerWarp;
  if (row0 >= m) return;
  const int64_t chunk = blockIdx.y;
  const int64_t cb = chunk * chunk_cols;
  const int64_t ce = min(n, cb + chunk_cols);
  const int64_t gb = cb >> 2, ge = ce >> 2;           // whole groups of this chunk
  const uint8_t* rowp[kNRowsPerWarp];
#pragma unroll
  for (int r = 0; r < kNRowsPerWarp; ++r) rowp[r] = A + min(row0 + r, m - 1) * lda * K;

  double v[kNRowsPerWarp];
  bool ok[kNRowsPerWarp];
#pragma unroll
  for (int r = 0; r < kNRowsPerWarp; ++r) { v[r] = 0.0; ok[r] = fast != 0; }
  if (fast) {
    DW2 acc[kNRowsPerWarp][2];
    uint32_t vmax[kNRowsPerWarp];
#pragma unroll
    for (int r = 0; r < kNRowsPerWarp; ++r) {
      vmax[r] = 0u;
      dw2_zero(acc[r][0]);
      dw2_zero(acc[r][1]);
    }
    int64_t g = gb + lane;
    auto load_batch = [&](int64_t g0, ulonglong2 (&xa)[kNUnroll], ulonglong2 (&xb)[kNUnroll],
                          uint32_t (&w)[kNUnroll][kNRowsPerWarp][K]) {
#pragma unroll
      for (int u = 0; u < kNUnroll; ++u) {
        const int64_t gu = g0 + 32 * u;
        xa[u] = __ldg(reinterpret_cast<const ulonglong2*>(x1) + gu);
        xb[u] = __ldg(reinterpret_cast<const ulonglong2*>(x2) + gu);
#pragma unroll
        for (int r = 0; r < kNRowsPerWarp; ++r) load_grp<K, UA>(rowp[r] + gu * (4 * K), w[u][r]);
      }
    };
    for (; g + 32 * (kNUnroll - 1) < ge; g += 32 * kNUnroll) {
      ulonglong2 xa[kNUnroll], xb[kNUnroll];
      uint32_t w[kNUnroll][kNRowsPerWarp][K];
      load_batch(g, xa, xb, w);
#pragma unroll
      for (int u = 0; u < kNUnroll; ++u) {
        const f2 X1[2] = {xa[u].x, xa[u].y}, N1[2] = {f2_neg(xa[u].x), f2_neg(xa[u].y)}, X2[2] = {xb[u].x, xb[u].y};
#pragma unroll
        for (int r = 0; r < kNRowsPerWarp; ++r) fold_group2<BASE, K, LAZY>(w[u][r], X1, N1, X2, acc[r], vmax[r]);
      }
    }
    for (; g < ge; g += 32) {
      const ulonglong2 xa = __ldg(reinterpret_cast<const ulonglong2*>(x1) + g);
      const ulonglong2 xb = __ldg(reinterpret_cast<const ulonglong2*>(x2) + g);
      const f2 X1[2] = {xa.x, xa.y}, N1[2] = {f2_neg(xa.x), f2_neg(xa.y)}, X2[2] = {xb.x, xb.y};
#pragma unroll
      for (int r = 0; r < kNRowsPerWarp; ++r) {
        uint32_t w[K];
        load_grp<K, UA>(rowp[r] + g * (4 * K), w);
        fold_group2<BASE, K, LAZY>(w, X1, N1, X2, acc[r], vmax[r]);
      }
    }
    const int64_t j = (ge << 2) + lane;               // trailing n % 4 elements (last chunk only)
    if (j < ce) {
#pragma unroll
      for (int r = 0; r < kNRowsPerWarp; ++r) {
        const uint64_t q = load_code_bytes<K>(rowp[r] + j * K);
        fold_one2<BASE, K, LAZY>(widen<BASE, K>(q), x1[j], x2[j], acc[r][0], vmax[r]);
      }
    }
#pragma unroll
    for (int r = 0; r < kNRowsPerWarp; ++r) {
      DW slots[4];
      dw2_slots(acc[r], slots);
      const double t = row_total(slots);
      v[r] = t;
      ok[r] = __all_sync(0xFFFFFFFFu, vmax[r] < window_limit<BASE>()) && isfinite(t);
    }
  }
#pragma unroll
  for (int r = 0; r < kNRowsPerWarp; ++r) {
    const int64_t row = row0 + r;
    if (row >= m) break;
    if (!ok[r]) {
      // binary64 FMAs over the raw bytes of this row and chunk
      const uint8_t* Ar = A + row * lda * K;
      double s = 0.0;
      for (int64_t c = cb + lane; c < ce; c += 32)
        s = fma(code_to_double<BASE, K>(load_code_bytes<K>(Ar + c * K)), x[c * incx], s);
      v[r] = warp_sum(s);
    }
    if (lane == 0) {
      if (direct) {
        y[row * incy] = epilogue(v[r], alpha, beta, y + row * incy);
      } else {
        partial[row * nchunks + chunk] = v[r];
      }
    }
  }
}

// Row sums over the chunks in chunk order, then the epilogue.
__global__ void __launch_bounds__(256) gemv_n_finish(const double* __restrict__ partial, int64_t nchunks,
                                                     int64_t m, double alpha, double beta,
                                                     double* __restrict__ y, int64_t incy) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= m) return;
  double t = 0.0;
  for (int64_t c = 0; c < nchunks; ++c) t += partial[i * nchunks + c];
  y[i * incy] = epilogue(t, alpha, beta, y + i * incy);
}

// The same with y stored as double-based flytes of KY bytes: the epilogue
// reads the old code (unless beta == 0), forms fma(alpha, t, beta y) in
// binary64 and packs it with the integer rounding of flyte_pack.
template <int KY>
__device__ __forceinline__ void epilogue_packed(double t, double alpha, double beta, uint8_t* yp, int mode) {
  const double yo = beta == 0.0 ? 0.0 : code_to_double<FLYTE_F64, KY>(load_code_bytes<KY>(yp));
  const double r = beta == 0.0 ? alpha * t : fma(alpha, t, beta * yo);
  store_code_bytes<KY>(yp, narrow<FLYTE_F64, KY>(uint64_t(__double_as_longlong(r)), mode));
}

template <int KY>
__global__ void __launch_bounds__(256) gemv_n_finish_packed(const double* __restrict__ partial, int64_t nchunks,
                                                            int64_t m, double alpha, double beta,
                                                            uint8_t* __restrict__ y, int64_t incy, int mode) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= m) return;
  double t = 0.0;
  for (int64_t c = 0; c < nchunks; ++c) t += partial[i * nchunks + c];
  epilogue_packed<KY>(t, alpha, beta, y + i * incy * KY, mode);
}

// ---- gemv T ---------------------------------------------------------------------

constexpr int kTThreads = 128;
// resident blocks per SM that the 'T' kernel's register use must allow
template <int K>
constexpr int t_min_blocks() {
#ifdef FLYTE_T_MIN_BLOCKS
  return FLYTE_T_MIN_BLOCKS;
#else
  return K == 4 ? 4 : 5;
#endif
}
constexpr int kTRowsPerIter = FLYTE_T_ROWS;   // rows loaded per iteration (a multiple of 4)

// Every fold_rows rows the two row-parity chains of each column are
// renormalised, added, and added into the column's running double-word total
// (two dw_add_dw levels per fold), then restarted.
__device__ __forceinline__ void fold_parities(DW (&acc)[2][4], DW (&tot)[4]) {
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    DW a = acc[0][e], b = acc[1][e];
    dw_norm(a);
    dw_norm(b);
    dw_add_dw(a, b);
    dw_add_dw(tot[e], a);
    dw_zero(acc[0][e]);
    dw_zero(acc[1][e]);
  }
}

// The same for pair accumulators: acc[parity][q] holds columns 2q and 2q + 1.
__device__ __forceinline__ void fold_parities2(DW2 (&acc)[2][2], DW (&tot)[4]) {
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    DW a[2], b[2];
    dw2_split(acc[0][q], a[0], a[1]);
    dw2_split(acc[1][q], b[0], b[1]);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      dw_norm(a[h]);
      dw_norm(b[h]);
      dw_add_dw(a[h], b[h]);
      dw_add_dw(tot[2 * q + h], a[h]);
    }
    dw2_zero(acc[0][q]);
    dw2_zero(acc[1][q]);
  }
}

template <int BASE, int K, bool LAZY, bool UA>
__global__ void __launch_bounds__(kTThreads, t_min_blocks<K>()) gemv_t_kernel(
    const uint8_t* __restrict__ A, int64_t lda, int64_t m, int64_t n, const float* __restrict__ x1,
    const float* __restrict__ x2, const double* __restrict__ x, int64_t incx, int64_t rb,
    int64_t fold_rows, double* __restrict__ partial, int fast) {
  constexpr int U = kTRowsPerIter;
  const int64_t cg = int64_t(blockIdx.x) * kTThreads + threadIdx.x;
  const int64_t c0 = cg * 4;
  if (c0 >= n) return;
  const int64_t i0 = int64_t(blockIdx.y) * rb;
  const int64_t i1 = min(m, i0 + rb);
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  bool ok = fast && c0 + 4 <= n;
  // Pairs of columns on the f32x2 pipe for double-based k = 4 (0.220 -> 0.208 ms at 16384^2); the
  // scalar fold elsewhere, where the pair fold measured slower (k = 3: 0.232 -> 0.244 ms, k = 5:
  // 0.303 -> 0.368 ms, same GPU and build)
  constexpr bool kPairs = BASE == FLYTE_F64 && K == 4;
  if constexpr (kPairs) {
    if (ok) {
      const uint8_t* colp = A + c0 * K;
      DW2 acc[2][2];
      DW tot[4];
      uint32_t vmax = 0u;
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        dw2_zero(acc[0][q]);
        dw2_zero(acc[1][q]);
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) dw_zero(tot[e]);
      int64_t since = 0;
      int64_t i = i0;
      auto load_batch = [&](int64_t r, uint32_t (&w)[U][K], float (&b1)[U], float (&b2)[U]) {
#pragma unroll
        for (int u = 0; u < U; u += 4) {
          const float4 p = __ldg(reinterpret_cast<const float4*>(x1 + r + u));
          const float4 q = __ldg(reinterpret_cast<const float4*>(x2 + r + u));
          b1[u] = p.x; b1[u + 1] = p.y; b1[u + 2] = p.z; b1[u + 3] = p.w;
          b2[u] = q.x; b2[u + 1] = q.y; b2[u + 2] = q.z; b2[u + 3] = q.w;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) load_grp<K, UA>(colp + (r + u) * lda * K, w[u]);
      };
#if FLYTE_GEMV_PREFETCH_T
      // software pipeline: the next batch of rows is in flight while this one is folded
      uint32_t wn[U][K];
      float n1[U], n2[U];
      if (i + U <= i1) load_batch(i, wn, n1, n2);
#endif
      for (; i + U <= i1; i += U) {
        uint32_t w[U][K];
        float a1[U], a2[U];
#if FLYTE_GEMV_PREFETCH_T
#pragma unroll
        for (int u = 0; u < U; ++u) {
          a1[u] = n1[u];
          a2[u] = n2[u];
#pragma unroll
          for (int j = 0; j < K; ++j) w[u][j] = wn[u][j];
        }
        if (i + 2 * U <= i1) load_batch(i + U, wn, n1, n2);
#else
        load_batch(i, w, a1, a2);
#endif
#pragma unroll
        for (int u = 0; u < U; ++u) {
          // the row's x for all four columns of the thread
          const f2 X1 = f2_pack(a1[u], a1[u]), X2 = f2_pack(a2[u], a2[u]);
          const f2 X1s[2] = {X1, X1}, N1s[2] = {f2_neg(X1), f2_neg(X1)}, X2s[2] = {X2, X2};
          fold_group2<BASE, K, LAZY>(w[u], X1s, N1s, X2s, acc[u & 1], vmax);
        }
        since += U;
        if (since >= fold_rows) {
          fold_parities2(acc, tot);
          since = 0;
        }
      }
      for (; i < i1; ++i) {
        uint32_t w[K];
        load_grp<K, UA>(colp + i * lda * K, w);
        const f2 X1 = f2_pack(x1[i], x1[i]), X2 = f2_pack(x2[i], x2[i]);
        const f2 X1s[2] = {X1, X1}, N1s[2] = {f2_neg(X1), f2_neg(X1)}, X2s[2] = {X2, X2};
        fold_group2<BASE, K, LAZY>(w, X1s, N1s, X2s, acc[0], vmax);
      }
      fold_parities2(acc, tot);
      ok = vmax < window_limit<BASE>();
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        v[e] = dw_value(tot[e]);      // exact: tot is normalised
        ok = ok && isfinite(v[e]);
      }
    }
  } else {
    if (ok) {
      const uint8_t* colp = A + c0 * K;
      DW acc[2][4], tot[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        dw_zero(acc[0][e]);
        dw_zero(acc[1][e]);
        dw_zero(tot[e]);
      }
      int64_t since = 0;
      int64_t i = i0;
      auto load_batch = [&](int64_t r, uint32_t (&w)[U][K], float (&b1)[U], float (&b2)[U]) {
#pragma unroll
        for (int u = 0; u < U; u += 4) {
          const float4 p = __ldg(reinterpret_cast<const float4*>(x1 + r + u));
          const float4 q = __ldg(reinterpret_cast<const float4*>(x2 + r + u));
          b1[u] = p.x; b1[u + 1] = p.y; b1[u + 2] = p.z; b1[u + 3] = p.w;
          b2[u] = q.x; b2[u + 1] = q.y; b2[u + 2] = q.z; b2[u + 3] = q.w;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) load_grp<K, UA>(colp + (r + u) * lda * K, w[u]);
      };
#if FLYTE_GEMV_PREFETCH_T
      // software pipeline: the next batch of rows is in flight while this one is folded
      uint32_t wn[U][K];
      float n1[U], n2[U];
      if (i + U <= i1) load_batch(i, wn, n1, n2);
#endif
      for (; i + U <= i1; i += U) {
        uint32_t w[U][K];
        float a1[U], a2[U];
#if FLYTE_GEMV_PREFETCH_T
#pragma unroll
        for (int u = 0; u < U; ++u) {
          a1[u] = n1[u];
          a2[u] = n2[u];
#pragma unroll
          for (int j = 0; j < K; ++j) w[u][j] = wn[u][j];
        }
        if (i + 2 * U <= i1) load_batch(i + U, wn, n1, n2);
#else
        load_batch(i, w, a1, a2);
#endif
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
          for (int e = 0; e < 4; ++e)
            fold<BASE, K, LAZY>(extract_widened<BASE, K>(w[u], e), a1[u], a2[u], acc[u & 1][e], ok);
        since += U;
        if (since >= fold_rows) {
          fold_parities(acc, tot);
          since = 0;
        }
      }
      for (; i < i1; ++i) {
        uint32_t w[K];
        load_grp<K, UA>(colp + i * lda * K, w);
        const float a1 = x1[i], a2 = x2[i];
#pragma unroll
        for (int e = 0; e < 4; ++e) fold<BASE, K, LAZY>(extract_widened<BASE, K>(w, e), a1, a2, acc[0][e], ok);
      }
      fold_parities(acc, tot);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        v[e] = dw_value(tot[e]);      // exact: tot is normalised
        ok = ok && isfinite(v[e]);
      }
    }
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

// Column sums over the tiles: lane = column, warps take tiles w, w+8, ...;
// the 8 warp sums are added in warp order, so the result is deterministic.
// Sum of column j over the tiles warp, warp + 8, ... in that order; four loads are issued before
// their additions so that the column's reads overlap (the order, hence the result, is unchanged).
__device__ __forceinline__ double tile_column_sum(const double* __restrict__ partial, int64_t ntiles, int64_t n,
                                                  int64_t j, int warp) {
  double t = 0.0;
  if (j >= n) return t;
  int64_t s = warp;
  for (; s + 24 < ntiles; s += 32) {
    const double a0 = partial[s * n + j], a1 = partial[(s + 8) * n + j];
    const double a2 = partial[(s + 16) * n + j], a3 = partial[(s + 24) * n + j];
    t += a0;
    t += a1;
    t += a2;
    t += a3;
  }
  for (; s < ntiles; s += 8) t += partial[s * n + j];
  return t;
}

__global__ void __launch_bounds__(256) gemv_t_finish(const double* __restrict__ partial, int64_t ntiles, int64_t n,
                                                     double alpha, double beta, double* __restrict__ y,
                                                     int64_t incy) {
  __shared__ double red[8][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t j = int64_t(blockIdx.x) * 32 + lane;
  const double t = tile_column_sum(partial, ntiles, n, j, warp);
  red[warp][lane] = t;
  __syncthreads();
  if (warp == 0 && j < n) {
    double sum = 0.0;
    for (int w = 0; w < 8; ++w) sum += red[w][lane];
    y[j * incy] = epilogue(sum, alpha, beta, y + j * incy);
  }
}

template <int KY>
__global__ void __launch_bounds__(256) gemv_t_finish_packed(const double* __restrict__ partial, int64_t ntiles,
                                                            int64_t n, double alpha, double beta,
                                                            uint8_t* __restrict__ y, int64_t incy, int mode) {
  __shared__ double red[8][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t j = int64_t(blockIdx.x) * 32 + lane;
  const double t = tile_column_sum(partial, ntiles, n, j, warp);
  red[warp][lane] = t;
  __syncthreads();
  if (warp == 0 && j < n) {
    double sum = 0.0;
    for (int w = 0; w < 8; ++w) sum += red[w][lane];
    epilogue_packed<KY>(sum, alpha, beta, y + j * incy * KY, mode);
  }
}

// ---- producer/consumer 'N' --------------------------------------------------------------
//
// A persistent block of kPcWarps consumer warps and one producer warp walks
// the (row block, column chunk) tiles tau = blockIdx.x, blockIdx.x + grid, ...
// The producer streams, per stage, SC columns of x1, x2 and of the tile's
// kPcRowsBlock rows into a ring of shared-memory stages with large bulk
// copies, running ahead across tile boundaries; the consumers fold each stage
// from shared memory (kPcRows rows per warp), release it, and at the end of a
// tile reduce and write their rows.  Registers then hold only accumulators,
// the bytes in flight per SM are set by the ring rather than by occupancy,
// and the ring is filled once per block instead of once per tile.

#ifndef FLYTE_PC_WARPS
#define FLYTE_PC_WARPS 8               // consumer warps per block
#endif
#ifndef FLYTE_PC_ROWS
#define FLYTE_PC_ROWS 2                // rows per consumer warp
#endif
#ifndef FLYTE_PC_SMEM
#define FLYTE_PC_SMEM 75000            // ring budget per block, k <= 4: three blocks per SM
#endif
#ifndef FLYTE_PC_SMEM_LARGE_K
#define FLYTE_PC_SMEM_LARGE_K 200000   // ring budget per block, k = 5, 6: one block per SM
#endif
#ifndef FLYTE_PC_SMEM_K78
#define FLYTE_PC_SMEM_K78 110000       // ring budget per block, k = 7, 8: two blocks per SM
#endif
#ifndef FLYTE_PC_UNROLL_FULL
#define FLYTE_PC_UNROLL_FULL 1         // unroll the group loop of a full stage
#endif
#ifndef FLYTE_PC_WARPS_LARGE_K
#define FLYTE_PC_WARPS_LARGE_K 16      // consumer warps per block, k = 5, 6
#endif
#ifndef FLYTE_PC_WARPS_K78
#define FLYTE_PC_WARPS_K78 12          // consumer warps per block, k = 7, 8
#endif

// k > 4 runs one block per SM; warps of one row hide latency better there
// than 8 warps of two rows (k = 5: 0.331 -> 0.302 ms with 16 warps, k = 8:
// 0.387 -> ~0.36 ms with 12), while k <= 4, with three blocks per SM, is faster
// with 8 warps of two rows (k = 3: 0.256 against 0.282 ms with 16 of one).
template <int K>
__host__ __device__ constexpr int pc_warps() {
  return K <= 4 ? FLYTE_PC_WARPS : (K <= 6 ? FLYTE_PC_WARPS_LARGE_K : FLYTE_PC_WARPS_K78);
}
template <int K>
__host__ __device__ constexpr int pc_rows() { return K <= 4 ? FLYTE_PC_ROWS : 1; }
template <int K>
__host__ __device__ constexpr int pc_rows_block() { return pc_warps<K>() * pc_rows<K>(); }
template <int K>
__host__ __device__ constexpr int pc_threads() { return (pc_warps<K>() + 1) * 32; }

template <int K>
__host__ __device__ constexpr int pc_cols() {
  // k = 7, 8 keep 512 columns: two stages of 1024 would not fit in shared memory
  return K <= 4 ? FLYTE_PC_COLS_SMALL_K : (K <= 6 ? FLYTE_PC_COLS_LARGE_K : 512);
}
template <int K>
__host__ __device__ constexpr int pc_stage_bytes() { return 8 * pc_cols<K>() + pc_rows_block<K>() * pc_cols<K>() * K; }
template <int K>
__host__ __device__ constexpr int pc_stages() {
  constexpr int s = (K <= 4 ? FLYTE_PC_SMEM : (K <= 6 ? FLYTE_PC_SMEM_LARGE_K : FLYTE_PC_SMEM_K78)) / pc_stage_bytes<K>();
  return s < 2 ? 2 : (s > 8 ? 8 : s);
}
template <int K>
__host__ __device__ constexpr int pc_smem() { return pc_stages<K>() * pc_stage_bytes<K>() + 16 * pc_stages<K>() + 128; }

template <int BASE, int K, bool LAZY>
__global__ void __launch_bounds__(pc_threads<K>()) gemv_n_pc(
    const uint8_t* __restrict__ A, int64_t lda, int64_t m, int64_t n, const float* __restrict__ x1,
    const float* __restrict__ x2, const double* __restrict__ x, int64_t incx, int64_t chunk_cols,
    int64_t nchunks, double* __restrict__ partial, double alpha, double beta, double* __restrict__ y,
    int64_t incy, int* __restrict__ status, int direct) {
  constexpr int SC = pc_cols<K>();
  constexpr int S = pc_stages<K>();
  constexpr int kStage = pc_stage_bytes<K>();
  constexpr int kRowBytes = SC * K;
  constexpr int kPcWarps = pc_warps<K>();
  constexpr int kPcRows = pc_rows<K>();
  constexpr int kPcRowsBlock = pc_rows_block<K>();
  static_assert(kPcRowsBlock + 2 <= 64, "the producer warp issues at most two copies per lane and stage");
  static_assert(pc_threads<K>() <= 1024, "block too large");
  extern __shared__ __align__(128) uint8_t smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + S * kStage);
  uint64_t* empty = full + S;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t ntiles = ((m + kPcRowsBlock - 1) / kPcRowsBlock) * nchunks;

  if (threadIdx.x == 0) {
    for (int i = 0; i < S; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], kPcWarps);
    }
    mbar_init_fence();
  }
  __syncthreads();

  if (warp == kPcWarps) {
    // producer: every stage of every tile of this block, in order
    uint32_t it = 0;
    bool ok = true;
    for (int64_t tau = blockIdx.x; tau < ntiles && ok; tau += gridDim.x) {
      const int64_t rb0 = (tau / nchunks) * kPcRowsBlock;
      const int64_t cb = (tau % nchunks) * chunk_cols;
      const int64_t ce = min(n, cb + chunk_cols);
      const int64_t cfull = cb + ((ce - cb) >> 7 << 7);   // whole 128-column steps go through the ring
      for (int64_t c0 = cb; c0 < cfull; c0 += SC, ++it) {
        const int st = int(it % S);
        const int cols = int(min(int64_t(SC), cfull - c0));
        if (lane == 0 && it >= S) ok = mbar_wait(&empty[st], ((it / S) - 1) & 1, status);
        ok = __shfl_sync(0xFFFFFFFFu, ok, 0);
        if (!ok) break;
        if (lane == 0) mbar_arrive_expect_tx(&full[st], uint32_t(8 * cols + kPcRowsBlock * cols * K));
        __syncwarp();
        uint8_t* d = smem + st * kStage;
        fence_proxy_async_smem();
#pragma unroll
        for (int c = lane; c < kPcRowsBlock + 2; c += 32) {
          if (c == 0) {
            bulk_g2s(d, x1 + c0, uint32_t(4 * cols), &full[st]);
          } else if (c == 1) {
            bulk_g2s(d + 4 * SC, x2 + c0, uint32_t(4 * cols), &full[st]);
          } else {
            const int r = c - 2;
            const int64_t row = min(rb0 + r, m - 1);
            bulk_g2s(d + 8 * SC + r * kRowBytes, A + (row * lda + c0) * K, uint32_t(cols * K), &full[st]);
          }
        }
      }
    }
    // The copies of the last S stages land before this warp leaves: after a
    // consumer gave up on a wait, nothing else keeps the block alive while
    // they are in flight (in normal operation these waits return at once or
    // when the consumers could proceed anyway).
    if (lane == 0) {
      for (uint32_t j = it > uint32_t(S) ? it - S : 0; j < it; ++j) mbar_wait(&full[j % S], (j / S) & 1, nullptr);
    }
    return;
  }

  // consumer warp: rows rb0 + warp * kPcRows + r of each tile.  After a wait
  // that gave up (the status word is set), the warp waits for nothing more
  // and writes NaN for its rows of this and every later tile, so that the
  // rows it could not compute are visible as such in y.
  uint32_t it = 0;
  bool failed = false;
  for (int64_t tau = blockIdx.x; tau < ntiles; tau += gridDim.x) {
    const int64_t row0 = (tau / nchunks) * kPcRowsBlock + warp * kPcRows;
    const int64_t chunk = tau % nchunks;
    const int64_t cb = chunk * chunk_cols;
    const int64_t ce = min(n, cb + chunk_cols);
    const int64_t ge = ce >> 2;
    const int64_t cfull = cb + ((ce - cb) >> 7 << 7);
    DW2 acc[kPcRows][2];
    uint32_t vmax[kPcRows];
#pragma unroll
    for (int r = 0; r < kPcRows; ++r) {
      vmax[r] = 0u;
      dw2_zero(acc[r][0]);
      dw2_zero(acc[r][1]);
    }
    for (int64_t c0 = cb; c0 < cfull && !failed; c0 += SC, ++it) {
      const int st = int(it % S);
      const bool got = mbar_wait(&full[st], (it / S) & 1, status);
      if (!__all_sync(0xFFFFFFFFu, got)) {   // the producer stops at its next bounded wait
        failed = true;
        break;
      }
      const uint8_t* d = smem + st * kStage;
      const int cols = int(min(int64_t(SC), cfull - c0));
      auto group = [&](int g) {
        const ulonglong2 xa = reinterpret_cast<const ulonglong2*>(d)[g];
        const ulonglong2 xb = reinterpret_cast<const ulonglong2*>(d + 4 * SC)[g];
        const f2 X1[2] = {xa.x, xa.y}, N1[2] = {f2_neg(xa.x), f2_neg(xa.y)}, X2[2] = {xb.x, xb.y};
#pragma unroll
        for (int r = 0; r < kPcRows; ++r) {
          uint32_t w[K];
          lds_group<K>(d + 8 * SC + (warp * kPcRows + r) * kRowBytes + g * 4 * K, w);
          fold_group2<BASE, K, LAZY>(w, X1, N1, X2, acc[r], vmax[r]);
        }
      };
      if (FLYTE_PC_UNROLL_FULL && cols == SC) {
        // a full stage: a fixed number of groups per lane, unrolled
#pragma unroll
        for (int j = 0; j < SC / 128; ++j) group(lane + 32 * j);
      } else {
        for (int g = lane; g < (cols >> 2); g += 32) group(g);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[st]);
    }
    const uint8_t* rowp[kPcRows];
#pragma unroll
    for (int r = 0; r < kPcRows; ++r) rowp[r] = A + min(row0 + r, m - 1) * lda * K;
    for (int64_t g = (cfull >> 2) + lane; g < ge && !failed; g += 32) {
      const ulonglong2 xa = __ldg(reinterpret_cast<const ulonglong2*>(x1) + g);
      const ulonglong2 xb = __ldg(reinterpret_cast<const ulonglong2*>(x2) + g);
      const f2 X1[2] = {xa.x, xa.y}, N1[2] = {f2_neg(xa.x), f2_neg(xa.y)}, X2[2] = {xb.x, xb.y};
#pragma unroll
      for (int r = 0; r < kPcRows; ++r) {
        uint32_t w[K];
        load_group<K>(rowp[r] + g * (4 * K), w);
        fold_group2<BASE, K, LAZY>(w, X1, N1, X2, acc[r], vmax[r]);
      }
    }
    const int64_t j = (ge << 2) + lane;
    if (j < ce && !failed) {
#pragma unroll
      for (int r = 0; r < kPcRows; ++r) {
        const uint64_t q = load_code_bytes<K>(rowp[r] + j * K);
        fold_one2<BASE, K, LAZY>(widen<BASE, K>(q), x1[j], x2[j], acc[r][0], vmax[r]);
      }
    }
#pragma unroll
    for (int r = 0; r < kPcRows; ++r) {
      DW slots[4];
      dw2_slots(acc[r], slots);
      double t = failed ? __longlong_as_double(0x7FF8000000000000ll) : row_total(slots);
      const bool good = failed || (__all_sync(0xFFFFFFFFu, vmax[r] < window_limit<BASE>()) && isfinite(t));
      const int64_t row = row0 + r;
      if (row >= m) break;
      if (!good) {
        const uint8_t* Ar = A + row * lda * K;
        double s2 = 0.0;
        for (int64_t c = cb + lane; c < ce; c += 32)
          s2 = fma(code_to_double<BASE, K>(load_code_bytes<K>(Ar + c * K)), x[c * incx], s2);
        t = warp_sum(s2);
      }
      if (lane == 0) {
        if (direct) {
          y[row * incy] = epilogue(t, alpha, beta, y + row * incy);
        } else {
          partial[row * nchunks + chunk] = t;
        }
      }
    }
  }
}

__global__ void scale_y(double* __restrict__ y, int64_t len, int64_t incy, double beta) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < len; j += stride)
    y[j * incy] = beta == 0.0 ? 0.0 : beta * y[j * incy];
}

// Row tile of gemv T: a multiple of 16 rows in [96, 160], chosen per call so
// that the grid (column blocks x row tiles) fills its last wave of resident
// blocks well: the smallest (waves rounded up) x (rows per tile), ties to the
// larger tile (fewer partial sums).  At 16384 x 16384 fixed tiles measured
// 144 rows (4.8 waves) 1-2.5 % faster than 128 (5.4 waves), 136 (5.1) the
// slowest; allowing up to 256 rows picked 176 there (1 % slower than 144)
// and 208 at 12288 x 12288 (1 % slower than the 144 chosen within 160).
// Defining FLYTE_T_ROW_TILE fixes the tile instead.
#ifndef FLYTE_T_ROW_TILE_MAX
#define FLYTE_T_ROW_TILE_MAX 160
#endif
constexpr int64_t kTRowTileMin = 96, kTRowTileMax = FLYTE_T_ROW_TILE_MAX;

int64_t t_row_tile(int64_t m, int64_t n, int64_t resident) {
#ifdef FLYTE_T_ROW_TILE
  (void)m, (void)n, (void)resident;
  return FLYTE_T_ROW_TILE;
#else
  const int64_t cb = (n + 4 * kTThreads - 1) / (4 * kTThreads);
  int64_t best = kTRowTileMin, best_cost = -1;
  for (int64_t rb = kTRowTileMin; rb <= kTRowTileMax; rb += 16) {
    const int64_t blocks = cb * ((m + rb - 1) / rb);
    const int64_t cost = (blocks + resident - 1) / max(resident, int64_t(1)) * rb;
    if (best_cost < 0 || cost <= best_cost) {
      best_cost = cost;
      best = rb;
    }
  }
  return best;
#endif
}

int64_t align16(int64_t b) { return (b + 15) & ~int64_t(15); }

// Opt a kernel into more than 48 KiB of dynamic shared memory (the attribute
// is per function and device; setting it again is cheap and idempotent).
template <typename Kern>
bool set_smem_once(Kern kern, int bytes) {
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) == cudaSuccess;
}

struct Plan {
  bool fast, lazy;
  int64_t chunk_cols, nchunks;        // N
  int64_t rb, ntiles, fold_rows;      // T
  int64_t off_status, off_x1, off_x2, off_part, bytes;
};

// rb: the 'T' row tile; 0 sizes the plan for the smallest tile (the most
// partial sums), which is what the workspace query reports.
Plan plan_gemv(char trans, int64_t m, int64_t n, int64_t rb = 0) {
  Plan p{};
  const int64_t lenx = trans == 'N' ? n : m;
  p.off_status = 0;                   // int: error bits of the bulk-copy pipeline
  p.off_x1 = 16;
  p.off_x2 = p.off_x1 + align16(4 * lenx);
  p.off_part = p.off_x2 + align16(4 * lenx);
  if (trans == 'N') {
    // Chunks of at most kNChunkCols columns (whole 128-column warp steps),
    // halved while that lets the chains use the lazy accumulator.  Chain: one
    // term per 128-column step (+ one trailing element); double-word tree: 4
    // slots (2 levels) and 5 warp levels; binary64: the chunks.
    // Prefer the widest lazy plan, then the widest fast one.
    p.fast = p.lazy = false;
    bool have = false;
    for (int64_t cmax = kNChunkCols; cmax >= 512 && !p.lazy; cmax /= 2) {
      Plan q = p;
      q.nchunks = (n + cmax - 1) / cmax;
      q.chunk_cols = (((n + q.nchunks - 1) / q.nchunks) + 127) / 128 * 128;
      q.nchunks = (n + q.chunk_cols - 1) / q.chunk_cols;
      const int64_t L = q.chunk_cols / 128 + 1;
      const int64_t D = 2 + 5;
      const int64_t R = q.nchunks + 1;
      q.lazy = dw_lazy_bound_ok(n, L, R, 14, D);
      q.fast = q.lazy || dw_bound_ok(n, L, R, 14, D);
      if (!have || q.lazy || (q.fast && !p.fast)) {
        p = q;
        have = true;
      }
    }
    p.bytes = p.off_part + 8 * m * p.nchunks;   // partial sums (also for one chunk with a packed y)
  } else {
#ifdef FLYTE_T_ROW_TILE
    p.rb = FLYTE_T_ROW_TILE;
#else
    p.rb = rb > 0 ? rb : kTRowTileMin;
#endif
    p.ntiles = (m + p.rb - 1) / p.rb;
    // chain: fold_rows / 2 rows per parity (+ up to kTRowsPerIter trailing
    // rows); double-word: the parity sum and one total per fold (the folds of
    // the tile plus the trailing one); binary64: the tiles in gemv_t_finish
    // (at most ntiles / 8 + 8 additions in a row)
    const int64_t R = p.ntiles / 8 + 8 + 1;
    p.lazy = false;
    p.fast = false;
    p.fold_rows = p.rb;
    auto depth = [&](int64_t f) { return 1 + (p.rb + f - 1) / f + 1; };
    constexpr int64_t kTrail = kTRowsPerIter;   // terms per parity after the last fold (trailing rows)
    for (int64_t f = FLYTE_T_FOLD_MAX; f >= kTRowsPerIter && !p.fast; f /= 2) {
      if (dw_lazy_bound_ok(m, f / 2 + kTrail, R, 14, depth(f))) {
        p.fast = p.lazy = true;
        p.fold_rows = f;
      }
    }
    for (int64_t f = p.rb; f >= kTRowsPerIter && !p.fast; f /= 2) {
      if (dw_bound_ok(m, f / 2 + kTrail, R, 14, depth(f))) {
        p.fast = true;
        p.fold_rows = f;
      }
    }
    p.bytes = p.off_part + 8 * p.ntiles * n;
  }
  return p;
}

}  // namespace

size_t gemv_workspace_bytes(char trans, int64_t m, int64_t n, flyte_fmt f) {
  (void)f;
  return size_t(plan_gemv(trans, m, n).bytes);
}

namespace {

template <int KY>
__global__ void scale_y_packed(uint8_t* __restrict__ y, int64_t len, int64_t incy, double beta, int mode) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < len; j += stride) {
    uint8_t* p = y + j * incy * KY;
    if (beta == 0.0) {
      store_code_bytes<KY>(p, 0);
    } else {
      const double r = beta * code_to_double<FLYTE_F64, KY>(load_code_bytes<KY>(p));
      store_code_bytes<KY>(p, narrow<FLYTE_F64, KY>(uint64_t(__double_as_longlong(r)), mode));
    }
  }
}

// Epilogue launch: y <- alpha t + beta y from the partial sums, as binary64
// (ky == 0) or packed to ky-byte double-based flytes.
flyte_status finish_y(char trans, const double* part, int64_t parts, int64_t len, double alpha, double beta,
                      void* y, int ky, int64_t incy, int mode, cudaStream_t s) {
  const bool N = trans == 'N';
  const unsigned grid = N ? unsigned((len + 255) / 256) : unsigned((len + 31) / 32);
  if (ky == 0) {
    if (N) {
      gemv_n_finish<<<grid, 256, 0, s>>>(part, parts, len, alpha, beta, static_cast<double*>(y), incy);
    } else {
      gemv_t_finish<<<grid, 256, 0, s>>>(part, parts, len, alpha, beta, static_cast<double*>(y), incy);
    }
  } else {
    const flyte_fmt fy{ky, FLYTE_F64};
    return dispatch_fmt(fy, [&]<int BASE, int KY>() -> flyte_status {
      uint8_t* y8 = static_cast<uint8_t*>(y);
      if (N) {
        gemv_n_finish_packed<KY><<<grid, 256, 0, s>>>(part, parts, len, alpha, beta, y8, incy, mode);
      } else {
        gemv_t_finish_packed<KY><<<grid, 256, 0, s>>>(part, parts, len, alpha, beta, y8, incy, mode);
      }
      FLYTE_TRY_LAUNCH("gemv");
      return FLYTE_OK;
    });
  }
  FLYTE_TRY_LAUNCH("gemv");
  return FLYTE_OK;
}

}  // namespace

flyte_status launch_gemv(char trans, int64_t m, int64_t n, double alpha, const void* A, flyte_fmt fa,
                         int64_t lda, const double* x, int64_t incx, double beta, void* yv, int ky, int64_t incy,
                         int mode, void* ws, size_t ws_bytes, cudaStream_t s) {
  const int64_t leny = trans == 'N' ? m : n;
  if (alpha == 0.0) {
    if (beta == 1.0) return FLYTE_OK;
    if (ky == 0) {
      scale_y<<<grid_for(leny, 256), 256, 0, s>>>(static_cast<double*>(yv), leny, incy, beta);
      FLYTE_TRY_LAUNCH("gemv");
      return FLYTE_OK;
    }
    return dispatch_fmt(flyte_fmt{ky, FLYTE_F64}, [&]<int BASE, int KY>() -> flyte_status {
      scale_y_packed<KY><<<grid_for(leny, 256), 256, 0, s>>>(static_cast<uint8_t*>(yv), leny, incy, beta, mode);
      FLYTE_TRY_LAUNCH("gemv");
      return FLYTE_OK;
    });
  }
  Plan p = plan_gemv(trans, m, n);
  if (ws == nullptr || ws_bytes < size_t(p.bytes)) {
    set_error("gemv: workspace of %lld bytes required", (long long)p.bytes);
    return FLYTE_ERR_WORKSPACE;
  }
  if (reinterpret_cast<uintptr_t>(ws) % 16 != 0) {
    set_error("gemv: workspace must be 16-byte aligned");
    return FLYTE_ERR_WORKSPACE;
  }
  uint8_t* w8 = static_cast<uint8_t*>(ws);
  int* status = reinterpret_cast<int*>(w8 + p.off_status);
  float* x1 = reinterpret_cast<float*>(w8 + p.off_x1);
  float* x2 = reinterpret_cast<float*>(w8 + p.off_x2);
  double* part = reinterpret_cast<double*>(w8 + p.off_part);
  const int64_t lenx = trans == 'N' ? n : m;
  // the 'N' kernels write y themselves for one chunk and a binary64 y
  const int direct = (trans == 'N' && p.nchunks == 1 && ky == 0) ? 1 : 0;
  double* y = static_cast<double*>(yv);
  const flyte_status st = dispatch_fmt(fa, [&]<int BASE, int K>() -> flyte_status {
    if (trans == 'T') {
      // the row tile for this grid and the kernel's occupancy (no more partial sums than sized for)
      int per_sm = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gemv_t_kernel<BASE, K, true, false>, kTThreads, 0) !=
          cudaSuccess)
        return cuda_status(cudaGetLastError(), "gemv");
      p = plan_gemv(trans, m, n, t_row_tile(m, n, int64_t(max(per_sm, 1)) * sm_count()));
    }
    constexpr int S = group_bytes(K);
    // rows whose groups are not 4k-byte aligned take the funnel-shift loads (UA kernels)
    const bool ua = !(reinterpret_cast<uintptr_t>(A) % S == 0 && (lda * K) % S == 0);
    const int fast = p.fast ? 1 : 0;
    if (fast) {
      prep_x<<<grid_for(lenx, 256), 256, 0, s>>>(x, lenx, incx, x1, x2, status);
      FLYTE_TRY_LAUNCH("gemv");
    }
    const uint8_t* A8 = static_cast<const uint8_t*>(A);
    // the producer's bulk copies need A and every row start 16-byte aligned
    const bool pc = FLYTE_GEMV_PC && K <= FLYTE_GEMV_PC_KMAX && fast && !ua && reinterpret_cast<uintptr_t>(A) % 16 == 0 &&
                    (lda * K) % 16 == 0;
    if (trans == 'N') {
      dim3 grid(unsigned((m + kNRowsPerBlock - 1) / kNRowsPerBlock), unsigned(p.nchunks));
      if (pc) {
        constexpr int smem = pc_smem<K>();
        constexpr int rows_block = pc_rows_block<K>(), threads = pc_threads<K>();
        const int64_t ntiles = ((m + rows_block - 1) / rows_block) * p.nchunks;
        auto run = [&](auto kern) -> flyte_status {
          if (!set_smem_once(kern, smem)) return cuda_status(cudaGetLastError(), "gemv");
          int per_sm = 0;
          if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem) != cudaSuccess)
            return cuda_status(cudaGetLastError(), "gemv");
          const int64_t blocks = min(ntiles, int64_t(max(per_sm, 1)) * sm_count());
          kern<<<unsigned(blocks), threads, smem, s>>>(A8, lda, m, n, x1, x2, x, incx, p.chunk_cols, p.nchunks,
                                                         part, alpha, beta, y, incy, status, direct);
          return FLYTE_OK;
        };
        const flyte_status st = p.lazy ? run(gemv_n_pc<BASE, K, true>) : run(gemv_n_pc<BASE, K, false>);
        if (st != FLYTE_OK) return st;
      } else {
        auto run = [&](auto kern) {
          kern<<<grid, kNWarps * 32, 0, s>>>(A8, lda, m, n, x1, x2, x, incx, p.chunk_cols, p.nchunks, part, alpha,
                                             beta, y, incy, fast, direct);
        };
        if (ua) {
          p.lazy ? run(gemv_n_kernel<BASE, K, true, true>) : run(gemv_n_kernel<BASE, K, false, true>);
        } else {
          p.lazy ? run(gemv_n_kernel<BASE, K, true, false>) : run(gemv_n_kernel<BASE, K, false, false>);
        }
      }
      FLYTE_TRY_LAUNCH("gemv");
    } else {
      dim3 grid(unsigned((n + 4 * kTThreads - 1) / (4 * kTThreads)), unsigned(p.ntiles));
      auto run = [&](auto kern) {
        kern<<<grid, kTThreads, 0, s>>>(A8, lda, m, n, x1, x2, x, incx, p.rb, p.fold_rows, part, fast);
      };
      if (ua) {
        p.lazy ? run(gemv_t_kernel<BASE, K, true, true>) : run(gemv_t_kernel<BASE, K, false, true>);
      } else {
        p.lazy ? run(gemv_t_kernel<BASE, K, true, false>) : run(gemv_t_kernel<BASE, K, false, false>);
      }
      FLYTE_TRY_LAUNCH("gemv");
    }
    return FLYTE_OK;
  });
  if (st != FLYTE_OK || direct) return st;
  return finish_y(trans, part, trans == 'N' ? p.nchunks : p.ntiles, leny, alpha, beta, yv, ky, incy, mode, s);
}

}  // namespace flyte
