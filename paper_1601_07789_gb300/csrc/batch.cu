// batch.cu -- many uneven jobs of mixed widths as the tiles of one persistent kernel.
//
// flyte_batch_prepare splits each job into tiles (a range of elements, a
// block of gemv rows, or a block of gemv columns) and uploads a job table and
// a tile table into the caller's workspace.  flyte_batch_launch starts a
// small kernel that splits the x of every gemv 'N' job into its binary32 pair
// once, then one persistent kernel of (SMs x resident blocks) blocks; each
// block repeatedly
// takes the next tile from an atomic counter and runs it with all its
// threads, so short and long jobs share the machine without a launch per
// job.  A dot's tiles leave partial sums in the workspace; the block that
// completes a dot's last tile adds them in tile order, so the result does not
// depend on the schedule.  The last block to finish resets the counters, so
// a launch can be replayed from a CUDA graph.  The kernels have no
// inter-block waits.
//
// The arithmetic is that of the single-job kernels: exact widening and
// integer narrowing (flyte_internal.cuh), double-word accumulation for
// in-window data when the host has proven the error bound for the job
// (dwacc.cuh), binary64 FMAs otherwise.  gemv tiles stage x as binary32
// pairs in shared memory ('N' tiles copy the pair split once per launch, 'T'
// tiles split their own rows), which caps the batch gemv sides at 4096.
//
// Tile sizes come from a per-(operation, base, k) table: built-in defaults,
// replaced by the fastest candidates that flyte_batch_autotune measures.
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "axpy_exact.cuh"
#include "load_unaligned.cuh"
#include "dwacc.cuh"

namespace flyte {
namespace {

constexpr int kBThreads = 256;
constexpr int kBWarps = kBThreads / 32;
constexpr int64_t kMaxSide = 4096;          // gemv: x (split) is staged in shared memory
constexpr int kNOps = 5;

struct Item {
  int32_t job, tile;
  int64_t begin, end;                         // elements, rows ('N') or columns ('T')
};

struct JobDev {
  flyte_job j;
  int64_t tiles, part_base;
  int32_t fast;                               // dot/gemv: double-word path proven; unpack/axpy: group path
  int32_t fold_rows;                          // gemv 'T'
  int32_t row_chunks;                         // gemv 'T': row chunks per column block
  int32_t done_base;                          // first completion counter of the job
  int32_t ua;                                 // dot/gemv: groups not 4k-byte aligned (funnel-shift loads)
  int32_t tgroups;                            // gemv 'T': row groups per tile (1, 2, 4, 8, 16)
  int64_t xsplit;                             // gemv N (double-word path): address of its x1, x2 in ws
};

struct Header {
  int32_t njobs, nitems, ndone, pad;
  int64_t off_jobs, off_items, off_parts, off_done, off_xs;
  int32_t counter;   // next tile to take
  int32_t exited;    // blocks that have finished
};

int64_t up256(int64_t b) { return (b + 255) & ~int64_t(255); }

// ---- tile table ----------------------------------------------------------------------------

// tile size per (op, base, k): elements (UNPACK, DOT, AXPY), rows (GEMV_N, and the row chunk of the
// 1024-column 'T' tiles)
std::mutex g_tune_mu;
int64_t g_tile[kNOps][2][9];
bool g_tile_init = false;

int64_t default_tile(int op) {
  switch (op) {
    case FLYTE_JOB_UNPACK: return 65536;
    case FLYTE_JOB_DOT: return 65536;
    case FLYTE_JOB_AXPY: return 65536;
    case FLYTE_JOB_GEMV_N: return 16;
    default: return 256;
  }
}

int64_t tile_for(int op, flyte_fmt f) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  if (!g_tile_init) {
    for (int o = 0; o < kNOps; ++o)
      for (int b = 0; b < 2; ++b)
        for (int k = 0; k < 9; ++k) g_tile[o][b][k] = default_tile(o);
    g_tile_init = true;
  }
  return g_tile[op][f.base][f.k];
}

void set_tile(int op, flyte_fmt f, int64_t t) {
  tile_for(op, f);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tile[op][f.base][f.k] = t;
}

// ---- device helpers -----------------------------------------------------------------------

// f(BASE, K) for a format known at run time (block-uniform).
template <typename F>
__device__ __forceinline__ void with_fmt(flyte_fmt f, F&& fn) {
  if (f.base == FLYTE_F64) {
    switch (f.k) {
      case 1: fn.template operator()<FLYTE_F64, 1>(); break;
      case 2: fn.template operator()<FLYTE_F64, 2>(); break;
      case 3: fn.template operator()<FLYTE_F64, 3>(); break;
      case 4: fn.template operator()<FLYTE_F64, 4>(); break;
      case 5: fn.template operator()<FLYTE_F64, 5>(); break;
      case 6: fn.template operator()<FLYTE_F64, 6>(); break;
      case 7: fn.template operator()<FLYTE_F64, 7>(); break;
      default: fn.template operator()<FLYTE_F64, 8>(); break;
    }
  } else {
    switch (f.k) {
      case 1: fn.template operator()<FLYTE_F32, 1>(); break;
      case 2: fn.template operator()<FLYTE_F32, 2>(); break;
      case 3: fn.template operator()<FLYTE_F32, 3>(); break;
      default: fn.template operator()<FLYTE_F32, 4>(); break;
    }
  }
}

template <int BASE>
__device__ __forceinline__ double native_to_double(typename Native<BASE>::bits u) {
  if constexpr (BASE == FLYTE_F64) {
    return __longlong_as_double((long long)u);
  } else {
    return double(__uint_as_float(u));
  }
}

// binary32 pieces of an element (see dbl_to_pair); false outside the window
template <int BASE, int K>
__device__ __forceinline__ bool pieces(typename Native<BASE>::bits u, float& hi, float& lo) {
  if constexpr (BASE == FLYTE_F64) {
    return dbl_to_pair<K>(uint32_t(u >> 32), uint32_t(u), hi, lo);
  } else {
    hi = __uint_as_float(u);
    lo = 0.f;
    return flt_in_window(u);
  }
}

template <int K>
__device__ __forceinline__ void load_group_any(const uint8_t* p, uint32_t (&w)[K], int ua) {
  if (ua) {
    load_group_unaligned<K>(p, w);
  } else {
    load_group<K>(p, w);
  }
}

// ---- UNPACK -------------------------------------------------------------------------------

template <int BASE, int K>
__device__ void unpack_tile(const JobDev& jd, int64_t b, int64_t e) {
  using Bits = typename Native<BASE>::bits;
  const uint8_t* src = static_cast<const uint8_t*>(jd.j.a);
  Bits* dst = static_cast<Bits*>(jd.j.y);
  int64_t i0 = b;
  if (jd.fast) {
    // b is a multiple of 4; whole groups [b/4, e/4)
    for (int64_t g = b / 4 + threadIdx.x; g < e / 4; g += kBThreads) {
      uint32_t w[K];
      load_group<K>(src + g * (4 * K), w);
#pragma unroll
      for (int q = 0; q < 4; ++q) dst[4 * g + q] = extract_widened<BASE, K>(w, q);
    }
    i0 = e / 4 * 4;
  }
  for (int64_t i = i0 + threadIdx.x; i < e; i += kBThreads) dst[i] = widen<BASE, K>(load_code_bytes<K>(src + i * K));
}

// ---- AXPY ---------------------------------------------------------------------------------

template <int BASE, int K>
__device__ __forceinline__ uint64_t axpy_elem(typename Native<BASE>::bits ux, typename Native<BASE>::bits uy,
                                              double alpha, int mode) {
  if constexpr (BASE == FLYTE_F64) {
    const double r = fma(alpha, __longlong_as_double((long long)ux), __longlong_as_double((long long)uy));
    return narrow<BASE, K>(uint64_t(__double_as_longlong(r)), mode);
  } else {
    const float r = __fmaf_rn(__double2float_rn(alpha), __uint_as_float(ux), __uint_as_float(uy));
    return narrow<BASE, K>(__float_as_uint(r), mode);
  }
}

// Groups [b/4, e/4) with the exact binary32 elements of axpy_exact.cuh (double-based k <= 4, alpha
// in the window; the host sets fast = 2 when alpha is a binary32 number, 3 otherwise), binary64 for
// a group that needs it.
template <int K, int MODE, bool SPLIT>
__device__ void axpy_groups_exact(const JobDev& jd, int64_t b, int64_t e) {
  const uint8_t* X = static_cast<const uint8_t*>(jd.j.a);
  uint8_t* Y = static_cast<uint8_t*>(jd.j.y);
  const float af = __double2float_rn(jd.j.alpha);
  const float a2 = __double2float_rn(jd.j.alpha - double(af));
  const float a3 = __double2float_rn(jd.j.alpha - double(af) - double(a2));
  for (int64_t g = b / 4 + threadIdx.x; g < e / 4; g += kBThreads) {
    uint32_t wx[K], wy[K], wo[K];
    load_group<K>(X + g * (4 * K), wx);
    load_group_rw<K>(Y + g * (4 * K), wy);
#pragma unroll
    for (int j = 0; j < K; ++j) wo[j] = 0;
    uint64_t c[4];
    bool ok = true;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint64_t ux = extract_widened<FLYTE_F64, K>(wx, q), uy = extract_widened<FLYTE_F64, K>(wy, q);
      if constexpr (SPLIT) {
        ok &= axpy_exact_f32x2<K, MODE>(ux, uy, af, a2, a3, c[q]);
      } else {
        ok &= axpy_exact_f32<K, MODE>(ux, uy, af, c[q]);
      }
    }
    if (!ok) {
#pragma unroll
      for (int q = 0; q < 4; ++q)
        c[q] = axpy_elem<FLYTE_F64, K>(extract_widened<FLYTE_F64, K>(wx, q), extract_widened<FLYTE_F64, K>(wy, q),
                                       jd.j.alpha, MODE);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) deposit_code<K>(wo, q, c[q]);
    store_group<K>(Y + g * (4 * K), wo);
  }
}

// y has format (BASE, K); x has the same base and width kx (any)
template <int BASE, int K>
__device__ void axpy_tile(const JobDev& jd, int64_t b, int64_t e) {
  using Bits = typename Native<BASE>::bits;
  constexpr int W = Native<BASE>::W;
  const uint8_t* X = static_cast<const uint8_t*>(jd.j.a);
  uint8_t* Y = static_cast<uint8_t*>(jd.j.y);
  const int kx = jd.j.fx.k;
  int64_t i0 = b;
  if constexpr (BASE == FLYTE_F64 && K >= 2 && K <= 4) {
    if (jd.fast == 2) {
      switch (jd.j.mode) {
        case FLYTE_RNE: axpy_groups_exact<K, FLYTE_RNE, false>(jd, b, e); break;
        case FLYTE_RTZ: axpy_groups_exact<K, FLYTE_RTZ, false>(jd, b, e); break;
        case FLYTE_HALF_UP: axpy_groups_exact<K, FLYTE_HALF_UP, false>(jd, b, e); break;
        default: axpy_groups_exact<K, FLYTE_RTO, false>(jd, b, e); break;
      }
      i0 = e / 4 * 4;
    } else if (jd.fast == 3) {
      switch (jd.j.mode) {
        case FLYTE_RNE: axpy_groups_exact<K, FLYTE_RNE, true>(jd, b, e); break;
        case FLYTE_RTZ: axpy_groups_exact<K, FLYTE_RTZ, true>(jd, b, e); break;
        case FLYTE_HALF_UP: axpy_groups_exact<K, FLYTE_HALF_UP, true>(jd, b, e); break;
        default: axpy_groups_exact<K, FLYTE_RTO, true>(jd, b, e); break;
      }
      i0 = e / 4 * 4;
    }
  }
  if (jd.fast == 1) {
    for (int64_t g = b / 4 + threadIdx.x; g < e / 4; g += kBThreads) {
      uint32_t wx[K], wy[K], wo[K];
      load_group<K>(X + g * (4 * K), wx);
      load_group_rw<K>(Y + g * (4 * K), wy);
#pragma unroll
      for (int j = 0; j < K; ++j) wo[j] = 0;
#pragma unroll
      for (int q = 0; q < 4; ++q)
        deposit_code<K>(wo, q, axpy_elem<BASE, K>(extract_widened<BASE, K>(wx, q), extract_widened<BASE, K>(wy, q),
                                                  jd.j.alpha, jd.j.mode));
      store_group<K>(Y + g * (4 * K), wo);
    }
    i0 = e / 4 * 4;
  }
  for (int64_t i = i0 + threadIdx.x; i < e; i += kBThreads) {
    const uint64_t qx = load_code_bytes_rt(X + i * kx, kx);
    const Bits ux = kx * 8 == W ? Bits(qx) : Bits(qx << (W - 8 * kx));
    uint8_t* py = Y + i * K;
    store_code_bytes<K>(py, axpy_elem<BASE, K>(ux, widen<BASE, K>(load_code_bytes<K>(py)), jd.j.alpha, jd.j.mode));
  }
}

// ---- DOT ----------------------------------------------------------------------------------

// Partial sum of x_i y_i over [b, e) for equal formats (BASE, K); every thread returns its share.
template <int BASE, int K>
__device__ double dot_share(const JobDev& jd, int64_t b, int64_t e) {
  const uint8_t* X = static_cast<const uint8_t*>(jd.j.a);
  const uint8_t* Y = static_cast<const uint8_t*>(jd.j.y);
  DW acc[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) dw_zero(acc[q]);
  double acc64 = 0.0;
  int64_t i0 = b;
  if (jd.fast) {
    for (int64_t g = b / 4 + threadIdx.x; g < e / 4; g += kBThreads) {
      uint32_t wx[K], wy[K];
      load_group_any<K>(X + g * (4 * K), wx, jd.ua);
      load_group_any<K>(Y + g * (4 * K), wy, jd.ua);
      typename Native<BASE>::bits ux[4], uy[4];
      bool ok = true;
      float p[4], s[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        ux[q] = extract_widened<BASE, K>(wx, q);
        uy[q] = extract_widened<BASE, K>(wy, q);
        float xh, xl, yh, yl;
        ok &= pieces<BASE, K>(ux[q], xh, xl);
        ok &= pieces<BASE, K>(uy[q], yh, yl);
        pair_times_pair(xh, xl, yh, yl, p[q], s[q]);
      }
      if (ok) {
#pragma unroll
        for (int q = 0; q < 4; ++q) dw_add(acc[q], p[q], s[q]);
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) acc64 = fma(native_to_double<BASE>(ux[q]), native_to_double<BASE>(uy[q]), acc64);
      }
    }
    i0 = e / 4 * 4;
  }
  for (int64_t i = i0 + threadIdx.x; i < e; i += kBThreads)
    acc64 = fma(code_to_double<BASE, K>(load_code_bytes<K>(X + i * K)),
                code_to_double<BASE, K>(load_code_bytes<K>(Y + i * K)), acc64);
  double v = acc64;
#pragma unroll
  for (int q = 0; q < 4; ++q) v += dw_value(acc[q]);
  return v;
}

// mixed formats: binary64 FMAs over the raw bytes
__device__ double dot_share_generic(const JobDev& jd, int64_t b, int64_t e) {
  const uint8_t* X = static_cast<const uint8_t*>(jd.j.a);
  const uint8_t* Y = static_cast<const uint8_t*>(jd.j.y);
  const flyte_fmt fx = jd.j.fx, fy = jd.j.fy;
  double acc = 0.0;
  for (int64_t i = b + threadIdx.x; i < e; i += kBThreads)
    acc = fma(code_to_double_rt(load_code_bytes_rt(X + i * fx.k, fx.k), fx.k, fx.base),
              code_to_double_rt(load_code_bytes_rt(Y + i * fy.k, fy.k), fy.k, fy.base), acc);
  return acc;
}

// ---- GEMV ---------------------------------------------------------------------------------

// x1 = RN32(x), x2 = RN32(x - x1) for x = 0 or 2^-40 <= |x| < 2^40; else x1 = NaN (marks the job's
// tile for the binary64 path), as prep_x of the single-job gemv.
__device__ void split_x(const double* __restrict__ x, int64_t len, float* x1, float* x2) {
  for (int64_t j = threadIdx.x; j < len; j += kBThreads) {
    const double v = x[j];
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

// Elements [b, e) of a job's split x (x1 at xg, x2 at xg + len, written by batch_split_x) into the
// tile's shared x1, x2.
__device__ __forceinline__ void stage_x(const float* __restrict__ xg, int64_t len, int64_t b, int64_t e, float* x1,
                                        float* x2) {
  for (int64_t j = b + threadIdx.x; j < e; j += kBThreads) {
    x1[j - b] = xg[j];
    x2[j - b] = xg[len + j];
  }
}

template <int BASE, int K>
__device__ __forceinline__ void fold_elem(typename Native<BASE>::bits u, float x1, float x2, DW& acc, bool& ok) {
  float hi, lo, p, e;
  ok &= pieces<BASE, K>(u, hi, lo);
  pair_times_x(hi, lo, x1, x2, p, e);
  dw_add(acc, p, e);
}

__device__ __forceinline__ double gemv_epilogue(double t, double alpha, double beta, const double* yp) {
  return beta == 0.0 ? alpha * t : fma(alpha, t, beta * *yp);
}

// Rows [r0, r1) of y <- alpha A x + beta y: warp w takes rows r0 + w, r0 + w + 8, ...
template <int BASE, int K>
__device__ void gemv_n_tile(const JobDev& jd, int64_t r0, int64_t r1, float* x1, float* x2) {
  const int64_t n = jd.j.n;
  const uint8_t* A = static_cast<const uint8_t*>(jd.j.a);
  const double* x = jd.j.xv;
  double* y = static_cast<double*>(jd.j.y);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (jd.fast) {
    stage_x(reinterpret_cast<const float*>(jd.xsplit), n, 0, n, x1, x2);
    __syncthreads();
  }
  for (int64_t r = r0 + warp; r < r1; r += kBWarps) {
    const uint8_t* Ar = A + r * n * K;
    double t = 0.0;
    bool good = false;
    if (jd.fast) {
      DW acc[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) dw_zero(acc[q]);
      bool ok = true;
      for (int64_t g = lane; g < n / 4; g += 32) {
        uint32_t w[K];
        load_group_any<K>(Ar + g * (4 * K), w, jd.ua);
#pragma unroll
        for (int q = 0; q < 4; ++q)
          fold_elem<BASE, K>(extract_widened<BASE, K>(w, q), x1[4 * g + q], x2[4 * g + q], acc[q], ok);
      }
      for (int64_t c = n / 4 * 4 + lane; c < n; c += 32)
        fold_elem<BASE, K>(widen<BASE, K>(load_code_bytes<K>(Ar + c * K)), x1[c], x2[c], acc[0], ok);
      if (jd.fast == 1) {
        // long rows: double-word tree, one conversion
        const DW s = dw_warp_sum(dw_sum4(acc[0], acc[1], acc[2], acc[3]));
        t = __shfl_sync(0xFFFFFFFFu, dw_value(s), 0);
      } else {
        // short rows: the four slots and the warp reduced in binary64 (a tighter bound)
        t = warp_sum(dw_value(acc[0]) + dw_value(acc[1]) + dw_value(acc[2]) + dw_value(acc[3]));
      }
      good = __all_sync(0xFFFFFFFFu, ok) && isfinite(t);
    }
    if (!good) {
      double s2 = 0.0;
      for (int64_t c = lane; c < n; c += 32) s2 = fma(code_to_double<BASE, K>(load_code_bytes<K>(Ar + c * K)), x[c], s2);
      t = warp_sum(s2);
    }
    if (lane == 0) y[r] = gemv_epilogue(t, jd.j.alpha, jd.j.beta, y + r);
  }
}

// Tile (column block cb, row chunk rc) of y <- alpha A^T x + beta y: thread t owns columns
// 1024 cb + 4t .. + 3 over rows [r0, r1) and writes their partial sums; the block that completes the
// column block's last row chunk adds the chunks in order and applies the epilogue.
template <int BASE, int K>
__device__ void gemv_t_tile(const JobDev& jd, int tile, int64_t r0, int64_t r1, float* x1, float* x2,
                            double* parts, int* done, int* s_last) {
  const int64_t n = jd.j.n;
  const uint8_t* A = static_cast<const uint8_t*>(jd.j.a);
  const double* x = jd.j.xv;
  double* y = static_cast<double*>(jd.j.y);
  const int nrc = jd.row_chunks;
  const int cb = tile / nrc, rc = tile % nrc;
  // G row groups of nthr threads: a narrow matrix (n below 4 x 256 columns) keeps every thread busy
  // by giving each group an even share of the chunk's rows; group 0 adds the groups' sums in order
  const int G = jd.tgroups, nthr = kBThreads / G;
  const int tg = threadIdx.x / nthr, tc = threadIdx.x % nthr;
  const int64_t c0 = int64_t(cb) * (4 * nthr);
  if (jd.fast) {
    split_x(x + r0, r1 - r0, x1, x2);
    __syncthreads();
  }
  const int64_t sub = ((r1 - r0 + G - 1) / G + 1) & ~int64_t(1);
  const int64_t ra = min(r1, r0 + tg * sub), rb = min(r1, ra + sub);
  const int64_t c = c0 + 4 * tc;
  const int nc = int(max(int64_t(0), min(int64_t(4), n - c)));
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  bool ok = jd.fast && nc == 4;
  if (ok) {
    DW acc[2][4];
#pragma unroll
    for (int q = 0; q < 4; ++q) dw_zero(acc[0][q]), dw_zero(acc[1][q]);
    const uint8_t* colp = A + c * K;
    int since = 0;
    int64_t i = ra;
    // two rows per step, both loads in flight before the folds (the chains, their order and the
    // fold points are those of the one-row loop below: fold_rows is even)
    for (; i + 1 < rb; i += 2) {
      uint32_t w0[K], w1[K];
      load_group_any<K>(colp + i * n * K, w0, jd.ua);
      load_group_any<K>(colp + (i + 1) * n * K, w1, jd.ua);
      const float a1 = x1[i - r0], a2 = x2[i - r0], b1 = x1[i + 1 - r0], b2 = x2[i + 1 - r0];
#pragma unroll
      for (int q = 0; q < 4; ++q) fold_elem<BASE, K>(extract_widened<BASE, K>(w0, q), a1, a2, acc[i & 1][q], ok);
#pragma unroll
      for (int q = 0; q < 4; ++q)
        fold_elem<BASE, K>(extract_widened<BASE, K>(w1, q), b1, b2, acc[(i + 1) & 1][q], ok);
      since += 2;
      if (since == jd.fold_rows) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          v[q] += dw_value(acc[0][q]) + dw_value(acc[1][q]);
          dw_zero(acc[0][q]);
          dw_zero(acc[1][q]);
        }
        since = 0;
      }
    }
    for (; i < rb; ++i) {
      uint32_t w[K];
      load_group_any<K>(colp + i * n * K, w, jd.ua);
      const float a1 = x1[i - r0], a2 = x2[i - r0];
#pragma unroll
      for (int q = 0; q < 4; ++q) fold_elem<BASE, K>(extract_widened<BASE, K>(w, q), a1, a2, acc[i & 1][q], ok);
      if (++since == jd.fold_rows) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          v[q] += dw_value(acc[0][q]) + dw_value(acc[1][q]);
          dw_zero(acc[0][q]);
          dw_zero(acc[1][q]);
        }
        since = 0;
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      v[q] += dw_value(acc[0][q]) + dw_value(acc[1][q]);
      ok = ok && isfinite(v[q]);
    }
  }
  if (!ok) {
    for (int q = 0; q < nc; ++q) {
      double s2 = 0.0;
      for (int64_t i = ra; i < rb; ++i)
        s2 = fma(code_to_double<BASE, K>(load_code_bytes<K>(A + (i * n + c + q) * K)), x[i], s2);
      v[q] = s2;
    }
  }
  if (G > 1) {
    // the groups' sums through shared memory (above the tile's x1: at most 1024 rows), in group order
    double* pp = reinterpret_cast<double*>(x1 + 1024);
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) pp[4 * threadIdx.x + q] = v[q];
    __syncthreads();
    if (tg == 0) {
      for (int g2 = 1; g2 < G; ++g2) {
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] += pp[4 * (g2 * nthr + tc) + q];
      }
    }
  }
  double* mine = parts + jd.part_base + (int64_t(cb) * nrc + rc) * (4 * kBThreads) + 4 * tc;
  if (tg == 0)
    for (int q = 0; q < nc; ++q) mine[q] = v[q];
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) *s_last = atomicAdd(&done[jd.done_base + cb], 1) == nrc - 1;
  __syncthreads();
  if (*s_last && tg == 0) {
    __threadfence();
    const double* col = parts + jd.part_base + int64_t(cb) * nrc * (4 * kBThreads) + 4 * tc;
    for (int q = 0; q < nc; ++q) {
      double t = 0.0;
      for (int r = 0; r < nrc; ++r) t += __ldcg(col + int64_t(r) * (4 * kBThreads) + q);
      y[c + q] = gemv_epilogue(t, jd.j.alpha, jd.j.beta, y + c + q);
    }
  }
}

// ---- x of the gemv jobs, split once per launch -------------------------------------------

// x1, x2 of every gemv N job on the double-word path, into the workspace (x1 then x2, n each),
// before the persistent kernel: its row tiles copy them instead of each splitting the whole x again
// (the splitting runs on the binary64 pipe; tiles of 16-32 rows repeated it for every tile).  'T'
// tiles split only their own rows of x, a small share of their work, and keep doing so.
__global__ void __launch_bounds__(kBThreads) batch_split_x(uint8_t* __restrict__ ws) {
  const Header* h = reinterpret_cast<const Header*>(ws);
  const JobDev* jobs = reinterpret_cast<const JobDev*>(ws + h->off_jobs);
  for (int i = blockIdx.x; i < h->njobs; i += gridDim.x) {
    const JobDev& jd = jobs[i];
    if (jd.j.op != FLYTE_JOB_GEMV_N || !jd.fast || jd.tiles == 0) continue;
    float* x1 = reinterpret_cast<float*>(jd.xsplit);
    split_x(jd.j.xv, jd.j.n, x1, x1 + jd.j.n);
  }
}

// ---- the persistent kernel ----------------------------------------------------------------

__global__ void __launch_bounds__(kBThreads, 4) batch_kernel(uint8_t* __restrict__ ws) {
  extern __shared__ __align__(16) float xs[];   // x1, x2 of the current gemv tile
  __shared__ int s_item, s_last;
  __shared__ double s_red[kBWarps];
  Header* h = reinterpret_cast<Header*>(ws);
  const JobDev* jobs = reinterpret_cast<const JobDev*>(ws + h->off_jobs);
  const Item* items = reinterpret_cast<const Item*>(ws + h->off_items);
  double* parts = reinterpret_cast<double*>(ws + h->off_parts);
  int* done = reinterpret_cast<int*>(ws + h->off_done);
  const int nitems = h->nitems;
  if (blockIdx.x == 0) {
    // a dot of length 0 has no tile: its result is written here
    for (int i = threadIdx.x; i < h->njobs; i += kBThreads)
      if (jobs[i].j.op == FLYTE_JOB_DOT && jobs[i].tiles == 0) *jobs[i].j.result = 0.0;
  }
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(&h->counter, 1);
    __syncthreads();
    const int it = s_item;
    __syncthreads();
    if (it >= nitems) break;
    const Item item = items[it];
    const JobDev& jd = jobs[item.job];
    const int op = jd.j.op;
    if (op == FLYTE_JOB_UNPACK) {
      with_fmt(jd.j.fx, [&]<int B, int K>() { unpack_tile<B, K>(jd, item.begin, item.end); });
    } else if (op == FLYTE_JOB_AXPY) {
      with_fmt(jd.j.fy, [&]<int B, int K>() { axpy_tile<B, K>(jd, item.begin, item.end); });
    } else if (op == FLYTE_JOB_DOT) {
      double v = 0.0;
      if (jd.j.fx.k == jd.j.fy.k && jd.j.fx.base == jd.j.fy.base) {
        with_fmt(jd.j.fx, [&]<int B, int K>() { v = dot_share<B, K>(jd, item.begin, item.end); });
      } else {
        v = dot_share_generic(jd, item.begin, item.end);
      }
      v = block_sum(v, s_red);
      if (threadIdx.x == 0) {
        parts[jd.part_base + item.tile] = v;
        __threadfence();
        if (atomicAdd(&done[jd.done_base], 1) == int(jd.tiles) - 1) {
          __threadfence();
          double s = 0.0;
          for (int64_t t = 0; t < jd.tiles; ++t) s += __ldcg(&parts[jd.part_base + t]);
          *jd.j.result = s;
        }
      }
    } else if (op == FLYTE_JOB_GEMV_N) {
      with_fmt(jd.j.fx, [&]<int B, int K>() { gemv_n_tile<B, K>(jd, item.begin, item.end, xs, xs + kMaxSide); });
    } else {
      with_fmt(jd.j.fx, [&]<int B, int K>() {
        gemv_t_tile<B, K>(jd, item.tile, item.begin, item.end, xs, xs + kMaxSide, parts, done, &s_last);
      });
    }
    __syncthreads();   // shared x and s_red are reused by the next tile
  }
  // The last block to finish resets the counters for the next launch (every
  // other block has taken its last tile and finished it by then).
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&h->exited, 1) == int(gridDim.x) - 1) {
      for (int i = 0; i < h->ndone; ++i) done[i] = 0;
      h->counter = 0;
      __threadfence();
      h->exited = 0;
    }
  }
}

constexpr int kBatchSmem = 2 * kMaxSide * 4;   // x1, x2

// ---- planning -------------------------------------------------------------------------------

bool aligned_to(const void* p, int b) { return reinterpret_cast<uintptr_t>(p) % b == 0; }

struct Plan {
  std::vector<JobDev> jobs;
  std::vector<Item> items;
  int64_t nparts = 0;
  int32_t ndone = 0;
  int64_t bytes = 0;
  Header hdr{};
};

flyte_status check_job(const flyte_job& j, int idx) {
  auto bad = [&](const char* what) {
    set_error("batch job %d: %s", idx, what);
    return FLYTE_ERR_INVALID_ARG;
  };
  if (j.op < FLYTE_JOB_UNPACK || j.op > FLYTE_JOB_GEMV_T) return bad("unknown op");
  if (!valid_fmt(j.fx)) return bad("format fx");
  if ((j.op == FLYTE_JOB_DOT || j.op == FLYTE_JOB_AXPY) && !valid_fmt(j.fy)) return bad("format fy");
  if (j.n < 0 || ((j.op == FLYTE_JOB_GEMV_N || j.op == FLYTE_JOB_GEMV_T) && j.m < 0)) return bad("negative size");
  if (j.op == FLYTE_JOB_AXPY) {
    if (j.fx.base != j.fy.base) {
      set_error("batch job %d: axpy x and y must share the base", idx);
      return FLYTE_ERR_UNSUPPORTED;
    }
    if (j.mode < FLYTE_RNE || j.mode > FLYTE_RTO) return bad("rounding mode");
  }
  if (j.op == FLYTE_JOB_GEMV_N || j.op == FLYTE_JOB_GEMV_T) {
    const int64_t lenx = j.op == FLYTE_JOB_GEMV_N ? j.n : j.m;
    if (lenx > kMaxSide) {
      set_error("batch job %d: gemv x longer than %lld (use flyte_gemv)", idx, (long long)kMaxSide);
      return FLYTE_ERR_UNSUPPORTED;
    }
  }
  const bool empty = j.n == 0 || ((j.op == FLYTE_JOB_GEMV_N || j.op == FLYTE_JOB_GEMV_T) && j.m == 0);
  if (!empty && (!j.a || !j.y)) return bad("null pointer");
  if (!empty && j.op == FLYTE_JOB_DOT && !j.result) return bad("null result");
  if (!empty && (j.op == FLYTE_JOB_GEMV_N || j.op == FLYTE_JOB_GEMV_T) && !j.xv) return bad("null x");
  return FLYTE_OK;
}

flyte_status make_plan(const flyte_job* jobs, int njobs, Plan& p) {
  if (njobs < 0 || (njobs > 0 && !jobs)) {
    set_error("batch: bad job list");
    return FLYTE_ERR_INVALID_ARG;
  }
  for (int i = 0; i < njobs; ++i) {
    const flyte_status st = check_job(jobs[i], i);
    if (st != FLYTE_OK) return st;
  }
  p.jobs.resize(size_t(njobs));
  for (int i = 0; i < njobs; ++i) {
    const flyte_job& j = jobs[i];
    JobDev& d = p.jobs[size_t(i)];
    std::memset(&d, 0, sizeof(d));
    d.j = j;
    const int op = j.op;
    const int64_t tile = tile_for(op, op == FLYTE_JOB_AXPY ? j.fy : j.fx);
    auto add_items = [&](int64_t total, int64_t step) {
      int32_t t = 0;
      for (int64_t b = 0; b < total; b += step, ++t) p.items.push_back(Item{i, t, b, std::min(total, b + step)});
      d.tiles = t;
    };
    if (op == FLYTE_JOB_GEMV_N || op == FLYTE_JOB_GEMV_T) {
      if (j.m == 0 || j.n == 0) continue;
      const int K = j.fx.k;
      // rows whose groups are not 4k-byte aligned are read with funnel-shift loads
      d.ua = !(aligned_to(j.a, group_bytes(K)) && (j.n * K) % group_bytes(K) == 0);
      if (op == FLYTE_JOB_GEMV_N) {
        // chains of n/128 + 1 terms per slot; then a double-word tree (2 + 5 levels, one binary64
        // step) or, for rows too short for its bound, binary64 (3 + 5 levels)
        const int64_t L = j.n / 128 + 2;
        d.fast = dw_bound_ok(j.n, L, 1, 14, 7) ? 1 : (dw_bound_ok(j.n, L, 9, 14) ? 2 : 0);
        add_items(j.m, tile);
      } else {
        // tiles: 1024-column blocks x chunks of `tile` rows; parity chains of fold/2 + 1 terms folded
        // into binary64 every fold rows; binary64 levels: the folds of a chunk, then the chunks in order
        const int64_t rows = std::max<int64_t>(4, tile);
        const int64_t nrc = (j.m + rows - 1) / rows;
        // threads per row group: 4 columns each, a power of two covering n (at least 16); the
        // block's other threads take further shares of the chunk's rows (chunks of <= 1024 rows)
        int64_t nthr = kBThreads;
        while (rows <= 1024 && nthr > 16 && 4 * (nthr / 2) >= j.n) nthr /= 2;
        const int64_t G = kBThreads / nthr;
        d.tgroups = int32_t(G);
        const int64_t ncb = (j.n + 4 * nthr - 1) / (4 * nthr);
        d.fast = 0;
        d.fold_rows = 64;
        for (int64_t f = 64; f >= 2; f /= 2) {
          // + G: the groups' sums added in binary64
          if (dw_bound_ok(j.m, f / 2 + 1, 2 * (rows / f) + 4 + nrc + G, 14)) {
            d.fast = 1;
            d.fold_rows = int32_t(f);
            break;
          }
        }
        d.row_chunks = int32_t(nrc);
        int32_t t = 0;
        for (int64_t cb = 0; cb < ncb; ++cb)
          for (int64_t rc = 0; rc < nrc; ++rc, ++t)
            p.items.push_back(Item{i, t, rc * rows, std::min(j.m, (rc + 1) * rows)});
        d.tiles = t;
        d.part_base = p.nparts;
        p.nparts += ncb * nrc * 4 * kBThreads;
        d.done_base = p.ndone;
        p.ndone += int32_t(ncb);
      }
    } else {
      if (j.n == 0) continue;
      const int64_t step = (tile + 3) / 4 * 4;
      if (op == FLYTE_JOB_UNPACK) {
        d.fast = aligned_to(j.a, group_bytes(j.fx.k)) && aligned_to(j.y, j.fx.base == FLYTE_F64 ? 8 : 4);
      } else if (op == FLYTE_JOB_AXPY) {
        d.fast = j.fx.k == j.fy.k && aligned_to(j.a, group_bytes(j.fy.k)) && aligned_to(j.y, group_bytes(j.fy.k));
        // alpha inside the window, double-based k = 2..4: the exact binary32 paths (2: alpha is a
        // binary32 number, 3: two binary32 parts)
        if (d.fast && j.fy.base == FLYTE_F64 && j.fy.k >= 2 && j.fy.k <= 4 && std::fabs(j.alpha) >= 0x1p-40 &&
            std::fabs(j.alpha) < 0x1p40)
          d.fast = double(float(j.alpha)) == j.alpha ? 2 : 3;
      } else {
        // per thread: 4 slots, (step / 4) / threads groups each; block sum (3 + 5 levels) and the tiles
        const int64_t L = step / (4 * kBThreads) + 1;
        const int64_t tiles = (j.n + step - 1) / step;
        d.fast = j.fx.k == j.fy.k && j.fx.base == j.fy.base && dw_bound_ok(j.n, L, 4 + 8 + tiles + 1, 20);
        d.ua = !(aligned_to(j.a, group_bytes(j.fx.k)) && aligned_to(j.y, group_bytes(j.fx.k)));
      }
      add_items(j.n, step);
      if (op == FLYTE_JOB_DOT) {
        d.part_base = p.nparts;
        p.nparts += d.tiles;
        d.done_base = p.ndone;
        p.ndone += 1;
      }
    }
  }
  p.hdr.njobs = njobs;
  p.hdr.nitems = int32_t(p.items.size());
  p.hdr.ndone = p.ndone;
  p.hdr.off_jobs = 256;
  p.hdr.off_items = p.hdr.off_jobs + up256(int64_t(sizeof(JobDev)) * njobs);
  p.hdr.off_parts = p.hdr.off_items + up256(int64_t(sizeof(Item)) * int64_t(p.items.size()));
  p.hdr.off_done = p.hdr.off_parts + up256(8 * p.nparts);
  // x1, x2 (binary32) of each gemv N job on the double-word path
  int64_t xs = 0;
  for (JobDev& d : p.jobs) {
    if (d.j.op != FLYTE_JOB_GEMV_N || !d.fast || d.tiles == 0) continue;
    d.xsplit = xs;   // an offset from off_xs here; flyte_batch_prepare makes it an address
    xs += (8 * d.j.n + 15) / 16 * 16;
  }
  p.hdr.off_xs = p.hdr.off_done + up256(4 * int64_t(p.ndone));
  p.bytes = p.hdr.off_xs + up256(xs);
  return FLYTE_OK;
}

// Resident blocks per SM the persistent grid uses: the occupancy limit, or fewer when the
// autotuner measured fewer to be faster (g_tuned_per_sm > 0).
int g_tuned_per_sm = 0;

int max_blocks_per_sm() {
  static int per_sm = -1;
  if (per_sm < 0) {
    int v = 0;
    cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kBatchSmem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, batch_kernel, kBThreads, kBatchSmem) != cudaSuccess) v = 1;
    per_sm = v < 1 ? 1 : v;
  }
  return per_sm;
}

int blocks_per_sm() {
  const int mx = max_blocks_per_sm();
  std::lock_guard<std::mutex> lk(g_tune_mu);
  return g_tuned_per_sm > 0 && g_tuned_per_sm < mx ? g_tuned_per_sm : mx;
}

int batch_blocks() { return blocks_per_sm() * sm_count(); }

}  // namespace

size_t batch_workspace_bytes(const flyte_job* jobs, int njobs) {
  Plan p;
  if (make_plan(jobs, njobs, p) != FLYTE_OK) return size_t(-1);
  return size_t(p.bytes);
}

flyte_status batch_prepare(const flyte_job* jobs, int njobs, void* ws, size_t ws_bytes, cudaStream_t s) {
  Plan p;
  const flyte_status st = make_plan(jobs, njobs, p);
  if (st != FLYTE_OK) return st;
  if (ws == nullptr || ws_bytes < size_t(p.bytes) || reinterpret_cast<uintptr_t>(ws) % 256 != 0) {
    set_error("batch: workspace of %lld bytes (256-byte aligned) required", (long long)p.bytes);
    return FLYTE_ERR_WORKSPACE;
  }
  // the gemv N jobs' split-x slots as addresses inside ws
  for (JobDev& d : p.jobs) {
    if (d.j.op == FLYTE_JOB_GEMV_N && d.fast && d.tiles > 0)
      d.xsplit = int64_t(reinterpret_cast<uintptr_t>(ws)) + p.hdr.off_xs + d.xsplit;
  }
  // header, jobs and tiles; the dot partials need no initial value; done counters start at 0
  std::vector<uint8_t> host(size_t(p.bytes), 0);
  std::memcpy(host.data(), &p.hdr, sizeof(Header));
  if (!p.jobs.empty()) std::memcpy(host.data() + p.hdr.off_jobs, p.jobs.data(), sizeof(JobDev) * p.jobs.size());
  if (!p.items.empty()) std::memcpy(host.data() + p.hdr.off_items, p.items.data(), sizeof(Item) * p.items.size());
  if (cudaMemcpyAsync(ws, host.data(), host.size(), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return cuda_status(cudaGetLastError(), "batch");
  return FLYTE_OK;
}

flyte_status batch_launch(void* ws, cudaStream_t s) {
  if (ws == nullptr || reinterpret_cast<uintptr_t>(ws) % 256 != 0) {
    set_error("batch: workspace must be the prepared, 256-byte aligned buffer");
    return FLYTE_ERR_WORKSPACE;
  }
  const int blocks = batch_blocks();
  batch_split_x<<<2 * sm_count(), kBThreads, 0, s>>>(static_cast<uint8_t*>(ws));
  FLYTE_TRY_LAUNCH("batch");
  batch_kernel<<<blocks, kBThreads, kBatchSmem, s>>>(static_cast<uint8_t*>(ws));
  FLYTE_TRY_LAUNCH("batch");
  return FLYTE_OK;
}

// ---- autotuning ----------------------------------------------------------------------------

namespace {

// Codes of in-window values (|v| in [1, 2) with random sign and mantissa) so that the timed path is
// the double-word one, as for typical data.
__global__ void fill_codes(uint8_t* p, int64_t n, int k, int base, uint32_t seed) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
    uint64_t r = uint64_t(i) * 0x9E3779B97F4A7C15ull + seed;
    r ^= r >> 29;
    r *= 0xBF58476D1CE4E5B9ull;
    r ^= r >> 32;
    const int bits = 8 * k;
    const int ebits = base == FLYTE_F64 ? 11 : 8;
    const uint64_t bias = base == FLYTE_F64 ? 1023 : 127;
    uint64_t code;
    if (bits > 1 + ebits) {
      const int mbits = bits - 1 - ebits;
      code = ((r >> 63) << (bits - 1)) | (bias << mbits) | (r & ((uint64_t(1) << mbits) - 1));
    } else {
      code = (r >> 63) << (bits - 1) | (bias >> (ebits + 1 - bits));   // k = 1: the exponent's top bits
    }
    for (int b = 0; b < k; ++b) p[i * k + b] = uint8_t(code >> (8 * b));
  }
}

__global__ void fill_ones(double* p, int64_t n) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) p[i] = 1.0 + 1e-3 * double(i % 97);
}

constexpr int64_t kTuneJobs = 16;
constexpr int64_t kTuneLen = int64_t(1) << 18;   // elements per streaming job
constexpr int64_t kTuneSide = 1024;               // gemv jobs: 1024 x 1024
constexpr int64_t kTuneData = 2 * kTuneJobs * kTuneLen * 8 + kTuneJobs * kTuneLen * 8;   // x, y streams, outputs
constexpr int64_t kTuneWs = int64_t(8) << 20;

}  // namespace

size_t batch_autotune_bytes() { return size_t(kTuneData + kTuneWs + 4096); }

flyte_status batch_autotune(void* ws, size_t ws_bytes, cudaStream_t s) {
  if (ws == nullptr || ws_bytes < batch_autotune_bytes() || reinterpret_cast<uintptr_t>(ws) % 256 != 0) {
    set_error("batch autotune: %zu bytes of 256-byte aligned scratch required", batch_autotune_bytes());
    return FLYTE_ERR_WORKSPACE;
  }
  uint8_t* w8 = static_cast<uint8_t*>(ws);
  uint8_t* xs = w8;                                        // x streams (or A), up to 8 bytes per element
  uint8_t* ys = xs + kTuneJobs * kTuneLen * 8;             // y streams (or gemv x, y)
  uint8_t* out = ys + kTuneJobs * kTuneLen * 8;            // unpack outputs, dot results
  uint8_t* bws = out + kTuneJobs * kTuneLen * 8;           // batch workspace
  const flyte_fmt fmts[12] = {{1, 1}, {2, 1}, {3, 1}, {4, 1}, {5, 1}, {6, 1}, {7, 1}, {8, 1},
                              {1, 0}, {2, 0}, {3, 0}, {4, 0}};
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return cuda_status(cudaGetLastError(), "batch autotune");
  flyte_status result = FLYTE_OK;
  for (int op : {FLYTE_JOB_UNPACK, FLYTE_JOB_DOT, FLYTE_JOB_AXPY, FLYTE_JOB_GEMV_N, FLYTE_JOB_GEMV_T}) {
    for (const flyte_fmt& f : fmts) {
      const bool gemv = op == FLYTE_JOB_GEMV_N || op == FLYTE_JOB_GEMV_T;
      const int64_t len = gemv ? kTuneSide * kTuneSide : kTuneLen;
      const int64_t njob = gemv ? (kTuneJobs * kTuneLen * 8) / (len * f.k) : kTuneJobs;
      fill_codes<<<grid_for(njob * len, 256), 256, 0, s>>>(xs, njob * len, f.k, f.base, 11u);
      fill_codes<<<grid_for(kTuneJobs * kTuneLen, 256), 256, 0, s>>>(ys, kTuneJobs * kTuneLen, f.k, f.base, 12u);
      if (gemv) fill_ones<<<grid_for(kTuneJobs * kTuneLen, 256), 256, 0, s>>>(reinterpret_cast<double*>(ys),
                                                                              kTuneJobs * kTuneLen);
      std::vector<flyte_job> jobs(static_cast<size_t>(njob));
      for (int64_t i = 0; i < njob; ++i) {
        flyte_job& j = jobs[size_t(i)];
        std::memset(&j, 0, sizeof(j));
        j.op = op;
        j.fx = f;
        j.fy = f;
        j.mode = FLYTE_RNE;
        j.alpha = 1e-9;
        j.beta = 0.0;
        if (gemv) {
          j.m = j.n = kTuneSide;
          j.a = xs + i * len * f.k;
          j.xv = reinterpret_cast<const double*>(ys);
          j.y = out + i * kTuneSide * 8;
        } else {
          j.n = len;
          j.a = xs + i * len * f.k;
          j.y = op == FLYTE_JOB_UNPACK ? static_cast<void*>(out + i * len * 8) : static_cast<void*>(ys + i * len * f.k);
          j.result = reinterpret_cast<double*>(out) + i;
        }
      }
      const int64_t cands_stream[3] = {16384, 65536, 262144};
      const int64_t cands_rows[3] = {8, 16, 32};
      const int64_t cands_chunks[3] = {128, 256, 512};
      const int64_t* cands = op == FLYTE_JOB_GEMV_T ? cands_chunks : (gemv ? cands_rows : cands_stream);
      int64_t best = cands[1];
      float best_ms = 1e30f;
      for (int c = 0; c < 3 && result == FLYTE_OK; ++c) {
        set_tile(op, f, cands[c]);
        if ((result = batch_prepare(jobs.data(), int(njob), bws, size_t(kTuneWs), s)) != FLYTE_OK) break;
        if ((result = batch_launch(bws, s)) != FLYTE_OK) break;   // warm-up
        cudaEventRecord(e0, s);
        for (int r = 0; r < 3; ++r)
          if ((result = batch_launch(bws, s)) != FLYTE_OK) break;
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
          result = cuda_status(cudaGetLastError(), "batch autotune");
          break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) {
          best_ms = ms;
          best = cands[c];
        }
      }
      set_tile(op, f, best);
      if (result != FLYTE_OK) break;
    }
    if (result != FLYTE_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return result;
}

// Tuning on the caller's own batch: coordinate descent, first over the resident blocks per SM,
// then over the tile size of every (operation, base, k) that occurs in the jobs, each candidate
// timed as the whole batch (prepare, one untimed launch, three timed launches); a candidate is
// kept only when it is at least 1 % faster than the best so far.
flyte_status batch_autotune_jobs(const flyte_job* jobs, int njobs, void* ws, size_t ws_bytes, cudaStream_t s) {
  if (jobs == nullptr || njobs <= 0) return FLYTE_OK;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return cuda_status(cudaGetLastError(), "batch autotune");
  flyte_status result = FLYTE_OK;
  // time of the batch with the current table; +inf when it does not fit in ws
  auto run = [&](float& ms) -> flyte_status {
    ms = 1e30f;
    Plan p;
    flyte_status st = make_plan(jobs, njobs, p);
    if (st != FLYTE_OK) return st;
    if (size_t(p.bytes) > ws_bytes) return FLYTE_OK;
    if ((st = batch_prepare(jobs, njobs, ws, ws_bytes, s)) != FLYTE_OK) return st;
    if ((st = batch_launch(ws, s)) != FLYTE_OK) return st;
    cudaEventRecord(e0, s);
    for (int r = 0; r < 3; ++r)
      if ((st = batch_launch(ws, s)) != FLYTE_OK) return st;
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) return cuda_status(cudaGetLastError(), "batch autotune");
    cudaEventElapsedTime(&ms, e0, e1);
    return FLYTE_OK;
  };
  float best = 1e30f;
  result = run(best);
  // resident blocks per SM
  if (result == FLYTE_OK) {
    const int mx = max_blocks_per_sm();
    int keep = 0;
    for (int b = mx - 1; b >= 1 && b >= mx - 2 && result == FLYTE_OK; --b) {
      {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned_per_sm = b;
      }
      float ms;
      result = run(ms);
      if (ms < 0.99f * best) {
        best = ms;
        keep = b;
      }
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned_per_sm = keep;
  }
  // tile sizes of the (operation, base, k) present
  bool seen[kNOps][2][9] = {};
  for (int i = 0; i < njobs && result == FLYTE_OK; ++i) {
    const flyte_job& j = jobs[i];
    if (j.op < 0 || j.op >= kNOps || !valid_fmt(j.fx)) continue;
    const flyte_fmt f = (j.op == FLYTE_JOB_AXPY) ? j.fy : j.fx;
    if (!valid_fmt(f) || seen[j.op][f.base][f.k]) continue;
    seen[j.op][f.base][f.k] = true;
    const int64_t cs[5] = {16384, 32768, 65536, 131072, 262144};
    const int64_t cr[4] = {4, 8, 16, 32};
    const int64_t cc[3] = {128, 256, 512};
    const bool gn = j.op == FLYTE_JOB_GEMV_N, gt = j.op == FLYTE_JOB_GEMV_T;
    const int64_t* cand = gt ? cc : (gn ? cr : cs);
    const int nc = gt ? 3 : (gn ? 4 : 5);
    const int64_t cur = tile_for(j.op, f);
    int64_t keep = cur;
    for (int c = 0; c < nc && result == FLYTE_OK; ++c) {
      if (cand[c] == cur) continue;
      set_tile(j.op, f, cand[c]);
      float ms;
      result = run(ms);
      if (ms < 0.99f * best) {
        best = ms;
        keep = cand[c];
      }
    }
    set_tile(j.op, f, keep);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return result;
}

int64_t batch_tile_size(int op, flyte_fmt f) {
  if (op < 0 || op >= kNOps || !valid_fmt(f)) return -1;
  return tile_for(op, f);
}

int batch_resident_blocks() { return blocks_per_sm(); }

}  // namespace flyte
