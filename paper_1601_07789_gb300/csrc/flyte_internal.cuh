// flyte_internal.cuh -- shared definitions of the CUDA library (not part of the ABI).
//
// Format traits, the bit-exact narrowing of Sec. 5 written on integer
// patterns, and the byte-stream helpers of Sec. 4 used by every kernel.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/flyte.h"

namespace flyte {

// ---- status plumbing -------------------------------------------------------

void set_error(const char* fmt, ...);
flyte_status cuda_status(cudaError_t e, const char* what);
// The argument checks of flyte_gemv (FLYTE_OK or FLYTE_ERR_INVALID_ARG with
// the message set), shared by the entry points that take its arguments.
flyte_status check_gemv_args(char trans, int64_t m, int64_t n, double alpha, const void* A, flyte_fmt fa,
                             int64_t lda, const double* x, int64_t incx, const void* y, int64_t incy);

#define FLYTE_TRY_LAUNCH(what)                                   \
  do {                                                           \
    cudaError_t _e = cudaGetLastError();                         \
    if (_e != cudaSuccess) return ::flyte::cuda_status(_e, what); \
  } while (0)

// ---- format traits (Sec. 3.1, Table 1) ------------------------------------

template <int BASE>
struct Native;
template <>
struct Native<FLYTE_F32> {
  using bits = uint32_t;
  using value = float;
  static constexpr int W = 32;        // native width in bits
  static constexpr int E = 8;         // exponent bits, same as the built-in type
};
template <>
struct Native<FLYTE_F64> {
  using bits = uint64_t;
  using value = double;
  static constexpr int W = 64;
  static constexpr int E = 11;
};

template <int BASE, int K>
struct Fmt {
  using N = Native<BASE>;
  using bits = typename N::bits;
  static constexpr int W = N::W;
  static constexpr int E = N::E;
  static constexpr int D = W - 8 * K;                 // dropped low bits
  static constexpr bits SIGN = bits(1) << (W - 1);
  static constexpr bits MAG = SIGN - 1;
  static constexpr bits INF = ((bits(1) << E) - 1) << (W - 1 - E);
  static constexpr uint64_t CODE_SIGN = uint64_t(1) << (8 * K - 1);
  // quiet bit of the flyte: its most significant mantissa bit (K >= 2)
  static constexpr uint64_t QUIET = K >= 2 ? (uint64_t(1) << (8 * K - 2 - E)) : 0;
};

// ---- narrowing (Sec. 5), integer-only -----------------------------------
//
// Every mode works on the magnitude m = |u| as an unsigned integer.  NaNs
// are recognised first (m > INF), keep their high payload and get the quiet
// bit.  Nearest-even uses the bias form t = (m + half - 1 + lsb) >> D, which
// carries into the exponent exactly when IEEE rounding does (Sec. 5.3).
// k = 1 has no Inf/NaN codes: specials map to 0x7F and the magnitude is
// clamped at 0x7F.

template <int BASE, int K>
__device__ __forceinline__ uint64_t narrow(typename Fmt<BASE, K>::bits u, int mode) {
  using F = Fmt<BASE, K>;
  using B = typename F::bits;
  if constexpr (F::D == 0) {
    return uint64_t(u);
  } else {
    const B m = u & F::MAG;
    const uint64_t s = (u & F::SIGN) ? F::CODE_SIGN : 0;
    const B half = B(1) << (F::D - 1);
    const B kept = m >> F::D;
    B t;
    if (mode == FLYTE_RNE) {
      t = (m + (half - 1) + (kept & 1)) >> F::D;
    } else if (mode == FLYTE_RTZ) {
      t = kept;
    } else if (mode == FLYTE_HALF_UP) {
      t = (m + half) >> F::D;
    } else {  // FLYTE_RTO
      t = kept | B((m & ((half << 1) - 1)) != 0);
    }
    if constexpr (K == 1) {
      if (m >= F::INF) t = 0x7F;
      t = t > B(0x7F) ? B(0x7F) : t;
    } else {
      if (m > F::INF) t = kept | B(F::QUIET);
    }
    return s | uint64_t(t);
  }
}

template <int BASE, int K>
__device__ __forceinline__ typename Fmt<BASE, K>::bits widen(uint64_t q) {
  using F = Fmt<BASE, K>;
  return typename F::bits(q) << F::D;
}

// ---- byte buffers held in 32-bit registers (Sec. 4.1, 4.3) --------------------
//
// A group of G consecutive elements occupies G*K bytes = NW words.  get4<P>()
// returns bytes [P, P+4) of the buffer (bytes outside read as zero); the
// positions are compile-time constants after unrolling, so this lowers to
// one funnel shift or a register move.

template <int NW>
__device__ __forceinline__ uint32_t word_at(const uint32_t (&w)[NW], int i) {
  return (i < 0 || i >= NW) ? 0u : w[i];
}

template <int NW>
__device__ __forceinline__ uint32_t get4(const uint32_t (&w)[NW], int pos) {
  const int wi = pos >= 0 ? pos / 4 : -((-pos + 3) / 4);
  const int r = pos - 4 * wi;
  const uint32_t lo = word_at(w, wi);
  if (r == 0) return lo;
  const uint32_t hi = word_at(w, wi + 1);
  return __funnelshift_r(lo, hi, 8 * r);
}

// Element e of a K-byte group buffer, returned as its native bit pattern
// (the code shifted up by D bits: the zero padding of Fig. 1).
template <int BASE, int K, int NW>
__device__ __forceinline__ typename Fmt<BASE, K>::bits extract_widened(const uint32_t (&w)[NW], int e) {
  using F = Fmt<BASE, K>;
  constexpr int NB = F::W / 8;                 // native bytes
  const int p = e * K + K - NB;                // buffer position of the native's byte 0
  if constexpr (BASE == FLYTE_F32) {
    uint32_t v = get4(w, p);
    if constexpr (F::D > 0) v &= ~((1u << F::D) - 1u);
    return v;
  } else {
    uint32_t lo = get4(w, p);
    uint32_t hi = get4(w, p + 4);
    if constexpr (F::D >= 32) {
      lo = 0;
      if constexpr (F::D > 32) hi &= ~((1u << (F::D - 32)) - 1u);
    } else if constexpr (F::D > 0) {
      lo &= ~((1u << F::D) - 1u);
    }
    return (uint64_t(hi) << 32) | lo;
  }
}

// Element e of the buffer as its raw K-byte code (low 8K bits).
template <int K, int NW>
__device__ __forceinline__ uint64_t extract_code(const uint32_t (&w)[NW], int e) {
  const int p = e * K;
  uint64_t lo = get4(w, p);
  if constexpr (K <= 4) {
    return K == 4 ? lo : (lo & ((uint64_t(1) << (8 * K)) - 1));
  } else {
    uint64_t hi = get4(w, p + 4);
    uint64_t v = lo | (hi << 32);
    return K == 8 ? v : (v & ((uint64_t(1) << (8 * K)) - 1));
  }
}

// OR code c (low 8K bits) into the buffer at element e.
template <int K, int NW>
__device__ __forceinline__ void deposit_code(uint32_t (&w)[NW], int e, uint64_t c) {
  const int p = e * K;  // first byte
#pragma unroll
  for (int j = 0; j < NW; ++j) {
    const int off = p - 4 * j;  // byte offset of the code relative to word j
    if (off >= 4 || off + K <= 0) continue;
    if (off >= 0) {
      w[j] |= uint32_t(c << (8 * off));
    } else {
      w[j] |= uint32_t(c >> (8 * (-off)));
    }
  }
}

// ---- 4-element groups: aligned vector access to 4k packed bytes ----------------------

// Widest power-of-two access (<= 16 bytes) that divides a 4k-byte group; the
// fast paths need the stream (and every row start) aligned to it.
__host__ __device__ constexpr int group_bytes(int K) {
  return (4 * K) % 16 == 0 ? 16 : ((4 * K) % 8 == 0 ? 8 : 4);
}

template <int K>
__device__ __forceinline__ void load_group(const uint8_t* p, uint32_t (&w)[K]) {
  constexpr int S = group_bytes(K);
  if constexpr (S == 16) {
#pragma unroll
    for (int i = 0; i < K / 4; ++i) {
      uint4 v = __ldg(reinterpret_cast<const uint4*>(p) + i);
      w[4 * i] = v.x; w[4 * i + 1] = v.y; w[4 * i + 2] = v.z; w[4 * i + 3] = v.w;
    }
  } else if constexpr (S == 8) {
#pragma unroll
    for (int i = 0; i < K / 2; ++i) {
      uint2 v = __ldg(reinterpret_cast<const uint2*>(p) + i);
      w[2 * i] = v.x; w[2 * i + 1] = v.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < K; ++i) w[i] = __ldg(reinterpret_cast<const uint32_t*>(p) + i);
  }
}

// Same, for a stream that the kernel also writes (no read-only cache path).
template <int K>
__device__ __forceinline__ void load_group_rw(const uint8_t* p, uint32_t (&w)[K]) {
  constexpr int S = group_bytes(K);
  if constexpr (S == 16) {
#pragma unroll
    for (int i = 0; i < K / 4; ++i) {
      uint4 v = reinterpret_cast<const uint4*>(p)[i];
      w[4 * i] = v.x; w[4 * i + 1] = v.y; w[4 * i + 2] = v.z; w[4 * i + 3] = v.w;
    }
  } else if constexpr (S == 8) {
#pragma unroll
    for (int i = 0; i < K / 2; ++i) {
      uint2 v = reinterpret_cast<const uint2*>(p)[i];
      w[2 * i] = v.x; w[2 * i + 1] = v.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < K; ++i) w[i] = reinterpret_cast<const uint32_t*>(p)[i];
  }
}

template <int K>
__device__ __forceinline__ void store_group(uint8_t* p, const uint32_t (&w)[K]) {
  constexpr int S = group_bytes(K);
  if constexpr (S == 16) {
#pragma unroll
    for (int i = 0; i < K / 4; ++i)
      reinterpret_cast<uint4*>(p)[i] = make_uint4(w[4 * i], w[4 * i + 1], w[4 * i + 2], w[4 * i + 3]);
  } else if constexpr (S == 8) {
#pragma unroll
    for (int i = 0; i < K / 2; ++i) reinterpret_cast<uint2*>(p)[i] = make_uint2(w[2 * i], w[2 * i + 1]);
  } else {
#pragma unroll
    for (int i = 0; i < K; ++i) reinterpret_cast<uint32_t*>(p)[i] = w[i];
  }
}

// ---- scalar byte access for the generic (any stride / alignment) paths ----------

template <int K>
__device__ __forceinline__ uint64_t load_code_bytes(const uint8_t* p) {
  uint64_t q = 0;
#pragma unroll
  for (int b = K - 1; b >= 0; --b) q = (q << 8) | uint64_t(p[b]);
  return q;
}

template <int K>
__device__ __forceinline__ void store_code_bytes(uint8_t* p, uint64_t q) {
#pragma unroll
  for (int b = 0; b < K; ++b) p[b] = uint8_t(q >> (8 * b));
}

// Exact binary64 value of a k-byte code.
template <int BASE, int K>
__device__ __forceinline__ double code_to_double(uint64_t q) {
  if constexpr (BASE == FLYTE_F64) {
    return __longlong_as_double((long long)widen<BASE, K>(q));
  } else {
    return double(__uint_as_float(widen<BASE, K>(q)));
  }
}

// Runtime-format variants for the generic paths.
__device__ __forceinline__ uint64_t load_code_bytes_rt(const uint8_t* p, int k) {
  uint64_t q = 0;
  for (int b = k - 1; b >= 0; --b) q = (q << 8) | uint64_t(p[b]);
  return q;
}

__device__ __forceinline__ double code_to_double_rt(uint64_t q, int k, int base) {
  if (base == FLYTE_F64) {
    return __longlong_as_double((long long)(k == 8 ? q : (q << (64 - 8 * k))));
  }
  return double(__uint_as_float(uint32_t(k == 4 ? q : (q << (32 - 8 * k)))));
}

__device__ __forceinline__ void store_code_bytes_rt(uint8_t* p, uint64_t q, int k) {
  for (int b = 0; b < k; ++b) p[b] = uint8_t(q >> (8 * b));
}

// narrow<BASE, k> for a k known only at run time (warp-uniform in every caller).
template <int BASE>
__device__ __forceinline__ uint64_t narrow_rt(typename Native<BASE>::bits u, int k, int mode) {
  switch (k) {
    case 1: return narrow<BASE, 1>(u, mode);
    case 2: return narrow<BASE, 2>(u, mode);
    case 3: return narrow<BASE, 3>(u, mode);
    case 4: return narrow<BASE, 4>(u, mode);
  }
  if constexpr (BASE == FLYTE_F64) {
    switch (k) {
      case 5: return narrow<BASE, 5>(u, mode);
      case 6: return narrow<BASE, 6>(u, mode);
      case 7: return narrow<BASE, 7>(u, mode);
      default: return narrow<BASE, 8>(u, mode);
    }
  }
  return uint64_t(u);
}

// ---- launch geometry -----------------------------------------------------------

int sm_count();   // streaming multiprocessors of the current device (cached per device)

inline unsigned grid_for(int64_t work_items, int per_block, int max_blocks_per_sm = 8) {
  int64_t blocks = (work_items + per_block - 1) / per_block;
  int64_t cap = int64_t(sm_count()) * max_blocks_per_sm;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  return unsigned(blocks);
}

// ---- format dispatch -------------------------------------------------------------

// Calls f.template operator()<BASE, K>() for the runtime (base, k).
template <typename Fn>
flyte_status dispatch_fmt(flyte_fmt f, Fn&& fn) {
  if (f.base == FLYTE_F32) {
    switch (f.k) {
      case 1: return fn.template operator()<FLYTE_F32, 1>();
      case 2: return fn.template operator()<FLYTE_F32, 2>();
      case 3: return fn.template operator()<FLYTE_F32, 3>();
      case 4: return fn.template operator()<FLYTE_F32, 4>();
    }
  } else {
    switch (f.k) {
      case 1: return fn.template operator()<FLYTE_F64, 1>();
      case 2: return fn.template operator()<FLYTE_F64, 2>();
      case 3: return fn.template operator()<FLYTE_F64, 3>();
      case 4: return fn.template operator()<FLYTE_F64, 4>();
      case 5: return fn.template operator()<FLYTE_F64, 5>();
      case 6: return fn.template operator()<FLYTE_F64, 6>();
      case 7: return fn.template operator()<FLYTE_F64, 7>();
      case 8: return fn.template operator()<FLYTE_F64, 8>();
    }
  }
  return FLYTE_ERR_INVALID_ARG;
}

inline bool valid_fmt(flyte_fmt f) {
  return (f.base == FLYTE_F32 && f.k >= 1 && f.k <= 4) || (f.base == FLYTE_F64 && f.k >= 1 && f.k <= 8);
}

// ---- launchers (one per operation, defined in the kernel files) ---------------------

flyte_status launch_pack(void* dst, const void* src, int64_t n, flyte_fmt f, int64_t inc_dst,
                         int64_t inc_src, int mode, cudaStream_t s);
flyte_status launch_unpack(void* dst, const void* src, int64_t n, flyte_fmt f, int64_t inc_dst,
                           int64_t inc_src, cudaStream_t s);
flyte_status launch_gemv(char trans, int64_t m, int64_t n, double alpha, const void* A, flyte_fmt fa,
                         int64_t lda, const double* x, int64_t incx, double beta, void* y, int ky, int64_t incy,
                         int mode, void* ws, size_t ws_bytes, cudaStream_t s);
size_t gemv_workspace_bytes(char trans, int64_t m, int64_t n, flyte_fmt f);
flyte_status launch_dot(double* result, int64_t n, const void* x, flyte_fmt fx, int64_t incx, const void* y,
                        flyte_fmt fy, int64_t incy, void* ws, size_t ws_bytes, cudaStream_t s);
size_t dot_workspace_bytes(int64_t n);
flyte_status launch_axpy(int64_t n, double alpha, const void* x, flyte_fmt fx, int64_t incx, void* y,
                         flyte_fmt fy, int64_t incy, int mode, cudaStream_t s);
flyte_status launch_scal(int64_t n, double alpha, void* x, flyte_fmt fx, int64_t incx, int mode, cudaStream_t s);
flyte_status launch_gemm(int64_t m, int64_t n, int64_t kdim, double alpha, const void* A, flyte_fmt fa,
                         int64_t lda, const void* B, int64_t ldb, double beta, void* C, int kc, int64_t ldc,
                         int mode, void* ws, size_t ws_bytes, cudaStream_t s);
size_t gemm_workspace_bytes(int64_t m, int64_t n, int64_t kdim, flyte_fmt f);
flyte_status launch_refine(int64_t n, const double* A64, int64_t lda64, const void* Ak, flyte_fmt fa, int64_t lda,
                           const double* b, double* x, double tol, int max_outer, int inner, void* ws,
                           size_t ws_bytes, cudaStream_t s, int* iters_out, double* relres_out);
size_t refine_workspace_bytes(int64_t n);
size_t batch_workspace_bytes(const flyte_job* jobs, int njobs);
flyte_status batch_prepare(const flyte_job* jobs, int njobs, void* ws, size_t ws_bytes, cudaStream_t s);
flyte_status batch_launch(void* ws, cudaStream_t s);
size_t batch_autotune_bytes();
flyte_status batch_autotune(void* ws, size_t ws_bytes, cudaStream_t s);
flyte_status batch_autotune_jobs(const flyte_job* jobs, int njobs, void* ws, size_t ws_bytes, cudaStream_t s);
int64_t batch_tile_size(int op, flyte_fmt f);
int batch_resident_blocks();

}  // namespace flyte
