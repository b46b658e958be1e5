// dwacc.cuh -- binary64-accurate dot products on the binary32 pipe.
//
// GB300 executes binary64 FMAs at 1/64 of the binary32 rate, too slow to keep
// up with a k-byte stream from HBM.  The BLAS kernels therefore widen each
// flyte to binary32 instead of binary64 (exactly: a double-based flyte with
// k <= 4 has at most 21 significant bits; k >= 5 is split into an exact
// high/low pair) whenever its exponent lies in a safe window, and accumulate
// in double-word ("float-float") arithmetic built from error-free
// transformations:
//
//   p + e       = a * x1          (TwoProd with an FMA; exact)
//   e'          = RN(a * x2 + e)  (low part of a*x, x = x1 + x2 + O(u^2 x))
//   s + t       = S + p           (TwoSum; exact)
//   v           = RN(RN(C + t) + e')
//   (S, C)      = Fast2Sum(s, v)  (exact: |C| <= u|S| and |v| <= 5u max(|S|,|p|)
//                                  make s a multiple of ulp(v) whenever |s| < |v|)
//
// With u = 2^-24, one step adds at most 6 u^2 P to the error, P the running
// sum of |a x| of that accumulator, and the product adds at most 14 u^2 |a x|
// (3 u^2 for k <= 4).  A chain of L terms therefore errs by at most
// (6L + 14) u^2 sum|a x|; the kernels keep L small by spreading a dot product
// over many independent accumulators.  Combining the accumulators in binary64
// adds at most R 2^-53 sum|a x|, R the depth of the reduction, and the
// epilogue fma(alpha, t, beta y) 2 2^-53 (|alpha t| + |beta y|).  The host only
// takes this path when
//   (6L + 14) * 32 + R <= 4 n                 (u^2 = 32 * 2^-53)
// so that the result meets |y - y_exact| <= 4 (n + 2) 2^-53 (|alpha| sum|a x| + |beta y|).
// Elements outside the window (zero, subnormal, huge, Inf, NaN) are detected
// with one integer compare each; the affected row, tile or group is then
// summed with binary64 FMAs instead, which also gives IEEE Inf/NaN semantics.
//
// All binary32 operations use the _rn intrinsics so that the compiler cannot
// contract them into FMAs and break the error-free transformations.
#pragma once

#include "flyte_internal.cuh"

namespace flyte {

struct DW {
  float hi, lo;
};

__device__ __forceinline__ void dw_zero(DW& a) { a.hi = 0.f; a.lo = 0.f; }

// (S, C) <- (S, C) + (p + e) with the algorithm above.
__device__ __forceinline__ void dw_add(DW& acc, float p, float e) {
  const float s = __fadd_rn(acc.hi, p);
  const float bp = __fsub_rn(s, acc.hi);
  const float ap = __fsub_rn(s, bp);
  const float t = __fadd_rn(__fsub_rn(acc.hi, ap), __fsub_rn(p, bp));
  const float v = __fadd_rn(__fadd_rn(acc.lo, t), e);
  const float hi = __fadd_rn(s, v);
  acc.lo = __fsub_rn(v, __fsub_rn(hi, s));
  acc.hi = hi;
}

// Lazy variant for short chains: the low word only collects the error terms
// and is never renormalised.  With |t_i| <= u P and |e'_i| <= 4u |a_i x_i|,
// after i steps |C| <= (i + 4) u P, so the two additions into C cost at most
// (2i + 12) u^2 P at step i and a chain of L terms errs by at most
// (L^2 + 13L) u^2 sum|a x| (instead of 6L u^2 with renormalisation), for 8
// binary32 operations per term instead of 11.
__device__ __forceinline__ void dw_add_lazy(DW& acc, float p, float e) {
  const float s = __fadd_rn(acc.hi, p);
  const float bp = __fsub_rn(s, acc.hi);
  const float ap = __fsub_rn(s, bp);
  const float t = __fadd_rn(__fsub_rn(acc.hi, ap), __fsub_rn(p, bp));
  acc.lo = __fadd_rn(__fadd_rn(acc.lo, t), e);
  acc.hi = s;
}

// Binary64 value of a double-word accumulator (one rounding at most; exact
// when the pair is normalised, |lo| <= ulp(hi) / 2, since hi + lo then has at
// most 49 significant bits).
__device__ __forceinline__ double dw_value(const DW& a) { return double(a.hi) + double(a.lo); }

// Exact renormalisation (TwoSum of the two words): afterwards |lo| <= ulp(hi) / 2.
// A lazy accumulator can have |lo| > |hi| after cancellation, so the
// ordering-free TwoSum is used rather than Fast2Sum.
__device__ __forceinline__ void dw_norm(DW& a) {
  const float s = __fadd_rn(a.hi, a.lo);
  const float bp = __fsub_rn(s, a.hi);
  const float ap = __fsub_rn(s, bp);
  a.lo = __fadd_rn(__fsub_rn(a.hi, ap), __fsub_rn(a.lo, bp));
  a.hi = s;
}

// acc <- acc + b for normalised acc and b: one dw_add step with p = b.hi and
// e = b.lo (|e| <= u |p|, inside the premises above), so it errs by at most
// 6 u^2 (|acc| + |b|) and leaves acc normalised.  Combining accumulators in a
// tree of depth D this way costs at most 6 D u^2 sum|a x| and no binary64
// instruction (binary64 runs at 1/64 of the binary32 rate on this GPU, and a
// warp-wide binary64 reduction per row stalled the pipe in profiles).
__device__ __forceinline__ void dw_add_dw(DW& acc, const DW& b) { dw_add(acc, b.hi, b.lo); }

// Normalise and add the four slot accumulators of a thread: depth 2.
__device__ __forceinline__ DW dw_sum4(DW a0, DW a1, DW a2, DW a3) {
  dw_norm(a0);
  dw_norm(a1);
  dw_norm(a2);
  dw_norm(a3);
  dw_add_dw(a0, a1);
  dw_add_dw(a2, a3);
  dw_add_dw(a0, a2);
  return a0;
}

// Warp sum of normalised double-word values over an xor tree (depth 5); the
// value in lane 0 is the one used.
__device__ __forceinline__ DW dw_warp_sum(DW a) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    DW b;
    b.hi = __shfl_xor_sync(0xFFFFFFFFu, a.hi, o);
    b.lo = __shfl_xor_sync(0xFFFFFFFFu, a.lo, o);
    dw_add_dw(a, b);
  }
  return a;
}

// ---- exponent window ------------------------------------------------------
//
// A value is "in window" when 2^-40 <= |v| < 2^40.  Products of two in-window
// values (or of one and a scaled x in [2^-40, 2)) stay within [2^-80, 2^81),
// so every error term of the double-word algorithm is a normal binary32
// number and no partial sum can overflow.

constexpr int kWinLog2 = 40;

// Double-based flyte element, widened to its 64-bit pattern (hi word h, low
// word l), as binary32 pieces: value = hi + lo exactly for k <= 7 (lo = 0 for
// k <= 4); for k = 8 lo keeps 23 of the 29 remaining bits (|error| < 2^-46 |v|).
// Returns false when the value is outside the window (including zero).
template <int K>
__device__ __forceinline__ bool dbl_to_pair(uint32_t h, uint32_t l, float& hi, float& lo) {
  constexpr uint32_t kElo = 1023 - kWinLog2;               // lowest exponent field in window
  const uint32_t v = (h << 1) - (kElo << 21);
  const bool ok = v < (uint32_t(2 * kWinLog2) << 21);
  // binary32 pattern: sign | (e - 896) << 23 | top 23 mantissa bits (valid in window)
  uint32_t mag;
  if constexpr (K <= 4) {
    mag = (h << 3) - (896u << 23);
  } else {
    mag = __funnelshift_l(l, h, 3) - (896u << 23);
  }
  const uint32_t hb = mag | (h & 0x80000000u);
  hi = __uint_as_float(hb);
  if constexpr (K <= 4) {
    lo = 0.f;
  } else {
    // the bits below hi's last one, l[28:0] (at most 23 of them kept), as the
    // exact difference (Sterbenz) of two binary32 numbers with hi's sign and an
    // exponent 23 below hi's: one with those bits as its leading fraction bits,
    // one with fraction 0 (in window the exponent stays normal)
    constexpr int kBits = 8 * (K - 4) - 3;                   // 5, 13, 21, 29
    constexpr int kKeep = kBits > 23 ? 23 : kBits;
    const uint32_t sbase = (hb & 0xFF800000u) - (23u << 23);
    const uint32_t frac = ((l & 0x1FFFFFFFu) >> (29 - kKeep)) << (23 - kKeep);
    lo = __fsub_rn(__uint_as_float(sbase | frac), __uint_as_float(sbase));
  }
  return ok;
}

// Float-based flyte element widened to its binary32 pattern f.
__device__ __forceinline__ bool flt_in_window(uint32_t f) {
  constexpr uint32_t kElo = 127 - kWinLog2;
  return ((f << 1) - (kElo << 24)) < (uint32_t(2 * kWinLog2) << 24);
}

// ---- pairs of binary32 values (f32x2) ------------------------------------------
//
// sm_100-family GPUs add, subtract, multiply and fma two binary32 values held
// in one 64-bit register with one instruction (add/sub/mul/fma.rn.f32x2),
// each value rounded exactly as the scalar _rn operation rounds it.  The
// binary32 rate per value is unchanged (measured on GB300: about 135 value
// operations per clock and SM for fma.rn.f32 and for fma.rn.f32x2 alike), but
// a pair costs one issue slot instead of two, which is what the issue-bound
// gemv kernels need.  The error-free transformations below are the scalar
// ones of this file applied to both values of a pair.

using f2 = unsigned long long;

__device__ __forceinline__ f2 f2_pack(float a, float b) {
  f2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void f2_unpack(f2 v, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ f2 f2_add(f2 a, f2 b) {
  f2 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2 f2_sub(f2 a, f2 b) {
  f2 r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2 f2_mul(f2 a, f2 b) {
  f2 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2 f2_fma(f2 a, f2 b, f2 c) {
  f2 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
__device__ __forceinline__ f2 f2_neg(f2 a) { return a ^ 0x8000000080000000ull; }

struct DW2 {
  f2 hi, lo;   // two double-word accumulators, one per value of the pair
};

__device__ __forceinline__ void dw2_zero(DW2& a) { a.hi = 0ull; a.lo = 0ull; }

// The two double-word accumulators held by a pair, as scalar DW values.
__device__ __forceinline__ void dw2_split(const DW2& a, DW& d0, DW& d1) {
  f2_unpack(a.hi, d0.hi, d1.hi);
  f2_unpack(a.lo, d0.lo, d1.lo);
}

// acc <- acc + (p + e), given pn = -p (negation is exact): dw_add_lazy on both values
// (s + t = S + p by TwoSum written with -pn, then C <- (C + t) + e').
__device__ __forceinline__ void dw2_add_lazy_neg(DW2& acc, f2 pn, f2 e) {
  const f2 s = f2_sub(acc.hi, pn);
  const f2 bp = f2_sub(s, acc.hi);
  const f2 ap = f2_sub(s, bp);
  const f2 t = f2_sub(f2_sub(acc.hi, ap), f2_add(pn, bp));
  acc.lo = f2_add(f2_add(acc.lo, t), e);
  acc.hi = s;
}

// The renormalising step (dw_add) on both values, with pn = -p.
__device__ __forceinline__ void dw2_add_neg(DW2& acc, f2 pn, f2 e) {
  const f2 s = f2_sub(acc.hi, pn);
  const f2 bp = f2_sub(s, acc.hi);
  const f2 ap = f2_sub(s, bp);
  const f2 t = f2_sub(f2_sub(acc.hi, ap), f2_add(pn, bp));
  const f2 v = f2_add(f2_add(acc.lo, t), e);
  const f2 hi = f2_add(s, v);
  acc.lo = f2_sub(v, f2_sub(hi, s));
  acc.hi = hi;
}

// Product of an in-window element (hi + lo) with x = x1 + x2 as (p, e').
__device__ __forceinline__ void pair_times_x(float ahi, float alo, float x1, float x2, float& p,
                                             float& e) {
  p = __fmul_rn(ahi, x1);
  float t = __fmaf_rn(ahi, x1, -p);
  t = __fmaf_rn(alo, x1, t);
  e = __fmaf_rn(ahi, x2, t);
}

// Product of two in-window split elements (ahi + alo)(bhi + blo) as (p, e');
// the alo*blo term (< 4u^2 |ab|) is dropped.
__device__ __forceinline__ void pair_times_pair(float ahi, float alo, float bhi, float blo, float& p,
                                                float& e) {
  p = __fmul_rn(ahi, bhi);
  float t = __fmaf_rn(ahi, bhi, -p);
  t = __fmaf_rn(alo, bhi, t);
  e = __fmaf_rn(ahi, blo, t);
}

__device__ __forceinline__ void single_times_x(float a, float x1, float x2, float& p, float& e) {
  p = __fmul_rn(a, x1);
  const float t = __fmaf_rn(a, x1, -p);
  e = __fmaf_rn(a, x2, t);
}

// ---- warp / block reductions in binary64 (fixed order: deterministic) ----------

// True when a length-n dot product summed in chains of at most L terms,
// combined by a double-word tree of depth D (dw_add_dw) and then by a
// binary64 reduction of depth R, meets the bound above.  P is the
// product-error constant: 14 when one operand is binary64 x = x1 + x2, 20
// when both operands are flytes split into high/low pairs (flyte_dot).
__host__ __device__ constexpr bool dw_bound_ok(int64_t n, int64_t L, int64_t R, int64_t P = 14, int64_t D = 0) {
  return (6 * L + P + 6 * D) * 32 + R <= 4 * n;
}
// The same for chains accumulated with dw_add_lazy.
__host__ __device__ constexpr bool dw_lazy_bound_ok(int64_t n, int64_t L, int64_t R, int64_t P = 14,
                                                    int64_t D = 0) {
  return (L * L + 13 * L + P + 6 * D) * 32 + R <= 4 * n;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  return v;
}

// Sum over the block (blockDim.x / 32 warps) in a fixed order; result in thread 0.
__device__ __forceinline__ double block_sum(double v, double* smem) {
  v = warp_sum(v);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) smem[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0) {
    for (int w = 0; w < int(blockDim.x >> 5); ++w) t += smem[w];
  }
  return t;
}

}  // namespace flyte
