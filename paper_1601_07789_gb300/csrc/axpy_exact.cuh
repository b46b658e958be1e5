// axpy_exact.cuh -- the binary64-free exact axpy elements (used by blas1.cu and batch.cu).
//
// binary64 FMAs run at a small fraction of the binary32 rate on this GPU and
// bound the kernel above (its fp64 pipe is ~82 % busy at a third of the HBM
// rate).  When alpha is a binary32 number (1.5, -2, 0.75, ...) and the
// format is double-based with k <= 4 (x, y then have <= 21 significant bits
// and are exact binary32 numbers inside the window), s = alpha x + y is
// obtained EXACTLY as h + L + Le with error-free transformations on the
// binary32 pipe, and the code of pack(RN64(s)) is decided from it:
//   p + e = alpha x (TwoProd), s1 + t1 = p + y, s2 + t2 = t1 + e,
//   h + l = s1 + s2, L + Le = l + t2               (TwoSum each; all exact;
//   Le is formed only when needed, see below)
// The k-byte result keeps the top m = 8k - 12 mantissa bits of h (magnitude
// code Q) and depends only on the sign of f - B, where f u_h = (dropped bits
// of h) u_h + L + Le is the exact remainder above Q's value and B is 0
// (toward zero, round to odd) or half a code ulp (nearest even, half-up).
// That sign is read exactly from w = RN((D - B) u_h + L) and Le.  RN64(s)
// can differ from s only by 2^-27 u_h, so it cannot move s across a boundary
// unless s lies within that distance of it; such elements (|w| <= 2^-20 u_h,
// not exactly on the boundary), exact zeros and anything outside the window
// send their group to the binary64 FMA instead.  Any other binary64 alpha in
// the window is split into two binary32 parts (axpy_exact_f32x2 below): the
// same chain with one more product, and a guard widened by a bound on the few
// terms it leaves out.
#pragma once

#include "dwacc.cuh"

namespace flyte {

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& t) {
  s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  const float ap = __fsub_rn(s, bp);
  t = __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp));
}

// The parts of the product left out of the chain when alpha is split (a2, a3 and the products'
// pieces), used only for a decision that falls on a rounding boundary.
struct SplitRest {
  float a2, a3, xf, p, p2, eB;
};

// The code of pack(RN64(s)) for s = h + l + t2 + r, where h + l + t2 comes from the TwoSum chain
// below and |r| <= margin (SPLIT = false: r = 0).  False sends the element to the binary64 path.
template <int K, int MODE, bool SPLIT>
__device__ __forceinline__ bool axpy_decide(float h, float l, float t2, float margin, const SplitRest& rest,
                                            uint64_t& code) {
  constexpr int m = 8 * K - 12;          // mantissa bits of the code
  constexpr int d = 23 - m;              // bits of h below the code's last bit
  constexpr bool kNearest = MODE == FLYTE_RNE || MODE == FLYTE_HALF_UP;
  constexpr float kB = kNearest ? float(1u << (d - 1)) : 0.f;   // boundary, in ulps of h
  // t2 != 0 needs p + y inexact, hence no cancellation in it, so |t2| <= 2^-23 ulp(s1) and
  // |l + t2| <= ulp(h) / 2 + tiny: L = RN(l + t2) errs by at most 2^-23 ulp(h), far inside the
  // 2^-20 ulp(h) guard below; the exact error is formed only when a decision falls on a boundary.
  const float L = __fadd_rn(l, t2);
  const uint32_t hb = __float_as_uint(h);
  const uint32_t E = (hb >> 23) & 0xFFu;
  bool ok = E >= 24u;                    // zero or too small for the exact code path: binary64
  const uint32_t M = hb & 0x7FFFFFu;
  const uint32_t D = M & ((1u << d) - 1u);
  const uint64_t Q = (uint64_t(E + 896u) << m) | (M >> d);
  const float uh = __uint_as_float(max(E, 24u) - 23u << 23);
  // r must stay below u_h / 4, so that s stays within the boundaries next to h: heavy
  // cancellation (|alpha x| above ~2^20 |s|) goes to binary64
  ok &= margin < __fmul_rn(uh, 0.25f);
  const bool neg = hb >> 31;
  const float Df = __fsub_rn(__uint_as_float(0x4B000000u | D), 8388608.0f);   // D exactly
  const float z = __fmul_rn(__fsub_rn(Df, kB), uh);                            // (D - B) u_h exactly
  const float w = __fadd_rn(z, neg ? -L : L);
  int sg = (w > 0.f) - (w < 0.f);                                              // sign of f - B
  if (!(fabsf(w) > __fmaf_rn(uh, 0x1p-20f, margin))) {
    float L2, Le;
    two_sum(l, t2, L2, Le);
    if constexpr (!SPLIT) {
      // s = h + l + t2 exactly: decided only when exactly on the boundary (these elements are
      // frequent with short x, y and a binary32 alpha, so this branch stays short)
      ok &= w == 0.f && Le == 0.f;
      sg = 0;
    } else {
      // Here |w| < u_h / 4 forces z = 0 or a cancellation, so w = z + L exactly, and s lies
      // F = w + Le + r (oriented like w) above the boundary, with Le the error of L and r the
      // terms left out of the chain.  The boundary lies within 0.6 u_h of h, so in h's binade
      // (or, when h is a power of two, at h itself), where half a binary64 ulp is
      // hu = 2^-53 2^e(h) (hu / 2 just below a power of two).  The binary64 fma rounds s onto
      // the boundary when |F| is below that and strictly to the side of F when |F| is above hu;
      // at hu binary64 decides.  r = eB + (a2 x - p2) + a3 x + (less than 2^-70 |p|), formed
      // as rc within re.
      const float e2 = __fmaf_rn(rest.a2, rest.xf, -rest.p2);
      const float p3 = __fmul_rn(rest.a3, rest.xf);
      const float rc = __fadd_rn(__fadd_rn(rest.eB, e2), p3);
      const float sa = __fadd_rn(__fadd_rn(fabsf(rest.eB), fabsf(e2)), fabsf(p3));
      const float re = __fadd_rn(__fmaf_rn(sa, 0x1p-22f, __fmul_rn(fabsf(rest.p), 0x1p-66f)), 0x1p-126f);
      const float F = __fadd_rn(__fadd_rn(w, neg ? -Le : Le), neg ? -rc : rc);
      const float eF = __fmaf_rn(__fadd_rn(__fadd_rn(fabsf(w), fabsf(Le)), fabsf(rc)), 0x1p-23f, re);
      const float hu = __uint_as_float(max(E, 54u) - 53u << 23);
      const bool snap = __fadd_rn(fabsf(F), eF) < (M == 0u ? __fmul_rn(hu, 0.5f) : hu);
      const bool beyond = __fsub_rn(fabsf(F), eF) > hu;
      ok &= E >= 100u && fabsf(w) < __fmul_rn(uh, 0.25f) && (snap || beyond);
      sg = snap ? 0 : (F > 0.f ? 1 : -1);
    }
  }
  uint64_t q;
  if constexpr (MODE == FLYTE_RNE) {
    q = sg < 0 ? Q : (sg > 0 ? Q + 1 : Q + (Q & 1));
  } else if constexpr (MODE == FLYTE_RTZ) {
    q = sg < 0 ? Q - 1 : Q;
  } else if constexpr (MODE == FLYTE_HALF_UP) {
    q = sg < 0 ? Q : Q + 1;
  } else {
    q = sg == 0 ? Q : ((sg < 0 ? Q - 1 : Q) | 1u);                            // round to odd
  }
  code = (uint64_t(neg) << (8 * K - 1)) | q;
  return ok;
}

// alpha a binary32 number af: s = p + e + y exactly.
template <int K, int MODE>
__device__ __forceinline__ bool axpy_exact_f32(uint64_t ux, uint64_t uy, float af, uint64_t& code) {
  float xf, yf, unused;
  bool ok = dbl_to_pair<K>(uint32_t(ux >> 32), 0u, xf, unused);
  ok &= dbl_to_pair<K>(uint32_t(uy >> 32), 0u, yf, unused);
  const float p = __fmul_rn(af, xf);
  const float e = __fmaf_rn(af, xf, -p);
  float s1, t1, s2, t2, h, l;
  two_sum(p, yf, s1, t1);
  two_sum(t1, e, s2, t2);
  two_sum(s1, s2, h, l);
  return axpy_decide<K, MODE, false>(h, l, t2, 0.f, SplitRest{}, code) && ok;
}

// scal, alpha a binary32 number af: s = af x = p + e exactly (TwoProd), |e| <= ulp(p) / 2, so
// (h, l, t2) = (p, e, 0) meets the premises of axpy_decide.
template <int K, int MODE>
__device__ __forceinline__ bool scal_exact_f32(uint64_t ux, float af, uint64_t& code) {
  float xf, unused;
  const bool ok = dbl_to_pair<K>(uint32_t(ux >> 32), 0u, xf, unused);
  const float p = __fmul_rn(af, xf);
  const float e = __fmaf_rn(af, xf, -p);
  return axpy_decide<K, MODE, false>(p, e, 0.f, 0.f, SplitRest{}, code) && ok;
}

// Any binary64 alpha inside the window, split as a1 = RN32(alpha), a2 = RN32(alpha - a1),
// a3 = RN32(alpha - a1 - a2) (|alpha - a1 - a2 - a3| <= 2^-72 |alpha|).  With p + e1 = a1 x
// (TwoProd), p2 = RN(a2 x) and eA + eB = e1 + p2 (TwoSum), the chain of the binary32 case runs on
// p, y and eA; the terms left out, eB, a2 x - p2 and (alpha - a1 - a2) x, are each at most about
// 2^-47 |p|, so |r| <= 2^-45 |p| bounds them, and a decision away from a boundary is taken only
// outside the guard widened by it.
template <int K, int MODE>
__device__ __forceinline__ bool axpy_exact_f32x2(uint64_t ux, uint64_t uy, float a1, float a2, float a3,
                                                 uint64_t& code) {
  float xf, yf, unused;
  bool ok = dbl_to_pair<K>(uint32_t(ux >> 32), 0u, xf, unused);
  ok &= dbl_to_pair<K>(uint32_t(uy >> 32), 0u, yf, unused);
  const float p = __fmul_rn(a1, xf);
  const float e1 = __fmaf_rn(a1, xf, -p);
  const float p2 = __fmul_rn(a2, xf);
  float eA, eB;
  two_sum(e1, p2, eA, eB);
  float s1, t1, s2, t2, h, l;
  two_sum(p, yf, s1, t1);
  two_sum(t1, eA, s2, t2);
  two_sum(s1, s2, h, l);
  return axpy_decide<K, MODE, true>(h, l, t2, __fmul_rn(fabsf(p), 0x1p-45f), SplitRest{a2, a3, xf, p, p2, eB},
                                    code) &&
         ok;
}

// Double-based k = 5, 6, 7 with a binary32 alpha a.  x and y have 29 to 45
// significant bits, so each is an exact binary32 pair (xh + xl, yh + yl:
// dbl_to_pair), and s = a x + y is carried exactly as
//   p1 + e1 = a xh, p2 + e2 = a xl                     (TwoProd)
//   s1 + t1 = p1 + yh, s2 + t2 = e1 + p2, s3 + t3 = s2 + yl,
//   s4 + t4 = s3 + t1, h + l = s1 + s4                  (TwoSum)
//   s = h + l + (t2 + t3 + t4 + e2)                     (exactly)
// with the last group, r, of order 2^-47 |a x|, formed in binary32 within
// 2^-21 of the sum of its terms' magnitudes.  The code keeps m = 8k - 12
// mantissa bits, more than h's 23, so h lies on the code grid and the
// rounding point falls inside l: in units U of the code's last bit,
// l / U = n + fl (n = floor, fl in [0, 1), both exact) and s lies fl + r/U
// code ulps above h + n U.  The decision reads that against the mode's
// boundary (1/2 for nearest-even and half-up; 0 and 1 for toward zero and
// round to odd), outside a guard of 2^(m-52) code ulps (twice the largest
// move of RN64, which precedes the pack) plus the error of r; exactly on a
// boundary (r = 0) it is exact, since such an s has at most m + 1 bits and
// RN64 leaves it alone.  Anything else goes to the binary64 fma: zero or
// out-of-window results, |r| >= U / 4 (heavy cancellation), s just below a
// power of two (a finer code grid), and elements within the guard.
// A randomised CPU mirror of this decision (13.2M elements: k = 5..7, all
// four modes, 11 binary32 alphas, N(0,1) data, short integers and planted
// near-cancellations) matched the oracle on every decided element; on
// N(0,1) data it sends 0.009 % (k = 5), 0.004 % (k = 6) and 0.23 % (k = 7) of
// the elements to binary64.
// HAS_Y = false: s = a x (scal), with yh = yl = 0 (the chain stays exact).
template <int K, int MODE, bool HAS_Y = true>
__device__ __forceinline__ bool axpy_exact_wide(uint64_t ux, uint64_t uy, float a, uint64_t& code) {
  static_assert(K >= 5 && K <= 7, "double-based k = 5..7");
  constexpr int m = 8 * K - 12;
  float xh, xl, yh = 0.f, yl = 0.f;
  bool ok = dbl_to_pair<K>(uint32_t(ux >> 32), uint32_t(ux), xh, xl);
  if constexpr (HAS_Y) ok &= dbl_to_pair<K>(uint32_t(uy >> 32), uint32_t(uy), yh, yl);
  const float p1 = __fmul_rn(a, xh), e1 = __fmaf_rn(a, xh, -p1);
  const float p2 = __fmul_rn(a, xl), e2 = __fmaf_rn(a, xl, -p2);
  float s1, t1, s2, t2, s3, t3, s4, t4, h, l;
  two_sum(p1, yh, s1, t1);
  two_sum(e1, p2, s2, t2);
  two_sum(s2, yl, s3, t3);
  two_sum(s3, t1, s4, t4);
  two_sum(s1, s4, h, l);
  float r = __fadd_rn(__fadd_rn(__fadd_rn(t2, t3), t4), e2);
  const float rmag = __fadd_rn(__fadd_rn(__fadd_rn(fabsf(t2), fabsf(t3)), fabsf(t4)), fabsf(e2));
  const uint32_t hb = __float_as_uint(h);
  const bool neg = hb >> 31;
  const uint32_t E = (hb >> 23) & 0xFFu, M = hb & 0x7FFFFFu;
  ok &= E >= 60u && E <= 200u;
  if (neg) {
    l = -l;
    r = -r;
  }
  ok &= !(M == 0u && (l < 0.f || (l == 0.f && r < 0.f)));
  // U = 2^(E - 127 - m); scaling by 1/U is exact (a power of two, normal for E in [60, 200])
  const float sc = __uint_as_float(uint32_t(254 + m - int(max(min(E, 200u), 60u))) << 23);
  const float lU = __fmul_rn(l, sc), rU = __fmul_rn(r, sc);
  const float eR = __fmul_rn(__fmul_rn(rmag, sc), 0x1p-21f);
  const float nf = floorf(lU);
  const float fl = __fsub_rn(lU, nf);
  constexpr float G = m == 28 ? 0x1p-24f : (m == 36 ? 0x1p-16f : 0x1p-8f);   // 2^(m - 52)
  const float guard = __fadd_rn(G, eR);
  ok &= fabsf(rU) < 0.25f;
  const int64_t Q = (int64_t(E + 896u) << m) | (int64_t(M) << (m - 23));
  const int64_t base = Q + int64_t(nf);
  int64_t q;
  if constexpr (MODE == FLYTE_RNE || MODE == FLYTE_HALF_UP) {
    const float w = __fadd_rn(__fsub_rn(fl, 0.5f), rU);
    if (fabsf(w) > guard) {
      q = base + (w > 0.f ? 1 : 0);
    } else {
      ok &= fl == 0.5f && r == 0.f;                     // exactly halfway
      q = MODE == FLYTE_HALF_UP ? base + 1 : base + (base & 1);
    }
  } else {
    const float f = __fadd_rn(fl, rU);
    if (f > guard && f < __fsub_rn(1.f, guard)) {
      q = MODE == FLYTE_RTO ? (base | 1) : base;
    } else {
      ok &= fl == 0.f && r == 0.f;                      // exactly on the grid
      q = base;
    }
  }
  code = (uint64_t(neg) << (8 * K - 1)) | uint64_t(q);
  return ok;
}

}  // namespace flyte
