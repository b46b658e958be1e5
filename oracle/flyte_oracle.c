/*
 * flyte_oracle.c -- plain, slow, scalar CPU oracle for the flyte multibyte
 * floating-point scheme of Anderson & Gregg, "Vectorization of Multibyte
 * Floating Point Data Formats" (PACT 2016).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the checker the GPU library is
 * compared against.  Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg may load it.  It shares no code, header, table or constant
 * generator with the CUDA library, and includes none of its headers.
 *
 * Everything here is written for a reader who checks it against the paper by
 * eye: one element at a time, in the order the paper's sections describe,
 * no blocking, no fusion.  Compile with -O2 -ffp-contract=off (no fast-math):
 * the only fused multiply-adds are the explicit fma() calls.
 *
 * Conventions (integer codes so the Python side can pass plain ints):
 *   base 0 = binary32-based flyte (k = 1..4), base 1 = binary64-based (k = 1..8)
 *   mode 0 = round to nearest, ties to even (Sec. 5.2)
 *   mode 1 = round toward zero / truncation (Sec. 5.1, the mode of Sec. 6)
 *   mode 2 = add half an ULP then truncate (the heuristic of Fig. 6)
 *   mode 3 = round to odd (Sec. 7 names it, after Boldo & Melquiond, as a
 *            narrowing that avoids double-rounding errors): truncate, and
 *            set the last kept bit if any dropped bit was set
 * A flyte code q is the top 8k bits of the native IEEE-754 pattern u
 * (Sec. 3.1, Table 1: sign and the full native exponent are kept, only low
 * mantissa bits are dropped).  Codes are stored back to back, k bytes each,
 * least significant byte first (Fig. 1's packed bit-field on a little-endian
 * machine; Sec. 4.1).
 *
 * Readings of the paper used here (where it is silent):
 *   - NaN in, NaN out for every mode: the format's quiet bit is forced, the
 *     sign and the high payload bits are kept (Sec. 5.1 and 5.3 say a NaN
 *     should stay NaN and that truncation may otherwise turn a signalling
 *     NaN into an infinity).
 *   - k = 1 keeps only 7 of the exponent bits, so it has no Inf/NaN codes:
 *     rounding is done on the bit pattern and the magnitude saturates at
 *     0x7F (Inf and NaN pack to sign|0x7F).  Table 1 does not list k = 1.
 *   - k = 8 (double) and k = 4 (float) pack is the identity, NaNs included.
 *   - Status: functions return 0 on success, -1 on a bad argument.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---- format parameters (Table 1) -------------------------------------- */

static int orc_valid(int base, int k)
{
    if (base == 0) return k >= 1 && k <= 4;
    if (base == 1) return k >= 1 && k <= 8;
    return 0;
}

/* W: width of the next largest built-in type in bits (Sec. 3.1). */
static int native_bits(int base) { return base == 0 ? 32 : 64; }
/* E: exponent width, the same as the built-in type's (Sec. 3.1). */
static int exp_bits(int base) { return base == 0 ? 8 : 11; }

static uint64_t low_mask(int bits)
{
    return bits >= 64 ? ~(uint64_t)0 : (((uint64_t)1 << bits) - 1);
}

/* ---- byte stream (Fig. 1, Sec. 4.1) ------------------------------------ */

/* Element of k bytes, least significant byte first. */
uint64_t orc_read_code(const uint8_t *p, int k)
{
    uint64_t q = 0;
    for (int b = k - 1; b >= 0; --b) q = (q << 8) | p[b];
    return q;
}

void orc_write_code(uint8_t *p, int k, uint64_t q)
{
    for (int b = 0; b < k; ++b) {
        p[b] = (uint8_t)(q & 0xFF);
        q >>= 8;
    }
}

/* ---- unpack (Fig. 1: "num << 8"; Sec. 4.1: shift and pad with zeros) ---- */

/* Widen a k-byte code to the native W-bit pattern: exact, no rounding. */
uint64_t orc_unpack_code(int base, int k, uint64_t q)
{
    int d = native_bits(base) - 8 * k;    /* dropped low bits */
    return (q << d) & low_mask(native_bits(base));
}

/* ---- pack (Sec. 5) ------------------------------------------------------ */

/* Narrow a native W-bit pattern u to a k-byte code with the given mode. */
uint64_t orc_pack_bits(int base, int k, int mode, uint64_t u)
{
    const int W = native_bits(base);
    const int E = exp_bits(base);
    const int d = W - 8 * k;                      /* bits dropped */
    const int M = W - 1 - E;                      /* native mantissa bits */

    u &= low_mask(W);
    if (d == 0) return u;                         /* full width: identity */

    const uint64_t sign = u >> (W - 1);
    const uint64_t mag = u & low_mask(W - 1);
    const uint64_t exp_field = mag >> M;
    const uint64_t mant_field = mag & low_mask(M);
    const int is_special = exp_field == low_mask(E);       /* Inf or NaN */
    const int is_nan = is_special && mant_field != 0;

    const uint64_t half = (uint64_t)1 << (d - 1);           /* 1/2 ULP of the flyte */
    const uint64_t dropped = mag & low_mask(d);
    uint64_t t = mag >> d;                                   /* truncated magnitude */

    if (k == 1) {
        /* Only 7 exponent bits survive: no Inf/NaN codes exist.  Round the
         * bit pattern as an integer and saturate the magnitude at 0x7F so
         * that a carry never reaches the sign bit. */
        if (is_special) {
            t = 0x7F;
        } else {
            if (mode == 0) {
                if (dropped > half || (dropped == half && (t & 1))) t += 1;
            } else if (mode == 2) {
                if (dropped >= half) t += 1;
            } else if (mode == 3) {
                if (dropped != 0) t |= 1;
            }
            if (t > 0x7F) t = 0x7F;
        }
        return (sign << 7) | t;
    }

    if (is_nan) {
        /* NaN stays NaN: keep the high payload and force the quiet bit,
         * which is the most significant mantissa bit of the flyte. */
        const uint64_t quiet = (uint64_t)1 << (8 * k - 2 - E);
        return (sign << (8 * k - 1)) | t | quiet;
    }

    if (mode == 0) {
        /* Round to nearest, ties to even (Sec. 5.2): above half rounds up,
         * exactly half rounds to the even neighbour.  A carry out of the
         * mantissa moves into the exponent, which is the correctly rounded
         * result (a subnormal may become the smallest normal, the largest
         * finite value may become infinity, Sec. 5.3). */
        if (dropped > half || (dropped == half && (t & 1))) t += 1;
    } else if (mode == 2) {
        /* Fig. 6: add half an ULP of the flyte, then truncate. */
        t = (mag + half) >> d;
    } else if (mode == 3) {
        /* Round to odd: a dropped nonzero part makes the kept value odd. */
        if (dropped != 0) t |= 1;
    }
    /* mode 1 (round toward zero, Sec. 5.1): plain truncation, t as is. */
    return (sign << (8 * k - 1)) | t;
}

/* ---- array conversion -------------------------------------------------- */

static uint64_t load_native(int base, const void *src, int64_t i)
{
    if (base == 0) {
        uint32_t v;
        memcpy(&v, (const uint8_t *)src + 4 * i, 4);
        return v;
    } else {
        uint64_t v;
        memcpy(&v, (const uint8_t *)src + 8 * i, 8);
        return v;
    }
}

static void store_native(int base, void *dst, int64_t i, uint64_t v)
{
    if (base == 0) {
        uint32_t w = (uint32_t)v;
        memcpy((uint8_t *)dst + 4 * i, &w, 4);
    } else {
        memcpy((uint8_t *)dst + 8 * i, &v, 8);
    }
}

/* dst[i*inc_dst] = unpack(src element i*inc_src); strides in elements. */
int orc_unpack(int base, int k, const uint8_t *src, int64_t n, int64_t inc_src,
               void *dst, int64_t inc_dst)
{
    if (!orc_valid(base, k) || n < 0 || inc_src < 1 || inc_dst < 1) return -1;
    for (int64_t i = 0; i < n; ++i) {
        uint64_t q = orc_read_code(src + (size_t)(i * inc_src) * (size_t)k, k);
        store_native(base, dst, i * inc_dst, orc_unpack_code(base, k, q));
    }
    return 0;
}

/* dst element i*inc_dst = pack(src[i*inc_src]). */
int orc_pack(int base, int k, int mode, const void *src, int64_t n, int64_t inc_src,
             uint8_t *dst, int64_t inc_dst)
{
    if (!orc_valid(base, k) || mode < 0 || mode > 3 || n < 0 || inc_src < 1 || inc_dst < 1)
        return -1;
    for (int64_t i = 0; i < n; ++i) {
        uint64_t u = load_native(base, src, i * inc_src);
        orc_write_code(dst + (size_t)(i * inc_dst) * (size_t)k, k, orc_pack_bits(base, k, mode, u));
    }
    return 0;
}

/* Value of the flyte element at p, widened exactly to double. */
static double code_value(int base, int k, const uint8_t *p)
{
    uint64_t u = orc_unpack_code(base, k, orc_read_code(p, k));
    if (base == 0) {
        uint32_t w = (uint32_t)u;
        float f;
        memcpy(&f, &w, 4);
        return (double)f;
    }
    double v;
    memcpy(&v, &u, 8);
    return v;
}

double orc_code_value(int base, int k, const uint8_t *p) { return code_value(base, k, p); }

/* ---- error-free transformations (Ogita, Rump & Oishi 2005) ------------- */

static void two_sum(double a, double b, double *s, double *e)
{
    double x = a + b;
    double z = x - a;
    *e = (a - (x - z)) + (b - z);
    *s = x;
}

static void two_prod(double a, double b, double *p, double *e)
{
    double x = a * b;
    *e = fma(a, b, -x);
    *p = x;
}

/* Dot2: the dot product computed as if in twice the working precision.
 * The error-free transformations are only defined for finite terms (the
 * TwoProduct of an infinity yields inf - inf = NaN), so when any product is
 * Inf or NaN the plain binary64 sum is returned instead: NaN if a term is
 * NaN or infinities of both signs occur, else the signed infinity, as the
 * special-value rules of Sec. 5.3 require. */
static double dot2(int64_t n, const double *x, const double *y, double *naive, double *absum)
{
    double p = 0.0, s = 0.0, nv = 0.0, ab = 0.0;
    int finite = 1;
    for (int64_t i = 0; i < n; ++i) {
        double h, r, q;
        if (!isfinite(x[i] * y[i])) finite = 0;
        two_prod(x[i], y[i], &h, &r);
        two_sum(p, h, &p, &q);
        s = s + (q + r);
        nv = nv + x[i] * y[i];
        ab = ab + fabs(x[i] * y[i]);
    }
    if (naive) *naive = nv;
    if (absum) *absum = ab;
    return finite ? p + s : nv;
}

/* ---- dot (BLAS level 1; accumulation AT_LEAST the flyte, Sec. 4.4) ------ */

/* out[0] = Dot2 reference, out[1] = naive FP64 loop, out[2] = sum |x_i y_i|. */
int orc_dot(int64_t n, const uint8_t *x, int bx, int kx, int64_t incx,
            const uint8_t *y, int by, int ky, int64_t incy, double *out)
{
    if (!orc_valid(bx, kx) || !orc_valid(by, ky) || n < 0 || incx < 1 || incy < 1) return -1;
    double *xv = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *yv = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!xv || !yv) { free(xv); free(yv); return -1; }
    for (int64_t i = 0; i < n; ++i) {
        xv[i] = code_value(bx, kx, x + (size_t)(i * incx) * (size_t)kx);
        yv[i] = code_value(by, ky, y + (size_t)(i * incy) * (size_t)ky);
    }
    out[0] = dot2(n, xv, yv, &out[1], &out[2]);
    free(xv);
    free(yv);
    return 0;
}

/* ---- axpy (BLAS level 1; FP_CONTRACT on, Sec. 4.4 and 6) ---------------- */

/* y_i <- pack(fma(alpha, x_i, y_i)), in place on the k-byte stream y.  The
 * arithmetic is done in the formats' native type (Sec. 3.1: a flyte is
 * converted to the next largest built-in type before computation): binary64
 * for double-based formats, binary32 (alpha rounded to binary32) for
 * float-based ones.  x and y must share the base. */
int orc_axpy(int64_t n, double alpha, const uint8_t *x, int bx, int kx, int64_t incx,
             uint8_t *y, int by, int ky, int64_t incy, int mode)
{
    if (!orc_valid(bx, kx) || !orc_valid(by, ky) || bx != by || n < 0 || incx < 1 || incy < 1 ||
        mode < 0 || mode > 3)
        return -1;
    const float alpha_f = (float)alpha;
    for (int64_t i = 0; i < n; ++i) {
        uint8_t *py = y + (size_t)(i * incy) * (size_t)ky;
        double xi = code_value(bx, kx, x + (size_t)(i * incx) * (size_t)kx);
        double yi = code_value(by, ky, py);
        uint64_t u;
        if (by == 0) {
            float r = fmaf(alpha_f, (float)xi, (float)yi);   /* both exact in binary32 */
            uint32_t w;
            memcpy(&w, &r, 4);
            u = w;
        } else {
            double r = fma(alpha, xi, yi);
            memcpy(&u, &r, 8);
        }
        orc_write_code(py, ky, orc_pack_bits(by, ky, mode, u));
    }
    return 0;
}

/* ---- scal (the in-place "scale" benchmark of Sec. 6) -------------------- */

/* x_i <- pack(alpha * x_i), in place on the k-byte stream x.  The product is
 * rounded once in the native type, as in orc_axpy: binary64 for double-based
 * formats, binary32 with alpha rounded to binary32 for float-based ones. */
int orc_scal(int64_t n, double alpha, uint8_t *x, int bx, int kx, int64_t incx, int mode)
{
    if (!orc_valid(bx, kx) || n < 0 || incx < 1 || mode < 0 || mode > 3) return -1;
    const float alpha_f = (float)alpha;
    for (int64_t i = 0; i < n; ++i) {
        uint8_t *px = x + (size_t)(i * incx) * (size_t)kx;
        double xi = code_value(bx, kx, px);
        uint64_t u;
        if (bx == 0) {
            float r = alpha_f * (float)xi;
            uint32_t w;
            memcpy(&w, &r, 4);
            u = w;
        } else {
            double r = alpha * xi;
            memcpy(&u, &r, 8);
        }
        orc_write_code(px, kx, orc_pack_bits(bx, kx, mode, u));
    }
    return 0;
}

/* ---- gemv (BLAS level 2, Sec. 6.3.2) ------------------------------------ */

/* Row-major A (m x n, leading dimension lda elements, k-byte codes).
 * trans 'N': y_i <- alpha * sum_j A_ij x_j + beta * y_i, i < m
 * trans 'T': y_j <- alpha * sum_i A_ij x_i + beta * y_j, j < n
 * The dot products use Dot2; absum (length of y) receives sum |A x| terms. */
int orc_gemv(char trans, int64_t m, int64_t n, double alpha, const uint8_t *A, int base, int k,
             int64_t lda, const double *x, int64_t incx, double beta, double *y, int64_t incy,
             double *absum)
{
    if (!orc_valid(base, k) || m < 0 || n < 0 || lda < (n > 1 ? n : 1) || incx < 1 || incy < 1)
        return -1;
    if (trans != 'N' && trans != 'T') return -1;
    const int64_t leny = trans == 'N' ? m : n;
    const int64_t lenx = trans == 'N' ? n : m;
    double *a = (double *)malloc(sizeof(double) * (size_t)(lenx > 0 ? lenx : 1));
    double *xv = (double *)malloc(sizeof(double) * (size_t)(lenx > 0 ? lenx : 1));
    if (!a || !xv) { free(a); free(xv); return -1; }
    for (int64_t j = 0; j < lenx; ++j) xv[j] = x[j * incx];
    for (int64_t i = 0; i < leny; ++i) {
        double t = 0.0, ab = 0.0;
        if (alpha != 0.0) {
            for (int64_t j = 0; j < lenx; ++j) {
                int64_t r = trans == 'N' ? i : j;
                int64_t c = trans == 'N' ? j : i;
                a[j] = code_value(base, k, A + (size_t)(r * lda + c) * (size_t)k);
            }
            t = dot2(lenx, a, xv, NULL, &ab);
        }
        double *yi = &y[i * incy];
        if (absum) absum[i] = ab;
        if (beta == 0.0) {
            *yi = alpha * t;                 /* y is not read when beta = 0 */
        } else if (alpha == 0.0) {
            *yi = beta * *yi;                /* A and x are not read when alpha = 0 */
        } else {
            *yi = fma(alpha, t, beta * *yi);
        }
    }
    free(a);
    free(xv);
    return 0;
}

/* ---- mixed-precision iterative refinement ------------------------------- */

/* Solve A x = b with the residual on the binary64 matrix A64 (read as k = 8
 * double-based codes) and Jacobi-Richardson correction sweeps on the k-byte
 * copy Ak, in the order of the library's description:
 *   r = b - A64 x; stop if ||r|| <= tol ||b|| or after max_outer corrections;
 *   d = 0; inner times: d = d + (r - Ak d) / diag(A64); x = x + d.
 * Products use orc_gemv (Dot2); norms are plain binary64 sums of squares.
 * x holds the initial guess and receives the result. */
int orc_refine_jacobi(int64_t n, const uint8_t *A64, int64_t lda64, const uint8_t *Ak, int base, int k,
                      int64_t lda, const double *b, double *x, double tol, int max_outer, int inner,
                      int *iters, double *relres)
{
    if (!orc_valid(base, k) || n < 0 || lda64 < n || lda < n || max_outer < 0 || inner < 1) return -1;
    double *r = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *t = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *d = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *diag = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!r || !t || !d || !diag) { free(r); free(t); free(d); free(diag); return -1; }
    double bb = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        bb += b[i] * b[i];
        diag[i] = code_value(1, 8, A64 + (size_t)(i * lda64 + i) * 8u);
    }
    const double bnorm = sqrt(bb);
    int it = 0;
    double rel = 0.0;
    for (;; ++it) {
        memcpy(r, b, sizeof(double) * (size_t)n);
        orc_gemv('N', n, n, -1.0, A64, 1, 8, lda64, x, 1, 1.0, r, 1, NULL);
        double rr = 0.0;
        for (int64_t i = 0; i < n; ++i) rr += r[i] * r[i];
        rel = bnorm > 0.0 ? sqrt(rr) / bnorm : sqrt(rr);
        if (!(rel > tol) || it >= max_outer) break;
        for (int64_t i = 0; i < n; ++i) d[i] = 0.0;
        for (int j = 0; j < inner; ++j) {
            memcpy(t, r, sizeof(double) * (size_t)n);
            if (j > 0) orc_gemv('N', n, n, -1.0, Ak, base, k, lda, d, 1, 1.0, t, 1, NULL);
            for (int64_t i = 0; i < n; ++i) d[i] = d[i] + t[i] / diag[i];
        }
        for (int64_t i = 0; i < n; ++i) x[i] += d[i];
    }
    if (iters) *iters = it;
    if (relres) *relres = rel;
    free(r); free(t); free(d); free(diag);
    return 0;
}

/* ---- gemm (BLAS level 3, Sec. 6.3.3) ------------------------------------ */

/* C_ij for the listed (i, j) pairs of row-major C = alpha*A*B + beta*C0, with
 * A m x kk (lda), B kk x n (ldb), both k-byte codes of their own format.  The
 * sum uses Dot2.  cin holds C0_ij (may be NULL when beta = 0); out receives
 * the reference and absum the sum |A_il B_lj|. */
int orc_gemm_entries(int64_t npairs, const int64_t *rows, const int64_t *cols, int64_t kk,
                     double alpha, const uint8_t *A, int ba, int ka, int64_t lda,
                     const uint8_t *B, int bb, int kb, int64_t ldb, double beta,
                     const double *cin, double *out, double *absum)
{
    if (!orc_valid(ba, ka) || !orc_valid(bb, kb) || kk < 0 || npairs < 0) return -1;
    double *a = (double *)malloc(sizeof(double) * (size_t)(kk > 0 ? kk : 1));
    double *b = (double *)malloc(sizeof(double) * (size_t)(kk > 0 ? kk : 1));
    if (!a || !b) { free(a); free(b); return -1; }
    for (int64_t p = 0; p < npairs; ++p) {
        const int64_t i = rows[p], j = cols[p];
        double t = 0.0, ab = 0.0;
        if (alpha != 0.0) {
            for (int64_t l = 0; l < kk; ++l) {
                a[l] = code_value(ba, ka, A + (size_t)(i * lda + l) * (size_t)ka);
                b[l] = code_value(bb, kb, B + (size_t)(l * ldb + j) * (size_t)kb);
            }
            t = dot2(kk, a, b, NULL, &ab);
        }
        double c0 = (beta != 0.0 && cin) ? cin[p] : 0.0;
        if (beta == 0.0) out[p] = alpha * t;
        else if (alpha == 0.0) out[p] = beta * c0;
        else out[p] = fma(alpha, t, beta * c0);
        if (absum) absum[p] = ab;
    }
    free(a);
    free(b);
    return 0;
}
