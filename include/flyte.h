/*
 * flyte.h -- C ABI of the GB300 flyte library (libflyte.so).
 *
 * A flyte (Anderson & Gregg, "Vectorization of Multibyte Floating Point Data
 * Formats", PACT 2016) stores an IEEE-754 value in its top k bytes: the sign
 * and the full exponent of the next larger built-in type are kept and only
 * low mantissa bits are dropped (Sec. 3.1, Table 1).  Float-based flytes
 * widen to binary32 (k = 1..4), double-based ones to binary64 (k = 1..8).
 * Arrays of flytes are packed back to back, k bytes per element, least
 * significant byte first (Fig. 1, Sec. 4.1).
 *
 * Conventions for every entry point:
 *  - Data pointers are DEVICE pointers owned by the caller.  The library
 *    never allocates device memory; scratch space comes from the caller
 *    (see flyte_workspace_bytes).
 *  - Calls are asynchronous on `stream` (0 = the legacy default stream) and
 *    return once the work is enqueued.  No host synchronisation.
 *  - Strides (inc*, ld*) count ELEMENTS, not bytes, and must be >= 1.
 *  - A length or dimension of 0 is a no-op returning FLYTE_OK.
 *  - Argument errors are detected on the host before anything is launched
 *    and return a status; nothing is written in that case.  CUDA launch
 *    errors return FLYTE_ERR_CUDA.  flyte_last_error_string() describes the
 *    last failure of the calling thread.
 *  - Any pointer alignment is accepted; 16-byte aligned pointers (and, for
 *    matrices, rows that start on 16-byte boundaries) take the fastest
 *    paths.  dot and gemv keep their double-word arithmetic for any
 *    alignment (unaligned 4-element groups are assembled from aligned word
 *    loads); pack, unpack, axpy and scal fall back to per-element code.
 *  - Outputs must not overlap inputs, except y in flyte_axpy and x in
 *    flyte_scal, which are updated in place.
 *  - Kernels that stream through shared-memory copy rings (gemv 'N', gemm)
 *    bound every wait (200 ms).  A wait that gives up (a stalled copy
 *    engine; it does not happen in normal operation) sets the call's status
 *    word nonzero -- the first 4 bytes of its workspace, which the call
 *    resets to 0 -- and the outputs the call could not compute are written
 *    as NaN, so the failure is visible in the results too (for
 *    flyte_gemv_static, whose status word lies inside the library, only
 *    there).
 */
#ifndef FLYTE_H
#define FLYTE_H

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Native type a flyte widens to (Sec. 3.1: "the next largest built-in type"). */
typedef enum { FLYTE_F32 = 0, FLYTE_F64 = 1 } flyte_base;

/* Narrowing modes (Sec. 5).
 *  FLYTE_RNE      round to nearest, ties to even (Sec. 5.2), with IEEE
 *                 overflow to infinity and gradual underflow (Sec. 5.3).
 *  FLYTE_RTZ      round toward zero, i.e. truncation (Sec. 5.1); the mode
 *                 of the paper's experiments (Sec. 6).
 *  FLYTE_HALF_UP  add half an ULP and truncate (Fig. 6).
 *  FLYTE_RTO      round to odd (Sec. 7, after Boldo & Melquiond).
 * In every mode a NaN stays NaN: sign and high payload are kept and the
 * format's quiet bit is set (Sec. 5.3.4).  For k = 1, which keeps only 7
 * exponent bits and has no Inf/NaN codes, the magnitude saturates at 0x7F. */
typedef enum {
  FLYTE_RNE = 0,
  FLYTE_RTZ = 1,
  FLYTE_HALF_UP = 2,
  FLYTE_RTO = 3
} flyte_round;

typedef enum {
  FLYTE_OK = 0,
  FLYTE_ERR_INVALID_ARG = 1,   /* bad k/base/mode, null pointer, n < 0, stride < 1, lda too small */
  FLYTE_ERR_UNSUPPORTED = 2,   /* a valid combination this library does not implement */
  FLYTE_ERR_ALIGNMENT = 3,     /* reserved: an operation that requires an alignment */
  FLYTE_ERR_CUDA = 4,          /* a CUDA call or launch failed */
  FLYTE_ERR_WORKSPACE = 5      /* workspace pointer null or smaller than flyte_workspace_bytes() */
} flyte_status;

/* Format of a flyte operand: k bytes per element, widening to `base`.
 * Valid: base FLYTE_F32 with k in 1..4, base FLYTE_F64 with k in 1..8
 * (Table 1 lists 16..32 and 40..64 bits; the other widths follow the same
 * "top k bytes" rule).  k = 4 (F32) and k = 8 (F64) are the native types. */
typedef struct flyte_fmt {
  int32_t k;
  int32_t base; /* flyte_base */
} flyte_fmt;

/* ---- conversion (Sec. 3-5) ------------------------------------------------ */

/* Pack: dst element i (k bytes at byte (i*inc_dst)*k) = round(src[i*inc_src]).
 * src: n values of the native type of f.base (float or double), device.
 * dst: packed k-byte stream, device.  Bit-exact: rounding is done on the
 * integer pattern (Sec. 5), never through floating-point arithmetic, so NaN
 * payloads and subnormals are handled exactly.  The GPU writes each output
 * byte once; elements of different threads never share a store. */
flyte_status flyte_pack(void* dst, const void* src, int64_t n, flyte_fmt f, int64_t inc_dst,
                        int64_t inc_src, flyte_round mode, cudaStream_t stream);

/* Unpack: dst[i*inc_dst] (float or double per f.base) = the k-byte element
 * i*inc_src of src shifted left and padded with zero bits (Fig. 1: the
 * 24-bit pattern "num << 8"; Sec. 4.1).  Exact, no rounding. */
flyte_status flyte_unpack(void* dst, const void* src, int64_t n, flyte_fmt f, int64_t inc_dst,
                          int64_t inc_src, cudaStream_t stream);

/* ---- BLAS level 1 (Sec. 6) --------------------------------------------------- */

/* dot: *result_dev = sum_i x_i * y_i over the unpacked values, accumulated
 * at least in binary64 (the AT_LEAST rule of Sec. 4.4) whatever the bases.
 * result_dev: one double in device memory.  ws: device scratch of at least
 * flyte_workspace_bytes("dot", n, 0, 0, fx) bytes, 16-byte aligned.
 * Accuracy: |result - exact| <= 4 n 2^-53 sum |x_i y_i| for finite data;
 * NaN if any term is NaN or infinities of both signs occur, else +-Inf.
 * Deterministic: the same inputs give the same bits on every call. */
flyte_status flyte_dot(double* result_dev, int64_t n, const void* x, flyte_fmt fx, int64_t incx,
                       const void* y, flyte_fmt fy, int64_t incy, void* ws, size_t ws_bytes,
                       cudaStream_t stream);

/* axpy, in place: y_i <- pack(fma(alpha, x_i, y_i), mode) (FP_CONTRACT on,
 * Sec. 4.4 and 6).  The fma runs in the formats' native type: binary64 for
 * double-based, binary32 (alpha rounded to float) for float-based; fx.base
 * must equal fy.base (else FLYTE_ERR_UNSUPPORTED).  Bit-exact against a
 * correctly rounded fma followed by the pack of flyte_pack. */
flyte_status flyte_axpy(int64_t n, double alpha, const void* x, flyte_fmt fx, int64_t incx, void* y,
                        flyte_fmt fy, int64_t incy, flyte_round mode, cudaStream_t stream);

/* scal, in place: x_i <- pack(alpha * x_i, mode), the in-place "scale"
 * benchmark of Sec. 6 (reads and writes of the stream overlap).  The product
 * is rounded once in the format's native type: binary64 for double-based,
 * binary32 (alpha rounded to float) for float-based; then packed as
 * flyte_pack does.  Bit-exact. */
flyte_status flyte_scal(int64_t n, double alpha, void* x, flyte_fmt fx, int64_t incx, flyte_round mode,
                        cudaStream_t stream);

/* ---- BLAS level 2 (Sec. 6.3.2) ----------------------------------------------- */

/* gemv on a row-major k-byte matrix A (m rows, n columns, row i starts at
 * element i*lda, lda >= n):
 *   trans 'N': y_i <- alpha * sum_j A_ij x_j + beta * y_i,   i < m, x has n entries
 *   trans 'T': y_j <- alpha * sum_i A_ij x_i + beta * y_j,   j < n, x has m entries
 * x, y: binary64 device vectors with strides incx, incy.  Sums are formed
 * to binary64 accuracy; the epilogue is fma(alpha, t, beta * y).  BLAS quick
 * returns: beta == 0 means y is not read; alpha == 0 means A and x are not
 * read.  Accuracy: |y - y_exact| <= 4 (len + 2) 2^-53 (|alpha| sum |A x| + |beta y|).
 * ws: scratch of flyte_workspace_bytes("gemv_n" or "gemv_t", m, n, 0, fa) bytes. */
flyte_status flyte_gemv(char trans, int64_t m, int64_t n, double alpha, const void* A, flyte_fmt fa,
                        int64_t lda, const double* x, int64_t incx, double beta, double* y,
                        int64_t incy, void* ws, size_t ws_bytes, cudaStream_t stream);

/* gemv with y stored as double-based flytes (fy.base must be FLYTE_F64,
 * else FLYTE_ERR_UNSUPPORTED; fy.k = 1..8): the write path of Sec. 4.3 and
 * 5 applied to a BLAS result.  y_i (k bytes at element offset i*incy of the
 * byte stream y) is read as unpack(y_i) unless beta == 0, the binary64 value
 * fma(alpha, t_i, beta * unpack(y_i)) is formed as in flyte_gemv, and packed
 * with `mode` in the same kernel that forms it: the result equals
 * flyte_pack(flyte_gemv(..., unpack(y), ...)) bit for bit.  alpha == 0 gives
 * pack(beta * unpack(y)) (beta == 0: zero codes).  Same arguments, workspace
 * and errors as flyte_gemv otherwise. */
flyte_status flyte_gemv_packed_y(char trans, int64_t m, int64_t n, double alpha, const void* A, flyte_fmt fa,
                                 int64_t lda, const double* x, int64_t incx, double beta, void* y, flyte_fmt fy,
                                 int64_t incy, flyte_round mode, void* ws, size_t ws_bytes, cudaStream_t stream);

/* gemv without a workspace argument.  The paper has no counterpart: this is
 * for callers that cannot allocate device memory themselves (a plug-in inside
 * a framework that owns all device allocations, or a serving loop that must
 * not call cudaMalloc after start-up).  Same operation, arguments, accuracy
 * and errors as flyte_gemv, with the scratch taken from a 4 MiB array built
 * into the library (held by every GPU that loads it until exit):
 *  - a call needing more than 4 MiB (flyte_workspace_bytes("gemv_n" or
 *    "gemv_t", m, n, 0, fa)) returns FLYTE_ERR_WORKSPACE, launching nothing;
 *  - the first call on each device looks up the array's address
 *    (cudaGetSymbolAddress) with that device current: make it before any
 *    stream capture;
 *  - all calls share the array; nothing in it needs to start at zero, but
 *    calls whose kernels overlap on the GPU (different streams or threads)
 *    race on it.
 * Allocates nothing: no cudaMalloc, cudaFree or allocating library call. */
flyte_status flyte_gemv_static(char trans, int64_t m, int64_t n, double alpha, const void* A,
                               flyte_fmt fa, int64_t lda, const double* x, int64_t incx, double beta,
                               double* y, int64_t incy, cudaStream_t stream);

/* ---- BLAS level 3 (Sec. 6.3.3) ----------------------------------------------- */

/* gemm, row-major: C <- alpha * A B + beta * C with A m x k_ (lda >= k_),
 * B k_ x n (ldb >= n), C m x n (ldc >= n).  fa and fb must be equal.
 *   float-based k = 2: codes are bfloat16 bit patterns, tensor cores, FP32 accumulation
 *   float-based k = 3: each value split exactly into two bfloat16 terms, all
 *                      four cross products on tensor cores, FP32 accumulation
 *   float-based k = 4: binary32 inputs split into three bfloat16 terms
 *   float-based k = 1: the codes are the top byte of a bfloat16 pattern (exact)
 *   double-based: binary64 tensor-core (DMMA) products, binary64 C
 * C is float for float-based formats and double for double-based ones.
 * Accuracy (float-based): |C - C_exact| <= 2^-22 (|alpha| sum_l |A_il B_lj| + |beta C_ij|), for
 * operands of mixed signs and of one sign alike (checked up to K = 8192; the worst measured error
 * is 0.6-0.8 of the bound on one-signed data).  The tensor core accumulates in binary32 with
 * truncation; the library limits that error to short chunks of the K loop, adds the chunks
 * exactly, and for k <= 2 starts each chunk below zero so that its truncation errors cancel.
 * An Inf or NaN input gives the entries it meets the IEEE class of their sum (Sec. 5.3): NaN if a
 * term is NaN (or Inf * 0) or infinities of both signs meet, else the signed infinity.
 * (double-based): 4 k_ 2^-53 (same sums).
 * beta == 0: C is not read. */
flyte_status flyte_gemm(int64_t m, int64_t n, int64_t k_, double alpha, const void* A, flyte_fmt fa,
                        int64_t lda, const void* B, flyte_fmt fb, int64_t ldb, double beta, void* C,
                        int64_t ldc, void* ws, size_t ws_bytes, cudaStream_t stream);

/* gemm with C stored as flytes of the base of A and B (fc.base == fa.base,
 * else FLYTE_ERR_UNSUPPORTED; fc.k = 1..4 float-based, 1..8 double-based):
 * C_ij (fc.k bytes at element offset i*ldc + j of the byte stream C) is read
 * as unpack(C_ij) unless beta == 0, alpha * (A B)_ij + beta * unpack(C_ij) is
 * formed in C's native type exactly as flyte_gemm forms it, and packed with
 * `mode` by the thread that formed it (the write path of Sec. 4.3 and 5
 * fused into the epilogue): the result equals the pack of flyte_gemm's C for
 * C0 = unpack(C) bit for bit.  Same arguments, workspace and accuracy before
 * the final rounding as flyte_gemm. */
flyte_status flyte_gemm_packed_c(int64_t m, int64_t n, int64_t k_, double alpha, const void* A, flyte_fmt fa,
                                 int64_t lda, const void* B, flyte_fmt fb, int64_t ldb, double beta, void* C,
                                 flyte_fmt fc, int64_t ldc, flyte_round mode, void* ws, size_t ws_bytes,
                                 cudaStream_t stream);

/* ---- mixed-precision iterative refinement ------------------------------------ */

/* Solve A x = b (n x n, row-major) for a diagonally dominant A, keeping A
 * twice: A64 in binary64 (lda64) for the residual and Ak, the same matrix as
 * k-byte flytes (fa, lda), for the correction sweeps -- the paper's premise
 * (Sec. 1-2) that storage precision can follow what the algorithm needs.
 *   repeat:  r = b - A64 x  (flyte_gemv with k = 8);  stop if ||r||_2 <= tol ||b||_2
 *            or after max_outer corrections;
 *            d = 0; `inner` times: d <- d + D^-1 (r - Ak d)  (Jacobi-Richardson,
 *            flyte_gemv on Ak; D = diag(A64));  x <- x + d
 * x: device vector, the initial guess on entry, the solution on return.
 * ws: flyte_workspace_bytes("refine", n, n, 0, fa) bytes, 256-byte aligned.
 * *iters (may be NULL): corrections applied; *relres (may be NULL): the last
 * ||r||_2 / ||b||_2.  Unlike the other entry points this call is synchronous:
 * it reads one norm back to the host per outer iteration (stream s). */
flyte_status flyte_refine_jacobi(int64_t n, const double* A64, int64_t lda64, const void* Ak, flyte_fmt fa,
                                 int64_t lda, const double* b, double* x, double tol, int max_outer, int inner,
                                 void* ws, size_t ws_bytes, cudaStream_t stream, int* iters, double* relres);

/* ---- batches of uneven jobs in one persistent launch ------------------------ */

/* Many small operations of mixed widths amortise launch latency when they
 * run as the tiles of one persistent kernel (the GPU counterpart of the
 * paper's unrolled loops over mixed data, Sec. 6).  A job is one of: */
typedef enum {
  FLYTE_JOB_UNPACK = 0, /* y[i] = unpack(x_i), i < n; y native (float/double per fx.base) */
  FLYTE_JOB_DOT = 1,    /* *result = sum_i x_i y_i over two flyte streams (fx, fy), i < n */
  FLYTE_JOB_AXPY = 2,   /* y_i <- pack(fma(alpha, x_i, y_i), mode), i < n (fx.base == fy.base) */
  FLYTE_JOB_GEMV_N = 3, /* y <- alpha A x + beta y; A m x n k-byte (fx), lda = n; x, y binary64 */
  FLYTE_JOB_GEMV_T = 4  /* y <- alpha A^T x + beta y; same A */
} flyte_job_op;

/* One job (88 bytes, host memory when handed to flyte_batch_prepare).  All
 * strides are 1 and matrices are dense (lda = n).  Semantics, accuracy and
 * quick returns are those of flyte_unpack / flyte_dot / flyte_axpy /
 * flyte_gemv. */
typedef struct flyte_job {
  int32_t op;         /* flyte_job_op */
  int32_t mode;       /* flyte_round (AXPY) */
  flyte_fmt fx;       /* x stream (UNPACK, DOT, AXPY) or A (GEMV) */
  flyte_fmt fy;       /* y stream (DOT, AXPY); unused otherwise */
  int64_t m, n;       /* GEMV: A is m x n; others: n elements (m unused) */
  const void* a;      /* UNPACK/DOT/AXPY: x stream; GEMV: A */
  const double* xv;   /* GEMV: x (n entries for N, m for T) */
  void* y;            /* UNPACK: output; DOT: y stream; AXPY: y stream (in/out); GEMV: y */
  double* result;     /* DOT: one double in device memory */
  double alpha, beta; /* AXPY: alpha; GEMV: alpha, beta */
} flyte_job;

/* Plan a batch: split every job into tiles (tile sizes per (operation, k,
 * base) from the table that flyte_batch_autotune fills, or built-in
 * defaults), and upload the job and tile tables into ws (device, 256-byte
 * aligned, flyte_batch_workspace_bytes(jobs, njobs) bytes).  Validates every
 * job first (FLYTE_ERR_INVALID_ARG / FLYTE_ERR_UNSUPPORTED naming the job).
 * Synchronous: returns when the tables are on the device.  Not capturable in
 * a CUDA graph; the launch below is. */
flyte_status flyte_batch_prepare(const flyte_job* jobs, int32_t njobs, void* ws, size_t ws_bytes,
                                 cudaStream_t stream);
size_t flyte_batch_workspace_bytes(const flyte_job* jobs, int32_t njobs);

/* Run a prepared batch: a small kernel that splits the x of every gemv 'N'
 * job once into its binary32 pair (into ws), then one persistent kernel (one
 * block per resident slot) whose blocks take tiles from a counter in ws
 * until none are left; a dot's partial sums are added in tile order by the
 * block that finishes its last tile, so results are deterministic.  Asynchronous, allocates nothing and
 * may be captured in a CUDA graph and replayed (ws must stay untouched
 * between prepare and the last replay).  Jobs in one batch must not write
 * memory that another job of the batch reads or writes. */
flyte_status flyte_batch_launch(void* ws, cudaStream_t stream);

/* Time the candidate tile sizes of each (operation, k, base) on synthetic
 * jobs (scratch from ws_bytes of device memory at ws, at least
 * flyte_batch_autotune_bytes()) and keep the fastest in the library's tile
 * table, which later flyte_batch_prepare calls use.  Synchronous. */
flyte_status flyte_batch_autotune(void* ws, size_t ws_bytes, cudaStream_t stream);
size_t flyte_batch_autotune_bytes(void);

/* Tune the same table, and the number of resident blocks per SM of the
 * persistent launch, on the caller's own batch (the GPU counterpart of the
 * paper's unrolling study, Sec. 6, on the workload itself): first the
 * resident blocks per SM, then the tile size of every (operation, k, base)
 * present in jobs, each candidate timed as the whole batch (prepare, one
 * untimed and three timed launches); a candidate is kept when it is at least
 * 1 % faster.  Tile candidates: 16384..262144 elements (unpack, dot, axpy),
 * 4..32 rows (gemv N), 128..512 rows per 1024-column block (gemv T); those
 * whose tables do not fit in ws_bytes are skipped.  ws: device, 256-byte
 * aligned.  The jobs run several times, so in-place outputs (axpy y) change:
 * tune on scratch copies or re-initialise them.  Synchronous. */
flyte_status flyte_batch_autotune_jobs(const flyte_job* jobs, int32_t njobs, void* ws, size_t ws_bytes,
                                       cudaStream_t stream);

/* The current tile size of (op, f) in the table (elements, or rows for gemv), or -1 for an
 * invalid pair; and the resident blocks per SM the persistent launch uses. */
int64_t flyte_batch_tile_size(int32_t op, flyte_fmt f);
int32_t flyte_batch_resident_blocks(void);

/* ---- helpers ---------------------------------------------------------------- */

/* Scratch bytes an operation needs for the given sizes: op is "dot",
 * "gemv_n", "gemv_t", "gemm" or "refine" (m, n, k_ as in that call; unused
 * ones 0).
 * Returns 0 for an operation that needs none and (size_t)-1 for an unknown
 * op.  The amount depends only on the arguments, never on the device. */
size_t flyte_workspace_bytes(const char* op, int64_t m, int64_t n, int64_t k_, flyte_fmt f);

/* Description of the last failure on the calling host thread ("" if none). */
const char* flyte_last_error_string(void);

/* Library version, major * 10000 + minor * 100 + patch. */
int flyte_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FLYTE_H */
