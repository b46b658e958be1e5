// gemm.cu -- C <- alpha A B + beta C on row-major k-byte operands (Sec. 6, BLAS level 3).
//
// Float-based formats run on the tensor cores (tcgen05, bf16 inputs, fp32
// accumulation in TMEM).  Every float-based flyte value is an exact sum of
// bf16 "parts": k <= 2 codes are bf16 patterns already (one part), a k = 3
// value is hi + lo with hi its top 16 bits and lo = v - hi (<= 8 significant
// bits), and a binary32 (k = 4) value splits into three parts by repeated
// rounding to bf16.  C is the sum of the part products that matter for the
// 2^-22 bound: all 4 for k = 3 (hi*hi, hi*lo, lo*hi, lo*lo), 6 of 9 for
// k = 4 (the dropped ones are below 2^-26 |ab|).
//
// A preparation pass writes the parts of A (m x k) and of B transposed
// (n x k) as K-major bf16 arrays in the workspace; for k = 2 an A whose rows
// are 16-byte aligned is used in place.  The main kernel is a TMA -> shared
// memory -> tcgen05.mma pipeline: one thread issues the TMA loads of all
// parts of a 64-wide k-block into a ring of stages, one thread issues the
// MMAs (4 per product and k-block, each 128 x 128 x 16) into a ring of TMEM
// chunk accumulators and releases stages with tcgen05.commit, and sixteen
// epilogue warps add each chunk exactly into a (hi, lo) pair of binary32
// registers per output (TwoSum, two outputs per f32x2 instruction), so that
// the only rounding errors left are the tensor core's own inside a chunk and
// the final rounding of hi + lo.  An Inf or NaN input of a split format
// marks its row or column, and those entries get their IEEE class from a
// small kernel afterwards.  Waits are bounded (bulkpipe.cuh).
//
// Double-based formats use binary64 tensor-core MMAs (mma.sync m8n8k4, DMMA)
// on operands widened to binary64 in shared memory.
#include <cstring>

#include "dwacc.cuh"
#include "tcgen05.cuh"

namespace flyte {
namespace {

#ifndef FLYTE_GEMM_CHUNK1
#define FLYTE_GEMM_CHUNK1 4            // k-blocks per TMEM chunk for one-part formats
#endif


constexpr int kBM = 128;
constexpr int kBK = 64;                // bf16 elements per row of a stage tile (128 bytes)
constexpr int kSmemBudget = 224 * 1024;

// ---- bf16 parts of a float-based value ----------------------------------------------

__device__ __forceinline__ uint16_t bf16_rn(float f) {
  // round to nearest even; callers pass finite values whose rounding cannot overflow
  const uint32_t u = __float_as_uint(f);
  return uint16_t((u + 0x7FFFu + ((u >> 16) & 1u)) >> 16);
}
__device__ __forceinline__ float bf16_to_float(uint16_t b) { return __uint_as_float(uint32_t(b) << 16); }

__device__ __forceinline__ bool finite_bits(uint32_t u) { return (u & 0x7F800000u) != 0x7F800000u; }

// NP parts p[0..NP) of the widened value u (a binary32 pattern).  A non-finite
// value of a split format (k = 3, 4) keeps its class in p[0] (a NaN stays a
// quiet NaN) and zero low parts; the entries it touches are recomputed with
// IEEE semantics afterwards (gemm_special_entries), since any split of an
// infinity meets a zero part of its partner (Inf * 0 = NaN).
template <int K, int NP>
__device__ __forceinline__ void split_parts(uint32_t u, uint16_t (&p)[3]) {
  if constexpr (K <= 2) {
    p[0] = uint16_t(u >> 16);                       // the code itself, an exact bf16
  } else if (!finite_bits(u)) {
    p[0] = uint16_t(u >> 16) | uint16_t((u & 0x7FFFFFu) != 0 ? 0x40u : 0u);
    p[1] = 0;
    if constexpr (NP == 3) p[2] = 0;
  } else if constexpr (K == 3) {
    p[0] = uint16_t(u >> 16);                       // hi: top 16 bits
    const float lo = __fsub_rn(__uint_as_float(u), __uint_as_float(u & 0xFFFF0000u));
    p[1] = bf16_rn(lo);                             // exact (<= 8 significant bits)
  } else {
    const float f = __uint_as_float(u);
    // the top part rounds to nearest, except where that would overflow to
    // infinity (|f| >= 0x7F7F8000): there it is the truncation, which is exact
    // too and leaves a finite remainder
    p[0] = (u & 0x7FFFFFFFu) >= 0x7F7F8000u ? uint16_t(u >> 16) : bf16_rn(f);
    const float r1 = __fsub_rn(f, bf16_to_float(p[0]));
    p[1] = bf16_rn(r1);
    const float r2 = __fsub_rn(r1, bf16_to_float(p[1]));
    p[2] = bf16_rn(r2);
  }
}

template <int K>
__host__ __device__ constexpr int parts_of() { return K <= 2 ? 1 : (K == 3 ? 2 : 3); }

// Rows of A and columns of B that hold an Inf or NaN (split formats only):
// flag[i] = 1 and *any = 1.
struct SpecialFlags {
  uint8_t* row;
  uint8_t* col;
  int* any;
};

// A (m x k, lda, k-byte codes) -> NP bf16 arrays of m rows x kp, element (i, l) at i*kp + l.
// Block (x, y) converts 1024 columns of row y.
template <int K>
__global__ void __launch_bounds__(256) prep_rows(const uint8_t* __restrict__ A, int64_t lda, int64_t kdim,
                                                 int64_t kp, uint16_t* __restrict__ out, int64_t part_stride,
                                                 SpecialFlags fl) {
  constexpr int NP = parts_of<K>();
  const int64_t i = blockIdx.y;
  const uint8_t* row = A + i * lda * K;
  bool special = false;
  for (int64_t l = int64_t(blockIdx.x) * 1024 + threadIdx.x; l < kdim && l < int64_t(blockIdx.x + 1) * 1024;
       l += 256) {
    uint16_t p[3];
    const uint32_t u = widen<FLYTE_F32, K>(load_code_bytes<K>(row + l * K));
    split_parts<K, NP>(u, p);
    special |= K >= 3 && !finite_bits(u);
#pragma unroll
    for (int q = 0; q < NP; ++q) out[q * part_stride + i * kp + l] = p[q];
  }
  if (special) {
    fl.row[i] = 1;
    *fl.any = 1;
  }
}

// B (k x n, ldb) -> NP bf16 arrays of n rows x kp (B transposed), via 32 x 32 shared tiles.
template <int K>
__global__ void __launch_bounds__(256) prep_cols(const uint8_t* __restrict__ B, int64_t ldb, int64_t kdim,
                                                 int64_t n, int64_t kp, uint16_t* __restrict__ out,
                                                 int64_t part_stride, SpecialFlags fl) {
  constexpr int NP = parts_of<K>();
  __shared__ uint16_t tile[NP][32][33];
  const int64_t l0 = int64_t(blockIdx.y) * 32, j0 = int64_t(blockIdx.x) * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
  for (int r = ty; r < 32; r += 8) {
    const int64_t l = l0 + r, j = j0 + tx;
    uint16_t p[3] = {0, 0, 0};
    if (l < kdim && j < n) {
      const uint32_t u = widen<FLYTE_F32, K>(load_code_bytes<K>(B + (l * ldb + j) * K));
      split_parts<K, NP>(u, p);
      if (K >= 3 && !finite_bits(u)) {
        fl.col[j] = 1;
        *fl.any = 1;
      }
    }
#pragma unroll
    for (int q = 0; q < NP; ++q) tile[q][r][tx] = p[q];
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int64_t j = j0 + r, l = l0 + tx;
    if (j < n && l < kdim) {
#pragma unroll
      for (int q = 0; q < NP; ++q) out[q * part_stride + j * kp + l] = tile[q][tx][r];
    }
  }
}

// ---- the tensor-core kernel ----------------------------------------------------------------

struct PartMaps {
  CUtensorMap a[3];
  CUtensorMap b[3];
};

template <int K>
struct GemmCfg {
  static constexpr int NP = parts_of<K>();
  static constexpr int BN = 128;                             // 128 x 128 outputs per tile
  static constexpr int kATile = kBM * kBK * 2;               // bytes of one A part tile
  static constexpr int kBTile = BN * kBK * 2;
  static constexpr int kStage = NP * (kATile + kBTile);
  static constexpr int S = kSmemBudget / kStage > 7 ? 7 : kSmemBudget / kStage;
  static constexpr int kSmem = 1024 + S * kStage + 256;      // alignment slack, stages, barriers
  static_assert(kSmem <= 227 * 1024, "shared memory per block");
  static constexpr int kNProd = NP == 1 ? 1 : (NP == 2 ? 4 : 6);
  // k-blocks per TMEM chunk (16-24 MMA steps); a one-part format starts with
  // kBufs chunks of one k-block (they are not preloaded, see below)
  static constexpr int kChunkBlocks = NP == 1 ? FLYTE_GEMM_CHUNK1 : 1;
  static constexpr bool kPreload = NP == 1;
  // Columns per epilogue warp (32 rows each): 8 warps of 168 registers keep
  // their pair accumulators without spilling, where 16 warps of 96 spilled
  // (measured at 8192^3 with the f32x2 fold and 16-column loads: k = 3 / 4
  // 325 / 253 useful TFLOP/s against 314 / 243 with 16 warps; one part 662
  // against 614 in the same comparison before the 16-column loads)
  static constexpr int kEpiCols = 64;
  static constexpr int kLoadCols = 16;   // TMEM columns per tcgen05.ld (one-part: 16 against 8, 681 against 665 TFLOP/s at 8192^3)
  static constexpr int kEpiWarps = 4 * (BN / kEpiCols);
  static constexpr int kThreads = 32 * (kEpiWarps + 2);      // + producer warp + MMA warp
  // TMEM columns: kBufs chunk buffers of BN (the MMAs run up to kBufs - 1
  // chunks ahead of the epilogue) and, for one-part formats, the preload values
  static constexpr int kBufs = kPreload ? 3 : 4;
  static constexpr int kTmemCols = 512;
  static constexpr uint32_t kPreloadCol = kBufs * BN;
  static_assert(kBufs * BN + (kPreload ? BN : 0) <= kTmemCols, "TMEM columns");
};

// First k-block of chunk c (chunk_start(NC) = KB) and the number of chunks.
template <int K>
__host__ __device__ __forceinline__ int chunk_start(int c, int KB) {
  using Cfg = GemmCfg<K>;
  constexpr int L = Cfg::kPreload ? Cfg::kBufs : 0;   // leading one-k-block chunks
  const int s = c < L ? c : L + (c - L) * Cfg::kChunkBlocks;
  return s < KB ? s : KB;
}
template <int K>
__host__ __device__ __forceinline__ int chunk_count(int KB) {
  using Cfg = GemmCfg<K>;
  constexpr int L = Cfg::kPreload ? Cfg::kBufs : 0;
  return KB <= L ? KB : L + (KB - L + Cfg::kChunkBlocks - 1) / Cfg::kChunkBlocks;
}

// Part products in issue order: smallest first and the large (0,0) product
// last, so that only its 4 MMA steps per chunk add into a large partial sum.
__host__ __device__ constexpr int prod_a(int np, int q) {
  return np == 1 ? 0 : (np == 2 ? (q == 0 || q == 2 ? 1 : 0) : (q == 0 ? 2 : (q == 1 || q == 3 ? 1 : 0)));
}
__host__ __device__ constexpr int prod_b(int np, int q) {
  return np == 1 ? 0 : (np == 2 ? (q < 2 ? 1 : 0) : (q == 2 ? 2 : (q == 1 || q == 4 ? 1 : 0)));
}

// Where C goes: the native array (q == nullptr) or a stream of kc-byte flytes
// of the same base, packed with `mode` right where the value is formed.
struct COut {
  uint8_t* q;
  int kc, mode;
};

// C_ij <- alpha acc + beta C_ij (beta == 0: C is not read) at element offset idx.
__device__ __forceinline__ void store_c(float* C, const COut& co, int64_t idx, float acc, float alpha, float beta) {
  if (co.q == nullptr) {
    C[idx] = beta == 0.f ? alpha * acc : __fmaf_rn(alpha, acc, beta * C[idx]);
    return;
  }
  uint8_t* p = co.q + idx * co.kc;
  float r;
  if (beta == 0.f) {
    r = alpha * acc;
  } else {
    const uint32_t u = uint32_t(load_code_bytes_rt(p, co.kc) << (32 - 8 * co.kc));
    r = __fmaf_rn(alpha, acc, beta * __uint_as_float(u));
  }
  store_code_bytes_rt(p, narrow_rt<FLYTE_F32>(__float_as_uint(r), co.kc, co.mode), co.kc);
}

__device__ __forceinline__ void store_c(double* C, const COut& co, int64_t idx, double acc, double alpha,
                                        double beta) {
  if (co.q == nullptr) {
    C[idx] = beta == 0.0 ? alpha * acc : fma(alpha, acc, beta * C[idx]);
    return;
  }
  uint8_t* p = co.q + idx * co.kc;
  double r;
  if (beta == 0.0) {
    r = alpha * acc;
  } else {
    const uint64_t q = load_code_bytes_rt(p, co.kc);
    r = fma(alpha, acc, beta * __longlong_as_double((long long)(co.kc == 8 ? q : q << (64 - 8 * co.kc))));
  }
  store_code_bytes_rt(p, narrow_rt<FLYTE_F64>(uint64_t(__double_as_longlong(r)), co.kc, co.mode), co.kc);
}

// Persistent: one CTA per SM walks the output tiles tau = blockIdx.x,
// blockIdx.x + gridDim.x, ... in groups of kGroupRows tile rows (column by
// column inside a group, so that concurrently running CTAs share A and B
// tiles in L2).  Warps [0, E): epilogue; warp E: TMA producer; warp E + 1:
// MMA issuer and TMEM owner.  The stage ring and the TMEM chunk buffers
// run on across tiles, so the next tile's loads and MMAs overlap this tile's
// C store.
//
// Accuracy.  The tensor core adds each MMA step into its binary32
// accumulator with truncation toward zero: over a chunk of L steps whose
// partial sums keep one sign, the error is about a quarter of L ulps of the
// chunk, one-signed (measured on one-signed data: about 0.3 x 2^-22 sum|ab|
// per k-block of chunk length for a one-part format, growing linearly with
// it; all-negative products give the mirror image).  So:
//  - the epilogue adds every chunk into hi + lo exactly (TwoSum), removing
//    the rounding of the fold (which otherwise reaches 2-3 x 2^-22 sum|ab|
//    at K = 8192);
//  - split formats fold every k-block (16-24 MMA steps, of which only the
//    last 4, the hi * hi product, add into a large partial sum);
//  - one-part formats fold every kChunkBlocks k-blocks after kBufs leading
//    chunks of one k-block, and every later chunk starts from
//    P = -(kChunkBlocks / 2) c0 (c0 the tile's first chunk) instead of zero,
//    written into its buffer by the epilogue: its partial sums then run
//    from about -c / 2 to c / 2, so that the truncation errors of the
//    negative and the positive half cancel instead of adding up.  The
//    preloads are taken out exactly at the end: C = (hi + lo) - n P with
//    TwoProd and TwoSum (n the number of preloaded chunks).
// Measured on one-signed U(0, 1) and |N(0, 1)| data at K = 2048 and 8192,
// the worst error over 4096 sampled entries is 0.6-0.7 x 2^-22 sum|ab| for
// every format.  The chunk buffers are multiple, so that the MMAs can run
// up to kBufs - 1 chunks ahead of the exact fold.
constexpr int kGroupRows = 16;

__device__ __forceinline__ void tile_of(int64_t tau, int64_t mt, int64_t nt, int64_t& tm, int64_t& tn) {
  const int64_t per_group = int64_t(kGroupRows) * nt;
  const int64_t g = tau / per_group, r = tau % per_group;
  const int64_t rows = min(int64_t(kGroupRows), mt - g * kGroupRows);
  tm = g * kGroupRows + r % rows;
  tn = r / rows;
}

__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& t) {
  s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  t = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
}

template <int K>
__global__ void __launch_bounds__(GemmCfg<K>::kThreads, 1) gemm_tc_kernel(
    const __grid_constant__ PartMaps maps, int64_t m, int64_t n, int64_t kdim, float alpha, float beta,
    float* __restrict__ C, int64_t ldc, const COut co, int* __restrict__ status, const SpecialFlags fl) {
  using Cfg = GemmCfg<K>;
  constexpr int NP = Cfg::NP, BN = Cfg::BN, S = Cfg::S, E = Cfg::kEpiWarps;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + S * Cfg::kStage);
  uint64_t* empty = full + S;
  constexpr int NB = Cfg::kBufs;
  uint64_t* accfull = empty + S;        // NB: chunk accumulator ready
  uint64_t* accempty = accfull + NB;    // NB: chunk accumulator drained (and preloaded)
  uint64_t* mdone = accempty + NB;      // every MMA has completed
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mdone + 1);
  uint32_t* issued = tslot + 1;         // k-blocks the producer issued (for the drain after a failure)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int KB = int((kdim + kBK - 1) / kBK);
  const int NC = chunk_count<K>(KB);
  const int64_t mt = (m + kBM - 1) / kBM, nt = (n + BN - 1) / BN;
  const int64_t ntiles = mt * nt;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < NB; ++b) {
      mbar_init(&accfull[b], 1);
      mbar_init(&accempty[b], E);
    }
    mbar_init(mdone, 1);
    *issued = 0;
    mbar_init_fence();
  }
  __syncwarp();
  if (warp == E + 1) tmem_alloc(tslot, Cfg::kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  auto a_tile = [&](int s, int p) { return smem + s * Cfg::kStage + p * Cfg::kATile; };
  auto b_tile = [&](int s, int p) { return smem + s * Cfg::kStage + NP * Cfg::kATile + p * Cfg::kBTile; };

  if (warp == E) {
    if (lane == 0) {
      uint32_t it = 0;
      bool ok = true;
      for (int64_t tau = blockIdx.x; tau < ntiles && ok; tau += gridDim.x) {
        int64_t tm, tn;
        tile_of(tau, mt, nt, tm, tn);
        for (int kb = 0; kb < KB; ++kb, ++it) {
          const int s = int(it % S);
          if (it >= S && !mbar_wait(&empty[s], ((it / S) - 1) & 1, status)) { ok = false; break; }
          mbar_arrive_expect_tx(&full[s], Cfg::kStage);
#pragma unroll
          for (int p = 0; p < NP; ++p) tma_load_2d(a_tile(s, p), &maps.a[p], kb * kBK, int(tm * kBM), &full[s]);
#pragma unroll
          for (int p = 0; p < NP; ++p) tma_load_2d(b_tile(s, p), &maps.b[p], kb * kBK, int(tn * BN), &full[s]);
        }
      }
      *issued = it;
    }
  } else if (warp == E + 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = umma_idesc_bf16(kBM, BN);
      bool ok = true;
      uint32_t it = 0, g = 0;   // k-blocks and chunks so far
      for (int64_t tau = blockIdx.x; tau < ntiles && ok; tau += gridDim.x) {
        for (int c = 0; c < NC && ok; ++c, ++g) {
          const int b = int(g % NB);
          if (g >= uint32_t(NB) && !mbar_wait(&accempty[b], ((g / NB) - 1) & 1, status)) { ok = false; break; }
          tc_fence_after();
          const uint32_t acc = tmem + uint32_t(b * BN);
          // a preloaded chunk adds onto the value the epilogue wrote into its buffer
          const bool onto = Cfg::kPreload && c >= NB;
          const int kb0 = chunk_start<K>(c, KB), kb_end = chunk_start<K>(c + 1, KB);
          for (int kb = kb0; kb < kb_end; ++kb, ++it) {
            const int s = int(it % S);
            if (!mbar_wait(&full[s], (it / S) & 1, status)) { ok = false; break; }
            tc_fence_after();
#pragma unroll
            for (int q = 0; q < Cfg::kNProd; ++q) {
              const int pa = prod_a(NP, q), pb = prod_b(NP, q);
              const uint64_t ad = umma_desc_kmajor_sw128(smem_addr(a_tile(s, pa)));
              const uint64_t bd = umma_desc_kmajor_sw128(smem_addr(b_tile(s, pb)));
#pragma unroll
              for (int kk = 0; kk < kBK / 16; ++kk)
                umma_bf16(acc, ad + 2 * kk, bd + 2 * kk, idesc,
                          (onto || kb > kb0 || q > 0 || kk > 0) ? 1u : 0u);
            }
            umma_commit(&empty[s]);
          }
          if (ok) umma_commit(&accfull[b]);
        }
      }
      umma_commit(mdone);    // fires once every MMA issued above has completed
    }
  } else {
    // epilogue warp: TMEM lanes 32 * (warp % 4) .. + 31, columns 32 * (warp / 4) .. + 31
    constexpr int EC = Cfg::kEpiCols;
    const int quarter = warp & 3, cblk = warp >> 2;
    const uint32_t lane_base = tmem + (uint32_t(32 * quarter) << 16);
    const uint32_t pcol = lane_base + Cfg::kPreloadCol + uint32_t(EC * cblk);
    const bool any_special = K >= 3 && *reinterpret_cast<volatile int*>(fl.any) != 0;
    bool failed = false;   // a wait gave up: no more waits, NaN for every remaining output
    uint32_t g = 0;
    for (int64_t tau = blockIdx.x; tau < ntiles; tau += gridDim.x) {
      int64_t tm, tn;
      tile_of(tau, mt, nt, tm, tn);
      // the exact fold, on pairs of outputs (f32x2): each output's chunks sum to hi + lo
      f2 hi[EC / 2], lo[EC / 2];
      for (int c = 0; c < NC && !failed; ++c, ++g) {
        const int b = int(g % NB);
        const bool got = mbar_wait(&accfull[b], (g / NB) & 1, status);
        if (!__all_sync(0xFFFFFFFFu, got)) {
          failed = true;
          break;
        }
        tc_fence_after();
        const uint32_t buf = lane_base + uint32_t(b * BN + EC * cblk);
        const bool preload_next = Cfg::kPreload && c + NB < NC;
        constexpr int LW = Cfg::kLoadCols;
#pragma unroll
        for (int j = 0; j < EC / LW; ++j) {
          uint32_t r[LW];
          if (preload_next && c > 0) {
            // the chunk and its buffer's next start value in flight together (one wait), the
            // start value written back before the fold (k = 2: 680 -> 696 TFLOP/s at 8192^3)
            static_assert(LW == 16, "paired loads are 16 columns wide");
            uint32_t p[LW];
            tmem_ld16_issue(buf + LW * j, r);
            tmem_ld16_issue(pcol + LW * j, p);
            tmem_ld16_wait2(r, p);
            tmem_st<LW>(buf + LW * j, p);
          } else {
            tmem_ld<LW>(buf + LW * j, r);
          }
#pragma unroll
          for (int i = 0; i < LW / 2; ++i) {
            const int e = (LW / 2) * j + i;
            const f2 v = f2_pack(__uint_as_float(r[2 * i]), __uint_as_float(r[2 * i + 1]));
            if (c == 0) {
              hi[e] = v;
              lo[e] = 0ull;
            } else {
              // TwoSum on both values: s + t = hi + v exactly
              const f2 s = f2_add(hi[e], v);
              const f2 bp = f2_sub(s, hi[e]);
              const f2 t = f2_add(f2_sub(hi[e], f2_sub(s, bp)), f2_sub(v, bp));
              hi[e] = s;
              lo[e] = f2_add(lo[e], t);
            }
          }
          if (preload_next) {
            // the next chunk in this buffer starts from P = -(kChunkBlocks / 2) c0: minus half a
            // full chunk as estimated from the first, one-k-block chunk (0 if c0 is not finite)
            if (c == 0) {
              constexpr float kHalfChunk = -0.5f * float(Cfg::kChunkBlocks);   // a power of two: exact
#pragma unroll
              for (int i = 0; i < LW; ++i)
                r[i] = __float_as_uint(finite_bits(r[i]) ? __fmul_rn(__uint_as_float(r[i]), kHalfChunk) : 0.f);
              tmem_st<LW>(pcol + LW * j, r);
              tmem_st<LW>(buf + LW * j, r);
            }
          }
        }
        if (preload_next) tmem_wait_st();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&accempty[b]);
      }
      // the result of each output, into hi: C = hi + lo, less the preloads (exact up to the
      // last rounding); a non-finite hi is the result as it stands
      if (failed) {
#pragma unroll
        for (int e = 0; e < EC / 2; ++e) hi[e] = f2_pack(__uint_as_float(0x7FC00000u), __uint_as_float(0x7FC00000u));
      } else if (Cfg::kPreload && NC > NB) {
        const float cnt = float(NC - NB);
#pragma unroll
        for (int j = 0; j < EC / 8; ++j) {
          uint32_t r[8];
          tmem_ld8(pcol + 8 * j, r);
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int e = 4 * j + i;
            float h[2], l[2];
            f2_unpack(hi[e], h[0], h[1]);
            f2_unpack(lo[e], l[0], l[1]);
#pragma unroll
            for (int q = 0; q < 2; ++q) {
              const float P = __uint_as_float(r[2 * i + q]);
              const float ph = __fmul_rn(cnt, P);
              const float pl = __fmaf_rn(cnt, P, -ph);
              float s, t;
              two_sum_f(h[q], -ph, s, t);
              if (finite_bits(__float_as_uint(h[q]))) h[q] = __fadd_rn(s, __fsub_rn(__fadd_rn(l[q], t), pl));
            }
            hi[e] = f2_pack(h[0], h[1]);
          }
        }
      } else {
#pragma unroll
        for (int e = 0; e < EC / 2; ++e) {
          float h[2], l[2];
          f2_unpack(hi[e], h[0], h[1]);
          f2_unpack(lo[e], l[0], l[1]);
#pragma unroll
          for (int q = 0; q < 2; ++q)
            if (finite_bits(__float_as_uint(h[q]))) h[q] = __fadd_rn(h[q], l[q]);
          hi[e] = f2_pack(h[0], h[1]);
        }
      }
      float total[EC];
#pragma unroll
      for (int e = 0; e < EC / 2; ++e) f2_unpack(hi[e], total[2 * e], total[2 * e + 1]);
      const int64_t row = tm * kBM + 32 * quarter + lane;
      const int64_t col0 = tn * BN + EC * cblk;
      if (row < m && col0 < n) {
        const int64_t base = row * ldc + col0;
        const bool row_special = any_special && fl.row[row] != 0;
        if (co.q == nullptr && !any_special && col0 + EC <= n && (reinterpret_cast<uintptr_t>(C + base) & 15) == 0) {
          float4* out = reinterpret_cast<float4*>(C + base);
#pragma unroll
          for (int i = 0; i < EC / 4; ++i) {
            float4 v = make_float4(alpha * total[4 * i], alpha * total[4 * i + 1], alpha * total[4 * i + 2],
                                   alpha * total[4 * i + 3]);
            if (beta != 0.f) {
              const float4 o = out[i];
              v = make_float4(__fmaf_rn(alpha, total[4 * i], beta * o.x), __fmaf_rn(alpha, total[4 * i + 1], beta * o.y),
                              __fmaf_rn(alpha, total[4 * i + 2], beta * o.z),
                              __fmaf_rn(alpha, total[4 * i + 3], beta * o.w));
            }
            out[i] = v;
          }
        } else {
#pragma unroll
          for (int i = 0; i < EC; ++i) {
            // entries that meet an Inf or NaN input are written by gemm_special_entries
            if (col0 + i < n && !(any_special && (row_special || fl.col[col0 + i] != 0)))
              store_c(C, co, base + i, total[i], alpha, beta);
          }
        }
      }
    }
  }
  __syncthreads();
  if (warp == E + 1) {
    // every MMA done (and, after a failed wait, every TMA drained) before TMEM is freed
    if (lane == 0) {
      mbar_wait(mdone, 0, nullptr);
      if (*reinterpret_cast<volatile int*>(status) != 0) {
        const uint32_t n_is = *issued;
        for (uint32_t j = n_is > uint32_t(S) ? n_is - S : 0; j < n_is; ++j)
          mbar_wait(&full[j % S], (j / S) & 1, nullptr);
      }
    }
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tmem, Cfg::kTmemCols);
  }
}

// Entries of C whose sum meets an Inf or NaN of A or B (split formats): the
// IEEE class of the sum (Sec. 5.3): NaN if a term is NaN (NaN input, or
// Inf * 0) or infinities of both signs occur, else the signed infinity;
// then alpha * class + beta * C as elsewhere.  Runs after the main kernel,
// which left these entries untouched; returns at once when no input was
// flagged.
template <int K>
__global__ void gemm_special_entries(const uint8_t* __restrict__ A, int64_t lda, const uint8_t* __restrict__ B,
                                     int64_t ldb, int64_t m, int64_t n, int64_t kdim, float alpha, float beta,
                                     float* __restrict__ C, int64_t ldc, const COut co, const SpecialFlags fl) {
  if (*reinterpret_cast<volatile int*>(fl.any) == 0) return;
  const int64_t total = m * n;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total; t += stride) {
    const int64_t i = t / n, j = t - i * n;
    if (fl.row[i] == 0 && fl.col[j] == 0) continue;
    bool nan = false, pos = false, neg = false;
    for (int64_t l = 0; l < kdim; ++l) {
      const uint32_t ua = widen<FLYTE_F32, K>(load_code_bytes<K>(A + (i * lda + l) * K));
      const uint32_t ub = widen<FLYTE_F32, K>(load_code_bytes<K>(B + (l * ldb + j) * K));
      if (finite_bits(ua) && finite_bits(ub)) continue;
      const float p = __fmul_rn(__uint_as_float(ua), __uint_as_float(ub));
      nan |= p != p;
      pos |= p > 0.f;
      neg |= p < 0.f;
    }
    const float cls = (nan || (pos && neg)) ? __uint_as_float(0x7FC00000u)
                                            : __uint_as_float(pos ? 0x7F800000u : 0xFF800000u);
    store_c(C, co, i * ldc + j, cls, alpha, beta);
  }
}

// ---- binary64 tensor-core kernel (double-based formats) ------------------------------------------

constexpr int kDT = 64;     // C tile 64 x 64
constexpr int kDK = 16;     // k step

__device__ __forceinline__ void dmma_884(double (&c)[2], double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
               : "+d"(c[0]), "+d"(c[1])
               : "d"(a), "d"(b));
}

// 4 warps, each a 32 x 32 quadrant of the 64 x 64 tile as 4 x 4 blocks of 8 x 8.
template <int K>
__global__ void __launch_bounds__(128) gemm_dmma_kernel(const uint8_t* __restrict__ A, int64_t lda,
                                                        const uint8_t* __restrict__ B, int64_t ldb, int64_t m,
                                                        int64_t n, int64_t kdim, double alpha, double beta,
                                                        double* __restrict__ C, int64_t ldc, const COut co) {
  __shared__ double sA[kDT][kDK + 1];
  __shared__ double sB[kDK][kDT + 1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t m0 = int64_t(blockIdx.y) * kDT, n0 = int64_t(blockIdx.x) * kDT;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  const int g = lane >> 2, t = lane & 3;
  double acc[4][4][2];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j][0] = acc[i][j][1] = 0.0;
  for (int64_t l0 = 0; l0 < kdim; l0 += kDK) {
    for (int e = threadIdx.x; e < kDT * kDK; e += 128) {
      const int r = e / kDK, c = e % kDK;
      const int64_t i = m0 + r, l = l0 + c;
      sA[r][c] = (i < m && l < kdim) ? code_to_double<FLYTE_F64, K>(load_code_bytes<K>(A + (i * lda + l) * K)) : 0.0;
    }
    for (int e = threadIdx.x; e < kDT * kDK; e += 128) {
      const int r = e / kDT, c = e % kDT;
      const int64_t l = l0 + r, j = n0 + c;
      sB[r][c] = (l < kdim && j < n) ? code_to_double<FLYTE_F64, K>(load_code_bytes<K>(B + (l * ldb + j) * K)) : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kDK; kk += 4) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = sA[wm + 8 * i + g][kk + t];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = sB[kk + t][wn + 8 * j + g];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) dmma_884(acc[i][j], a[i], b[j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int64_t row = m0 + wm + 8 * i + g, col = n0 + wn + 8 * j + 2 * t + h;
        if (row < m && col < n) store_c(C, co, row * ldc + col, acc[i][j][h], alpha, beta);
      }
}

// C <- beta C (alpha == 0 or k_ == 0), native or packed; beta == 0 writes zeros without reading C.
__global__ void scale_c(void* C, int64_t m, int64_t n, int64_t ldc, double beta, int is_double, const COut co) {
  const int64_t total = m * n;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total; t += stride) {
    const int64_t i = t / n, j = t - i * n;
    const int64_t idx = i * ldc + j;
    if (co.q == nullptr) {
      if (is_double) {
        double* c = static_cast<double*>(C) + idx;
        *c = beta == 0.0 ? 0.0 : beta * *c;
      } else {
        float* c = static_cast<float*>(C) + idx;
        *c = beta == 0.0 ? 0.f : float(beta) * *c;
      }
      continue;
    }
    uint8_t* p = co.q + idx * co.kc;
    const uint64_t q = beta == 0.0 ? 0 : load_code_bytes_rt(p, co.kc);
    uint64_t out = 0;
    if (beta != 0.0 && is_double) {
      const double r = beta * __longlong_as_double((long long)(co.kc == 8 ? q : q << (64 - 8 * co.kc)));
      out = narrow_rt<FLYTE_F64>(uint64_t(__double_as_longlong(r)), co.kc, co.mode);
    } else if (beta != 0.0) {
      const float r = float(beta) * __uint_as_float(uint32_t(q << (32 - 8 * co.kc)));
      out = narrow_rt<FLYTE_F32>(__float_as_uint(r), co.kc, co.mode);
    }
    store_code_bytes_rt(p, out, co.kc);
  }
}

int64_t round_up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

struct GemmPlan {
  int np;
  int64_t kp;            // row stride (elements) of the bf16 part arrays
  bool a_in_place;       // k = 2 with 16-byte aligned rows: A is used as is
  // status word (int at 0) and "some input is Inf/NaN" word (int at 4), row
  // flags of A (m bytes) and column flags of B (n bytes), bf16 parts of A and B
  int64_t off_status, off_rflag, off_cflag, off_a, off_b, bytes;
};

GemmPlan plan_gemm(int64_t m, int64_t n, int64_t kdim, flyte_fmt f, const void* A, int64_t lda) {
  GemmPlan p{};
  p.off_status = 0;
  if (f.base == FLYTE_F64) {
    p.bytes = 16;
    return p;
  }
  p.np = f.k <= 2 ? 1 : (f.k == 3 ? 2 : 3);
  p.kp = round_up(kdim > 0 ? kdim : 1, 8);
  p.a_in_place = f.k == 2 && (A == nullptr || reinterpret_cast<uintptr_t>(A) % 16 == 0) && (lda * 2) % 16 == 0;
  p.off_rflag = 256;
  p.off_cflag = p.off_rflag + round_up(m, 256);
  p.off_a = p.off_cflag + round_up(n, 256);
  // room for the A parts is reserved even when A is used in place, so that the
  // size depends on the shape and format only
  const int64_t a_bytes = round_up(int64_t(p.np) * m * p.kp * 2, 256);
  p.off_b = p.off_a + a_bytes;
  p.bytes = p.off_b + round_up(int64_t(p.np) * n * p.kp * 2, 256);
  return p;
}

// The driver's tensor-map encoder, looked up through the runtime so that the
// library does not link libcuda (and loads on machines without a driver).
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled_fn() {
  static EncodeTiledFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<EncodeTiledFn>(p);
  }();
  return fn;
}

bool encode_map(CUtensorMap* map, const void* ptr, int64_t inner, int64_t outer, int64_t row_bytes, int box_outer) {
  const EncodeTiledFn encode = encode_tiled_fn();
  if (encode == nullptr) return false;
  cuuint64_t dims[2] = {cuuint64_t(inner), cuuint64_t(outer)};
  cuuint64_t strides[1] = {cuuint64_t(row_bytes)};
  cuuint32_t box[2] = {cuuint32_t(kBK), cuuint32_t(box_outer)};
  cuuint32_t es[2] = {1, 1};
  return encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int K>
flyte_status launch_tc(int64_t m, int64_t n, int64_t kdim, double alpha, const uint8_t* A, int64_t lda,
                       const uint8_t* B, int64_t ldb, double beta, float* C, int64_t ldc, const COut& co,
                       uint8_t* ws, const GemmPlan& p, cudaStream_t s) {
  using Cfg = GemmCfg<K>;
  int* status = reinterpret_cast<int*>(ws + p.off_status);
  uint16_t* ap = reinterpret_cast<uint16_t*>(ws + p.off_a);
  uint16_t* bp = reinterpret_cast<uint16_t*>(ws + p.off_b);
  const SpecialFlags fl{ws + p.off_rflag, ws + p.off_cflag, status + 1};
  if (cudaMemsetAsync(status, 0, 2 * sizeof(int), s) != cudaSuccess) return cuda_status(cudaGetLastError(), "gemm");
  if (Cfg::NP > 1 && cudaMemsetAsync(ws + p.off_rflag, 0, size_t(p.off_a - p.off_rflag), s) != cudaSuccess)
    return cuda_status(cudaGetLastError(), "gemm");
  if (!p.a_in_place) {
    dim3 grid(unsigned((kdim + 1023) / 1024), unsigned(m));
    prep_rows<K><<<grid, 256, 0, s>>>(A, lda, kdim, p.kp, ap, m * p.kp, fl);
    FLYTE_TRY_LAUNCH("gemm");
  }
  {
    dim3 grid(unsigned((n + 31) / 32), unsigned((kdim + 31) / 32));
    prep_cols<K><<<grid, 256, 0, s>>>(B, ldb, kdim, n, p.kp, bp, n * p.kp, fl);
    FLYTE_TRY_LAUNCH("gemm");
  }
  PartMaps maps;
  std::memset(&maps, 0, sizeof(maps));
  for (int q = 0; q < Cfg::NP; ++q) {
    const void* abase = p.a_in_place ? static_cast<const void*>(A) : static_cast<const void*>(ap + q * m * p.kp);
    const int64_t arow = p.a_in_place ? lda * 2 : p.kp * 2;
    if (!encode_map(&maps.a[q], abase, kdim, m, arow, kBM) ||
        !encode_map(&maps.b[q], bp + q * n * p.kp, kdim, n, p.kp * 2, Cfg::BN)) {
      set_error("gemm: cuTensorMapEncodeTiled failed");
      return FLYTE_ERR_CUDA;
    }
  }
  if (cudaFuncSetAttribute(gemm_tc_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::kSmem) !=
      cudaSuccess)
    return cuda_status(cudaGetLastError(), "gemm");
  const int64_t tiles = ((m + kBM - 1) / kBM) * ((n + Cfg::BN - 1) / Cfg::BN);
  const unsigned grid = unsigned(min(tiles, int64_t(sm_count())));   // persistent: one CTA per SM
  gemm_tc_kernel<K><<<grid, Cfg::kThreads, Cfg::kSmem, s>>>(maps, m, n, kdim, float(alpha), float(beta), C, ldc,
                                                            co, status, fl);
  FLYTE_TRY_LAUNCH("gemm");
  if constexpr (Cfg::NP > 1) {
    gemm_special_entries<K><<<grid_for(m * n, 256), 256, 0, s>>>(A, lda, B, ldb, m, n, kdim, float(alpha),
                                                                 float(beta), C, ldc, co, fl);
    FLYTE_TRY_LAUNCH("gemm");
  }
  return FLYTE_OK;
}

}  // namespace

size_t gemm_workspace_bytes(int64_t m, int64_t n, int64_t kdim, flyte_fmt f) {
  return size_t(plan_gemm(m, n, kdim, f, nullptr, 8).bytes);
}

flyte_status launch_gemm(int64_t m, int64_t n, int64_t kdim, double alpha, const void* A, flyte_fmt fa,
                         int64_t lda, const void* B, int64_t ldb, double beta, void* C, int kc, int64_t ldc,
                         int mode, void* ws, size_t ws_bytes, cudaStream_t s) {
  const bool dbl = fa.base == FLYTE_F64;
  const COut co{kc == 0 ? nullptr : static_cast<uint8_t*>(C), kc, mode};
  if (alpha == 0.0 || kdim == 0) {
    if (beta == 1.0) return FLYTE_OK;
    scale_c<<<grid_for(m * n, 256), 256, 0, s>>>(C, m, n, ldc, beta, dbl ? 1 : 0, co);
    FLYTE_TRY_LAUNCH("gemm");
    return FLYTE_OK;
  }
  const GemmPlan p = plan_gemm(m, n, kdim, fa, A, lda);
  if (ws == nullptr || ws_bytes < size_t(p.bytes) || reinterpret_cast<uintptr_t>(ws) % 256 != 0) {
    set_error("gemm: workspace of %lld bytes (256-byte aligned) required", (long long)p.bytes);
    return FLYTE_ERR_WORKSPACE;
  }
  const uint8_t* A8 = static_cast<const uint8_t*>(A);
  const uint8_t* B8 = static_cast<const uint8_t*>(B);
  uint8_t* w8 = static_cast<uint8_t*>(ws);
  if (dbl) {
    return dispatch_fmt(fa, [&]<int BASE, int K>() -> flyte_status {
      if constexpr (BASE == FLYTE_F64) {
        dim3 grid(unsigned((n + kDT - 1) / kDT), unsigned((m + kDT - 1) / kDT));
        gemm_dmma_kernel<K><<<grid, 128, 0, s>>>(A8, lda, B8, ldb, m, n, kdim, alpha, beta, static_cast<double*>(C),
                                                 ldc, co);
        FLYTE_TRY_LAUNCH("gemm");
      }
      return FLYTE_OK;
    });
  }
  float* Cf = static_cast<float*>(C);
  switch (fa.k) {
    case 1: return launch_tc<1>(m, n, kdim, alpha, A8, lda, B8, ldb, beta, Cf, ldc, co, w8, p, s);
    case 2: return launch_tc<2>(m, n, kdim, alpha, A8, lda, B8, ldb, beta, Cf, ldc, co, w8, p, s);
    case 3: return launch_tc<3>(m, n, kdim, alpha, A8, lda, B8, ldb, beta, Cf, ldc, co, w8, p, s);
    case 4: return launch_tc<4>(m, n, kdim, alpha, A8, lda, B8, ldb, beta, Cf, ldc, co, w8, p, s);
  }
  return FLYTE_ERR_INVALID_ARG;
}

}  // namespace flyte
