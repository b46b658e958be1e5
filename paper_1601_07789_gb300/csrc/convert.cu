// convert.cu -- streaming pack and unpack of flyte arrays (Sec. 3-5 of the paper).
//
// Fast path (unit strides, suitably aligned pointers): each thread owns
// groups of 4 consecutive elements.  4 elements of k bytes are 4k bytes, a
// whole number of 32-bit words, so a thread reads (unpack) or writes (pack)
// its packed bytes with aligned vector accesses that never overlap another
// thread's: the GPU form of the paper's "compact, blend, then
// non-overlapping stores" (Sec. 4.3).  Inside the thread the bytes are split
// into lanes with funnel shifts (Sec. 4.1: shift and pad with zeros) or
// assembled from the rounded codes.  Native values move as 16-byte vectors.
// Each thread keeps UNROLL groups in flight to cover HBM latency.
//
// Generic path (any stride or alignment): one thread per element with byte
// loads and stores; elements never share a byte, so byte stores from
// different threads cannot conflict.
#include "flyte_internal.cuh"

namespace flyte {
namespace {

constexpr int kThreads = 256;
constexpr int kUnroll = 4;
// 128-element tiles in flight per warp in unpack_f64_tiles: 8 for k >= 3 (measured at 2^28: k = 3
// 0.516 -> 0.484 ms, k = 6 0.603 -> 0.569 ms), 4 below (8 was slower for k = 2)
template <int K>
__host__ __device__ constexpr int unpack_tile_unroll() { return K >= 3 ? 8 : 4; }
template <int K>
__host__ __device__ constexpr int unpack_tile_smem() { return (kThreads / 32) * unpack_tile_unroll<K>() * 1024; }

// Bit k set: double-based width k uses the warp-tile kernels below.
#ifndef FLYTE_PACK_TILES_MASK
#define FLYTE_PACK_TILES_MASK 0x8E   // k = 1, 2, 3, 7 (k = 4..6 measured 2-3 % faster without)
#endif
#ifndef FLYTE_UNPACK_TILES_MASK
#define FLYTE_UNPACK_TILES_MASK 0xFE
#endif

// 4 native values: 16 bytes (float) or 32 bytes (double).
template <int BASE>
struct Quad {
  typename Native<BASE>::bits v[4];
};

template <int BASE>
__device__ __forceinline__ void load_quad(const void* p, Quad<BASE>& q) {
  if constexpr (BASE == FLYTE_F32) {
    uint4 a = __ldg(reinterpret_cast<const uint4*>(p));
    q.v[0] = a.x; q.v[1] = a.y; q.v[2] = a.z; q.v[3] = a.w;
  } else {
    const uint4* s = reinterpret_cast<const uint4*>(p);
    uint4 a = __ldg(s), b = __ldg(s + 1);
    q.v[0] = (uint64_t(a.y) << 32) | a.x; q.v[1] = (uint64_t(a.w) << 32) | a.z;
    q.v[2] = (uint64_t(b.y) << 32) | b.x; q.v[3] = (uint64_t(b.w) << 32) | b.z;
  }
}

template <int BASE>
__device__ __forceinline__ void store_quad(void* p, const Quad<BASE>& q) {
  if constexpr (BASE == FLYTE_F32) {
    *reinterpret_cast<uint4*>(p) = make_uint4(q.v[0], q.v[1], q.v[2], q.v[3]);
  } else {
    uint4* d = reinterpret_cast<uint4*>(p);
    d[0] = make_uint4(uint32_t(q.v[0]), uint32_t(q.v[0] >> 32), uint32_t(q.v[1]), uint32_t(q.v[1] >> 32));
    d[1] = make_uint4(uint32_t(q.v[2]), uint32_t(q.v[2] >> 32), uint32_t(q.v[3]), uint32_t(q.v[3] >> 32));
  }
}

// ---- unpack ------------------------------------------------------------------

template <int BASE, int K>
__global__ void __launch_bounds__(kThreads) unpack_groups(const uint8_t* __restrict__ src,
                                                          void* __restrict__ dst, int64_t ngroups) {
  using Bits = typename Native<BASE>::bits;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  for (; g < ngroups; g += kUnroll * stride) {
    uint32_t w[kUnroll][K];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int64_t gu = g + u * stride;
      if (gu < ngroups) load_group<K>(src + gu * (4 * K), w[u]);
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int64_t gu = g + u * stride;
      if (gu < ngroups) {
        Quad<BASE> q;
#pragma unroll
        for (int e = 0; e < 4; ++e) q.v[e] = extract_widened<BASE, K>(w[u], e);
        store_quad<BASE>(static_cast<uint8_t*>(dst) + gu * (4 * sizeof(Bits)), q);
      }
    }
  }
}

// Double-based unpack with coalesced stores.  A lane's 4 doubles are 32
// contiguous bytes, so storing them directly makes every 16-byte store of a
// warp touch 1 KiB with gaps.  Here a warp converts 32 groups (128 elements,
// 1 KiB of output) at a time, passes them through a per-warp shared buffer
// (16-byte halves XOR-swizzled so that both the writes and the reads are free
// of bank conflicts) and stores them with two instructions that each cover
// 512 contiguous bytes.
template <int K>
__global__ void __launch_bounds__(kThreads) unpack_f64_tiles(const uint8_t* __restrict__ src,
                                                             uint8_t* __restrict__ dst, int64_t ntiles) {
  constexpr int kWarps = kThreads / 32;
  constexpr int kUnroll = unpack_tile_unroll<K>();
  extern __shared__ __align__(16) uint4 dyn_smem[];
  auto buf = reinterpret_cast<uint4(*)[kUnroll][64]>(dyn_smem);   // [warp][tile][16-byte chunk]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t wstride = int64_t(gridDim.x) * kWarps;
  const int sw = (lane >> 2) & 1;
  for (int64_t t = int64_t(blockIdx.x) * kWarps + warp; t < ntiles; t += kUnroll * wstride) {
    uint32_t w[kUnroll][K];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int64_t tu = t + u * wstride;
      if (tu < ntiles) load_group<K>(src + (tu * 32 + lane) * (4 * K), w[u]);
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      if (t + u * wstride < ntiles) {
        uint64_t v[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) v[e] = extract_widened<FLYTE_F64, K>(w[u], e);
        buf[warp][u][2 * lane + sw] = make_uint4(uint32_t(v[0]), uint32_t(v[0] >> 32), uint32_t(v[1]),
                                                 uint32_t(v[1] >> 32));
        buf[warp][u][2 * lane + (sw ^ 1)] = make_uint4(uint32_t(v[2]), uint32_t(v[2] >> 32), uint32_t(v[3]),
                                                       uint32_t(v[3] >> 32));
      }
    }
    __syncwarp();
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int64_t tu = t + u * wstride;
      if (tu < ntiles) {
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const int c = 32 * j + lane;                       // 16-byte chunk of the warp's 1 KiB
          const uint4 val = buf[warp][u][2 * (c >> 1) + ((c & 1) ^ ((c >> 3) & 1))];
          reinterpret_cast<uint4*>(dst + tu * 1024)[c] = val;
        }
      }
    }
    __syncwarp();
  }
}

template <int BASE, int K>
__global__ void __launch_bounds__(kThreads) unpack_generic(const uint8_t* __restrict__ src, int64_t inc_src,
                                                           void* __restrict__ dst, int64_t inc_dst,
                                                           int64_t first, int64_t n) {
  using Bits = typename Native<BASE>::bits;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t i = first + int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint64_t q = load_code_bytes<K>(src + i * inc_src * K);
    const Bits u = widen<BASE, K>(q);
    uint8_t* d = static_cast<uint8_t*>(dst) + i * inc_dst * int64_t(sizeof(Bits));
    if ((reinterpret_cast<uintptr_t>(d) & (sizeof(Bits) - 1)) == 0) {
      *reinterpret_cast<Bits*>(d) = u;
    } else {
#pragma unroll
      for (int b = 0; b < int(sizeof(Bits)); ++b) d[b] = uint8_t(u >> (8 * b));
    }
  }
}

// ---- pack --------------------------------------------------------------------

template <int BASE, int K>
__global__ void __launch_bounds__(kThreads) pack_groups(const void* __restrict__ src, uint8_t* __restrict__ dst,
                                                        int64_t ngroups, int mode) {
  using Bits = typename Native<BASE>::bits;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  for (; g < ngroups; g += kUnroll * stride) {
    Quad<BASE> q[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int64_t gu = g + u * stride;
      if (gu < ngroups) load_quad<BASE>(static_cast<const uint8_t*>(src) + gu * (4 * sizeof(Bits)), q[u]);
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int64_t gu = g + u * stride;
      if (gu < ngroups) {
        uint32_t w[K];
#pragma unroll
        for (int j = 0; j < K; ++j) w[j] = 0;
#pragma unroll
        for (int e = 0; e < 4; ++e) deposit_code<K>(w, e, narrow<BASE, K>(q[u].v[e], mode));
        store_group<K>(dst + gu * (4 * K), w);
      }
    }
  }
}

// Double-based pack with coalesced stores, the mirror of unpack_f64_tiles: a
// lane's 4 codes are 4k bytes at a 4k-byte stride, so storing them directly
// spreads every store instruction of a warp over 128k bytes (for k = 7 this
// halved the bandwidth).  A warp packs 32 groups (128 elements) into a
// per-warp shared buffer and writes the tile's 128k bytes as 16-byte chunks,
// consecutive lanes taking consecutive chunks.
template <int K>
__global__ void __launch_bounds__(kThreads) pack_f64_tiles(const uint8_t* __restrict__ src,
                                                           uint8_t* __restrict__ dst, int64_t ntiles, int mode) {
  constexpr int kWarps = kThreads / 32;
  constexpr int kChunks = 8 * K;                       // 16-byte chunks per tile (128 k bytes)
  __shared__ __align__(16) uint32_t buf[kWarps][kUnroll][32 * K];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t wstride = int64_t(gridDim.x) * kWarps;
  for (int64_t t = int64_t(blockIdx.x) * kWarps + warp; t < ntiles; t += kUnroll * wstride) {
    Quad<FLYTE_F64> q[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int64_t tu = t + u * wstride;
      if (tu < ntiles) load_quad<FLYTE_F64>(src + (tu * 32 + lane) * 32, q[u]);
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      if (t + u * wstride < ntiles) {
        uint32_t w[K];
#pragma unroll
        for (int j = 0; j < K; ++j) w[j] = 0;
#pragma unroll
        for (int e = 0; e < 4; ++e) deposit_code<K>(w, e, narrow<FLYTE_F64, K>(q[u].v[e], mode));
        store_group<K>(reinterpret_cast<uint8_t*>(buf[warp][u]) + lane * (4 * K), w);   // widest aligned stores
      }
    }
    __syncwarp();
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int64_t tu = t + u * wstride;
      if (tu < ntiles) {
#pragma unroll
        for (int c = lane; c < kChunks; c += 32)
          reinterpret_cast<uint4*>(dst + tu * (128 * K))[c] = reinterpret_cast<const uint4*>(buf[warp][u])[c];
      }
    }
    __syncwarp();
  }
}

template <int BASE, int K>
__global__ void __launch_bounds__(kThreads) pack_generic(const void* __restrict__ src, int64_t inc_src,
                                                         uint8_t* __restrict__ dst, int64_t inc_dst,
                                                         int64_t first, int64_t n, int mode) {
  using Bits = typename Native<BASE>::bits;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t i = first + int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint8_t* s = static_cast<const uint8_t*>(src) + i * inc_src * int64_t(sizeof(Bits));
    Bits u = 0;
    if ((reinterpret_cast<uintptr_t>(s) & (sizeof(Bits) - 1)) == 0) {
      u = *reinterpret_cast<const Bits*>(s);
    } else {
#pragma unroll
      for (int b = int(sizeof(Bits)) - 1; b >= 0; --b) u = (u << 8) | Bits(s[b]);
    }
    store_code_bytes<K>(dst + i * inc_dst * K, narrow<BASE, K>(u, mode));
  }
}

bool aligned(const void* p, int bytes) { return (reinterpret_cast<uintptr_t>(p) % bytes) == 0; }

}  // namespace

flyte_status launch_unpack(void* dst, const void* src, int64_t n, flyte_fmt f, int64_t inc_dst,
                           int64_t inc_src, cudaStream_t s) {
  return dispatch_fmt(f, [&]<int BASE, int K>() -> flyte_status {
    using Bits = typename Native<BASE>::bits;
    int64_t first = 0;
    const bool fast = inc_src == 1 && inc_dst == 1 && aligned(src, group_bytes(K)) && aligned(dst, 16);
    if constexpr (BASE == FLYTE_F64 && K < 8 && ((FLYTE_UNPACK_TILES_MASK >> K) & 1)) {
      if (fast && n >= 128) {
        const int64_t ntiles = n / 128;
        constexpr int smem = unpack_tile_smem<K>();
        if (cudaFuncSetAttribute(unpack_f64_tiles<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
            cudaSuccess)
          return cuda_status(cudaGetLastError(), "unpack");
        unpack_f64_tiles<K><<<grid_for(ntiles * 32, kThreads * unpack_tile_unroll<K>(), 6), kThreads, smem, s>>>(
            static_cast<const uint8_t*>(src), static_cast<uint8_t*>(dst), ntiles);
        FLYTE_TRY_LAUNCH("unpack");
        first = ntiles * 128;
      }
    }
    if (fast && n - first >= 4) {
      const int64_t ngroups = (n - first) / 4;
      unpack_groups<BASE, K><<<grid_for(ngroups, kThreads * kUnroll), kThreads, 0, s>>>(
          static_cast<const uint8_t*>(src) + first * K, static_cast<uint8_t*>(dst) + first * sizeof(Bits),
          ngroups);
      FLYTE_TRY_LAUNCH("unpack");
      first += ngroups * 4;
    }
    if (first < n) {
      unpack_generic<BASE, K><<<grid_for(n - first, kThreads), kThreads, 0, s>>>(
          static_cast<const uint8_t*>(src), inc_src, dst, inc_dst, first, n);
      FLYTE_TRY_LAUNCH("unpack");
    }
    (void)sizeof(Bits);
    return FLYTE_OK;
  });
}

flyte_status launch_pack(void* dst, const void* src, int64_t n, flyte_fmt f, int64_t inc_dst,
                         int64_t inc_src, int mode, cudaStream_t s) {
  return dispatch_fmt(f, [&]<int BASE, int K>() -> flyte_status {
    int64_t first = 0;
    using Bits = typename Native<BASE>::bits;
    const bool fast = inc_src == 1 && inc_dst == 1 && aligned(src, 16) && aligned(dst, group_bytes(K));
    if constexpr (BASE == FLYTE_F64 && K < 8 && ((FLYTE_PACK_TILES_MASK >> K) & 1)) {
      if (fast && aligned(dst, 16) && n >= 128) {
        const int64_t ntiles = n / 128;
        pack_f64_tiles<K><<<grid_for(ntiles * 32, kThreads * kUnroll, 6), kThreads, 0, s>>>(
            static_cast<const uint8_t*>(src), static_cast<uint8_t*>(dst), ntiles, mode);
        FLYTE_TRY_LAUNCH("pack");
        first = ntiles * 128;
      }
    }
    if (fast && n - first >= 4) {
      const int64_t ngroups = (n - first) / 4;
      pack_groups<BASE, K><<<grid_for(ngroups, kThreads * kUnroll), kThreads, 0, s>>>(
          static_cast<const uint8_t*>(src) + first * sizeof(Bits), static_cast<uint8_t*>(dst) + first * K, ngroups,
          mode);
      FLYTE_TRY_LAUNCH("pack");
      first += ngroups * 4;
    }
    if (first < n) {
      pack_generic<BASE, K><<<grid_for(n - first, kThreads), kThreads, 0, s>>>(
          src, inc_src, static_cast<uint8_t*>(dst), inc_dst, first, n, mode);
      FLYTE_TRY_LAUNCH("pack");
    }
    return FLYTE_OK;
  });
}

}  // namespace flyte
