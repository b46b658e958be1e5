// bulkpipe.cuh -- mbarrier and bulk-copy primitives of the shared-memory rings.
//
// A ring has S stages of shared memory, each with a "full" mbarrier (and,
// when producer and consumers are different warps, an "empty" one).  For
// each stage a producer lane arms the full barrier with the number of bytes
// expected, producer lanes issue cp.async.bulk copies (global -> shared,
// completion counted on the barrier), and the consumers wait on the
// barrier's phase before reading the stage, then arrive on the empty
// barrier.  Keeping S - 1 stages in flight makes the bytes in flight per SM
// independent of register pressure and occupancy (gemv 'N'; the gemm uses
// the same barriers with TMA tensor copies).
//
// Every wait is bounded: after 200 ms (or kWaitLimit polls, or as soon as
// another warp has already recorded a failure) the waiting lane records an
// error code in a device word (the operation's status word in the workspace)
// and the kernel abandons its work, after draining the copies it issued.
#pragma once

#include <cstdint>

#include "flyte_internal.cuh"

namespace flyte {

constexpr uint32_t kWaitLimit = 1u << 24;      // polls of try_wait (each may suspend briefly)
constexpr uint64_t kWaitNanos = 200000000ull;  // wall-clock limit of one wait
constexpr int kErrPipeTimeout = 1;

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Plain arrival (count-based phases).
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Wait for the given phase parity; false (and an error recorded in *err,
// when err is given) on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t it = 0; it < kWaitLimit; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255) == 255) {
      if (global_ns() - t0 > kWaitNanos) break;
      if (err && *reinterpret_cast<volatile int*>(err) != 0) break;
    }
  }
  if (err) atomicOr(err, kErrPipeTimeout);
  return false;
}

// Order this thread's earlier generic-proxy accesses of shared memory before
// its following async-proxy (bulk copy) accesses.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 1-D bulk copy global -> shared; bytes a multiple of 16, both addresses 16-byte aligned.
__device__ __forceinline__ void bulk_g2s(void* smem_dst, const void* gmem_src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(smem_dst)),
      "l"(gmem_src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Shared-memory loads of a lane's 4-element group (4k bytes at a 4k-byte
// aligned offset inside a 16-byte aligned stage).
template <int K>
__device__ __forceinline__ void lds_group(const uint8_t* p, uint32_t (&w)[K]) {
  constexpr int S = group_bytes(K);
  if constexpr (S == 16) {
#pragma unroll
    for (int i = 0; i < K / 4; ++i) {
      const uint4 v = reinterpret_cast<const uint4*>(p)[i];
      w[4 * i] = v.x; w[4 * i + 1] = v.y; w[4 * i + 2] = v.z; w[4 * i + 3] = v.w;
    }
  } else if constexpr (S == 8) {
#pragma unroll
    for (int i = 0; i < K / 2; ++i) {
      const uint2 v = reinterpret_cast<const uint2*>(p)[i];
      w[2 * i] = v.x; w[2 * i + 1] = v.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < K; ++i) w[i] = reinterpret_cast<const uint32_t*>(p)[i];
  }
}

}  // namespace flyte
