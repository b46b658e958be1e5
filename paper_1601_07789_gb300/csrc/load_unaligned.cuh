// load_unaligned.cuh -- a 4-element flyte group read at any byte address.
//
// The vector group loads need the group's 4k bytes to start on a 4k-byte
// boundary (16, 8 or 4 bytes).  A stream that starts at another element (a
// sub-vector, a row of a matrix whose row length is not a multiple of 4)
// is read here with aligned 32-bit loads of the words that hold the group
// and funnel shifts, so the double-word arithmetic still applies.  Every
// word read holds at least one byte of the group, so no read leaves the
// 4-byte words the group occupies.  Used by blas1.cu, gemv.cu and batch.cu.
#pragma once

#include <cstdint>

namespace flyte {

template <int K>
__device__ __forceinline__ void load_group_unaligned(const uint8_t* p, uint32_t (&w)[K]) {
  const uint32_t off = uint32_t(reinterpret_cast<uintptr_t>(p) & 3u);
  const uint32_t* b = reinterpret_cast<const uint32_t*>(p - off);
  if (off == 0) {
#pragma unroll
    for (int j = 0; j < K; ++j) w[j] = __ldg(b + j);
  } else {
    uint32_t v[K + 1];
#pragma unroll
    for (int j = 0; j <= K; ++j) v[j] = __ldg(b + j);
#pragma unroll
    for (int j = 0; j < K; ++j) w[j] = __funnelshift_r(v[j], v[j + 1], 8 * off);
  }
}

}  // namespace flyte
