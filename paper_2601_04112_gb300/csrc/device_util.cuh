// Warp-level helpers shared by the solve-phase kernels.
#pragma once

#include <cuda_runtime.h>

namespace amgdd {

// Sum over the aligned group of L lanes (L a power of two dividing 32) that
// the calling lane belongs to; every lane of the group gets the sum.
template <int L, class T>
__device__ __forceinline__ T group_sum(T v, unsigned mask) {
#pragma unroll
  for (int off = L / 2; off > 0; off >>= 1) v += __shfl_xor_sync(mask, v, off, L);
  return v;
}

template <int L>
__device__ __forceinline__ unsigned group_mask() {
  if constexpr (L == 32) {
    return 0xffffffffu;
  } else {
    const int g = (threadIdx.x & 31) / L;
    return ((1u << L) - 1u) << (g * L);
  }
}


__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

}  // namespace amgdd
