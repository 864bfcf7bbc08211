// Warp-level helpers shared by the solve-phase kernels.
#pragma once

#include <cuda_runtime.h>

#include <utility>

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


// Programmatic dependent launch.  Every solve-phase kernel begins with
// pdl_prologue(): it waits until the grids it depends on have completed and
// their memory is visible (a no-op for a launch without the attribute), then
// lets the next grid of the stream start its launch.  Nothing before the wait
// touches global memory, so a dependent grid that starts early only spends
// the wait resident on the SMs.
__device__ __forceinline__ void pdl_prologue() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" :::);
}

// Launch with the programmatic-stream-serialization attribute when `pdl`.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(bool pdl, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                            Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

constexpr long long kBarrierCycles = 4000000000LL;  // about 2 s at 2 GHz

// Grid barrier for a cooperative launch (all CTAs resident).  bar[0] counts
// arrivals, bar[1] is the generation.  The wait is bounded: on timeout, or if
// another CTA already reported one, it sets *err and returns, and every later
// barrier of the launch returns at once.
__device__ __forceinline__ void grid_barrier(unsigned* bar, int* err) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = bar + 1;
    volatile int* verr = err;
    const unsigned gen = *vgen;
    __threadfence();
    const unsigned arrived = atomicAdd(bar, 1u);
    if (arrived == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const long long t0 = clock64();
      while (*vgen == gen) {
        if (*verr != 0 || clock64() - t0 > kBarrierCycles) {
          atomicExch(err, 1);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

}  // namespace amgdd
