// Solve-phase kernels for K right-hand sides at once (K = 2, 4, 8, 16 or 32).
//
// Vectors hold the K columns interleaved by node: v[i * K + k].  Every
// matrix entry a gather-GEMV reads is applied to all the columns of its
// launch, so the matrices of a V-cycle (the smoother rows W_i, the coarse
// bases Z_i, the rows of A) stream once per K solves.  A gather-GEMV whose
// staged input would not fit shared memory at K columns takes the columns in
// tiles inside the launch (leading dimension K, tile t at column t * KT):
// each CTA stages one tile, applies its block rows, then the next tile, so
// the block's rows come again from L2 rather than DRAM.  The CG of each column is the same
// recurrence as the single right-hand-side solver, with its own scalars and
// convergence flag; a column that has converged keeps its iterate.
#include <cuda_runtime.h>

#include <cstdint>

#include "device_util.cuh"
#include "internal.h"

namespace amgdd {

namespace {

constexpr int kMultiThreads = 128;

template <class T, int K>
__device__ __forceinline__ void multi_out(SegMode mode, T* y, const T* c, int o, const T (&acc)[K], int ld, int k0) {
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int64_t at = (int64_t)o * ld + k0 + k;
    T* d = y + at;
    switch (mode) {
      case SEG_STORE: *d = acc[k]; break;
      case SEG_ADD: *d += acc[k]; break;
      case SEG_ATOMIC_ADD: atomicAdd(d, acc[k]); break;
      case SEG_ATOMIC_SUB: atomicAdd(d, -acc[k]); break;
      default: *d = c[at] - acc[k]; break;
    }
  }
}

// Lanes-per-row plans: one CTA per chunk (block b, rows r0..r1); the K
// columns of the gathered input are staged in shared memory, node-major.
template <class T, int L, int K>
__global__ void __launch_bounds__(kMultiThreads) k_seg_multi(const SegDesc* __restrict__ desc,
                                                             const int32_t* __restrict__ in_idx,
                                                             const int32_t* __restrict__ out_idx,
                                                             const T* __restrict__ M, const T* __restrict__ x,
                                                             T* __restrict__ y, const T* __restrict__ c, int mode,
                                                             const int* skip, int ld, int ntile) {
  pdl_prologue();
  if (skip != nullptr && *skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* xs = reinterpret_cast<T*>(smem_raw);
  const SegDesc dsc = desc[blockIdx.x];  // the chunk's block, in one dependent step
  const int r0 = dsc.r0;
  const int ncb = dsc.nc;
  const int r1 = dsc.r1;
  const int32_t* ii = in_idx + dsc.in_off;
  const int lane = threadIdx.x % L;
  const int grp = threadIdx.x / L;
  const int ngrp = blockDim.x / L;
  const unsigned mask = group_mask<L>();
  const T* Mb = M + dsc.m_off;
  const int32_t* oo = out_idx + dsc.out_off;
  for (int tile = 0; tile < ntile; ++tile) {
    const int k0 = tile * K;
    if (tile > 0) __syncthreads();  // every row of the previous tile has read xs
    for (int e = threadIdx.x; e < ncb * K; e += blockDim.x) {
      const int cc = e / K, k = e - cc * K;
      xs[e] = x[(int64_t)ii[cc] * ld + k0 + k];
    }
    __syncthreads();
    for (int r = r0 + grp; r < r1; r += ngrp) {
      const T* row = Mb + (int64_t)r * ncb;
      T acc[K];
#pragma unroll
      for (int k = 0; k < K; ++k) acc[k] = T(0);
      int cc = lane;
      for (; cc + 3 * L < ncb; cc += 4 * L) {  // four row entries per lane in flight
        T m[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) m[u] = row[cc + u * L];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int k = 0; k < K; ++k) acc[k] += m[u] * xs[(cc + u * L) * K + k];
      }
      for (; cc < ncb; cc += L) {
        const T m = row[cc];
#pragma unroll
        for (int k = 0; k < K; ++k) acc[k] += m * xs[cc * K + k];
      }
#pragma unroll
      for (int k = 0; k < K; ++k) acc[k] = group_sum<L>(acc[k], mask);
      if (lane == 0) multi_out<T, K>((SegMode)mode, y, c, oo[r], acc, ld, k0);
    }
  }
}

// Level-0 A by ELL rows for K interleaved columns: one thread per row reads
// each slot's index and value once and applies it to the K columns
// (consecutive in memory); y = A x, or y = c - A x (residual).
template <class T, int K, bool RESID>
__global__ void __launch_bounds__(256) k_ell_multi(const T* __restrict__ val, const int32_t* __restrict__ col, int w,
                                                   int64_t n, const T* __restrict__ x, T* __restrict__ y,
                                                   const T* __restrict__ c, const int* skip) {
  pdl_prologue();
  if (skip != nullptr && *skip) return;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  T acc[K];
#pragma unroll
  for (int k = 0; k < K; ++k) acc[k] = T(0);
  for (int q = 0; q < w; q += 4) {
    int ci[4];
    T v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      ci[u] = q + u < w ? col[(int64_t)(q + u) * n + i] : (int32_t)i;
      v[u] = q + u < w ? val[(int64_t)(q + u) * n + i] : T(0);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const T* xr = x + (int64_t)ci[u] * K;
#pragma unroll
      for (int k = 0; k < K; ++k) acc[k] += v[u] * xr[k];
    }
  }
#pragma unroll
  for (int k = 0; k < K; ++k) y[i * K + k] = RESID ? c[i * K + k] - acc[k] : acc[k];
}

// Row-per-lane plans over the block-wise transposed copy MT.
template <class T, int L, int K>
__global__ void __launch_bounds__(kMultiThreads) k_seg_rows_multi(
    const SegDesc* __restrict__ desc, int ntasks, int max_nc, const int32_t* __restrict__ in_idx, const int32_t* __restrict__ out_idx, const T* __restrict__ MT,
    const T* __restrict__ x, T* __restrict__ y, const T* __restrict__ c, int mode, const int* skip, int ld, int ntile) {
  pdl_prologue();
  if (skip != nullptr && *skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int grp = (int)threadIdx.x / L;
  const int t = blockIdx.x * (kMultiThreads / L) + grp;
  if (t >= ntasks) return;
  const int lane = threadIdx.x % L;
  const unsigned mask = group_mask<L>();
  T* xs = reinterpret_cast<T*>(smem_raw) + (size_t)grp * max_nc * K;
  const SegDesc dsc = desc[t];  // the task's block, in one dependent step
  const int r0 = dsc.r0;
  const int rows = dsc.r1 - dsc.r0;
  const int ncb = dsc.nc, nrb = dsc.nr;
  const int32_t* ii = in_idx + dsc.in_off;
  const int r = r0 + lane;
  const T* col = MT + dsc.m_off + r;
  for (int tile = 0; tile < ntile; ++tile) {
    const int k0 = tile * K;
    if (tile > 0) __syncwarp(mask);  // every lane of the group has read the previous tile
    for (int e = lane; e < ncb * K; e += L) {
      const int cc = e / K, k = e - cc * K;
      xs[e] = x[(int64_t)ii[cc] * ld + k0 + k];
    }
    __syncwarp(mask);
    if (lane < rows) {
      T acc[K];
#pragma unroll
      for (int k = 0; k < K; ++k) acc[k] = T(0);
      for (int cc = 0; cc < ncb; ++cc) {
        const T m = col[(int64_t)cc * nrb];
#pragma unroll
        for (int k = 0; k < K; ++k) acc[k] += m * xs[cc * K + k];
      }
      multi_out<T, K>((SegMode)mode, y, c, out_idx[dsc.out_off + r], acc, ld, k0);
    }
  }
}

// K dot products a_k . b_k (and a_k . c_k) per CTA; the grid stride is a
// multiple of K, so each thread stays on one column.
template <int K>
__global__ void __launch_bounds__(256) k_dot_multi(const double* __restrict__ a, const double* __restrict__ b,
                                                   const double* __restrict__ c, int64_t len,
                                                   double* __restrict__ partials, const int* skip) {
  pdl_prologue();
  if (skip != nullptr && *skip) return;
  double s0 = 0.0, s1 = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x) {
    const double ae = a[e];
    s0 += ae * b[e];
    if (c != nullptr) s1 += ae * c[e];
  }
  // lanes with equal (lane mod K) hold the same column
#pragma unroll
  for (int off = 16; off >= K; off >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, off);
    s1 += __shfl_xor_sync(0xffffffffu, s1, off);
  }
  __shared__ double sh0[8][K], sh1[8][K];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane < K) {
    sh0[w][lane] = s0;
    sh1[w][lane] = s1;
  }
  __syncthreads();
  if (threadIdx.x < K) {
    double v0 = 0.0, v1 = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      v0 += sh0[i][threadIdx.x];
      v1 += sh1[i][threadIdx.x];
    }
    partials[(int64_t)blockIdx.x * 2 * K + threadIdx.x] = v0;
    partials[(int64_t)blockIdx.x * 2 * K + K + threadIdx.x] = v1;
  }
}

// The scalar steps of CG for each of the K columns (warp k handles column
// k): the same recurrences as the single right-hand-side k_pcg_scalar.
// grp[0] = 1 once every column is done (the skip flag of the cycle).
template <int K>
__global__ void __launch_bounds__(32 * K) k_pcg_scalar_multi(int which, PcgState* st, int* grp,
                                                             const double* __restrict__ partials, int nblk,
                                                             cudaGraphConditionalHandle cond, int use_cond) {
  pdl_prologue();
  const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
  PcgState& S = st[k];
  const bool skip_col = which != 0 && which != 4 && S.done;
  double a = 0.0, bb = 0.0;
  if (!skip_col) {
    for (int i = lane; i < nblk; i += 32) {
      a += partials[(int64_t)i * 2 * K + k];
      bb += partials[(int64_t)i * 2 * K + K + k];
    }
    a = warp_sum_d(a);
    bb = warp_sum_d(bb);
  }
  if (lane == 0 && !skip_col) {
    switch (which) {
      case 0: S.rz = a; break;
      case 1:
        S.pq = a;
        if (!(a > 0.0)) {
          S.status = AMGDD_ERR_BREAKDOWN;
          S.done = 1;
        } else {
          S.alpha = S.rz / a;
        }
        break;
      case 2:
        S.rr = a;
        S.iters += 1;
        S.relres = S.bnorm2 > 0.0 ? sqrt(a / S.bnorm2) : 0.0;
        if (!(a == a)) {
          S.status = AMGDD_ERR_NONFINITE;
          S.done = 1;
        } else if (a <= S.tol2) {
          S.status = AMGDD_OK;
          S.done = 1;
        } else if (S.iters >= S.max_iter) {
          S.status = AMGDD_ERR_NO_CONVERGENCE;
          S.done = 1;
        } else if (S.flexible && S.iters % 10 == 0) {
          if (a > 0.81 * S.rr_mark) {  // FP32-cycle stall guard
            S.status = kStallStatus;
            S.done = 1;
          } else {
            S.rr_mark = a;
          }
        }
        break;
      case 3:
        S.rzn = a;
        S.rzo = bb;
        S.beta = S.flexible ? (a - bb) / S.rz : a / S.rz;
        S.rz = a;
        break;
      case 4:
        S.bnorm2 = a;
        S.rr_mark = a;
        S.tol2 = S.tol2 * a;
        S.iters = 0;
        S.relres = 1.0;
        S.status = AMGDD_OK;
        S.done = (a == 0.0) ? 1 : 0;
        if (a == 0.0) S.relres = 0.0;
        break;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int all = 1;
    for (int j = 0; j < K; ++j) all &= st[j].done != 0;
    grp[0] = all;
    if (which == 3 && use_cond) cudaGraphSetConditional(cond, all ? 0u : 1u);
  }
}

template <int K>
__global__ void k_update_xr_multi(const PcgState* __restrict__ st, const int* grp, double* __restrict__ x,
                                  double* __restrict__ r, const double* __restrict__ p, const double* __restrict__ q,
                                  int64_t len) {
  pdl_prologue();
  if (grp[0]) return;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x) {
    const PcgState& S = st[e % K];
    if (S.done) continue;
    x[e] += S.alpha * p[e];
    r[e] -= S.alpha * q[e];
  }
}

template <int K>
__global__ void k_update_p_multi(const PcgState* __restrict__ st, const int* grp, double* __restrict__ p,
                                 const double* __restrict__ z, double* __restrict__ zold, int64_t len) {
  pdl_prologue();
  if (grp[0]) return;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x) {
    const PcgState& S = st[e % K];
    if (S.done) continue;
    p[e] = z[e] + S.beta * p[e];
    if (zold != nullptr) zold[e] = z[e];
  }
}

// Column-major (n x K, leading dimension ld) <-> node-major interleaved.
__global__ void k_interleave(const double* __restrict__ src, int64_t ld, int ncols, double* __restrict__ dst, int64_t n,
                             int K) {
  pdl_prologue();
  const int64_t len = n * K;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / K;
    const int k = (int)(e - i * K);
    dst[e] = k < ncols ? src[(int64_t)k * ld + i] : 0.0;
  }
}

__global__ void k_deinterleave(const double* __restrict__ src, int64_t n, int K, double* __restrict__ dst, int64_t ld,
                               int ncols) {
  pdl_prologue();
  const int64_t len = n * ncols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = e / n;
    const int64_t i = e - k * n;
    dst[k * ld + i] = src[i * K + k];
  }
}

int grid_of(int64_t len, int threads) {
  const int64_t g = (len + threads - 1) / threads;
  return (int)std::min<int64_t>(std::max<int64_t>(g, 1), 152 * 16);
}

// Shared memory of one launch over KT columns.
size_t seg_multi_smem(const SegPlan& p, int KT, size_t esz) {
  const int per = p.rows_mode ? kMultiThreads / (p.kind == 8 ? 8 : (p.kind == 16 ? 16 : 32)) : 1;
  return (size_t)per * p.max_nc * KT * esz;
}

template <class T, int K>
int seg_multi_k(const SegPlan& p, const T* M, const T* MT, const T* x, T* y, SegMode mode, const T* c,
                const int* skip, cudaStream_t s, int ld, int ntile) {
  if (p.rows_mode) {
    if (MT == nullptr) {
      set_error("launch_seg_multi: row-per-lane plan needs the transposed operator");
      return AMGDD_ERR_INTERNAL;
    }
    auto go = [&](auto kern, int L) -> int {
      const int per = kMultiThreads / L;
      const size_t smem = (size_t)per * p.max_nc * K * sizeof(T);
      if (smem > 48 * 1024) AMGDD_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      AMGDD_CUDA(launch_k(g_pdl, kern, (p.ntasks + per - 1) / per, kMultiThreads, smem, s,
                          (const SegDesc*)p.task_desc.p, p.ntasks, p.max_nc, p.in_idx_ext, p.out_idx_ext, MT, x, y,
                          c, (int)mode, skip, ld, ntile));
      AMGDD_CUDA(cudaGetLastError());
      count_kernels(1);
      return AMGDD_OK;
    };
    switch (p.kind) {
      case 8: return go(k_seg_rows_multi<T, 8, K>, 8);
      case 16: return go(k_seg_rows_multi<T, 16, K>, 16);
      default: return go(k_seg_rows_multi<T, 32, K>, 32);
    }
  }
  auto go = [&](auto kern) -> int {
    const size_t smem = (size_t)p.max_nc * K * sizeof(T);
    if (smem > 48 * 1024) AMGDD_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    AMGDD_CUDA(launch_k(g_pdl, kern, p.nchunks, kMultiThreads, smem, s, (const SegDesc*)p.chunk_desc.p,
                        p.in_idx_ext, p.out_idx_ext, M, x, y, c, (int)mode, skip, ld, ntile));
    AMGDD_CUDA(cudaGetLastError());
    count_kernels(1);
    return AMGDD_OK;
  };
  switch (p.lanes) {
    case 4: return go(k_seg_multi<T, 4, K>);
    case 8: return go(k_seg_multi<T, 8, K>);
    case 16: return go(k_seg_multi<T, 16, K>);
    default: return go(k_seg_multi<T, 32, K>);
  }
}

// The columns of one staged tile: all K while the staged input stays within
// 64 KiB (wider tiles only where they leave room for several CTAs per SM),
// and within 200 KiB for K <= 8; the launch then walks K / KT tiles.
int seg_multi_tile(const SegPlan& p, int K, size_t esz) {
  int KT = K;
  while (KT > 8 && seg_multi_smem(p, KT, esz) > (size_t)64 * 1024) KT /= 2;
  while (KT > 2 && seg_multi_smem(p, KT, esz) > (size_t)200 * 1024) KT /= 2;
  return KT;
}

template <class T>
int seg_multi(const SegPlan& p, const T* M, const T* MT, const T* x, T* y, SegMode mode, const T* c, int K,
              const int* skip, cudaStream_t s) {
  if (K != 2 && K != 4 && K != 8 && K != 16 && K != 32) {
    set_error("launch_seg_multi: K must be 2, 4, 8, 16 or 32 (got %d)", K);
    return AMGDD_ERR_INTERNAL;
  }
  const int KT = seg_multi_tile(p, K, sizeof(T));
  const int nt = K / KT;
  switch (KT) {
    case 2: return seg_multi_k<T, 2>(p, M, MT, x, y, mode, c, skip, s, K, nt);
    case 4: return seg_multi_k<T, 4>(p, M, MT, x, y, mode, c, skip, s, K, nt);
    case 8: return seg_multi_k<T, 8>(p, M, MT, x, y, mode, c, skip, s, K, nt);
    case 16: return seg_multi_k<T, 16>(p, M, MT, x, y, mode, c, skip, s, K, nt);
    default: return seg_multi_k<T, 32>(p, M, MT, x, y, mode, c, skip, s, K, nt);
  }
}

}  // namespace

int launch_seg_multi(const SegPlan& p, const void* M, const void* MT, bool fp32, const void* x, void* y, SegMode mode,
                     const void* csrc, int K, const int* skip, cudaStream_t s) {
  if (p.rows_mode ? p.ntasks == 0 : p.nchunks == 0) return AMGDD_OK;
  if (mode == SEG_RESID && csrc == nullptr) {
    set_error("launch_seg_multi: the residual mode needs the right-hand side");
    return AMGDD_ERR_INTERNAL;
  }
  if (fp32)
    return seg_multi<float>(p, (const float*)M, (const float*)MT, (const float*)x, (float*)y, mode,
                            (const float*)csrc, K, skip, s);
  return seg_multi<double>(p, (const double*)M, (const double*)MT, (const double*)x, (double*)y, mode,
                           (const double*)csrc, K, skip, s);
}

int launch_dot_multi(const double* a, const double* b, const double* c, int64_t n, int K, double* partials,
                     const int* skip, cudaStream_t s) {
  const int64_t len = n * K;
  switch (K) {
    case 2: AMGDD_CUDA(launch_k(g_pdl, k_dot_multi<2>, kDotBlocks, 256, 0, s, a, b, c, len, partials, skip)); break;
    case 4: AMGDD_CUDA(launch_k(g_pdl, k_dot_multi<4>, kDotBlocks, 256, 0, s, a, b, c, len, partials, skip)); break;
    case 8: AMGDD_CUDA(launch_k(g_pdl, k_dot_multi<8>, kDotBlocks, 256, 0, s, a, b, c, len, partials, skip)); break;
    case 16: AMGDD_CUDA(launch_k(g_pdl, k_dot_multi<16>, kDotBlocks, 256, 0, s, a, b, c, len, partials, skip)); break;
    case 32: AMGDD_CUDA(launch_k(g_pdl, k_dot_multi<32>, kDotBlocks, 256, 0, s, a, b, c, len, partials, skip)); break;
    default: set_error("launch_dot_multi: K must be 2, 4, 8, 16 or 32"); return AMGDD_ERR_INTERNAL;
  }
  AMGDD_CUDA(cudaGetLastError());
  count_kernels(1);
  return AMGDD_OK;
}

int launch_pcg_scalar_multi(int which, PcgState* st, int* grp, const double* partials, int K, cudaStream_t s,
                            cudaGraphConditionalHandle cond, int use_cond) {
  switch (K) {
    case 2: AMGDD_CUDA(launch_k(g_pdl, k_pcg_scalar_multi<2>, 1, 64, 0, s, which, st, grp, partials, kDotBlocks, cond, use_cond)); break;
    case 4: AMGDD_CUDA(launch_k(g_pdl, k_pcg_scalar_multi<4>, 1, 128, 0, s, which, st, grp, partials, kDotBlocks, cond, use_cond)); break;
    case 8: AMGDD_CUDA(launch_k(g_pdl, k_pcg_scalar_multi<8>, 1, 256, 0, s, which, st, grp, partials, kDotBlocks, cond, use_cond)); break;
    case 16: AMGDD_CUDA(launch_k(g_pdl, k_pcg_scalar_multi<16>, 1, 512, 0, s, which, st, grp, partials, kDotBlocks, cond, use_cond)); break;
    case 32: AMGDD_CUDA(launch_k(g_pdl, k_pcg_scalar_multi<32>, 1, 1024, 0, s, which, st, grp, partials, kDotBlocks, cond, use_cond)); break;
    default: set_error("launch_pcg_scalar_multi: K must be 2, 4, 8, 16 or 32"); return AMGDD_ERR_INTERNAL;
  }
  AMGDD_CUDA(cudaGetLastError());
  count_kernels(1);
  return AMGDD_OK;
}

int launch_update_xr_multi(const PcgState* st, const int* grp, double* x, double* r, const double* p, const double* q,
                           int64_t n, int K, cudaStream_t s) {
  const int64_t len = n * K;
  const int g = grid_of(len, 256);
  switch (K) {
    case 2: AMGDD_CUDA(launch_k(g_pdl, k_update_xr_multi<2>, g, 256, 0, s, st, grp, x, r, p, q, len)); break;
    case 4: AMGDD_CUDA(launch_k(g_pdl, k_update_xr_multi<4>, g, 256, 0, s, st, grp, x, r, p, q, len)); break;
    case 8: AMGDD_CUDA(launch_k(g_pdl, k_update_xr_multi<8>, g, 256, 0, s, st, grp, x, r, p, q, len)); break;
    case 16: AMGDD_CUDA(launch_k(g_pdl, k_update_xr_multi<16>, g, 256, 0, s, st, grp, x, r, p, q, len)); break;
    case 32: AMGDD_CUDA(launch_k(g_pdl, k_update_xr_multi<32>, g, 256, 0, s, st, grp, x, r, p, q, len)); break;
    default: set_error("launch_update_xr_multi: K must be 2, 4, 8, 16 or 32"); return AMGDD_ERR_INTERNAL;
  }
  AMGDD_CUDA(cudaGetLastError());
  count_kernels(1);
  return AMGDD_OK;
}

int launch_update_p_multi(const PcgState* st, const int* grp, double* p, const double* z, double* zold, int64_t n,
                          int K, cudaStream_t s) {
  const int64_t len = n * K;
  const int g = grid_of(len, 256);
  switch (K) {
    case 2: AMGDD_CUDA(launch_k(g_pdl, k_update_p_multi<2>, g, 256, 0, s, st, grp, p, z, zold, len)); break;
    case 4: AMGDD_CUDA(launch_k(g_pdl, k_update_p_multi<4>, g, 256, 0, s, st, grp, p, z, zold, len)); break;
    case 8: AMGDD_CUDA(launch_k(g_pdl, k_update_p_multi<8>, g, 256, 0, s, st, grp, p, z, zold, len)); break;
    case 16: AMGDD_CUDA(launch_k(g_pdl, k_update_p_multi<16>, g, 256, 0, s, st, grp, p, z, zold, len)); break;
    case 32: AMGDD_CUDA(launch_k(g_pdl, k_update_p_multi<32>, g, 256, 0, s, st, grp, p, z, zold, len)); break;
    default: set_error("launch_update_p_multi: K must be 2, 4, 8, 16 or 32"); return AMGDD_ERR_INTERNAL;
  }
  AMGDD_CUDA(cudaGetLastError());
  count_kernels(1);
  return AMGDD_OK;
}

int launch_interleave(const double* src, int64_t ld, int ncols, double* dst, int64_t n, int K, cudaStream_t s) {
  AMGDD_CUDA(launch_k(g_pdl, k_interleave, grid_of(n * K, 256), 256, 0, s, src, ld, ncols, dst, n, K));
  AMGDD_CUDA(cudaGetLastError());
  count_kernels(1);
  return AMGDD_OK;
}

int launch_deinterleave(const double* src, int64_t n, int K, double* dst, int64_t ld, int ncols, cudaStream_t s) {
  AMGDD_CUDA(launch_k(g_pdl, k_deinterleave, grid_of(n * ncols, 256), 256, 0, s, src, n, K, dst, ld, ncols));
  AMGDD_CUDA(cudaGetLastError());
  count_kernels(1);
  return AMGDD_OK;
}

int launch_ell_multi(const Level& L, bool fp32, const void* x, void* y, const void* c, int K, const int* skip,
                     cudaStream_t s) {
  if (L.n <= 0) return AMGDD_OK;
  const int grid = (int)((L.n + 255) / 256);
  auto go = [&](auto kf32, auto kf64) -> int {
    if (fp32)
      AMGDD_CUDA(launch_k(g_pdl, kf32, grid, 256, 0, s, (const float*)L.ell32.p, (const int32_t*)L.ellc.p, L.ell_w,
                          L.n, (const float*)x, (float*)y, (const float*)c, skip));
    else
      AMGDD_CUDA(launch_k(g_pdl, kf64, grid, 256, 0, s, (const double*)L.ell64.p, (const int32_t*)L.ellc.p, L.ell_w,
                          L.n, (const double*)x, (double*)y, (const double*)c, skip));
    count_kernels(1);
    return AMGDD_OK;
  };
  const bool res = c != nullptr;
  switch (K) {
    case 2:
      return res ? go(k_ell_multi<float, 2, true>, k_ell_multi<double, 2, true>)
                 : go(k_ell_multi<float, 2, false>, k_ell_multi<double, 2, false>);
    case 4:
      return res ? go(k_ell_multi<float, 4, true>, k_ell_multi<double, 4, true>)
                 : go(k_ell_multi<float, 4, false>, k_ell_multi<double, 4, false>);
    case 8:
      return res ? go(k_ell_multi<float, 8, true>, k_ell_multi<double, 8, true>)
                 : go(k_ell_multi<float, 8, false>, k_ell_multi<double, 8, false>);
    case 16:
      return res ? go(k_ell_multi<float, 16, true>, k_ell_multi<double, 16, true>)
                 : go(k_ell_multi<float, 16, false>, k_ell_multi<double, 16, false>);
    case 32:
      return res ? go(k_ell_multi<float, 32, true>, k_ell_multi<double, 32, true>)
                 : go(k_ell_multi<float, 32, false>, k_ell_multi<double, 32, false>);
    default:
      set_error("launch_ell_multi: K must be 2, 4, 8, 16 or 32");
      return AMGDD_ERR_INVALID_ARG;
  }
}

}  // namespace amgdd
