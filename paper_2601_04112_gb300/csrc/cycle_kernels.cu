// Solve-phase kernels: everything one V-cycle and one CG iteration execute.
//
//  * k_seg      batched gather-GEMV-scatter (RAS, Eq. ras: x(omega_i) =
//               [A_i^{-1}](omega_i, :) r(Omega_i); RAS-T, Eq. ras-t:
//               x(Omega_i) += [A_i^{-1}](:, omega_i) s(omega_i); restriction
//               and prolongation with the block-diagonal P of Eq. mg-p; the
//               coarsest solve with the explicit inverse of A_L).
//  * k_apply    A-apply by row groups of G: y(S_g) -/+= R_g^T (R_g x(S_g)),
//               i.e. G then G^T (Eq. 1), with R_g the compressed rows of G
//               that share the support S_g.
//  * PCG vector kernels with deterministic two-stage reductions.
//
// All kernels take an optional device flag `skip`; when it is set (the CG
// iteration has converged) they return at once, so a captured batch of
// iterations is a no-op after convergence.
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"

namespace amgdd {

namespace {

constexpr int kSegThreads = 128;

template <class T>
__device__ __forceinline__ void atomic_add(T* p, T v) {
  atomicAdd(p, v);
}

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

// ---------------------------------------------------------------------------
// Batched gather-GEMV-scatter.  One CTA takes `rows_per_chunk` rows of one
// block; the gathered input x(in_idx) is staged once in shared memory and L
// lanes stream each row of the row-major block with coalesced loads.
template <class T>
struct Vec2 {};
template <>
struct Vec2<float> {
  using type = float4;
  static constexpr int width = 4;
};
template <>
struct Vec2<double> {
  using type = double2;
  static constexpr int width = 2;
};

__device__ __forceinline__ float vdot(const float4& a, const float4& b) {
  return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w;
}
__device__ __forceinline__ double vdot(const double2& a, const double2& b) { return a.x * b.x + a.y * b.y; }

// VEC: every row of every block starts on a 16-byte boundary and has a
// multiple of the vector width entries (checked when the plan is built);
// rows and the staged x are then read 16 bytes per lane.
template <class T, int L, int MODE, bool VEC>
__global__ void __launch_bounds__(kSegThreads) k_seg(const int32_t* __restrict__ chunk_blk,
                                                     const int32_t* __restrict__ chunk_row0, int rows_per_chunk,
                                                     const int64_t* __restrict__ m_off, const int32_t* __restrict__ nr,
                                                     const int32_t* __restrict__ nc,
                                                     const int64_t* __restrict__ in_off,
                                                     const int64_t* __restrict__ out_off,
                                                     const int32_t* __restrict__ in_idx,
                                                     const int32_t* __restrict__ out_idx, const T* __restrict__ M,
                                                     const T* __restrict__ x, T* __restrict__ y, const int* skip,
                                                     const T* __restrict__ csrc, T* __restrict__ cdst) {
  if (skip != nullptr && *skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* xs = reinterpret_cast<T*>(smem_raw);
  const int b = chunk_blk[blockIdx.x];
  const int r0 = chunk_row0[blockIdx.x];
  const int ncb = nc[b];
  const int r1 = min(nr[b], r0 + rows_per_chunk);
  const int32_t* ii = in_idx + in_off[b];
  for (int c = threadIdx.x; c < ncb; c += blockDim.x) xs[c] = x[ii[c]];
  __syncthreads();
  const int lane = threadIdx.x % L;
  const int grp = threadIdx.x / L;
  const int ngrp = blockDim.x / L;
  const unsigned mask = group_mask<L>();
  const T* Mb = M + m_off[b];
  const int32_t* oo = out_idx + out_off[b];
  for (int r = r0 + grp; r < r1; r += ngrp) {
    const T* row = Mb + (int64_t)r * ncb;
    T acc = T(0);
    if constexpr (VEC) {
      using V = typename Vec2<T>::type;
      constexpr int W = Vec2<T>::width;
      const V* rv = reinterpret_cast<const V*>(row);
      const V* xv = reinterpret_cast<const V*>(xs);
      const int nv = ncb / W;
      for (int c = lane; c < nv; c += L) acc += vdot(rv[c], xv[c]);
    } else {
      for (int c = lane; c < ncb; c += L) acc += row[c] * xs[c];
    }
    acc = group_sum<L>(acc, mask);
    if (lane == 0) {
      const int o = oo[r];
      T* dst = y + o;
      if (MODE == SEG_STORE)
        *dst = acc;
      else if (MODE == SEG_ADD)
        *dst += acc;
      else if (MODE == SEG_ATOMIC_ADD)
        atomic_add(dst, acc);
      else if (MODE == SEG_ATOMIC_SUB)
        atomic_add(dst, -acc);
      else
        *dst = csrc[o] - acc;
      if (MODE != SEG_RESID && cdst != nullptr) cdst[o] = csrc[o];
    }
  }
}

// Short rows, row per lane: a task (block, first row, up to L rows) belongs
// to L lanes; lane l owns output row r0 + l and streams column c of the
// block's transposed copy MT (nc x nr, row-major), so the L lanes read L
// consecutive values.  x(in_idx) is staged once per task in shared memory.
// Outputs, atomics and the fused copy are issued by all lanes at once.
template <class T, int L, int MODE>
__global__ void __launch_bounds__(128) k_seg_rows(const int32_t* __restrict__ task_blk,
                                                  const int32_t* __restrict__ task_row0,
                                                  const int32_t* __restrict__ task_nrow, int ntasks, int max_nc,
                                                  const int64_t* __restrict__ m_off, const int32_t* __restrict__ nr,
                                                  const int32_t* __restrict__ nc, const int64_t* __restrict__ in_off,
                                                  const int64_t* __restrict__ out_off,
                                                  const int32_t* __restrict__ in_idx,
                                                  const int32_t* __restrict__ out_idx, const T* __restrict__ MT,
                                                  const T* __restrict__ x, T* __restrict__ y, const int* skip,
                                                  const T* __restrict__ csrc, T* __restrict__ cdst) {
  if (skip != nullptr && *skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int grp = (int)threadIdx.x / L;
  const int t = blockIdx.x * (128 / L) + grp;
  if (t >= ntasks) return;
  const int lane = threadIdx.x % L;
  const unsigned mask = group_mask<L>();
  T* xs = reinterpret_cast<T*>(smem_raw) + (size_t)grp * max_nc;
  const int b = task_blk[t];
  const int r0 = task_row0[t];
  const int rows = task_nrow[t];
  const int ncb = nc[b], nrb = nr[b];
  const int32_t* ii = in_idx + in_off[b];
  for (int c = lane; c < ncb; c += L) xs[c] = x[ii[c]];
  __syncwarp(mask);
  if (lane >= rows) return;
  const int r = r0 + lane;
  const T* col = MT + m_off[b] + r;
  T acc = T(0);
  for (int c = 0; c < ncb; ++c) acc += col[(int64_t)c * nrb] * xs[c];
  const int o = out_idx[out_off[b] + r];
  T* dst = y + o;
  if (MODE == SEG_STORE)
    *dst = acc;
  else if (MODE == SEG_ADD)
    *dst += acc;
  else if (MODE == SEG_ATOMIC_ADD)
    atomic_add(dst, acc);
  else if (MODE == SEG_ATOMIC_SUB)
    atomic_add(dst, -acc);
  else
    *dst = csrc[o] - acc;
  if (MODE != SEG_RESID && cdst != nullptr) cdst[o] = csrc[o];
}

template <class T, int L, int MODE>
int seg_rows_launch(const SegPlan& p, const T* MT, const T* x, T* y, const int* skip, cudaStream_t s, const T* csrc,
                    T* cdst) {
  const int per = 128 / L;
  const int grid = (p.ntasks + per - 1) / per;
  const size_t smem = (size_t)per * p.max_nc * sizeof(T);
  auto kern = k_seg_rows<T, L, MODE>;
  if (smem > 48 * 1024) AMGDD_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<grid, 128, smem, s>>>(p.task_blk.p, p.task_row0.p, p.task_nrow.p, p.ntasks, p.max_nc, p.m_off.p, p.nr.p,
                               p.nc.p, p.in_off.p, p.out_off.p, p.in_idx_ext, p.out_idx_ext, MT, x, y, skip, csrc,
                               cdst);
  AMGDD_CUDA(cudaGetLastError());
  count_kernels(1);
  return AMGDD_OK;
}

template <class T, int L>
int seg_rows_mode(const SegPlan& p, const T* MT, const T* x, T* y, SegMode mode, const int* skip, cudaStream_t s,
                  const T* csrc, T* cdst) {
  switch (mode) {
    case SEG_STORE: return seg_rows_launch<T, L, SEG_STORE>(p, MT, x, y, skip, s, csrc, cdst);
    case SEG_ADD: return seg_rows_launch<T, L, SEG_ADD>(p, MT, x, y, skip, s, csrc, cdst);
    case SEG_ATOMIC_ADD: return seg_rows_launch<T, L, SEG_ATOMIC_ADD>(p, MT, x, y, skip, s, csrc, cdst);
    case SEG_ATOMIC_SUB: return seg_rows_launch<T, L, SEG_ATOMIC_SUB>(p, MT, x, y, skip, s, csrc, cdst);
    default: return seg_rows_launch<T, L, SEG_RESID>(p, MT, x, y, skip, s, csrc, cdst);
  }
}

template <class T, int L>
int seg_dispatch_mode(const SegPlan& p, const T* M, const T* x, T* y, SegMode mode, const int* skip,
                      cudaStream_t s, const T* csrc, T* cdst) {
  const size_t smem = (size_t)p.max_nc * sizeof(T);
  auto launch = [&](auto kern) -> int {
    if (smem > 48 * 1024) AMGDD_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<p.nchunks, kSegThreads, smem, s>>>(p.chunk_blk.p, p.chunk_row0.p, p.rows_per_chunk, p.m_off.p, p.nr.p,
                                              p.nc.p, p.in_off.p, p.out_off.p, p.in_idx_ext, p.out_idx_ext, M, x, y,
                                              skip, csrc, cdst);
    AMGDD_CUDA(cudaGetLastError());
    count_kernels(1);
    return AMGDD_OK;
  };
  if (p.vec) {
    switch (mode) {
      case SEG_STORE: return launch(k_seg<T, L, SEG_STORE, true>);
      case SEG_ADD: return launch(k_seg<T, L, SEG_ADD, true>);
      case SEG_ATOMIC_ADD: return launch(k_seg<T, L, SEG_ATOMIC_ADD, true>);
      case SEG_ATOMIC_SUB: return launch(k_seg<T, L, SEG_ATOMIC_SUB, true>);
      default: return launch(k_seg<T, L, SEG_RESID, true>);
    }
  }
  switch (mode) {
    case SEG_STORE: return launch(k_seg<T, L, SEG_STORE, false>);
    case SEG_ADD: return launch(k_seg<T, L, SEG_ADD, false>);
    case SEG_ATOMIC_ADD: return launch(k_seg<T, L, SEG_ATOMIC_ADD, false>);
    case SEG_ATOMIC_SUB: return launch(k_seg<T, L, SEG_ATOMIC_SUB, false>);
    default: return launch(k_seg<T, L, SEG_RESID, false>);
  }
}

template <class T>
int seg_dispatch(const SegPlan& p, const T* M, const T* MT, const T* x, T* y, SegMode mode, const int* skip,
                 cudaStream_t s, const T* csrc, T* cdst) {
  if (p.rows_mode) {
    if (MT == nullptr) {
      set_error("launch_seg: row-per-lane plan needs the transposed operator");
      return AMGDD_ERR_INTERNAL;
    }
    switch (p.kind) {
      case 8: return seg_rows_mode<T, 8>(p, MT, x, y, mode, skip, s, csrc, cdst);
      case 16: return seg_rows_mode<T, 16>(p, MT, x, y, mode, skip, s, csrc, cdst);
      default: return seg_rows_mode<T, 32>(p, MT, x, y, mode, skip, s, csrc, cdst);
    }
  }
  switch (p.lanes) {
    case 4: return seg_dispatch_mode<T, 4>(p, M, x, y, mode, skip, s, csrc, cdst);
    case 8: return seg_dispatch_mode<T, 8>(p, M, x, y, mode, skip, s, csrc, cdst);
    case 16: return seg_dispatch_mode<T, 16>(p, M, x, y, mode, skip, s, csrc, cdst);
    default: return seg_dispatch_mode<T, 32>(p, M, x, y, mode, skip, s, csrc, cdst);
  }
}

// ---------------------------------------------------------------------------
// A-apply by compressed row groups.  A task is (group, first row, rows);
// L lanes share it, lane l owning support columns l, l+L, ...  For each row
// t = R_row . x(S) (group reduction), then acc += R_row * t; finally the
// lanes scatter acc into y(S) with atomics (supports of different groups
// overlap).  Kinds: (L, J) with J = columns per lane held in registers.
struct ApplyArgs {
  const int32_t* task_grp;
  const int32_t* task_row0;
  const int32_t* task_nrow;
  const int64_t* g_ptr;
  const int32_t* g_idx;
  const int64_t* r_off;
  int nbuckets;
  int bucket_start[16];
  int bucket_kind[16];
  int bucket_task0[16];
  int bucket_tasks[16];
};

template <class T, int L, int J>
__device__ __forceinline__ void apply_task(const ApplyArgs& a, int task, const T* __restrict__ R,
                                           const T* __restrict__ x, T* __restrict__ y, T sign, unsigned mask) {
  const int g = a.task_grp[task];
  const int row0 = a.task_row0[task];
  const int nrow = a.task_nrow[task];
  const int64_t sp = a.g_ptr[g];
  const int s = (int)(a.g_ptr[g + 1] - sp);
  const int32_t* S = a.g_idx + sp;
  const T* Rg = R + a.r_off[g];
  const int lane = threadIdx.x % L;
  T xr[J], acc[J];
#pragma unroll
  for (int j = 0; j < J; ++j) {
    const int c = lane + L * j;
    xr[j] = c < s ? x[S[c]] : T(0);
    acc[j] = T(0);
  }
  for (int r = row0; r < row0 + nrow; ++r) {
    const T* row = Rg + (int64_t)r * s;
    T rv[J];
    T t = T(0);
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const int c = lane + L * j;
      rv[j] = c < s ? row[c] : T(0);
      t += rv[j] * xr[j];
    }
    t = group_sum<L>(t, mask);
#pragma unroll
    for (int j = 0; j < J; ++j) acc[j] += rv[j] * t;
  }
#pragma unroll
  for (int j = 0; j < J; ++j) {
    const int c = lane + L * j;
    if (c < s) atomic_add(y + S[c], sign * acc[j]);
  }
}

constexpr int kApplyThreads = 128;

// Supports of at most 4 nodes (every cell group of a 2D Q1 level 0): one
// thread owns a group, keeps x(S) and the rows of R_g in registers, and
// needs no shuffles.
template <class T>
__device__ __forceinline__ void apply_task_thread(const ApplyArgs& a, int task, const T* __restrict__ R,
                                                  const T* __restrict__ x, T* __restrict__ y, T sign) {
  const int g = a.task_grp[task];
  const int nrow = min(a.task_nrow[task], 4);
  const int64_t sp = a.g_ptr[g];
  const int s = (int)(a.g_ptr[g + 1] - sp);
  const int32_t* S = a.g_idx + sp;
  const T* Rg = R + a.r_off[g];
  // issue every load of the group before using any of them
  int idx[4];
  T xr[4], acc[4], rv[4][4];
#pragma unroll
  for (int c = 0; c < 4; ++c) idx[c] = c < s ? S[c] : 0;
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) rv[r][c] = (r < nrow && c < s) ? Rg[r * s + c] : T(0);
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    xr[c] = c < s ? x[idx[c]] : T(0);
    acc[c] = T(0);
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    T t = T(0);
#pragma unroll
    for (int c = 0; c < 4; ++c) t += rv[r][c] * xr[c];
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[c] += rv[r][c] * t;
  }
#pragma unroll
  for (int c = 0; c < 4; ++c)
    if (c < s) atomic_add(y + idx[c], sign * acc[c]);
}

// Grouped A-apply, two kernels so that the narrow kinds are not held to
// the register budget of the wide ones.  BIG = false: kind 0 (at most 4
// nodes, one thread per group) and kinds 1-3 (8, 16, 32 lanes, one column
// per lane).  BIG = true: kinds 4-7 (32 lanes, 2/4/8/16 columns per lane).
// Supports above 512 nodes go through two gather-GEMV passes instead.
template <class T, bool BIG>
__global__ void __launch_bounds__(kApplyThreads) k_apply(ApplyArgs a, const T* __restrict__ R,
                                                         const T* __restrict__ x, T* __restrict__ y, T sign,
                                                         const int* skip) {
  if (skip != nullptr && *skip) return;
  int bkt = 0;
  while (bkt + 1 < a.nbuckets && (int)blockIdx.x >= a.bucket_start[bkt + 1]) ++bkt;
  const int kind = a.bucket_kind[bkt];
  const int cta = blockIdx.x - a.bucket_start[bkt];
#define AMGDD_KIND(K, LL, JJ)                                                               \
  case K: {                                                                                 \
    const int t = cta * (kApplyThreads / LL) + (int)threadIdx.x / LL;                       \
    if (t < a.bucket_tasks[bkt])                                                            \
      apply_task<T, LL, JJ>(a, a.bucket_task0[bkt] + t, R, x, y, sign, group_mask<LL>());    \
    return;                                                                                 \
  }
  if constexpr (BIG) {
    switch (kind) {
      AMGDD_KIND(4, 32, 2)
      AMGDD_KIND(5, 32, 4)
      AMGDD_KIND(6, 32, 8)
      AMGDD_KIND(7, 32, 16)
      default: return;
    }
  } else {
    if (kind == 0) {
      // two groups per thread (independent work for latency hiding)
      const int t = cta * (2 * kApplyThreads) + (int)threadIdx.x;
      if (t < a.bucket_tasks[bkt]) apply_task_thread<T>(a, a.bucket_task0[bkt] + t, R, x, y, sign);
      if (t + kApplyThreads < a.bucket_tasks[bkt])
        apply_task_thread<T>(a, a.bucket_task0[bkt] + t + kApplyThreads, R, x, y, sign);
      return;
    }
    switch (kind) {
      AMGDD_KIND(1, 8, 1)
      AMGDD_KIND(2, 16, 1)
      AMGDD_KIND(3, 32, 1)
      default: return;
    }
  }
#undef AMGDD_KIND
}

// ---------------------------------------------------------------------------
template <class S, class D>
__global__ void k_cast(const S* __restrict__ src, D* __restrict__ dst, int64_t n, const int* skip) {
  if (skip != nullptr && *skip) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (D)src[i];
}

int grid_for(int64_t n, int threads) {
  int64_t g = (n + threads - 1) / threads;
  if (g > 152 * 16) g = 152 * 16;
  if (g < 1) g = 1;
  return (int)g;
}

// Deterministic dot products: fixed grid, fixed per-thread stride, tree
// reductions in a fixed order; stage 2 is done by k_pcg_scalar.
constexpr int kDotThreads = 256;

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

__global__ void __launch_bounds__(kDotThreads) k_dot_partial(const double* __restrict__ a, const double* __restrict__ b,
                                                             const double* __restrict__ c, int64_t n,
                                                             double* __restrict__ partials, const int* skip) {
  if (skip != nullptr && *skip) return;
  double s0 = 0.0, s1 = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double ai = a[i];
    s0 += ai * b[i];
    if (c != nullptr) s1 += ai * c[i];
  }
  __shared__ double sh0[kDotThreads / 32], sh1[kDotThreads / 32];
  s0 = warp_sum_d(s0);
  s1 = warp_sum_d(s1);
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    sh0[w] = s0;
    sh1[w] = s1;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    double v0 = threadIdx.x < kDotThreads / 32 ? sh0[threadIdx.x] : 0.0;
    double v1 = threadIdx.x < kDotThreads / 32 ? sh1[threadIdx.x] : 0.0;
    v0 = warp_sum_d(v0);
    v1 = warp_sum_d(v1);
    if (threadIdx.x == 0) {
      partials[2 * blockIdx.x] = v0;
      partials[2 * blockIdx.x + 1] = v1;
    }
  }
}

// Stage 2 of the dot products plus the scalar recurrences of CG.
//  which 0: rz = sum(r.z)                         (start)
//        1: pq = sum(p.q); alpha = rz / pq        (breakdown if pq <= 0)
//        2: rr = sum(r.r); convergence / iteration limit
//        3: rzn = sum(r.z_new), rzo = sum(r.z_old); beta; rz = rzn
//        4: bnorm2 = sum(b.b); tol2 = tol^2 bnorm2 (tol passed in st->tol2)
__global__ void __launch_bounds__(1024) k_pcg_scalar(int which, PcgState* st, const double* __restrict__ partials,
                                                     cudaGraphConditionalHandle cond, int use_cond) {
  if (which != 0 && which != 4 && st->done) {
    if (which == 3 && use_cond && threadIdx.x == 0) cudaGraphSetConditional(cond, 0u);
    return;
  }
  __shared__ double s0[1024], s1[1024];
  double v0 = 0.0, v1 = 0.0;
  for (int i = threadIdx.x; i < kDotBlocks; i += blockDim.x) {
    v0 += partials[2 * i];
    v1 += partials[2 * i + 1];
  }
  s0[threadIdx.x] = v0;
  s1[threadIdx.x] = v1;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) {
      s0[threadIdx.x] += s0[threadIdx.x + h];
      s1[threadIdx.x] += s1[threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  const double a = s0[0], b = s1[0];
  switch (which) {
    case 0:
      st->rz = a;
      break;
    case 1:
      st->pq = a;
      if (!(a > 0.0)) {
        st->status = AMGDD_ERR_BREAKDOWN;
        st->done = 1;
      } else {
        st->alpha = st->rz / a;
      }
      break;
    case 2:
      st->rr = a;
      st->iters += 1;
      st->relres = st->bnorm2 > 0.0 ? sqrt(a / st->bnorm2) : 0.0;
      if (!(a == a)) {
        st->status = AMGDD_ERR_NONFINITE;
        st->done = 1;
      } else if (a <= st->tol2) {
        st->status = AMGDD_OK;
        st->done = 1;
      } else if (st->iters >= st->max_iter) {
        st->status = AMGDD_ERR_NO_CONVERGENCE;
        st->done = 1;
      }
      break;
    case 3:
      st->rzn = a;
      st->rzo = b;
      st->beta = st->flexible ? (a - b) / st->rz : a / st->rz;
      st->rz = a;
      if (use_cond) cudaGraphSetConditional(cond, 1u);
      break;
    case 4:
      st->bnorm2 = a;
      st->tol2 = st->tol2 * a;
      st->iters = 0;
      st->relres = 1.0;
      st->status = AMGDD_OK;
      st->done = (a == 0.0) ? 1 : 0;
      if (a == 0.0) st->relres = 0.0;
      break;
  }
}

__global__ void k_update_xr(const PcgState* __restrict__ st, double* __restrict__ x, double* __restrict__ r,
                            const double* __restrict__ p, const double* __restrict__ q, int64_t n) {
  if (st->done) return;
  const double al = st->alpha;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    x[i] += al * p[i];
    r[i] -= al * q[i];
  }
}

__global__ void k_update_p(const PcgState* __restrict__ st, double* __restrict__ p, const double* __restrict__ z,
                           double* __restrict__ zold, int64_t n) {
  if (st->done) return;
  const double be = st->beta;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    p[i] = z[i] + be * p[i];
    if (zold != nullptr) zold[i] = z[i];
  }
}

}  // namespace

// ---------------------------------------------------------------------------
int launch_seg(const SegPlan& p, const void* M, bool m_fp32, const void* x, void* y, bool v_fp32, SegMode mode,
               const int* skip, cudaStream_t s, const void* csrc, void* cdst, const void* MT) {
  if (p.rows_mode ? p.ntasks == 0 : p.nchunks == 0) return AMGDD_OK;
  if (m_fp32 != v_fp32) {
    set_error("launch_seg: matrix and vector precision differ");
    return AMGDD_ERR_INTERNAL;
  }
  if (mode == SEG_RESID && csrc == nullptr) {
    set_error("launch_seg: the residual mode needs the right-hand side");
    return AMGDD_ERR_INTERNAL;
  }
  if (m_fp32)
    return seg_dispatch<float>(p, (const float*)M, (const float*)MT, (const float*)x, (float*)y, mode, skip, s,
                               (const float*)csrc, (float*)cdst);
  return seg_dispatch<double>(p, (const double*)M, (const double*)MT, (const double*)x, (double*)y, mode, skip, s,
                              (const double*)csrc, (double*)cdst);
}

int launch_apply(const ApplyPlan& p, const Level& L, bool fp32, const void* x, void* y, int sign, const int* skip,
                 cudaStream_t s) {
  // buckets are ordered by kind: kinds 0-3 run in the narrow kernel, 4-7 in the wide one
  for (int big = 0; big < 2 && p.ntasks > 0; ++big) {
    ApplyArgs a{};
    a.task_grp = p.task_grp.p;
    a.task_row0 = p.task_row0.p;
    a.task_nrow = p.task_nrow.p;
    a.g_ptr = L.d_g_ptr.p;
    a.g_idx = L.d_g_idx.p;
    a.r_off = L.d_h_off.p;
    int task0 = 0, cta = 0;
    a.nbuckets = 0;
    for (int b = 0; b < p.nbuckets; ++b) {
      if ((p.bucket_kind[b] >= 4) == (big == 1)) {
        const int k = a.nbuckets++;
        a.bucket_start[k] = cta;
        a.bucket_kind[k] = p.bucket_kind[b];
        a.bucket_task0[k] = task0;
        a.bucket_tasks[k] = p.bucket_tasks[b];
        cta += p.bucket_start[b + 1] - p.bucket_start[b];
      }
      task0 += p.bucket_tasks[b];
    }
    if (a.nbuckets == 0) continue;
    if (fp32) {
      if (big)
        k_apply<float, true><<<cta, kApplyThreads, 0, s>>>(a, L.d_R32.p, (const float*)x, (float*)y, (float)sign, skip);
      else
        k_apply<float, false><<<cta, kApplyThreads, 0, s>>>(a, L.d_R32.p, (const float*)x, (float*)y, (float)sign,
                                                             skip);
    } else {
      if (big)
        k_apply<double, true><<<cta, kApplyThreads, 0, s>>>(a, L.d_R64.p, (const double*)x, (double*)y,
                                                             (double)sign, skip);
      else
        k_apply<double, false><<<cta, kApplyThreads, 0, s>>>(a, L.d_R64.p, (const double*)x, (double*)y,
                                                              (double)sign, skip);
    }
    AMGDD_CUDA(cudaGetLastError());
    count_kernels(1);
  }
  if (L.t_len > 0) {
    const void* R = fp32 ? (const void*)L.d_R32.p : (const void*)L.d_R64.p;
    void* t = fp32 ? (void*)L.t32.p : (void*)L.t64.p;
    AMGDD_TRY(launch_seg(L.gt1, R, fp32, x, t, fp32, SEG_STORE, skip, s));
    AMGDD_TRY(launch_seg(L.gt2, nullptr, fp32, t, y, fp32, sign > 0 ? SEG_ATOMIC_ADD : SEG_ATOMIC_SUB, skip, s,
                         nullptr, nullptr, R));
  }
  return AMGDD_OK;
}

int launch_cast(const void* src, bool src32, void* dst, bool dst32, int64_t n, const int* skip, cudaStream_t s) {
  if (n == 0) return AMGDD_OK;
  const int g = grid_for(n, 256);
  if (src32 && !dst32)
    k_cast<float, double><<<g, 256, 0, s>>>((const float*)src, (double*)dst, n, skip);
  else if (!src32 && dst32)
    k_cast<double, float><<<g, 256, 0, s>>>((const double*)src, (float*)dst, n, skip);
  else if (src32)
    k_cast<float, float><<<g, 256, 0, s>>>((const float*)src, (float*)dst, n, skip);
  else
    k_cast<double, double><<<g, 256, 0, s>>>((const double*)src, (double*)dst, n, skip);
  AMGDD_CUDA(cudaGetLastError());
  count_kernels(1);
  return AMGDD_OK;
}

int launch_copy_vec(const void* src, void* dst, bool fp32, int64_t n, const int* skip, cudaStream_t s) {
  return launch_cast(src, fp32, dst, fp32, n, skip, s);
}

int launch_dot_partial(const double* a, const double* b, const double* c, int64_t n, double* partials,
                       const int* skip, cudaStream_t s) {
  k_dot_partial<<<kDotBlocks, kDotThreads, 0, s>>>(a, b, c, n, partials, skip);
  AMGDD_CUDA(cudaGetLastError());
  count_kernels(1);
  return AMGDD_OK;
}

int launch_pcg_scalar(int which, PcgState* st, const double* partials, cudaStream_t s,
                      cudaGraphConditionalHandle cond, int use_cond) {
  k_pcg_scalar<<<1, 1024, 0, s>>>(which, st, partials, cond, use_cond);
  AMGDD_CUDA(cudaGetLastError());
  count_kernels(1);
  return AMGDD_OK;
}

int launch_update_xr(PcgState* st, double* x, double* r, const double* p, const double* q, int64_t n,
                     cudaStream_t s) {
  k_update_xr<<<grid_for(n, 256), 256, 0, s>>>(st, x, r, p, q, n);
  AMGDD_CUDA(cudaGetLastError());
  count_kernels(1);
  return AMGDD_OK;
}

int launch_update_p(PcgState* st, double* p, const double* z, double* zold, int64_t n, cudaStream_t s) {
  k_update_p<<<grid_for(n, 256), 256, 0, s>>>(st, p, z, zold, n);
  AMGDD_CUDA(cudaGetLastError());
  count_kernels(1);
  return AMGDD_OK;
}

}  // namespace amgdd
