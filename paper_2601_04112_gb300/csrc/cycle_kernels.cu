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
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>
#include <map>
#include <mutex>
#include <cstdint>

#include "device_util.cuh"
#include "internal.h"

namespace amgdd {

namespace {

constexpr int kSegThreads = 128;

template <class T>
__device__ __forceinline__ void atomic_add(T* p, T v) {
  atomicAdd(p, v);
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

// Matrix entries of type TM against vector entries of type T: V is the
// 16-byte load of W = 16 / sizeof(TM) matrix entries, dot() its product with
// W consecutive entries of x (aligned: x + c W is a multiple of W elements).
// 16-bit matrices (the MIXED16 storage) are widened to FP32 and summed in
// FP32.
template <class T, class TM>
struct MV;
template <>
struct MV<float, float> {
  using V = float4;
  static constexpr int W = 4;
  static __device__ __forceinline__ float dot(const V& m, const float* x) {
    return vdot(m, *reinterpret_cast<const float4*>(x));
  }
};
template <>
struct MV<double, double> {
  using V = double2;
  static constexpr int W = 2;
  static __device__ __forceinline__ double dot(const V& m, const double* x) {
    return vdot(m, *reinterpret_cast<const double2*>(x));
  }
};
template <>
struct MV<float, __half> {
  using V = uint4;
  static constexpr int W = 8;
  static __device__ __forceinline__ float dot(const V& m, const float* x) {
    const float4 a = *reinterpret_cast<const float4*>(x);
    const float4 b = *reinterpret_cast<const float4*>(x + 4);
    const float2 f0 = __half22float2(*reinterpret_cast<const __half2*>(&m.x));
    const float2 f1 = __half22float2(*reinterpret_cast<const __half2*>(&m.y));
    const float2 f2 = __half22float2(*reinterpret_cast<const __half2*>(&m.z));
    const float2 f3 = __half22float2(*reinterpret_cast<const __half2*>(&m.w));
    return f0.x * a.x + f0.y * a.y + f1.x * a.z + f1.y * a.w + f2.x * b.x + f2.y * b.y + f3.x * b.z + f3.y * b.w;
  }
};
template <class T, class TM>
__device__ __forceinline__ T mval(TM v) {
  return T(v);
}
template <>
__device__ __forceinline__ float mval<float, __half>(__half v) {
  return __half2float(v);
}

// VK (vector kind) 0: scalar loads.  VK 1: every row of every block starts on
// a 16-byte boundary and has a multiple of the vector width W entries (checked
// when the plan is built); rows and the staged x are read 16 bytes per lane.
// VK 2 (any rows): a row starting a = (offset mod W) elements past a 16-byte
// boundary is read as aligned vectors from that boundary, against the copy of
// the staged x shifted right by a.  Shared memory then holds W copies of
// stride S = ceil(nc / W) W + W, zero outside the row, so the entries of the
// neighbouring rows that the aligned vectors take in (stored, finite values)
// are multiplied by zero.  A vector that would cross the end of the stored
// matrix (m_len entries) is read element by element up to that end.
// VK 3: every row padded with zeros to a whole number of vectors (row
// stride nc rounded up to W; the MIXED16 copies), read like VK 1 against
// one staged copy of x that is zero past nc.
// U = 4 (plans with long rows only): the gather and the row loop keep four
// independent loads per thread in flight.
template <class T, int VK, int W>
__device__ __forceinline__ void seg_stage(T* xs, int S, int c, T v) {
  if constexpr (VK == 2) {
#pragma unroll
    for (int k = 0; k < W; ++k) xs[k * S + c + k] = v;
  } else {
    xs[c] = v;
  }
}

template <class T, class TM, int L, int MODE, int VK, int U = 1>
__global__ void __launch_bounds__(kSegThreads) k_seg(const SegDesc* __restrict__ desc,
                                                     const int32_t* __restrict__ in_idx,
                                                     const int32_t* __restrict__ out_idx, const TM* __restrict__ M,
                                                     const T* __restrict__ x, T* __restrict__ y, const int* skip,
                                                     const T* __restrict__ csrc, T* __restrict__ cdst, int64_t m_len) {
  pdl_prologue();
  if (skip != nullptr && *skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using V = typename MV<T, TM>::V;
  constexpr int W = MV<T, TM>::W;
  T* xs = reinterpret_cast<T*>(smem_raw);
  const SegDesc dsc = desc[blockIdx.x];  // the chunk's block, in one dependent step
  const int r0 = dsc.r0;
  const int ncb = dsc.nc;
  const int r1 = dsc.r1;
  const int64_t mob = dsc.m_off;
  const int32_t* ii = in_idx + dsc.in_off;
  const int S = VK == 2 ? ((ncb + W - 1) / W) * W + W : 0;
  const int lane = threadIdx.x % L;
  const int grp = threadIdx.x / L;
  const int ngrp = blockDim.x / L;
  // shifted form: the group's first row is requested before the gather, so
  // that its loads overlap the gather's two dependent loads
  const int rf = r0 + grp;
  const int32_t* oo = out_idx + dsc.out_off;
  const bool need_c = MODE == SEG_RESID || cdst != nullptr;
  V pre[U];
  int po = 0;
  T pc = T(0), py = T(0);
  if constexpr (VK == 2) {
#pragma unroll
    for (int u = 0; u < U; ++u) pre[u] = V{};
    if (rf < r1) {
      const int64_t e0 = mob + (int64_t)rf * ncb;
      const int a = (int)(e0 & (W - 1));
      const int64_t base = e0 - a;
      int nv = (ncb + a + W - 1) / W;
      if (base + (int64_t)nv * W > m_len) --nv;
      const V* rv = reinterpret_cast<const V*>(M + base);
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (lane + u * L < nv) pre[u] = rv[lane + u * L];
      if (lane == 0) {
        po = oo[rf];
        if (need_c) pc = csrc[po];
        if (MODE == SEG_ADD) py = y[po];
      }
    }
  }
  if constexpr (VK == 2) {
    const int E = S - ncb;  // zeros per copy: k ahead of the row, E - k after it
    for (int t = threadIdx.x; t < W * E; t += blockDim.x) {
      const int k = t / E, e = t - k * E;
      xs[k * S + (e < k ? e : ncb + e)] = T(0);
    }
  }
  if constexpr (VK == 3) {  // padded rows: the staged x is zero up to the padded length
    for (int c = ncb + (int)threadIdx.x; c < ((ncb + W - 1) / W) * W; c += blockDim.x) xs[c] = T(0);
  }
  if constexpr (U == 1) {
    for (int c = threadIdx.x; c < ncb; c += blockDim.x) seg_stage<T, VK, W>(xs, S, c, x[ii[c]]);
  } else {
    const int step = (int)blockDim.x;
    int c = threadIdx.x;
    for (; c + (U - 1) * step < ncb; c += U * step) {
      int id[U];
#pragma unroll
      for (int u = 0; u < U; ++u) id[u] = ii[c + u * step];
      T v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) v[u] = x[id[u]];
#pragma unroll
      for (int u = 0; u < U; ++u) seg_stage<T, VK, W>(xs, S, c + u * step, v[u]);
    }
    for (; c < ncb; c += step) seg_stage<T, VK, W>(xs, S, c, x[ii[c]]);
  }
  __syncthreads();
  const unsigned mask = group_mask<L>();
  if constexpr (VK == 2) {
    // software pipeline over the group's rows: the next row's first U
    // vectors, output index, copied value and (add mode) old output are
    // requested before the current row is summed
    for (int r = rf; r < r1; r += ngrp) {
      const int64_t e0 = mob + (int64_t)r * ncb;
      const int a = (int)(e0 & (W - 1));
      const int64_t base = e0 - a;
      const V* rv = reinterpret_cast<const V*>(M + base);
      const T* xa = xs + a * S;
      int nv = (ncb + a + W - 1) / W;
      const bool cut = base + (int64_t)nv * W > m_len;  // last row of the matrix: one vector crosses its end
      if (cut) --nv;
      const int rn = r + ngrp;
      V nxt[U];
#pragma unroll
      for (int u = 0; u < U; ++u) nxt[u] = V{};
      int no = 0;
      T nc_ = T(0), ny = T(0);
      if (rn < r1) {
        const int64_t e1 = mob + (int64_t)rn * ncb;
        const int a1 = (int)(e1 & (W - 1));
        const int64_t base1 = e1 - a1;
        int nv1 = (ncb + a1 + W - 1) / W;
        if (base1 + (int64_t)nv1 * W > m_len) --nv1;
        const V* rv1 = reinterpret_cast<const V*>(M + base1);
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (lane + u * L < nv1) nxt[u] = rv1[lane + u * L];
        if (lane == 0) {
          no = oo[rn];
          if (need_c) nc_ = csrc[no];
          if (MODE == SEG_ADD) ny = y[no];
        }
      }
      T acc = T(0);
      if (cut && lane == 0) {
        for (int j = nv * W; base + j < m_len; ++j) acc += mval<T, TM>(M[base + j]) * xa[j];
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (lane + u * L < nv) acc += MV<T, TM>::dot(pre[u], xa + (lane + u * L) * W);
      int c = lane + U * L;
      {
        T q[U];
#pragma unroll
        for (int u = 0; u < U; ++u) q[u] = T(0);
        for (; c + (U - 1) * L < nv; c += U * L) {
          V m[U];
#pragma unroll
          for (int u = 0; u < U; ++u) m[u] = rv[c + u * L];
#pragma unroll
          for (int u = 0; u < U; ++u) q[u] += MV<T, TM>::dot(m[u], xa + (c + u * L) * W);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) acc += q[u];
      }
      for (; c < nv; c += L) acc += MV<T, TM>::dot(rv[c], xa + c * W);
      acc = group_sum<L>(acc, mask);
      if (lane == 0) {
        T* dst = y + po;
        if (MODE == SEG_STORE)
          *dst = acc;
        else if (MODE == SEG_ADD)
          *dst = py + acc;
        else if (MODE == SEG_ATOMIC_ADD)
          atomic_add(dst, acc);
        else if (MODE == SEG_ATOMIC_SUB)
          atomic_add(dst, -acc);
        else
          *dst = pc - acc;
        if (MODE != SEG_RESID && cdst != nullptr) cdst[po] = pc;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) pre[u] = nxt[u];
      po = no;
      pc = nc_;
      py = ny;
    }
  } else {
    for (int r = r0 + grp; r < r1; r += ngrp) {
      T acc = T(0);
      if constexpr (VK != 0) {
        // VK 1: aligned rows of whole vectors; VK 3: rows padded to whole vectors (stride rounded up)
        const int stride = VK == 3 ? ((ncb + W - 1) / W) * W : ncb;
        const V* rv = reinterpret_cast<const V*>(M + mob + (int64_t)r * stride);
        const int nv = stride / W;
        int c = lane;
        if constexpr (U > 1) {
          T a[U];
  #pragma unroll
          for (int u = 0; u < U; ++u) a[u] = T(0);
          for (; c + (U - 1) * L < nv; c += U * L) {
            V m[U];
  #pragma unroll
            for (int u = 0; u < U; ++u) m[u] = rv[c + u * L];
  #pragma unroll
            for (int u = 0; u < U; ++u) a[u] += MV<T, TM>::dot(m[u], xs + (c + u * L) * W);
          }
  #pragma unroll
          for (int u = 0; u < U; ++u) acc += a[u];
        }
        for (; c < nv; c += L) acc += MV<T, TM>::dot(rv[c], xs + c * W);
      } else {
        const TM* row = M + mob + (int64_t)r * ncb;
        int c = lane;
        if constexpr (U > 1) {
          T a[U];
  #pragma unroll
          for (int u = 0; u < U; ++u) a[u] = T(0);
          for (; c + (U - 1) * L < ncb; c += U * L) {
            T m[U];
  #pragma unroll
            for (int u = 0; u < U; ++u) m[u] = mval<T, TM>(row[c + u * L]);
  #pragma unroll
            for (int u = 0; u < U; ++u) a[u] += m[u] * xs[c + u * L];
          }
  #pragma unroll
          for (int u = 0; u < U; ++u) acc += a[u];
        }
        for (; c < ncb; c += L) acc += mval<T, TM>(row[c]) * xs[c];
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
}

// Short rows, row per lane: a task (block, first row, up to L rows) belongs
// to L lanes; lane l owns output row r0 + l and streams column c of the
// block's transposed copy MT (nc x nr, row-major), so the L lanes read L
// consecutive values.  x(in_idx) is staged once per task in shared memory.
// Outputs, atomics and the fused copy are issued by all lanes at once.
template <class T, class TM, int L, int MODE>
__global__ void __launch_bounds__(128) k_seg_rows(const SegDesc* __restrict__ desc, int ntasks, int max_nc,
                                                  const int32_t* __restrict__ in_idx,
                                                  const int32_t* __restrict__ out_idx, const TM* __restrict__ MT,
                                                  const T* __restrict__ x, T* __restrict__ y, const int* skip,
                                                  const T* __restrict__ csrc, T* __restrict__ cdst) {
  pdl_prologue();
  if (skip != nullptr && *skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int grp = (int)threadIdx.x / L;
  const int t = blockIdx.x * (128 / L) + grp;
  if (t >= ntasks) return;
  const int lane = threadIdx.x % L;
  const unsigned mask = group_mask<L>();
  T* xs = reinterpret_cast<T*>(smem_raw) + (size_t)grp * max_nc;
  const SegDesc dsc = desc[t];  // the task's block, in one dependent step
  const int r0 = dsc.r0;
  const int rows = dsc.r1 - dsc.r0;
  const int ncb = dsc.nc, nrb = dsc.nr;
  const int32_t* ii = in_idx + dsc.in_off;
  // the lane's first kPre column entries, its output index and the copied
  // value are requested before the gather, overlapping its dependent loads
  constexpr int kPre = 16;
  const bool act = lane < rows;
  const int r = r0 + lane;
  const TM* col = MT + dsc.m_off + r;
  T pre[kPre];
#pragma unroll
  for (int c = 0; c < kPre; ++c) pre[c] = (act && c < ncb) ? mval<T, TM>(col[(int64_t)c * nrb]) : T(0);
  const int o = act ? out_idx[dsc.out_off + r] : 0;
  const bool need_c = MODE == SEG_RESID || cdst != nullptr;
  const T cv = (act && need_c) ? csrc[o] : T(0);
  for (int c = lane; c < ncb; c += L) xs[c] = x[ii[c]];
  __syncwarp(mask);
  if (!act) return;
  T acc = T(0);
#pragma unroll
  for (int c = 0; c < kPre; ++c)
    if (c < ncb) acc += pre[c] * xs[c];
  for (int c = kPre; c < ncb; ++c) acc += mval<T, TM>(col[(int64_t)c * nrb]) * xs[c];
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
    *dst = cv - acc;
  if (MODE != SEG_RESID && cdst != nullptr) cdst[o] = cv;
}

// FP16 row per lane (MIXED16): lane l of a task owns output rows r0 + 2l and
// r0 + 2l + 1 and reads both at once as one half2 of the transposed FP16
// copy (columns of rows padded to an even count, so every half2 is aligned
// and the padding row is zero), widened to FP32 and summed in FP32.
template <int L, int MODE>
__global__ void __launch_bounds__(128) k_seg_rows16(const SegDesc* __restrict__ desc, int ntasks, int max_nc,
                                                    const int32_t* __restrict__ in_idx,
                                                    const int32_t* __restrict__ out_idx, const __half* __restrict__ MT,
                                                    const float* __restrict__ x, float* __restrict__ y,
                                                    const int* skip, const float* __restrict__ csrc,
                                                    float* __restrict__ cdst) {
  pdl_prologue();
  if (skip != nullptr && *skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int grp = (int)threadIdx.x / L;
  const int t = blockIdx.x * (128 / L) + grp;
  if (t >= ntasks) return;
  const int lane = threadIdx.x % L;
  const unsigned mask = group_mask<L>();
  float* xs = reinterpret_cast<float*>(smem_raw) + (size_t)grp * max_nc;
  const SegDesc dsc = desc[t];
  const int rows = dsc.r1 - dsc.r0;
  const int ncb = dsc.nc;
  const int nrp = (dsc.nr + 1) & ~1;
  const int32_t* ii = in_idx + dsc.in_off;
  const int ra = dsc.r0 + 2 * lane;
  const bool act0 = 2 * lane < rows, act1 = 2 * lane + 1 < rows;
  const __half2* col = reinterpret_cast<const __half2*>(MT + dsc.m_off + ra);
  const int64_t step = nrp / 2;
  constexpr int kPre = 16;
  float2 pre[kPre];
#pragma unroll
  for (int c = 0; c < kPre; ++c)
    pre[c] = (act0 && c < ncb) ? __half22float2(col[(int64_t)c * step]) : make_float2(0.f, 0.f);
  const bool need_c = MODE == SEG_RESID || cdst != nullptr;
  const int o0 = act0 ? out_idx[dsc.out_off + ra] : 0;
  const int o1 = act1 ? out_idx[dsc.out_off + ra + 1] : 0;
  const float cv0 = (act0 && need_c) ? csrc[o0] : 0.f;
  const float cv1 = (act1 && need_c) ? csrc[o1] : 0.f;
  for (int c = lane; c < ncb; c += L) xs[c] = x[ii[c]];
  __syncwarp(mask);
  if (!act0) return;
  float a0 = 0.f, a1 = 0.f;
#pragma unroll
  for (int c = 0; c < kPre; ++c)
    if (c < ncb) {
      a0 += pre[c].x * xs[c];
      a1 += pre[c].y * xs[c];
    }
  for (int c = kPre; c < ncb; ++c) {
    const float2 f = __half22float2(col[(int64_t)c * step]);
    a0 += f.x * xs[c];
    a1 += f.y * xs[c];
  }
  auto out = [&](int o, float acc, float cv) {
    float* dst = y + o;
    if (MODE == SEG_STORE)
      *dst = acc;
    else if (MODE == SEG_ADD)
      *dst += acc;
    else if (MODE == SEG_ATOMIC_ADD)
      atomic_add(dst, acc);
    else if (MODE == SEG_ATOMIC_SUB)
      atomic_add(dst, -acc);
    else
      *dst = cv - acc;
    if (MODE != SEG_RESID && cdst != nullptr) cdst[o] = cv;
  };
  out(o0, a0, cv0);
  if (act1) out(o1, a1, cv1);
}

// ---------------------------------------------------------------------------
// Staged gather-GEMV-scatter.  One item (a contiguous range of the stored
// matrix: consecutive whole blocks, or a row slice of one block) is moved to
// shared memory by a single bulk copy completing on an mbarrier, while the
// CTA gathers the item's inputs x(in_idx) with independent loads; rows are
// then computed from shared memory by groups of L lanes.

constexpr long long kWaitCycles = 2000000000LL;  // about 1 s at 2 GHz
constexpr int kItemThreads = 128;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// one bulk copy global -> shared of `bytes` (16-byte aligned addresses and
// size), completing the current phase of `bar`
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// bounded wait for phase `parity` of `bar`, backing off between polls so
// that a waiting warp takes few issue slots; false on timeout.  One thread
// waits and the CTA then meets at a barrier, which orders the copied data
// before every thread's reads.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
  const long long t0 = clock64();
  unsigned ns = 32;
  for (;;) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > kWaitCycles) return false;
    __nanosleep(ns);
    ns = ns < 256 ? 2 * ns : 256;
  }
}

// Shared memory of the staged kernels: mbarrier (16 bytes), tables (132
// ints), gathered inputs xs, per-row operand values cs (residual source or
// previous output) and cc (copied source), output indices os, then the
// staged matrix.
constexpr int kTabInts = 132;
__host__ __device__ constexpr size_t a16(size_t b) { return (b + 15) / 16 * 16; }
__host__ __device__ constexpr size_t staged_bytes(int max_in, int max_rows, int max_m, size_t esz) {
  return 16 + (size_t)kTabInts * 4 + a16((size_t)max_in * esz) + 2 * a16((size_t)max_rows * esz) +
         a16((size_t)max_rows * 4) + a16((size_t)max_m * esz);
}

// Processes item `it` of a staged phase.  `use` counts completed phases of
// `bar`.  Returns false after an expired wait (err set, copy waited for).
template <class T, int L>
__device__ bool item_run(const PhaseDesc& P, int it, unsigned char* smem, uint64_t* bar, unsigned& use, int* err) {
  constexpr int V = 16 / sizeof(T);
  using VT = typename Vec2<T>::type;
  int* tab = reinterpret_cast<int*>(smem + 16);
  T* xs = reinterpret_cast<T*>(smem + 16 + kTabInts * 4);
  T* cs = reinterpret_cast<T*>(reinterpret_cast<unsigned char*>(xs) + a16((size_t)P.max_in * sizeof(T)));
  T* cc = reinterpret_cast<T*>(reinterpret_cast<unsigned char*>(cs) + a16((size_t)P.max_rows * sizeof(T)));
  int* os = reinterpret_cast<int*>(reinterpret_cast<unsigned char*>(cc) + a16((size_t)P.max_rows * sizeof(T)));
  T* Ms = reinterpret_cast<T*>(reinterpret_cast<unsigned char*>(os) + a16((size_t)P.max_rows * 4));
  const ItemDesc d = P.items[it];
  const int64_t a0 = d.m_start & ~(int64_t)(V - 1);
  const int64_t a1 = (d.m_start + d.m_len + V - 1) & ~(int64_t)(V - 1);
  const int delta = (int)(d.m_start - a0);
  if (threadIdx.x == 0) bulk_load(Ms, (const T*)P.M + a0, (unsigned)((a1 - a0) * sizeof(T)), bar);
  const int ntab = 4 * d.nb + 3;
  for (int t = threadIdx.x; t < ntab; t += kItemThreads) tab[t] = P.tabs[d.tab + t];
  // inputs and per-row operands: all index loads, then all value loads
  {
    const T* x = (const T*)P.x;
    const bool need_c = P.mode == SEG_RESID || P.mode == SEG_ADD;
    const T* csrc = P.mode == SEG_ADD ? (const T*)P.y : (const T*)P.csrc;
    constexpr int U = 8;
    for (int base = 0; base < d.nin || base < d.nrows; base += U * kItemThreads) {
      int ix[U], io[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int c = base + u * kItemThreads + (int)threadIdx.x;
        ix[u] = c < d.nin ? P.gidx[d.xin + c] : -1;
        io[u] = c < d.nrows ? P.gout[d.out + c] : -1;
      }
      T xv[U], cv[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        xv[u] = ix[u] >= 0 ? __ldcg(x + ix[u]) : T(0);
        cv[u] = (need_c && io[u] >= 0) ? __ldcg(csrc + io[u]) : T(0);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int c = base + u * kItemThreads + (int)threadIdx.x;
        if (c < d.nin) xs[c] = xv[u];
        if (c < d.nrows) {
          os[c] = io[u];
          cs[c] = cv[u];
        }
      }
    }
    // the fused copy cdst = csrc (level-0 residual source) is rare: own loop
    if (P.cdst != nullptr && P.mode != SEG_RESID) {
      __syncthreads();
      for (int c = threadIdx.x; c < d.nrows; c += kItemThreads) cc[c] = __ldcg((const T*)P.csrc + os[c]);
    }
  }
  const bool ok = threadIdx.x != 0 || mbar_wait(bar, use & 1u);
  ++use;
  if (__syncthreads_or(!ok)) {
    if (threadIdx.x == 0) {
      atomicExch(err, 2);
      (void)mbar_wait(bar, (use - 1) & 1u);
    }
    return false;
  }
  // rows: group g of L lanes takes rows g, g + ngrp, ...
  const int nb = d.nb;
  const int* rp = tab;
  const int* mp = tab + nb + 1;
  const int* ip = mp + nb + 1;
  const int* ncs = ip + nb + 1;
  const int lane = (int)threadIdx.x % L;
  constexpr int ngrp = kItemThreads / L;
  const unsigned mask = group_mask<L>();
  T* y = (T*)P.y;
  int j = 0;
  for (int q = (int)threadIdx.x / L; q < d.nrows; q += ngrp) {
    while (rp[j + 1] <= q) ++j;
    const int rl = q - rp[j];
    const int ncb = ncs[j];
    const int moff = delta + mp[j] + rl * ncb;
    const T* row = Ms + moff;
    const T* xb = xs + ip[j];
    T acc = T(0);
    if (((moff | ip[j] | ncb) & (V - 1)) == 0) {
      const VT* rv = reinterpret_cast<const VT*>(row);
      const VT* xv = reinterpret_cast<const VT*>(xb);
      const int nv = ncb / V;
      for (int c = lane; c < nv; c += L) acc += vdot(rv[c], xv[c]);
    } else {
      for (int c = lane; c < ncb; c += L) acc += row[c] * xb[c];
    }
    acc = group_sum<L>(acc, mask);
    if (lane == 0) {
      const int o = os[q];
      switch (P.mode) {
        case SEG_STORE: y[o] = acc; break;
        case SEG_ADD: y[o] = cs[q] + acc; break;
        case SEG_ATOMIC_ADD: atomicAdd(y + o, acc); break;
        case SEG_ATOMIC_SUB: atomicAdd(y + o, -acc); break;
        default: y[o] = cs[q] - acc; break;
      }
      if (P.cdst != nullptr && P.mode != SEG_RESID) ((T*)P.cdst)[o] = cc[q];
    }
  }
  __syncthreads();
  return true;
}

template <class T, int L>
__global__ void __launch_bounds__(kItemThreads) k_seg_staged(const __grid_constant__ PhaseDesc P, const int* skip,
                                                             int* err) {
  pdl_prologue();
  if (skip != nullptr && *skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  if (threadIdx.x == 0) mbar_init(bar);
  __syncthreads();
  unsigned use = 0;
  (void)item_run<T, L>(P, blockIdx.x, smem_raw, bar, use, err);
}

template <class T, class TM, int L, int MODE>
int seg_rows_launch(const SegPlan& p, const TM* MT, const T* x, T* y, const int* skip, cudaStream_t s, const T* csrc,
                    T* cdst) {
  const int per = 128 / L;
  const int grid = (p.ntasks + per - 1) / per;
  const size_t smem = (size_t)per * p.max_nc * sizeof(T);
  auto kern = k_seg_rows<T, TM, L, MODE>;
  if (smem > 48 * 1024) AMGDD_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  AMGDD_CUDA(launch_k(g_pdl, kern, grid, 128, smem, s, (const SegDesc*)p.task_desc.p, p.ntasks, p.max_nc,
                      p.in_idx_ext, p.out_idx_ext, MT, x, y, skip, csrc, cdst));
  AMGDD_CUDA(cudaGetLastError());
  count_kernels(1);
  return AMGDD_OK;
}

template <class T, class TM, int L>
int seg_rows_mode(const SegPlan& p, const TM* MT, const T* x, T* y, SegMode mode, const int* skip, cudaStream_t s,
                  const T* csrc, T* cdst) {
  switch (mode) {
    case SEG_STORE: return seg_rows_launch<T, TM, L, SEG_STORE>(p, MT, x, y, skip, s, csrc, cdst);
    case SEG_ADD: return seg_rows_launch<T, TM, L, SEG_ADD>(p, MT, x, y, skip, s, csrc, cdst);
    case SEG_ATOMIC_ADD: return seg_rows_launch<T, TM, L, SEG_ATOMIC_ADD>(p, MT, x, y, skip, s, csrc, cdst);
    case SEG_ATOMIC_SUB: return seg_rows_launch<T, TM, L, SEG_ATOMIC_SUB>(p, MT, x, y, skip, s, csrc, cdst);
    default: return seg_rows_launch<T, TM, L, SEG_RESID>(p, MT, x, y, skip, s, csrc, cdst);
  }
}

template <class T, class TM, int L, int VK, int U>
int seg_launch_kind(const SegPlan& p, const TM* M, const T* x, T* y, SegMode mode, const int* skip, cudaStream_t s,
                    const T* csrc, T* cdst, size_t smem) {
  auto launch = [&](auto kern) -> int {
    if (smem > 48 * 1024) AMGDD_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    AMGDD_CUDA(launch_k(g_pdl, kern, p.nchunks, kSegThreads, smem, s, (const SegDesc*)p.chunk_desc.p,
                        p.in_idx_ext, p.out_idx_ext, M, x, y, skip, csrc, cdst, p.mat_len));
    AMGDD_CUDA(cudaGetLastError());
    count_kernels(1);
    return AMGDD_OK;
  };
  switch (mode) {
    case SEG_STORE: return launch(k_seg<T, TM, L, SEG_STORE, VK, U>);
    case SEG_ADD: return launch(k_seg<T, TM, L, SEG_ADD, VK, U>);
    case SEG_ATOMIC_ADD: return launch(k_seg<T, TM, L, SEG_ATOMIC_ADD, VK, U>);
    case SEG_ATOMIC_SUB: return launch(k_seg<T, TM, L, SEG_ATOMIC_SUB, VK, U>);
    default: return launch(k_seg<T, TM, L, SEG_RESID, VK, U>);
  }
}

// Shared memory of the shifted-vector form (W copies of the staged input).
template <class T, class TM>
size_t seg_shift_smem(const SegPlan& p) {
  constexpr int W = MV<T, TM>::W;
  return (size_t)W * (size_t)(((p.max_nc + W - 1) / W) * W + W) * sizeof(T);
}

template <class T, int L>
int seg_dispatch_mode(const SegPlan& p, const T* M, const T* x, T* y, SegMode mode, const int* skip,
                      cudaStream_t s, const T* csrc, T* cdst) {
  const size_t smem = (size_t)p.max_nc * sizeof(T);
  // the shifted form (always with the 4-way unrolled gather and row loops)
  // needs a 16-byte aligned base (device allocations are)
  if ((sizeof(T) == 4 ? p.shift : p.shift64) && !p.vec && ((uintptr_t)M & 15) == 0)
    return seg_launch_kind<T, T, L, 2, 4>(p, M, x, y, mode, skip, s, csrc, cdst, seg_shift_smem<T, T>(p));
  if constexpr (L == 32) {
    if (p.unroll)
      return p.vec ? seg_launch_kind<T, T, L, 1, 4>(p, M, x, y, mode, skip, s, csrc, cdst, smem)
                   : seg_launch_kind<T, T, L, 0, 4>(p, M, x, y, mode, skip, s, csrc, cdst, smem);
  }
  return p.vec ? seg_launch_kind<T, T, L, 1, 1>(p, M, x, y, mode, skip, s, csrc, cdst, smem)
               : seg_launch_kind<T, T, L, 0, 1>(p, M, x, y, mode, skip, s, csrc, cdst, smem);
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
      case 8: return seg_rows_mode<T, T, 8>(p, MT, x, y, mode, skip, s, csrc, cdst);
      case 16: return seg_rows_mode<T, T, 16>(p, MT, x, y, mode, skip, s, csrc, cdst);
      default: return seg_rows_mode<T, T, 32>(p, MT, x, y, mode, skip, s, csrc, cdst);
    }
  }
  switch (p.lanes) {
    case 4: return seg_dispatch_mode<T, 4>(p, M, x, y, mode, skip, s, csrc, cdst);
    case 8: return seg_dispatch_mode<T, 8>(p, M, x, y, mode, skip, s, csrc, cdst);
    case 16: return seg_dispatch_mode<T, 16>(p, M, x, y, mode, skip, s, csrc, cdst);
    default: return seg_dispatch_mode<T, 32>(p, M, x, y, mode, skip, s, csrc, cdst);
  }
}

// FP16 matrices (MIXED16 storage) against FP32 vectors: rows padded to
// whole 16-byte vectors (VK 3), one staged copy of x.
template <int L>
int seg16_lanes(const SegPlan& p, const float* x, float* y, SegMode mode, const int* skip, cudaStream_t s,
                const float* csrc, float* cdst) {
  constexpr int W = MV<float, __half>::W;
  const size_t smem = (size_t)((p.max_nc + W - 1) / W) * W * sizeof(float);
  auto launch = [&](auto kern) -> int {
    if (smem > 48 * 1024) AMGDD_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    AMGDD_CUDA(launch_k(g_pdl, kern, p.nchunks, kSegThreads, smem, s, (const SegDesc*)p.chunk_desc16.p,
                        p.in_idx_ext, p.out_idx_ext, (const __half*)p.m16.p, x, y, skip, csrc, cdst, p.mat_len16));
    AMGDD_CUDA(cudaGetLastError());
    count_kernels(1);
    return AMGDD_OK;
  };
  switch (mode) {
    case SEG_STORE: return launch(k_seg<float, __half, L, SEG_STORE, 3, 4>);
    case SEG_ADD: return launch(k_seg<float, __half, L, SEG_ADD, 3, 4>);
    case SEG_ATOMIC_ADD: return launch(k_seg<float, __half, L, SEG_ATOMIC_ADD, 3, 4>);
    case SEG_ATOMIC_SUB: return launch(k_seg<float, __half, L, SEG_ATOMIC_SUB, 3, 4>);
    default: return launch(k_seg<float, __half, L, SEG_RESID, 3, 4>);
  }
}

// ---------------------------------------------------------------------------
// Dense GEMV y = B x (the dense V-cycle tail).  S warps share a row (each
// takes every S-th run of 32 vectors), 8 / S rows per CTA of 256 threads;
// rows and x are read as 16-byte vectors straight from global memory (x is
// small and stays in L1/L2), four vectors per lane in flight, and the n mod
// W last columns element by element, so x is never read past n.  The S
// partial sums of a row meet in shared memory in a fixed order.
template <class T, int S>
__global__ void __launch_bounds__(256) k_dense(const T* __restrict__ B, int64_t ld, int n, const T* __restrict__ x,
                                               T* __restrict__ y, const int* skip) {
  pdl_prologue();
  if (skip != nullptr && *skip) return;
  using V = typename Vec2<T>::type;
  constexpr int W = Vec2<T>::width;
  constexpr int U = 4;
  __shared__ T part[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r = blockIdx.x * (8 / S) + warp / S;
  const int sub = warp % S;
  const int nv = n / W;
  T acc = T(0);
  if (r < n) {
    const T* row = B + (int64_t)r * ld;
    const V* rv = reinterpret_cast<const V*>(row);
    const V* xv = reinterpret_cast<const V*>(x);
    T a[U];
#pragma unroll
    for (int u = 0; u < U; ++u) a[u] = T(0);
    int c = sub * 32 + lane;
    for (; c + (U - 1) * 32 * S < nv; c += U * 32 * S) {
      V m[U], v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        m[u] = rv[c + u * 32 * S];
        v[u] = xv[c + u * 32 * S];
      }
#pragma unroll
      for (int u = 0; u < U; ++u) a[u] += vdot(m[u], v[u]);
    }
    acc = (a[0] + a[1]) + (a[2] + a[3]);
    for (; c < nv; c += 32 * S) acc += vdot(rv[c], xv[c]);
    if (sub == 0)
      for (int j = nv * W + lane; j < n; j += 32) acc += row[j] * x[j];
    acc = group_sum<32>(acc, 0xffffffffu);
  }
  if constexpr (S == 1) {
    if (r < n && lane == 0) y[r] = acc;
  } else {
    if (lane == 0) part[warp] = acc;
    __syncthreads();
    if (r < n && sub == 0 && lane == 0) {
      T t = part[warp];
#pragma unroll
      for (int k = 1; k < S; ++k) t += part[warp + k];
      y[r] = t;
    }
  }
}

// ---------------------------------------------------------------------------
// Deterministic RAS-T, second half: x_j += sum of the stored y entries of
// node j, in ascending position order (one thread per node and column).
template <class T, int K>
__global__ void __launch_bounds__(256) k_gather_add(const int64_t* __restrict__ ptr, const int32_t* __restrict__ pos,
                                                    const T* __restrict__ Y, T* __restrict__ x, int64_t n,
                                                    const int* skip) {
  pdl_prologue();
  if (skip != nullptr && *skip) return;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n * K) return;
  const int64_t j = t / K;
  const int k = (int)(t - j * K);
  T acc = T(0);
  for (int64_t q = ptr[j]; q < ptr[j + 1]; ++q) acc += Y[(int64_t)pos[q] * K + k];
  x[t] += acc;
}

// ---------------------------------------------------------------------------
// A-apply by rows in ELL form (level 0): one thread per row, the slots'
// column indices and values requested eight at a time before the gathered
// x entries; y = A x, or y = c - A x (residual).
template <class T, bool RESID>
__global__ void __launch_bounds__(256) k_ell(const T* __restrict__ val, const int32_t* __restrict__ col, int w,
                                             int64_t n, const T* __restrict__ x, T* __restrict__ y,
                                             const T* __restrict__ c, const int* skip) {
  pdl_prologue();
  if (skip != nullptr && *skip) return;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const T cv = RESID ? c[i] : T(0);
  T acc = T(0);
  int k = 0;
  for (; k + 8 <= w; k += 8) {
    int ci[8];
    T v[8], xv[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      ci[u] = col[(int64_t)(k + u) * n + i];
      v[u] = val[(int64_t)(k + u) * n + i];
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) xv[u] = x[ci[u]];
#pragma unroll
    for (int u = 0; u < 8; ++u) acc += v[u] * xv[u];
  }
  for (; k < w; ++k) acc += val[(int64_t)k * n + i] * x[col[(int64_t)k * n + i]];
  y[i] = RESID ? cv - acc : acc;
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
  pdl_prologue();
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
  pdl_prologue();
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


__global__ void __launch_bounds__(kDotThreads) k_dot_partial(const double* __restrict__ a, const double* __restrict__ b,
                                                             const double* __restrict__ c, int64_t n,
                                                             double* __restrict__ partials, const int* skip) {
  pdl_prologue();
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
// The scalar step `which` given the two reduced sums a, b (thread 0 only).
__device__ void pcg_scalar_step(int which, PcgState* st, double a, double b, cudaGraphConditionalHandle cond,
                                int use_cond) {
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
      } else if (st->flexible && st->iters % 10 == 0) {
        // FP32-cycle stall guard: ||r|| must fall by 10% every 10 iterations
        if (a > 0.81 * st->rr_mark) {
          st->status = kStallStatus;
          st->done = 1;
        } else {
          st->rr_mark = a;
        }
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
      st->rr_mark = a;
      st->tol2 = st->tol2 * a;
      st->iters = 0;
      st->relres = 1.0;
      st->status = AMGDD_OK;
      st->done = (a == 0.0) ? 1 : 0;
      if (a == 0.0) st->relres = 0.0;
      break;
  }
}

__global__ void __launch_bounds__(1024) k_pcg_scalar(int which, PcgState* st, const double* __restrict__ partials,
                                                     cudaGraphConditionalHandle cond, int use_cond) {
  pdl_prologue();
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
  pcg_scalar_step(which, st, s0[0], s1[0], cond, use_cond);
}

// Fused CG kernels: kDotBlocks CTAs of kDotThreads.  Each CTA writes its
// partial sums (s0, s1); the last CTA to finish (device-scope ticket) sums
// all partials in a fixed order, runs the scalar step and resets the ticket.
// The result does not depend on which CTA finishes last.
__device__ void cg_finish(double s0, double s1, double* partials, PcgState* st, int which,
                          cudaGraphConditionalHandle cond, int use_cond) {
  __shared__ double sh0[kDotThreads / 32], sh1[kDotThreads / 32];
  __shared__ int last;
  s0 = warp_sum_d(s0);
  s1 = warp_sum_d(s1);
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    sh0[w] = s0;
    sh1[w] = s1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double v0 = 0.0, v1 = 0.0;
    for (int k = 0; k < kDotThreads / 32; ++k) {
      v0 += sh0[k];
      v1 += sh1[k];
    }
    partials[2 * blockIdx.x] = v0;
    partials[2 * blockIdx.x + 1] = v1;
    __threadfence();
    last = atomicAdd(&st->ticket, 1u) == gridDim.x - 1 ? 1 : 0;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double v0 = 0.0, v1 = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
    v0 += __ldcg(partials + 2 * i);
    v1 += __ldcg(partials + 2 * i + 1);
  }
  v0 = warp_sum_d(v0);
  v1 = warp_sum_d(v1);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) {
    sh0[w] = v0;
    sh1[w] = v1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int k = 0; k < kDotThreads / 32; ++k) {
      a += sh0[k];
      b += sh1[k];
    }
    st->ticket = 0u;
    pcg_scalar_step(which, st, a, b, cond, use_cond);
  }
}

// q = A p over level 0's ELL rows; p.q; alpha
__global__ void __launch_bounds__(kDotThreads) k_cg_ap(const double* __restrict__ val, const int32_t* __restrict__ col,
                                                       int w, int64_t n, const double* __restrict__ p,
                                                       double* __restrict__ q, double* partials, PcgState* st) {
  pdl_prologue();
  if (st->done) return;
  double s0 = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    int k = 0;
    for (; k + 8 <= w; k += 8) {
      int ci[8];
      double v[8], xv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        ci[u] = col[(int64_t)(k + u) * n + i];
        v[u] = val[(int64_t)(k + u) * n + i];
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) xv[u] = p[ci[u]];
#pragma unroll
      for (int u = 0; u < 8; ++u) acc += v[u] * xv[u];
    }
    for (; k < w; ++k) acc += val[(int64_t)k * n + i] * p[col[(int64_t)k * n + i]];
    q[i] = acc;
    s0 += p[i] * acc;
  }
  cg_finish(s0, 0.0, partials, st, 1, 0, 0);
}

// x += alpha p, r -= alpha q (r32 = r when given); r.r; convergence
__global__ void __launch_bounds__(kDotThreads) k_cg_xr(double* __restrict__ x, double* __restrict__ r,
                                                       float* __restrict__ r32, const double* __restrict__ p,
                                                       const double* __restrict__ q, int64_t n, double* partials,
                                                       PcgState* st) {
  pdl_prologue();
  if (st->done) return;
  const double al = st->alpha;
  double s0 = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    x[i] += al * p[i];
    const double ri = r[i] - al * q[i];
    r[i] = ri;
    if (r32 != nullptr) r32[i] = (float)ri;
    s0 += ri * ri;
  }
  cg_finish(s0, 0.0, partials, st, 2, 0, 0);
}

// z = x32 when given; r.z and r.z_old; beta; graph condition
__global__ void __launch_bounds__(kDotThreads) k_cg_zdot(const float* __restrict__ x32, double* __restrict__ z,
                                                         const double* __restrict__ r,
                                                         const double* __restrict__ zold, int64_t n, double* partials,
                                                         PcgState* st, cudaGraphConditionalHandle cond, int use_cond) {
  pdl_prologue();
  if (st->done) {
    if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(cond, 0u);
    return;
  }
  double s0 = 0.0, s1 = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double zi;
    if (x32 != nullptr) {
      zi = (double)x32[i];
      z[i] = zi;
    } else {
      zi = z[i];
    }
    const double ri = r[i];
    s0 += ri * zi;
    if (zold != nullptr) s1 += ri * zold[i];
  }
  cg_finish(s0, s1, partials, st, 3, cond, use_cond);
}

__global__ void k_update_xr(const PcgState* __restrict__ st, double* __restrict__ x, double* __restrict__ r,
                            const double* __restrict__ p, const double* __restrict__ q, int64_t n) {
  pdl_prologue();
  if (st->done) return;
  const double al = st->alpha;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    x[i] += al * p[i];
    r[i] -= al * q[i];
  }
}

__global__ void k_update_p(const PcgState* __restrict__ st, double* __restrict__ p, const double* __restrict__ z,
                           double* __restrict__ zold, int64_t n) {
  pdl_prologue();
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
  // the staged kernel streams M itself; callers that pass only the
  // transposed copy (row-per-lane plans) keep the unstaged kernels
  if (p.staged && g_err_word != nullptr && M != nullptr) {
    const PhaseDesc d = seg_phase(p, M, MT, m_fp32, x, y, mode, csrc, cdst);
    const size_t smem = phase_smem(d);
    auto go = [&](auto kern) -> int {
      if (smem > 48 * 1024)
        AMGDD_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      AMGDD_CUDA(launch_k(g_pdl, kern, p.nitems, kItemThreads, smem, s, d, skip, g_err_word));
      AMGDD_CUDA(cudaGetLastError());
      count_kernels(1);
      return AMGDD_OK;
    };
    if (m_fp32) {
      switch (p.item_lanes) {
        case 4: return go(k_seg_staged<float, 4>);
        case 8: return go(k_seg_staged<float, 8>);
        case 16: return go(k_seg_staged<float, 16>);
        default: return go(k_seg_staged<float, 32>);
      }
    }
    switch (p.item_lanes) {
      case 4: return go(k_seg_staged<double, 4>);
      case 8: return go(k_seg_staged<double, 8>);
      case 16: return go(k_seg_staged<double, 16>);
      default: return go(k_seg_staged<double, 32>);
    }
  }
  if (m_fp32)
    return seg_dispatch<float>(p, (const float*)M, (const float*)MT, (const float*)x, (float*)y, mode, skip, s,
                               (const float*)csrc, (float*)cdst);
  return seg_dispatch<double>(p, (const double*)M, (const double*)MT, (const double*)x, (double*)y, mode, skip, s,
                              (const double*)csrc, (double*)cdst);
}

int launch_seg16(const SegPlan& p, const float* x, float* y, SegMode mode, const int* skip, cudaStream_t s,
                 const float* csrc, float* cdst) {
  if (mode == SEG_RESID && csrc == nullptr) {
    set_error("launch_seg16: the residual mode needs the right-hand side");
    return AMGDD_ERR_INTERNAL;
  }
  if (p.lanes16 > 0 && p.nchunks == 0) return AMGDD_OK;
  if (p.lanes16 > 0 && (p.m16.p == nullptr || p.chunk_desc16.p == nullptr)) {
    set_error("launch_seg16: the plan has no FP16 copy");
    return AMGDD_ERR_INTERNAL;
  }
  if (p.lanes16 < 0) {  // row per lane, -lanes16 lanes per task of up to 2 (-lanes16) rows
    if (p.mt16.p == nullptr || p.task_desc16.p == nullptr || p.ntasks16 == 0) {
      set_error("launch_seg16: the plan has no FP16 row-per-lane form");
      return AMGDD_ERR_INTERNAL;
    }
    auto go = [&](auto kern, int L) -> int {
      const int per = 128 / L;
      const size_t smem = (size_t)per * p.max_nc * sizeof(float);
      if (smem > 48 * 1024)
        AMGDD_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      AMGDD_CUDA(launch_k(g_pdl, kern, (p.ntasks16 + per - 1) / per, 128, smem, s,
                          (const SegDesc*)p.task_desc16.p, p.ntasks16, p.max_nc, p.in_idx_ext, p.out_idx_ext,
                          (const __half*)p.mt16.p, x, y, skip, csrc, cdst));
      AMGDD_CUDA(cudaGetLastError());
      count_kernels(1);
      return AMGDD_OK;
    };
    auto modes = [&](auto tag) -> int {
      constexpr int L = decltype(tag)::value;
      switch (mode) {
        case SEG_STORE: return go(k_seg_rows16<L, SEG_STORE>, L);
        case SEG_ADD: return go(k_seg_rows16<L, SEG_ADD>, L);
        case SEG_ATOMIC_ADD: return go(k_seg_rows16<L, SEG_ATOMIC_ADD>, L);
        case SEG_ATOMIC_SUB: return go(k_seg_rows16<L, SEG_ATOMIC_SUB>, L);
        default: return go(k_seg_rows16<L, SEG_RESID>, L);
      }
    };
    switch (-p.lanes16) {
      case 8: return modes(std::integral_constant<int, 8>{});
      case 16: return modes(std::integral_constant<int, 16>{});
      default: return modes(std::integral_constant<int, 32>{});
    }
  }
  switch (p.lanes16) {
    case 4: return seg16_lanes<4>(p, x, y, mode, skip, s, csrc, cdst);
    case 8: return seg16_lanes<8>(p, x, y, mode, skip, s, csrc, cdst);
    case 16: return seg16_lanes<16>(p, x, y, mode, skip, s, csrc, cdst);
    default: return seg16_lanes<32>(p, x, y, mode, skip, s, csrc, cdst);
  }
}

__global__ void k_pad16(const float* __restrict__ M32, const int64_t* __restrict__ m_off,
                        const int32_t* __restrict__ nr, const int32_t* __restrict__ nc,
                        const int64_t* __restrict__ m_off16, __half* __restrict__ dst) {
  const int b = blockIdx.x;
  const int r_n = nr[b], c_n = nc[b], cp = (c_n + 7) / 8 * 8;
  const float* src = M32 + m_off[b];
  __half* d = dst + m_off16[b];
  for (int64_t e = threadIdx.x; e < (int64_t)r_n * cp; e += blockDim.x) {
    const int r = (int)(e / cp), c = (int)(e % cp);
    d[e] = c < c_n ? __float2half_rn(src[(int64_t)r * c_n + c]) : __float2half_rn(0.0f);
  }
}

__global__ void k_pad16t(const float* __restrict__ MT32, const int64_t* __restrict__ m_off,
                         const int32_t* __restrict__ nr, const int32_t* __restrict__ nc,
                         const int64_t* __restrict__ m_off16, __half* __restrict__ dst) {
  const int b = blockIdx.x;
  const int r_n = nr[b], c_n = nc[b], rp = (r_n + 1) & ~1;
  const float* src = MT32 + m_off[b];
  __half* d = dst + m_off16[b];
  for (int64_t e = threadIdx.x; e < (int64_t)c_n * rp; e += blockDim.x) {
    const int c = (int)(e / rp), r = (int)(e % rp);
    d[e] = r < r_n ? __float2half_rn(src[(int64_t)c * r_n + r]) : __float2half_rn(0.0f);
  }
}

int launch_pad16t(const float* MT32, const int64_t* m_off, const int32_t* nr, const int32_t* nc,
                  const int64_t* m_off16, int nblocks, __half* dst, cudaStream_t s) {
  if (nblocks == 0) return AMGDD_OK;
  k_pad16t<<<nblocks, 128, 0, s>>>(MT32, m_off, nr, nc, m_off16, dst);
  AMGDD_CUDA(cudaGetLastError());
  count_kernels(1);
  return AMGDD_OK;
}

int launch_pad16(const float* M32, const int64_t* m_off, const int32_t* nr, const int32_t* nc,
                 const int64_t* m_off16, int nblocks, __half* dst, cudaStream_t s) {
  if (nblocks == 0) return AMGDD_OK;
  k_pad16<<<nblocks, 128, 0, s>>>(M32, m_off, nr, nc, m_off16, dst);
  AMGDD_CUDA(cudaGetLastError());
  count_kernels(1);
  return AMGDD_OK;
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
        AMGDD_CUDA(launch_k(g_pdl, k_apply<float, true>, cta, kApplyThreads, 0, s, a, L.d_R32.p, (const float*)x, (float*)y, (float)sign, skip));
      else
        AMGDD_CUDA(launch_k(g_pdl, k_apply<float, false>, cta, kApplyThreads, 0, s, a, L.d_R32.p, (const float*)x, (float*)y, (float)sign,
                                                             skip));
    } else {
      if (big)
        AMGDD_CUDA(launch_k(g_pdl, k_apply<double, true>, cta, kApplyThreads, 0, s, a, L.d_R64.p, (const double*)x, (double*)y,
                                                             (double)sign, skip));
      else
        AMGDD_CUDA(launch_k(g_pdl, k_apply<double, false>, cta, kApplyThreads, 0, s, a, L.d_R64.p, (const double*)x, (double*)y,
                                                              (double)sign, skip));
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

int launch_gather_add(const int64_t* ptr, const int32_t* pos, const void* Y, void* x, int64_t n, int K, bool fp32,
                      const int* skip, cudaStream_t s) {
  if (n <= 0) return AMGDD_OK;
  const int grid = (int)((n * K + 255) / 256);
  auto go = [&](auto kf, auto kd) -> int {
    if (fp32)
      AMGDD_CUDA(launch_k(g_pdl, kf, grid, 256, 0, s, ptr, pos, (const float*)Y, (float*)x, n, skip));
    else
      AMGDD_CUDA(launch_k(g_pdl, kd, grid, 256, 0, s, ptr, pos, (const double*)Y, (double*)x, n, skip));
    count_kernels(1);
    return AMGDD_OK;
  };
  switch (K) {
    case 1: return go(k_gather_add<float, 1>, k_gather_add<double, 1>);
    case 2: return go(k_gather_add<float, 2>, k_gather_add<double, 2>);
    case 4: return go(k_gather_add<float, 4>, k_gather_add<double, 4>);
    case 8: return go(k_gather_add<float, 8>, k_gather_add<double, 8>);
    case 16: return go(k_gather_add<float, 16>, k_gather_add<double, 16>);
    case 32: return go(k_gather_add<float, 32>, k_gather_add<double, 32>);
    default:
      set_error("launch_gather_add: K must be 1, 2, 4, 8, 16 or 32");
      return AMGDD_ERR_INVALID_ARG;
  }
}

int launch_ell(const Level& L, bool fp32, const void* x, void* y, const void* csrc, const int* skip,
               cudaStream_t s) {
  if (L.n <= 0) return AMGDD_OK;
  const int grid = (int)((L.n + 255) / 256);
  const bool res = csrc != nullptr;
  if (fp32) {
    if (res)
      AMGDD_CUDA(launch_k(g_pdl, k_ell<float, true>, grid, 256, 0, s, (const float*)L.ell32.p, (const int32_t*)L.ellc.p,
                          L.ell_w, L.n, (const float*)x, (float*)y, (const float*)csrc, skip));
    else
      AMGDD_CUDA(launch_k(g_pdl, k_ell<float, false>, grid, 256, 0, s, (const float*)L.ell32.p,
                          (const int32_t*)L.ellc.p, L.ell_w, L.n, (const float*)x, (float*)y, (const float*)nullptr,
                          skip));
  } else {
    if (res)
      AMGDD_CUDA(launch_k(g_pdl, k_ell<double, true>, grid, 256, 0, s, (const double*)L.ell64.p,
                          (const int32_t*)L.ellc.p, L.ell_w, L.n, (const double*)x, (double*)y, (const double*)csrc,
                          skip));
    else
      AMGDD_CUDA(launch_k(g_pdl, k_ell<double, false>, grid, 256, 0, s, (const double*)L.ell64.p,
                          (const int32_t*)L.ellc.p, L.ell_w, L.n, (const double*)x, (double*)y,
                          (const double*)nullptr, skip));
  }
  count_kernels(1);
  return AMGDD_OK;
}

int launch_dense(const void* B, int64_t ld, int n, bool fp32, const void* x, void* y, const int* skip,
                 cudaStream_t s) {
  if (n <= 0) return AMGDD_OK;
  if (ld % 4 != 0 || (((uintptr_t)B | (uintptr_t)x) & 15) != 0) {
    set_error("launch_dense: B, x and the leading dimension must be 16-byte aligned");
    return AMGDD_ERR_INTERNAL;
  }
  // warps per row: about 8 vectors per lane or more, at most 8 warps
  const int W = fp32 ? 4 : 2;
  const int64_t per = ((int64_t)n / W + 255) / 256;
  const int S = per >= 8 ? 8 : (per >= 4 ? 4 : (per >= 2 ? 2 : 1));
  const int grid = (int)(((int64_t)n * S + 7) / 8);
  auto go = [&](auto kf, auto kd) -> int {
    if (fp32)
      AMGDD_CUDA(launch_k(g_pdl, kf, grid, 256, 0, s, (const float*)B, ld, n, (const float*)x, (float*)y, skip));
    else
      AMGDD_CUDA(launch_k(g_pdl, kd, grid, 256, 0, s, (const double*)B, ld, n, (const double*)x, (double*)y, skip));
    count_kernels(1);
    return AMGDD_OK;
  };
  switch (S) {
    case 8: return go(k_dense<float, 8>, k_dense<double, 8>);
    case 4: return go(k_dense<float, 4>, k_dense<double, 4>);
    case 2: return go(k_dense<float, 2>, k_dense<double, 2>);
    default: return go(k_dense<float, 1>, k_dense<double, 1>);
  }
}

template <class T>
__global__ void k_count_nonfinite(const T* __restrict__ v, int64_t n, int* __restrict__ count) {
  int c = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (!isfinite(v[i])) ++c;
  if (c) atomicAdd(count, c);
}

int count_nonfinite(const void* v, int64_t n, bool fp32, int* d_count, cudaStream_t s) {
  if (n <= 0 || v == nullptr) return AMGDD_OK;
  const int grid = (int)std::min<int64_t>((n + 255) / 256, 152 * 8);
  if (fp32)
    k_count_nonfinite<float><<<grid, 256, 0, s>>>((const float*)v, n, d_count);
  else
    k_count_nonfinite<double><<<grid, 256, 0, s>>>((const double*)v, n, d_count);
  AMGDD_CUDA(cudaGetLastError());
  count_kernels(1);
  return AMGDD_OK;
}

int launch_cast(const void* src, bool src32, void* dst, bool dst32, int64_t n, const int* skip, cudaStream_t s) {
  if (n == 0) return AMGDD_OK;
  const int g = grid_for(n, 256);
  if (src32 && !dst32)
    AMGDD_CUDA(launch_k(g_pdl, k_cast<float, double>, g, 256, 0, s, (const float*)src, (double*)dst, n, skip));
  else if (!src32 && dst32)
    AMGDD_CUDA(launch_k(g_pdl, k_cast<double, float>, g, 256, 0, s, (const double*)src, (float*)dst, n, skip));
  else if (src32)
    AMGDD_CUDA(launch_k(g_pdl, k_cast<float, float>, g, 256, 0, s, (const float*)src, (float*)dst, n, skip));
  else
    AMGDD_CUDA(launch_k(g_pdl, k_cast<double, double>, g, 256, 0, s, (const double*)src, (double*)dst, n, skip));
  AMGDD_CUDA(cudaGetLastError());
  count_kernels(1);
  return AMGDD_OK;
}

int launch_copy_vec(const void* src, void* dst, bool fp32, int64_t n, const int* skip, cudaStream_t s) {
  return launch_cast(src, fp32, dst, fp32, n, skip, s);
}

int launch_dot_partial(const double* a, const double* b, const double* c, int64_t n, double* partials,
                       const int* skip, cudaStream_t s) {
  AMGDD_CUDA(launch_k(g_pdl, k_dot_partial, kDotBlocks, kDotThreads, 0, s, a, b, c, n, partials, skip));
  AMGDD_CUDA(cudaGetLastError());
  count_kernels(1);
  return AMGDD_OK;
}

int launch_pcg_scalar(int which, PcgState* st, const double* partials, cudaStream_t s,
                      cudaGraphConditionalHandle cond, int use_cond) {
  AMGDD_CUDA(launch_k(g_pdl, k_pcg_scalar, 1, 1024, 0, s, which, st, partials, cond, use_cond));
  AMGDD_CUDA(cudaGetLastError());
  count_kernels(1);
  return AMGDD_OK;
}

int launch_update_xr(PcgState* st, double* x, double* r, const double* p, const double* q, int64_t n,
                     cudaStream_t s) {
  AMGDD_CUDA(launch_k(g_pdl, k_update_xr, grid_for(n, 256), 256, 0, s, st, x, r, p, q, n));
  AMGDD_CUDA(cudaGetLastError());
  count_kernels(1);
  return AMGDD_OK;
}

int launch_update_p(PcgState* st, double* p, const double* z, double* zold, int64_t n, cudaStream_t s) {
  AMGDD_CUDA(launch_k(g_pdl, k_update_p, grid_for(n, 256), 256, 0, s, st, p, z, zold, n));
  AMGDD_CUDA(cudaGetLastError());
  count_kernels(1);
  return AMGDD_OK;
}

int launch_cg_ap(const Level& L0, PcgState* st, const double* p, double* q, double* partials, cudaStream_t s) {
  AMGDD_CUDA(launch_k(g_pdl, k_cg_ap, kDotBlocks, kDotThreads, 0, s, (const double*)L0.ell64.p,
                      (const int32_t*)L0.ellc.p, L0.ell_w, L0.n, p, q, partials, st));
  count_kernels(1);
  return AMGDD_OK;
}

int launch_cg_xr(PcgState* st, double* x, double* r, float* r32, const double* p, const double* q, int64_t n,
                 double* partials, cudaStream_t s) {
  AMGDD_CUDA(launch_k(g_pdl, k_cg_xr, kDotBlocks, kDotThreads, 0, s, x, r, r32, p, q, n, partials, st));
  count_kernels(1);
  return AMGDD_OK;
}

int launch_cg_zdot(PcgState* st, const float* x32, double* z, const double* r, const double* zold, int64_t n,
                   double* partials, cudaStream_t s, cudaGraphConditionalHandle cond, int use_cond) {
  AMGDD_CUDA(launch_k(g_pdl, k_cg_zdot, kDotBlocks, kDotThreads, 0, s, x32, z, r, zold, n, partials, st, cond,
                      use_cond));
  count_kernels(1);
  return AMGDD_OK;
}

// ---------------------------------------------------------------------------
// Persistent V-cycle tail (cooperative launch).  Vectors are written by other
// CTAs in earlier phases of the same launch, so they are read through L2
// (__ldcg) and never through the non-coherent read-only path; matrices and
// index arrays are read-only for the whole launch.
namespace {


// Failure-detection probe of the bounded waits: which 0, a grid barrier that
// the last CTA never reaches; which 1, an mbarrier phase that no copy or
// arrival completes.  Each wait gives up after its limit (about 2 s and 1 s)
// and sets the error word; no copy is in flight, nothing faults.
__global__ void k_wait_probe(unsigned* bar, int* err, int which) {
  if (which == 0) {
    if (blockIdx.x == gridDim.x - 1) return;  // the CTA that never arrives
    grid_barrier(bar, err);
  } else {
    __shared__ __align__(8) uint64_t mb;
    if (threadIdx.x == 0) mbar_init(&mb);
    __syncthreads();
    if (threadIdx.x == 0 && !mbar_wait(&mb, 0u)) atomicExch(err, 1);
    __syncthreads();
  }
}

template <class T>
__device__ __forceinline__ void phase_out(const PhaseDesc& P, int o, T acc) {
  T* y = (T*)P.y;
  switch (P.mode) {
    case SEG_STORE: y[o] = acc; break;
    case SEG_ADD: y[o] = __ldcg(y + o) + acc; break;
    case SEG_ATOMIC_ADD: atomicAdd(y + o, acc); break;
    case SEG_ATOMIC_SUB: atomicAdd(y + o, -acc); break;
    default: y[o] = __ldcg((const T*)P.csrc + o) - acc; break;
  }
  if (P.mode != SEG_RESID && P.cdst != nullptr) ((T*)P.cdst)[o] = __ldcg((const T*)P.csrc + o);
}

// One chunk of an unstaged lanes-per-row plan (the body of k_seg).
template <class T, int L, bool VEC>
__device__ __forceinline__ void phase_chunk(const PhaseDesc& P, int chunk, T* xs) {
  const int b = P.chunk_blk[chunk];
  const int r0 = P.chunk_row0[chunk];
  const int ncb = P.nc[b];
  const int r1 = min(P.nr[b], r0 + P.rows_per_chunk);
  const int32_t* ii = P.in_idx + P.in_off[b];
  const T* x = (const T*)P.x;
  for (int c = threadIdx.x; c < ncb; c += blockDim.x) xs[c] = __ldcg(x + ii[c]);
  __syncthreads();
  const int lane = threadIdx.x % L;
  const int grp = threadIdx.x / L;
  const int ngrp = blockDim.x / L;
  const unsigned mask = group_mask<L>();
  const T* Mb = (const T*)P.M + P.m_off[b];
  const int32_t* oo = P.out_idx + P.out_off[b];
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
    if (lane == 0) phase_out<T>(P, oo[r], acc);
  }
  __syncthreads();
}

// One task of an unstaged row-per-lane plan (the body of k_seg_rows).
template <class T, int L>
__device__ __forceinline__ void phase_task(const PhaseDesc& P, int t, T* xs, int lane, unsigned mask) {
  const int b = P.task_blk[t];
  const int r0 = P.task_row0[t];
  const int rows = P.task_nrow[t];
  const int ncb = P.nc[b], nrb = P.nr[b];
  const int32_t* ii = P.in_idx + P.in_off[b];
  const T* x = (const T*)P.x;
  for (int c = lane; c < ncb; c += L) xs[c] = __ldcg(x + ii[c]);
  __syncwarp(mask);
  if (lane < rows) {
    const int r = r0 + lane;
    const T* col = (const T*)P.MT + P.m_off[b] + r;
    T acc = T(0);
    for (int c = 0; c < ncb; ++c) acc += col[(int64_t)c * nrb] * xs[c];
    phase_out<T>(P, P.out_idx[P.out_off[b] + r], acc);
  }
  __syncwarp(mask);
}

template <class T, int L>
__device__ void run_chunks(const PhaseDesc& P, unsigned char* smem) {
  T* xs = reinterpret_cast<T*>(smem);
  if (P.vec) {
    for (int c = blockIdx.x; c < P.nwork; c += gridDim.x) phase_chunk<T, L, true>(P, c, xs);
  } else {
    for (int c = blockIdx.x; c < P.nwork; c += gridDim.x) phase_chunk<T, L, false>(P, c, xs);
  }
}

template <class T, int L>
__device__ void run_tasks(const PhaseDesc& P, unsigned char* smem) {
  const int per = (int)blockDim.x / L;
  const int grp = (int)threadIdx.x / L;
  const int lane = (int)threadIdx.x % L;
  const unsigned mask = group_mask<L>();
  T* xs = reinterpret_cast<T*>(smem) + (size_t)grp * P.max_nc;
  for (int tb = blockIdx.x; tb * per < P.nwork; tb += gridDim.x) {
    const int t = tb * per + grp;
    if (t < P.nwork) phase_task<T, L>(P, t, xs, lane, mask);
  }
}

template <class T>
__device__ void run_seg(const PhaseDesc& P, unsigned char* smem) {
  if (P.rows_mode) {
    switch (P.lanes) {
      case 8: run_tasks<T, 8>(P, smem); break;
      case 16: run_tasks<T, 16>(P, smem); break;
      default: run_tasks<T, 32>(P, smem); break;
    }
  } else {
    switch (P.lanes) {
      case 4: run_chunks<T, 4>(P, smem); break;
      case 8: run_chunks<T, 8>(P, smem); break;
      case 16: run_chunks<T, 16>(P, smem); break;
      default: run_chunks<T, 32>(P, smem); break;
    }
  }
}

__device__ void run_cast(const PhaseDesc& P) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P.n; i += stride) {
    const double v = P.src32 ? (double)__ldcg((const float*)P.x + i) : __ldcg((const double*)P.x + i);
    if (P.dst32)
      ((float*)P.y)[i] = (float)v;
    else
      ((double*)P.y)[i] = v;
  }
}

template <class T, int L>
__device__ bool run_items_l(const PhaseDesc& P, unsigned char* smem, uint64_t* bar, unsigned& use, int* err) {
  for (int it = blockIdx.x; it < P.nwork; it += gridDim.x)
    if (!item_run<T, L>(P, it, smem, bar, use, err)) return false;
  return true;
}

template <class T>
__device__ bool run_items(const PhaseDesc& P, unsigned char* smem, uint64_t* bar, unsigned& use, int* err) {
  switch (P.lanes) {
    case 4: return run_items_l<T, 4>(P, smem, bar, use, err);
    case 8: return run_items_l<T, 8>(P, smem, bar, use, err);
    case 16: return run_items_l<T, 16>(P, smem, bar, use, err);
    default: return run_items_l<T, 32>(P, smem, bar, use, err);
  }
}

// Every phase is a gather-GEMV (staged: CTAs loop over its items; unstaged:
// over its chunks or row tasks) or a cast; CTAs meet at a grid barrier
// between phases.
__global__ void __launch_bounds__(kItemThreads, 6) k_persistent(const PhaseDesc* __restrict__ phases, int nphases,
                                                               unsigned* bar, int* err, const int* skip) {
  pdl_prologue();
  if ((skip != nullptr && *skip) || *(volatile int*)err != 0) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem_raw);
  if (threadIdx.x == 0) mbar_init(mbar);
  __syncthreads();
  unsigned use = 0;
  bool alive = true;
  for (int k = 0; k < nphases; ++k) {
    const PhaseDesc& P = phases[k];
    if (alive) {
      if (P.op == PH_CAST)
        run_cast(P);
      else if (P.items != nullptr)
        alive = P.fp32 ? run_items<float>(P, smem_raw, mbar, use, err) : run_items<double>(P, smem_raw, mbar, use, err);
      else if (P.fp32)
        run_seg<float>(P, smem_raw + 16);
      else
        run_seg<double>(P, smem_raw + 16);
    }
    if (k + 1 < nphases) grid_barrier(bar, err);
  }
}

}  // namespace

int launch_wait_probe(int which, unsigned* bar, int* err, cudaStream_t s) {
  k_wait_probe<<<which == 0 ? 2 : 1, 32, 0, s>>>(bar, err, which);
  AMGDD_CUDA(cudaGetLastError());
  count_kernels(1);
  return AMGDD_OK;
}

PhaseDesc seg_phase(const SegPlan& p, const void* M, const void* MT, bool fp32, const void* x, void* y, SegMode mode,
                    const void* csrc, void* cdst) {
  PhaseDesc d;
  d.op = PH_SEG;
  d.fp32 = fp32 ? 1 : 0;
  d.mode = (int)mode;
  d.rows_mode = p.rows_mode ? 1 : 0;
  d.lanes = p.rows_mode ? p.kind : p.lanes;
  d.vec = p.vec ? 1 : 0;
  d.rows_per_chunk = p.rows_per_chunk;
  d.nwork = p.rows_mode ? p.ntasks : p.nchunks;
  d.max_nc = p.max_nc;
  d.chunk_blk = p.chunk_blk.p;
  d.chunk_row0 = p.chunk_row0.p;
  d.task_blk = p.task_blk.p;
  d.task_row0 = p.task_row0.p;
  d.task_nrow = p.task_nrow.p;
  d.m_off = p.m_off.p;
  d.in_off = p.in_off.p;
  d.out_off = p.out_off.p;
  d.nr = p.nr.p;
  d.nc = p.nc.p;
  d.in_idx = p.in_idx_ext;
  d.out_idx = p.out_idx_ext;
  d.M = M;
  d.MT = MT;
  d.x = x;
  d.y = y;
  d.csrc = csrc;
  d.cdst = cdst;
  if (p.staged && M != nullptr) {
    d.items = p.items.p;
    d.tabs = p.tabs.p;
    d.gidx = p.gidx.p;
    d.gout = p.gout.p;
    d.nwork = p.nitems;
    d.lanes = p.item_lanes;
    d.rows_mode = 0;
    d.max_in = p.item_max_in;
    d.max_m = p.item_max_m;
    d.max_rows = p.item_max_rows;
  }
  return d;
}

PhaseDesc cast_phase(const void* src, bool src32, void* dst, bool dst32, int64_t n) {
  PhaseDesc d;
  d.op = PH_CAST;
  d.x = src;
  d.y = dst;
  d.src32 = src32 ? 1 : 0;
  d.dst32 = dst32 ? 1 : 0;
  d.n = n;
  return d;
}

size_t staged_smem(int max_in, int max_rows, int max_m, size_t esz) {
  return staged_bytes(max_in, max_rows, max_m, esz);
}

size_t phase_smem(const PhaseDesc& d) {
  if (d.op != PH_SEG) return 16;
  const size_t esz = d.fp32 ? sizeof(float) : sizeof(double);
  if (d.items != nullptr) return staged_smem(d.max_in, d.max_rows, d.max_m, esz);
  return 16 + (size_t)d.max_nc * esz * (d.rows_mode ? (size_t)(kItemThreads / d.lanes) : 1);
}

int persistent_grid(size_t smem, int* grid) {
  int dev = 0, sms = 0, per_sm = 0;
  AMGDD_CUDA(cudaGetDevice(&dev));
  AMGDD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (smem > 48 * 1024)
    AMGDD_CUDA(cudaFuncSetAttribute(k_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  AMGDD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_persistent, kItemThreads, smem));
  if (per_sm < 1) {
    set_error("persistent V-cycle: no CTA fits with %zu bytes of shared memory", smem);
    return AMGDD_ERR_INTERNAL;
  }
  *grid = sms * std::min(per_sm, 16);
  return AMGDD_OK;
}

int launch_persistent(const PhaseDesc* d_phases, int nphases, size_t smem, int grid, unsigned* bar, int* err,
                      const int* skip, cudaStream_t s) {
  if (nphases == 0) return AMGDD_OK;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kItemThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  AMGDD_CUDA(cudaLaunchKernelEx(&cfg, k_persistent, d_phases, nphases, bar, err, skip));
  count_kernels(1);
  return AMGDD_OK;
}

}  // namespace amgdd
