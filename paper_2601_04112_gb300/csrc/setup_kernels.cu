// Setup kernels (FP64): the numeric steps of Algorithm 1.
//
//  k_gram_rows   H_g = sum of g^T g over the rows of one support group of G
//  k_pchol       rank-revealing (diagonally pivoted) Cholesky H_g = R_g^T R_g:
//                the compressed rows of G_l used by the A-apply
//  k_assemble    A_i = A(Omega_i, Omega_i) and the SPSD splitting block
//                A~_i = sum_{rows in nz_i} g^T g / M (Lemma)
//  k_chol        A_i = L L^T (the omega-first ordering makes the leading
//                block the Cholesky factor of A_ww)
//  k_schur       S~ = A~_ww - A~_wG A~_GG^+ A~_Gw (Eq. gevp-S) by eliminating
//                the Gamma pivots, largest diagonal first; pivots below
//                rtol * max diag are the null space of A~_GG
//  k_inv_rows    A_i^{-1}(:, omega_i): the RAS / RAS-T operators
//  k_gep         S~ u = mu A_ww u via C = L^{-1} S~ L^{-T}; cyclic Jacobi for
//                small blocks, Householder tridiagonalisation + implicit QL
//                for large ones;
//                ascending mu, selection, Z = L^{-T} V, sign convention
//  k_pack_z      Z_i and Z_i^T in FP64 and FP32
//  k_next_gram   Grams of G_{l+1} = G_l P_l, per new support group
//
// One CTA owns one matrix; matrices live in global memory (column-major
// unless stated otherwise) so that sizes from a handful to a few thousand
// rows use the same code.
#include <cuda_runtime.h>

#include <algorithm>

#include <cfloat>
#include <cstdint>

#include <cooperative_groups.h>

#include "internal.h"

namespace cg = cooperative_groups;

namespace amgdd {

namespace {

__device__ __forceinline__ double warp_max_idx(double v, int& idx) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, v, off);
    const int oi = __shfl_xor_sync(0xffffffffu, idx, off);
    if (ov > v || (ov == v && oi < idx)) {
      v = ov;
      idx = oi;
    }
  }
  return v;
}

__device__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = (int)threadIdx.x < nw ? sh[threadIdx.x] : 0.0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
    if (threadIdx.x == 0) sh[0] = t;
  }
  __syncthreads();
  t = sh[0];
  __syncthreads();
  return t;
}

// ---------------------------------------------------------------------------
__global__ void k_gram_rows(int64_t first, const int64_t* __restrict__ g_row0, const int64_t* __restrict__ g_row1,
                            const int64_t* __restrict__ g_ptr, const int64_t* __restrict__ h_off,
                            const int64_t* __restrict__ rowptr, const double* __restrict__ val,
                            double* __restrict__ H) {
  const int64_t g = first + blockIdx.x;
  const int s = (int)(g_ptr[g + 1] - g_ptr[g]);
  double* Hg = H + h_off[g];
  const int64_t r0 = g_row0[g], r1 = g_row1[g];
  for (int e = threadIdx.x; e < s * s; e += blockDim.x) {
    const int a = e / s, b = e % s;
    double acc = 0.0;
    for (int64_t r = r0; r < r1; ++r) {
      const double* v = val + rowptr[r];
      acc += v[a] * v[b];
    }
    Hg[e] = acc;
  }
}

__global__ void k_gram_diag(int64_t n, int64_t first_group, const int64_t* __restrict__ h_off,
                            const double* __restrict__ D1, double* __restrict__ H) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j < n) H[h_off[first_group + j]] = D1[j];
}

// Diagonally pivoted Cholesky of the PSD Gram H (s x s, row-major) on a
// scratch copy W.  Row k of R: R[k][piv_k] = sqrt(d_k), R[k][piv_j] =
// W[piv_j][piv_k] / sqrt(d_k) for later pivots, 0 for earlier ones; the
// columns stay in support order, so R^T R = H up to the dropped remainder.
// Stops when the largest remaining diagonal is <= max(s,16) * 4 eps * max
// diag(H) (rounding level).
__global__ void k_pchol(int64_t first, const int64_t* __restrict__ g_ptr, const int64_t* __restrict__ h_off,
                        const double* __restrict__ H, double* __restrict__ R64, float* __restrict__ R32,
                        int32_t* __restrict__ rank_out, double* __restrict__ scratch, int64_t scratch_per) {
  extern __shared__ int piv[];
  __shared__ double sh_best;
  __shared__ int sh_bidx;
  const int64_t g = first + blockIdx.x;
  const int s = (int)(g_ptr[g + 1] - g_ptr[g]);
  const double* Hg = H + h_off[g];
  double* R = R64 + h_off[g];
  float* R32g = R32 + h_off[g];
  double* W = scratch + (int64_t)blockIdx.x * scratch_per;
  for (int e = threadIdx.x; e < s * s; e += blockDim.x) W[e] = Hg[e];
  for (int j = threadIdx.x; j < s; j += blockDim.x) piv[j] = j;
  __syncthreads();
  double dmax0 = 0.0;
  for (int j = 0; j < s; ++j) dmax0 = fmax(dmax0, Hg[j * s + j]);
  const double tau = (double)max(s, 16) * 4.0 * DBL_EPSILON * dmax0;
  int rank = 0;
  for (int k = 0; k < s; ++k) {
    if (threadIdx.x < 32) {
      double best = -1.0;
      int bidx = s;
      for (int j = k + threadIdx.x; j < s; j += 32) {
        const double d = W[piv[j] * s + piv[j]];
        if (d > best || (d == best && j < bidx)) {
          best = d;
          bidx = j;
        }
      }
      best = warp_max_idx(best, bidx);
      if (threadIdx.x == 0) {
        sh_best = best;
        sh_bidx = bidx;
      }
    }
    __syncthreads();
    const double d = sh_best;
    if (!(d > tau)) break;
    if (threadIdx.x == 0) {
      const int t = piv[k];
      piv[k] = piv[sh_bidx];
      piv[sh_bidx] = t;
    }
    __syncthreads();
    const int pk = piv[k];
    const double l = sqrt(d);
    double* Rk = R + (int64_t)k * s;
    for (int j = threadIdx.x; j < s; j += blockDim.x) {
      double v;
      if (j < k)
        v = 0.0;
      else if (j == k)
        v = l;
      else
        v = W[piv[j] * s + pk] / l;
      Rk[piv[j]] = v;
      R32g[(int64_t)k * s + piv[j]] = (float)v;
    }
    __syncthreads();
    const int rem = s - k - 1;
    for (int e = threadIdx.x; e < rem * rem; e += blockDim.x) {
      const int i = piv[k + 1 + e / rem], j = piv[k + 1 + e % rem];
      W[i * s + j] -= Rk[i] * Rk[j];
    }
    __syncthreads();
    rank = k + 1;
  }
  if (threadIdx.x == 0) rank_out[g] = rank;
}

// ---------------------------------------------------------------------------
__global__ void k_assemble(const int32_t* __restrict__ mdim, const int64_t* __restrict__ a_off,
                           const int64_t* __restrict__ pair_ptr, const int32_t* __restrict__ pair_grp,
                           const int32_t* __restrict__ pair_nz, const int64_t* __restrict__ map_ptr,
                           const int32_t* __restrict__ map, const int64_t* __restrict__ g_ptr,
                           const int64_t* __restrict__ h_off, const double* __restrict__ H,
                           const int32_t* __restrict__ M, double* __restrict__ Apool, double* __restrict__ Atpool) {
  const int b = blockIdx.x;
  const int m = mdim[b];
  double* A = Apool + a_off[b];
  double* At = Atpool + a_off[b];
  for (int64_t e = threadIdx.x; e < (int64_t)m * m; e += blockDim.x) {
    A[e] = 0.0;
    At[e] = 0.0;
  }
  __syncthreads();
  for (int64_t p = pair_ptr[b]; p < pair_ptr[b + 1]; ++p) {
    const int g = pair_grp[p];
    const int s = (int)(g_ptr[g + 1] - g_ptr[g]);
    const double* Hg = H + h_off[g];
    const int32_t* mp = map + map_ptr[p];
    const bool nz = pair_nz[p] != 0;
    const double w = 1.0 / (double)M[g];
    for (int e = threadIdx.x; e < s * s; e += blockDim.x) {
      const int a = e / s, c = e % s;
      const int la = mp[a], lc = mp[c];
      if (la >= 0 && lc >= 0) {
        const double h = Hg[e];
        A[la + (int64_t)lc * m] += h;
        if (nz) At[la + (int64_t)lc * m] += h * w;
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// A "team" works on one matrix: one CTA, or CL CTAs of a thread-block
// cluster (large coarse-level blocks) that synchronise with cluster barriers.
// Reductions across the team go through a small global slot per matrix.
template <int CL>
struct Team {
  int cta, rank, size;
  __device__ Team() {
    if constexpr (CL > 1)
      cta = (int)cg::this_cluster().block_rank();
    else
      cta = 0;
    rank = cta * (int)blockDim.x + (int)threadIdx.x;
    size = CL * (int)blockDim.x;
  }
  __device__ void sync() const {
    if constexpr (CL > 1)
      cg::this_cluster().sync();
    else
      __syncthreads();
  }
  // deterministic team-wide sum; red holds CL doubles
  __device__ double sum(double v, double* sh, double* red) const {
    v = block_sum(v, sh);
    if constexpr (CL == 1) {
      return v;
    } else {
      if (threadIdx.x == 0) red[cta] = v;
      sync();
      double t = 0.0;
      for (int c = 0; c < CL; ++c) t += red[c];
      sync();
      return t;
    }
  }
};

// In-place right-looking Cholesky (lower, column-major).
template <int CL>
__global__ void k_chol(const int32_t* __restrict__ mdim, const int64_t* __restrict__ a_off, double* __restrict__ Apool,
                       int32_t* __restrict__ status) {
  const Team<CL> tm;
  const int b = blockIdx.x / CL;
  const int m = mdim[b];
  double* A = Apool + a_off[b];
  int bad = 0;
  for (int k = 0; k < m; ++k) {
    const double d = A[k + (int64_t)k * m];
    if (!(d > 0.0) || !isfinite(d)) {
      bad = k + 1;
      break;
    }
    const double l = sqrt(d);
    tm.sync();
    for (int i = k + 1 + tm.rank; i < m; i += tm.size) A[i + (int64_t)k * m] /= l;
    tm.sync();
    if (tm.rank == 0) A[k + (int64_t)k * m] = l;
    const int rem = m - k - 1;
    for (int64_t e = tm.rank; e < (int64_t)rem * rem; e += tm.size) {
      const int j = k + 1 + (int)(e / rem), i = k + 1 + (int)(e % rem);
      if (i >= j) A[i + (int64_t)j * m] -= A[i + (int64_t)k * m] * A[j + (int64_t)k * m];
    }
    tm.sync();
  }
  if (tm.rank == 0) status[b] = bad;
}

// Eliminate the Gamma pivots of the symmetric A~ (local indices no..m-1,
// lower triangle maintained) so that the omega block becomes the Schur
// complement.  Pivots are taken largest remaining Gamma diagonal first
// (diagonal pivoting, which reveals the rank of a singular PSD A~_GG) and
// elimination stops once the largest remaining one is <= rtol * the largest
// initial one: those directions are treated as the null space of A~_GG.
// Every CTA of the team chooses the same pivot from the same data.
template <int CL>
__global__ void k_schur(const int32_t* __restrict__ mdim, const int32_t* __restrict__ nodim,
                        const int64_t* __restrict__ a_off, double* __restrict__ Atpool, double rtol) {
  extern __shared__ int elim[];  // m - no flags, one per Gamma index
  __shared__ double sh_best;
  __shared__ int sh_p;
  const Team<CL> tm;
  const int b = blockIdx.x / CL;
  const int m = mdim[b], no = nodim[b];
  const int ng = m - no;
  double* A = Atpool + a_off[b];
  auto at = [&](int i, int j) -> double& { return i >= j ? A[i + (int64_t)j * m] : A[j + (int64_t)i * m]; };
  for (int q = threadIdx.x; q < ng; q += blockDim.x) elim[q] = 0;
  double dmax = 0.0;
  for (int p = no; p < m; ++p) dmax = fmax(dmax, A[p + (int64_t)p * m]);
  tm.sync();
  for (int step = 0; step < ng; ++step) {
    // argmax of the remaining Gamma diagonal (smallest index on ties), per CTA
    if (threadIdx.x < 32) {
      double best = -1.0;
      int bi = m;
      for (int q = threadIdx.x; q < ng; q += 32) {
        if (elim[q]) continue;
        const double d = A[(no + q) + (int64_t)(no + q) * m];
        if (d > best || (d == best && no + q < bi)) {
          best = d;
          bi = no + q;
        }
      }
      best = warp_max_idx(best, bi);
      if (threadIdx.x == 0) {
        sh_best = best;
        sh_p = bi;
      }
    }
    __syncthreads();
    const double d = sh_best;
    const int p = sh_p;
    if (!(d > rtol * dmax)) break;
    if (threadIdx.x == 0) elim[p - no] = 1;
    __syncthreads();
    // update every remaining pair (i >= j), i, j in omega or a live Gamma index
    for (int64_t e = tm.rank; e < (int64_t)m * m; e += tm.size) {
      const int j = (int)(e / m), i = (int)(e % m);
      if (i < j) continue;
      if ((i >= no && elim[i - no]) || (j >= no && elim[j - no])) continue;
      A[i + (int64_t)j * m] -= at(i, p) * at(j, p) / d;
    }
    tm.sync();
  }
  for (int64_t e = tm.rank; e < (int64_t)no * no; e += tm.size) {
    const int j = (int)(e / no), i = (int)(e % no);
    if (i < j) A[i + (int64_t)j * m] = A[j + (int64_t)i * m];
  }
}

// Columns [c0, c1) of X = A^{-1} E_omega = L^{-T} L^{-1} E_omega (m x no):
// the substitutions of different columns are independent, so each CTA takes
// one chunk of columns.  Writes W = X^T (no x m, row-major) and W^T = X
// (m x no, row-major), FP64 and FP32.
__global__ void k_inv_rows(const int32_t* __restrict__ chunk_b, const int32_t* __restrict__ chunk_c0, int cw,
                           const int32_t* __restrict__ mdim, const int32_t* __restrict__ nodim,
                           const int64_t* __restrict__ a_off, const double* __restrict__ Lpool,
                           const int64_t* __restrict__ w_off, double* __restrict__ W64, float* __restrict__ W32,
                           double* __restrict__ Wt64, float* __restrict__ Wt32, double* __restrict__ scratch) {
  const int b = chunk_b[blockIdx.x];
  const int c0 = chunk_c0[blockIdx.x];
  const int m = mdim[b], no = nodim[b];
  const int c1 = min(no, c0 + cw);
  const int nc = c1 - c0;
  const double* L = Lpool + a_off[b];
  double* Y = scratch + w_off[b];  // row-major m x no
  for (int64_t e = threadIdx.x; e < (int64_t)m * nc; e += blockDim.x) {
    const int i = (int)(e / nc), j = c0 + (int)(e % nc);
    Y[(int64_t)i * no + j] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  // forward: L Y = E (column j is zero above row j)
  for (int t = c0; t < m; ++t) {
    const double ltt = L[t + (int64_t)t * m];
    const int jn = min(c1, t + 1) - c0;
    for (int j = threadIdx.x; j < jn; j += blockDim.x) Y[(int64_t)t * no + c0 + j] /= ltt;
    __syncthreads();
    const int rem = m - t - 1;
    for (int64_t e = threadIdx.x; e < (int64_t)rem * jn; e += blockDim.x) {
      const int i = t + 1 + (int)(e / jn), j = c0 + (int)(e % jn);
      Y[(int64_t)i * no + j] -= L[i + (int64_t)t * m] * Y[(int64_t)t * no + j];
    }
    __syncthreads();
  }
  // backward: L^T X = Y
  for (int t = m - 1; t >= 0; --t) {
    const double ltt = L[t + (int64_t)t * m];
    for (int j = threadIdx.x; j < nc; j += blockDim.x) Y[(int64_t)t * no + c0 + j] /= ltt;
    __syncthreads();
    for (int64_t e = threadIdx.x; e < (int64_t)t * nc; e += blockDim.x) {
      const int i = (int)(e / nc), j = c0 + (int)(e % nc);
      Y[(int64_t)i * no + j] -= L[t + (int64_t)i * m] * Y[(int64_t)t * no + j];
    }
    __syncthreads();
  }
  const int64_t o = w_off[b];
  for (int64_t e = threadIdx.x; e < (int64_t)m * nc; e += blockDim.x) {
    const int i = (int)(e / nc), j = c0 + (int)(e % nc);
    const double v = Y[(int64_t)i * no + j];
    Wt64[o + (int64_t)i * no + j] = v;
    Wt32[o + (int64_t)i * no + j] = (float)v;
    W64[o + (int64_t)j * m + i] = v;
    W32[o + (int64_t)j * m + i] = (float)v;
  }
}

// Forward substitution L X = B on columns [c0, c1) of the column-major n x nc
// matrix X (ld n), L lower with leading dimension ldl.
__device__ void tri_fwd_cols(const double* __restrict__ L, int ldl, double* X, int n, int c0, int c1) {
  const int nc = c1 - c0;
  if (nc <= 0) return;
  for (int t = 0; t < n; ++t) {
    const double ltt = L[t + (int64_t)t * ldl];
    for (int j = threadIdx.x; j < nc; j += blockDim.x) X[t + (int64_t)(c0 + j) * n] /= ltt;
    __syncthreads();
    const int rem = n - t - 1;
    for (int64_t e = threadIdx.x; e < (int64_t)rem * nc; e += blockDim.x) {
      const int i = t + 1 + (int)(e % rem), j = c0 + (int)(e / rem);
      X[i + (int64_t)j * n] -= L[i + (int64_t)t * ldl] * X[t + (int64_t)j * n];
    }
    __syncthreads();
  }
}

// Backward substitution L^T X = B on columns [c0, c1).
__device__ void tri_bwd_cols(const double* __restrict__ L, int ldl, double* X, int n, int c0, int c1) {
  const int nc = c1 - c0;
  if (nc <= 0) return;
  for (int t = n - 1; t >= 0; --t) {
    const double ltt = L[t + (int64_t)t * ldl];
    for (int j = threadIdx.x; j < nc; j += blockDim.x) X[t + (int64_t)(c0 + j) * n] /= ltt;
    __syncthreads();
    for (int64_t e = threadIdx.x; e < (int64_t)t * nc; e += blockDim.x) {
      const int i = (int)(e % t), j = c0 + (int)(e / t);
      X[i + (int64_t)j * n] -= L[t + (int64_t)i * ldl] * X[t + (int64_t)j * n];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Generalized eigenproblem S~ u = mu A_ww u on one aggregate (one team).
// Global scratch per matrix: C, Cn, V, Vn, T (n x n each), perm (n ints),
// red (CL doubles), kslot.  Shared: rotation coefficients of one round.
template <int CL, bool QL>
__global__ void k_gep(const int32_t* __restrict__ mdim, const int32_t* __restrict__ nodim,
                      const int64_t* __restrict__ a_off, const double* __restrict__ Lpool,
                      const double* __restrict__ Spool, const int32_t* __restrict__ capv, double thresh,
                      const int64_t* __restrict__ mu_off, double* __restrict__ mu_out,
                      const int64_t* __restrict__ z_off_cap, double* __restrict__ Zcap, int32_t* __restrict__ kout,
                      double* __restrict__ scratch, const int64_t* __restrict__ scr_off,
                      int32_t* __restrict__ work_out, int ql_smem) {
  __shared__ double sh[32];
  int work = 0;  // Jacobi sweeps or QL rotations (for the setup flop count)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Team<CL> tm;
  const int b = blockIdx.x / CL;
  const int m = mdim[b], n = nodim[b];
  const double* L = Lpool + a_off[b];  // leading n x n block: chol(A_ww), ld m
  const double* S = Spool + a_off[b];  // leading n x n block: S~, ld m
  double* C = scratch + scr_off[b];
  double* Cn = C + (int64_t)n * n;
  double* V = Cn + (int64_t)n * n;
  double* Vn = V + (int64_t)n * n;
  double* T = Vn + (int64_t)n * n;
  int* perm = (int*)(T + (int64_t)n * n);
  double* red = (double*)(perm + n + (n & 1)) ;
  int* kslot = (int*)(red + CL);
  double* cself = reinterpret_cast<double*>(smem_raw);
  double* cpart = cself + n + 1;
  int* partner = reinterpret_cast<int*>(cpart + n + 1);
  // this CTA's contiguous column range for column-parallel phases
  const int per = (n + CL - 1) / CL;
  const int c0 = min(n, tm.cta * per), c1 = min(n, c0 + per);

  // T = L^{-1} S (column-major n x n)
  for (int64_t e = threadIdx.x; e < (int64_t)n * (c1 - c0); e += blockDim.x) {
    const int i = (int)(e % n), j = c0 + (int)(e / n);
    T[i + (int64_t)j * n] = S[i + (int64_t)j * m];
  }
  __syncthreads();
  tri_fwd_cols(L, m, T, n, c0, c1);
  tm.sync();
  // C = L^{-1} T^T
  for (int64_t e = threadIdx.x; e < (int64_t)n * (c1 - c0); e += blockDim.x) {
    const int i = (int)(e % n), j = c0 + (int)(e / n);
    C[i + (int64_t)j * n] = T[j + (int64_t)i * n];
  }
  __syncthreads();
  tri_fwd_cols(L, m, C, n, c0, c1);
  tm.sync();
  // symmetrise (upper from lower), V = I
  for (int64_t e = tm.rank; e < (int64_t)n * n; e += tm.size) {
    const int i = (int)(e % n), j = (int)(e / n);
    if (i > j) {
      const double v = 0.5 * (C[i + (int64_t)j * n] + C[j + (int64_t)i * n]);
      Cn[i + (int64_t)j * n] = v;
      Cn[j + (int64_t)i * n] = v;
    } else if (i == j) {
      Cn[e] = C[e];
    }
    V[e] = (i == j) ? 1.0 : 0.0;
  }
  tm.sync();
  {
    double* t0 = C;
    C = Cn;
    Cn = t0;
  }

  if constexpr (QL) {
    // Large blocks: Householder reduction to tridiagonal form, explicit
    // accumulation of the reflectors into V, then implicit QL sweeps with
    // Wilkinson shifts.  One thread computes each sweep's rotation chain; the
    // whole team applies the chain to its rows of V.
    double* d = Cn;
    double* e = d + n;
    double* tau = e + n;
    double* pv = tau + n;
    double* rc = pv + n;
    double* rs = rc + n;
    int* ri = reinterpret_cast<int*>(rs + n);
    int* ctl = ri + n;  // [0] rotations in the sweep, [1] finished
    for (int k = 0; k + 2 < n; ++k) {
      const int mm = n - k - 1;
      double* x = C + (k + 1) + (int64_t)k * n;  // column k below the diagonal
      double ss = 0.0;
      for (int i = tm.rank; i < mm; i += tm.size) ss += x[i] * x[i];
      ss = tm.sum(ss, sh, red);
      const double x0 = x[0];
      const double xn = sqrt(ss);
      // H = I - tk u u^T with u = x - alpha e_0, alpha = -sign(x0) ||x||,
      // u^T u = 2 (||x||^2 + |x0| ||x||)
      const double alpha = xn == 0.0 ? 0.0 : (x0 >= 0.0 ? -xn : xn);
      const double tk = xn == 0.0 ? 0.0 : 1.0 / (xn * (xn + fabs(x0)));
      tm.sync();
      if (tm.rank == 0) {
        x[0] = x0 - alpha;
        tau[k] = tk;
        e[k] = alpha;
        d[k] = C[k + (int64_t)k * n];
      }
      tm.sync();
      if (tk != 0.0) {
        double* A = C + (k + 1) + (int64_t)(k + 1) * n;  // trailing block, leading dimension n
        for (int i = tm.rank; i < mm; i += tm.size) {
          double acc = 0.0;
          for (int j = 0; j < mm; ++j) acc += A[i + (int64_t)j * n] * x[j];
          pv[i] = tk * acc;
        }
        tm.sync();
        double pu = 0.0;
        for (int i = tm.rank; i < mm; i += tm.size) pu += pv[i] * x[i];
        pu = tm.sum(pu, sh, red);
        const double K = 0.5 * tk * pu;
        for (int64_t q = tm.rank; q < (int64_t)mm * mm; q += tm.size) {
          const int i = (int)(q % mm), j = (int)(q / mm);
          A[i + (int64_t)j * n] -= x[i] * (pv[j] - K * x[j]) + (pv[i] - K * x[i]) * x[j];
        }
        tm.sync();
      }
    }
    if (tm.rank == 0) {
      if (n >= 2) {
        d[n - 2] = C[(n - 2) + (int64_t)(n - 2) * n];
        e[n - 2] = C[(n - 1) + (int64_t)(n - 2) * n];
      }
      d[n - 1] = C[(n - 1) + (int64_t)(n - 1) * n];
      e[n - 1] = 0.0;
    }
    tm.sync();
    // V = H_0 H_1 ... H_{n-3}, accumulated backwards
    for (int k = n - 3; k >= 0; --k) {
      const double tk = tau[k];
      if (tk == 0.0) continue;
      const int mm = n - k - 1;
      const double* u = C + (k + 1) + (int64_t)k * n;
      double* Q = V + (k + 1) + (int64_t)(k + 1) * n;
      for (int j = tm.rank; j < mm; j += tm.size) {
        double acc = 0.0;
        for (int i = 0; i < mm; ++i) acc += u[i] * Q[i + (int64_t)j * n];
        pv[j] = tk * acc;
      }
      tm.sync();
      for (int64_t q = tm.rank; q < (int64_t)mm * mm; q += tm.size) {
        const int i = (int)(q % mm), j = (int)(q / mm);
        Q[i + (int64_t)j * n] -= u[i] * pv[j];
      }
      tm.sync();
    }
    // implicit QL on (d, e): e[i] couples i and i+1.  This is the published
    // implicit QL method with Wilkinson shifts (Bowdler, Martin, Reinsch and
    // Wilkinson, Numer. Math. 11 (1968); EISPACK tql2): per sweep the shift g,
    // the chain of plane rotations from the bottom of the unreduced block up,
    // and the split test on |e|; rotations are accumulated into V by the team.
    // The chain is serial: warp 0 of the team's first CTA runs it (the split
    // test by the whole warp, 32 entries per ballot; the rotations by lane 0)
    // on copies of d and e in that CTA's shared memory when they fit
    // (ql_smem), then publishes the sweep's rotations for the team.
    const bool lead = tm.cta == 0;
    const bool shq = ql_smem != 0;
    double* sd = shq ? reinterpret_cast<double*>(smem_raw) : d;
    double* se = shq ? sd + n : e;
    double* qc = shq ? se + n : rc;
    double* qs = shq ? qc + n : rs;
    int* qi = shq ? reinterpret_cast<int*>(qs + n) : ri;
    if (shq && lead) {
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        sd[i] = d[i];
        se[i] = e[i];
      }
      __syncthreads();
    }
    int l = 0, iter = 0;  // kept by warp 0 of the first CTA (the same in every lane)
    for (int guard = 0; guard < 64 * n + 64; ++guard) {
      if (lead && threadIdx.x < 32) {
        const int lane = (int)threadIdx.x;
        int nrot = 0, fin = 0;
        for (;;) {
          if (l >= n) {
            fin = 1;
            break;
          }
          int mm = n - 1;  // the first small e[mm] at or after l
          for (int base = l; base < n - 1; base += 32) {
            const int idx = base + lane;
            const bool small =
                idx < n - 1 && fabs(se[idx]) <= DBL_EPSILON * (fabs(sd[idx]) + fabs(sd[idx + 1]));
            const unsigned bal = __ballot_sync(0xffffffffu, small);
            if (bal) {
              mm = base + __ffs(bal) - 1;
              break;
            }
          }
          if (mm == l || iter >= 60) {  // d[l] converged (or the iteration budget is spent)
            ++l;
            iter = 0;
            continue;
          }
          ++iter;
          if (lane == 0) {
            double g = (sd[l + 1] - sd[l]) / (2.0 * se[l]);
            double r = hypot(g, 1.0);
            g = sd[mm] - sd[l] + se[l] / (g + (g >= 0.0 ? r : -r));
            double sn = 1.0, cs = 1.0, p = 0.0;
            bool split = false;
            for (int i = mm - 1; i >= l; --i) {
              const double f = sn * se[i], bb = cs * se[i];
              r = hypot(f, g);
              se[i + 1] = r;
              if (r == 0.0) {  // the chain split: recheck convergence before finishing
                sd[i + 1] -= p;
                se[mm] = 0.0;
                split = true;
                break;
              }
              sn = f / r;
              cs = g / r;
              g = sd[i + 1] - p;
              r = (sd[i] - g) * sn + 2.0 * cs * bb;
              p = sn * r;
              sd[i + 1] = g + p;
              g = cs * r - bb;
              qc[nrot] = cs;
              qs[nrot] = sn;
              qi[nrot] = i;
              ++nrot;
            }
            if (!split) {
              sd[l] -= p;
              se[l] = g;
              se[mm] = 0.0;
            }
          }
          nrot = __shfl_sync(0xffffffffu, nrot, 0);
          __syncwarp();
          break;
        }
        if (lane == 0) {
          ctl[0] = nrot;
          ctl[1] = fin;
        }
      }
      if (shq && lead) {  // publish the sweep's rotations for the other CTAs
        __syncthreads();
        const int nr = ctl[0];
        for (int q = threadIdx.x; q < nr; q += blockDim.x) {
          rc[q] = qc[q];
          rs[q] = qs[q];
          ri[q] = qi[q];
        }
      }
      tm.sync();
      const int nrot = ctl[0];
      const int fin = ctl[1];
      work += nrot;
      if (fin) break;
      // The chain's rotations act on consecutive pairs (i, i + 1), i = ri[0],
      // ri[0] - 1, ...: rotation q finishes element i + 1 of a row and hands
      // its new element i to rotation q + 1, so that element stays in a
      // register and only the independent loads of element i touch memory.
      if (nrot > 0) {
        for (int row = tm.rank; row < n; row += tm.size) {
          double* vr = V + row;
          double hi = vr[(int64_t)(ri[0] + 1) * n];
#pragma unroll 4
          for (int q = 0; q < nrot; ++q) {
            const int i = ri[q];
            const double cs = rc[q], sn = rs[q];
            const double a0 = vr[(int64_t)i * n];
            vr[(int64_t)(i + 1) * n] = sn * a0 + cs * hi;
            hi = cs * a0 - sn * hi;
          }
          vr[(int64_t)ri[nrot - 1] * n] = hi;
        }
      }
      tm.sync();
    }
    if (shq && lead) {  // the eigenvalues back to d for the team
      for (int i = threadIdx.x; i < n; i += blockDim.x) d[i] = sd[i];
    }
    tm.sync();
    for (int i = tm.rank; i < n; i += tm.size) C[i + (int64_t)i * n] = d[i];
    tm.sync();
  } else {
    // Cyclic Jacobi, parallel (round-robin) ordering: each round applies n/2
    // disjoint rotations at once, C <- J^T C J, V <- V J.  Every CTA of the
    // team computes all rotation angles of a round (same inputs, same
    // results) and updates its share of the entries.
    const int ne = n + (n & 1);
    const int mr = ne - 1;
    const double tolf = 4.0 * (double)max(n, 16) * DBL_EPSILON;
    for (int sweep = 0; sweep < 40 && n > 1; ++sweep) {
      double off = 0.0, tot = 0.0;
      for (int64_t e = tm.rank; e < (int64_t)n * n; e += tm.size) {
        const int i = (int)(e % n), j = (int)(e / n);
        const double v = C[e] * C[e];
        tot += v;
        if (i != j) off += v;
      }
      off = tm.sum(off, sh, red);
      tot = tm.sum(tot, sh, red);
      if (!(off > tolf * tolf * tot)) break;
      ++work;
      for (int r = 0; r < mr; ++r) {
        for (int k = threadIdx.x; k < ne / 2; k += blockDim.x) {
          int p, q;
          if (k == 0) {
            p = 0;
            q = r + 1;
          } else {
            p = ((r + k) % mr) + 1;
            q = (((r - k) % mr) + mr) % mr + 1;
          }
          if (p > q) {
            const int t = p;
            p = q;
            q = t;
          }
          if (q >= n) {  // dummy partner (odd n)
            if (p < n) {
              partner[p] = p;
              cself[p] = 1.0;
              cpart[p] = 0.0;
            }
            continue;
          }
          const double app = C[p + (int64_t)p * n], aqq = C[q + (int64_t)q * n], apq = C[p + (int64_t)q * n];
          double c = 1.0, s = 0.0;
          if (apq != 0.0) {
            const double th = (aqq - app) / (2.0 * apq);
            const double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(1.0 + th * th));
            c = 1.0 / sqrt(1.0 + t * t);
            s = t * c;
          }
          partner[p] = q;
          partner[q] = p;
          cself[p] = c;
          cpart[p] = -s;
          cself[q] = c;
          cpart[q] = s;
        }
        __syncthreads();
        for (int64_t e = tm.rank; e < (int64_t)n * n; e += tm.size) {
          const int i = (int)(e % n), j = (int)(e / n);
          const int pi = partner[i], pj = partner[j];
          const double si = cself[i], ti = cpart[i], sj = cself[j], tj = cpart[j];
          double v = si * sj * C[i + (int64_t)j * n];
          if (pj != j) v += si * tj * C[i + (int64_t)pj * n];
          if (pi != i) v += ti * sj * C[pi + (int64_t)j * n];
          if (pi != i && pj != j) v += ti * tj * C[pi + (int64_t)pj * n];
          Cn[e] = v;
          double w = sj * V[i + (int64_t)j * n];
          if (pj != j) w += tj * V[i + (int64_t)pj * n];
          Vn[e] = w;
        }
        tm.sync();
        double* t0 = C;
        C = Cn;
        Cn = t0;
        double* t1 = V;
        V = Vn;
        Vn = t1;
      }
    }
  }
  if (tm.rank == 0) work_out[b] = work;
  // ascending mu (stable on ties)
  for (int i = tm.rank; i < n; i += tm.size) {
    const double di = C[i + (int64_t)i * n];
    int rk = 0;
    for (int j = 0; j < n; ++j) {
      const double dj = C[j + (int64_t)j * n];
      if (dj < di || (dj == di && j < i)) ++rk;
    }
    perm[rk] = i;
  }
  tm.sync();
  if (tm.rank == 0) {
    int cnt = 0;
    for (int i = 0; i < n; ++i) {
      const double mu = C[perm[i] + (int64_t)perm[i] * n];
      if (thresh <= 0.0 || mu <= 0.0 || mu < 1.0 / thresh) ++cnt;
    }
    const int kk = min(cnt, capv[b]);
    kout[b] = kk;
    *kslot = kk;
  }
  for (int i = tm.rank; i < n; i += tm.size) mu_out[mu_off[b] + i] = C[perm[i] + (int64_t)perm[i] * n];
  tm.sync();
  const int k = *kslot;
  // X = L^{-T} V(:, perm[0..k)) in T (column-major n x k); column chunks per CTA
  const int perk = (k + CL - 1) / CL;
  const int k0 = min(k, tm.cta * perk), k1 = min(k, k0 + perk);
  for (int64_t e = threadIdx.x; e < (int64_t)n * (k1 - k0); e += blockDim.x) {
    const int i = (int)(e % n), c = k0 + (int)(e / n);
    T[i + (int64_t)c * n] = V[i + (int64_t)perm[c] * n];
  }
  __syncthreads();
  tri_bwd_cols(L, m, T, n, k0, k1);
  // sign: the first entry within (1 - 1e-6) of the largest magnitude is
  // positive (robust when two entries tie in exact arithmetic)
  double* Z = Zcap + z_off_cap[b];  // column-major n x k
  for (int c = k0 + (int)threadIdx.x; c < k1; c += blockDim.x) {
    double best = 0.0;
    for (int i = 0; i < n; ++i) best = fmax(best, fabs(T[i + (int64_t)c * n]));
    int bi = 0;
    for (int i = 0; i < n; ++i)
      if (fabs(T[i + (int64_t)c * n]) >= (1.0 - 1e-6) * best) {
        bi = i;
        break;
      }
    const double sg = T[bi + (int64_t)c * n] < 0.0 ? -1.0 : 1.0;
    for (int i = 0; i < n; ++i) Z[i + (int64_t)c * n] = sg * T[i + (int64_t)c * n];
  }
}

__global__ void k_pack_z(const int32_t* __restrict__ nodim, const int32_t* __restrict__ kv,
                         const int64_t* __restrict__ z_off_cap, const double* __restrict__ Zcap,
                         const int64_t* __restrict__ z_off, double* __restrict__ Z64, float* __restrict__ Z32,
                         double* __restrict__ Zt64, float* __restrict__ Zt32) {
  const int b = blockIdx.x;
  const int n = nodim[b], k = kv[b];
  const double* Zc = Zcap + z_off_cap[b];
  const int64_t o = z_off[b];
  for (int64_t e = threadIdx.x; e < (int64_t)n * k; e += blockDim.x) {
    const int i = (int)(e % n), c = (int)(e / n);
    const double v = Zc[e];
    Z64[o + (int64_t)i * k + c] = v;  // Z: n x k row-major
    Z32[o + (int64_t)i * k + c] = (float)v;
    Zt64[o + (int64_t)c * n + i] = v;  // Z^T: k x n row-major
    Zt32[o + (int64_t)c * n + i] = (float)v;
  }
}

// ---------------------------------------------------------------------------
// Gram of one support group of G_{l+1} = G_l P_l:  H' = sum_g P_g^T H_g P_g.
// Row b of P_g (support node b of g) has k_b entries Z(row of node b, :) at
// columns [col_b, col_b + k_b) of the new support.
__global__ void k_next_gram(int64_t first, const int64_t* __restrict__ new_ptr, const int32_t* __restrict__ contrib,
                            const int64_t* __restrict__ new_sptr, const int64_t* __restrict__ new_hoff,
                            const int64_t* __restrict__ rowz_ptr, const int64_t* __restrict__ rowz_zoff,
                            const int32_t* __restrict__ rowz_k, const int32_t* __restrict__ rowz_col,
                            const int64_t* __restrict__ g_ptr, const int64_t* __restrict__ h_off,
                            const double* __restrict__ H, const double* __restrict__ Z64, double* __restrict__ Hn,
                            double* __restrict__ scratch, int64_t scratch_per) {
  const int64_t h = first + blockIdx.x;
  const int sn = (int)(new_sptr[h + 1] - new_sptr[h]);
  double* Hh = Hn + new_hoff[h];
  double* Tm = scratch + (int64_t)blockIdx.x * scratch_per;
  for (int64_t e = threadIdx.x; e < (int64_t)sn * sn; e += blockDim.x) Hh[e] = 0.0;
  __syncthreads();
  for (int64_t q = new_ptr[h]; q < new_ptr[h + 1]; ++q) {
    const int g = contrib[q];
    const int s = (int)(g_ptr[g + 1] - g_ptr[g]);
    const double* Hg = H + h_off[g];
    const int64_t rp = rowz_ptr[g];
    // Tm (s x sn, row-major) = H_g P_g
    for (int64_t e = threadIdx.x; e < (int64_t)s * sn; e += blockDim.x) {
      const int a = (int)(e / sn), d = (int)(e % sn);
      double acc = 0.0;
      for (int bb = 0; bb < s; ++bb) {
        const int cb = rowz_col[rp + bb];
        const int kb = rowz_k[rp + bb];
        if (d >= cb && d < cb + kb) acc += Hg[(int64_t)a * s + bb] * Z64[rowz_zoff[rp + bb] + (d - cb)];
      }
      Tm[e] = acc;
    }
    __syncthreads();
    // Hh += P_g^T Tm
    for (int64_t e = threadIdx.x; e < (int64_t)sn * sn; e += blockDim.x) {
      const int c = (int)(e / sn), d = (int)(e % sn);
      double acc = 0.0;
      for (int a = 0; a < s; ++a) {
        const int ca = rowz_col[rp + a];
        const int ka = rowz_k[rp + a];
        if (c >= ca && c < ca + ka) acc += Z64[rowz_zoff[rp + a] + (c - ca)] * Tm[(int64_t)a * sn + d];
      }
      Hh[e] += acc;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Rows of one support group of G_{l+1} = G_l P_l (Section 3.1), carried as
// rows: the stacked products R_g P_g of every contributing level-l group g
// (rank_g rows each, P_g as in k_next_gram) are reduced by Householder QR to
// their R factor, min(rows, sn) rows over the new support.  Q is orthogonal,
// so R^T R = sum_g P_g^T R_g^T R_g P_g (the Gram k_next_gram forms), while R
// keeps the small singular values of the rows to rounding relative to the
// largest, which the Gram of the rows would square away.
// T: stacked rows, column-major (ld = rows) in scratch at t_off[h].
template <int CL>
__global__ void k_next_rows(int64_t first, const int64_t* __restrict__ new_ptr, const int32_t* __restrict__ contrib,
                            const int64_t* __restrict__ new_sptr, const int64_t* __restrict__ new_hoff,
                            const int64_t* __restrict__ rowz_ptr, const int64_t* __restrict__ rowz_zoff,
                            const int32_t* __restrict__ rowz_k, const int32_t* __restrict__ rowz_col,
                            const int64_t* __restrict__ g_ptr, const int64_t* __restrict__ h_off,
                            const int32_t* __restrict__ rank, const double* __restrict__ R,
                            const double* __restrict__ Z64, const int64_t* __restrict__ t_off,
                            double* __restrict__ scratch, double* __restrict__ Rn64, float* __restrict__ Rn32,
                            int32_t* __restrict__ rank_out, double* __restrict__ red_pool) {
  __shared__ double sh[32];
  const Team<CL> tm;
  const int64_t h = first + blockIdx.x / CL;
  const int sn = (int)(new_sptr[h + 1] - new_sptr[h]);
  double* T = scratch + (t_off[h] - t_off[first]);
  double* red = red_pool + (h - first) * CL;
  const int nr = (int)(t_off[h + 1] - t_off[h]) / sn;
  // T = [R_g P_g; ...]
  int row = 0;
  for (int64_t q = new_ptr[h]; q < new_ptr[h + 1]; ++q) {
    const int g = contrib[q];
    const int s = (int)(g_ptr[g + 1] - g_ptr[g]);
    const int rk = rank[g];
    const double* Rg = R + h_off[g];
    const int64_t rp = rowz_ptr[g];
    for (int64_t e = tm.rank; e < (int64_t)rk * sn; e += tm.size) {
      const int r = (int)(e / sn), d = (int)(e % sn);
      double acc = 0.0;
      for (int bb = 0; bb < s; ++bb) {
        const int cb = rowz_col[rp + bb];
        const int kb = rowz_k[rp + bb];
        if (d >= cb && d < cb + kb) acc += Rg[(int64_t)r * s + bb] * Z64[rowz_zoff[rp + bb] + (d - cb)];
      }
      T[(row + r) + (int64_t)d * nr] = acc;
    }
    row += rk;
  }
  tm.sync();
  const int kmax = min(nr, sn);
  const int warp = tm.rank >> 5, lane = (int)threadIdx.x & 31, nw = tm.size >> 5;
  for (int k = 0; k < kmax; ++k) {
    const double* xk = T + (int64_t)k * nr;
    double part = 0.0;
    for (int i = k + tm.rank; i < nr; i += tm.size) part += xk[i] * xk[i];
    const double nb2 = tm.sum(part, sh, red);
    const double x0 = xk[k];
    const double xn = sqrt(nb2);
    const double alpha = x0 >= 0.0 ? -xn : xn;
    const double v0 = x0 - alpha;
    const double vtv = v0 * v0 + (nb2 - x0 * x0);
    if (vtv > 0.0) {
      for (int j = k + 1 + warp; j < sn; j += nw) {
        double* cj = T + (int64_t)j * nr;
        double acc = lane == 0 ? v0 * cj[k] : 0.0;
        for (int i = k + 1 + lane; i < nr; i += 32) acc += xk[i] * cj[i];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        const double f = 2.0 * acc / vtv;
        if (lane == 0) cj[k] -= f * v0;
        for (int i = k + 1 + lane; i < nr; i += 32) cj[i] -= f * xk[i];
      }
    }
    tm.sync();
    if (tm.rank == 0) T[k + (int64_t)k * nr] = vtv > 0.0 ? alpha : x0;
    tm.sync();
  }
  // R (row-major, ld sn): row k = T[k, k..sn-1], zeros left of the diagonal
  double* Rh = Rn64 + new_hoff[h];
  float* Rh32 = Rn32 + new_hoff[h];
  for (int64_t e = tm.rank; e < (int64_t)kmax * sn; e += tm.size) {
    const int k = (int)(e / sn), j = (int)(e % sn);
    const double v = j < k ? 0.0 : T[k + (int64_t)j * nr];
    Rh[e] = v;
    Rh32[e] = (float)v;
  }
  if (tm.rank == 0) rank_out[h] = kmax;
}

// Schur complement of Eq. gevp-S in row form: S~ = X^T (I - Pi) X with
// [X Y_G] = W^{1/2} G(nz_i, Omega_i) the rows of the splitting of the Lemma
// (each group g in nz_i contributes its rows R_g / sqrt(M_g)), X on omega_i,
// Y_G on Gamma_i, and Pi the orthogonal projector onto range(Y_G).
// Householder QR with column pivoting on the Gamma columns (largest remaining
// column norm first, the smallest index on ties) reveals the numerical rank
// of Y_G: it stops once the largest remaining column norm is at most
// max(rows, |Gamma_i|) eps times the first pivot's (those directions are its
// numerical null space).  The same reflections applied to X leave
// Q^T X = [X_1; X_2] with Pi X = Q [X_1; 0], so S~ = X_2^T X_2, formed from
// rows and never as a difference of Grams.  S~ replaces the omega block of
// At (column-major, ld m), which the eigensolver reads.
// Y: rows x m column-major at y_off[b]; nrm: m doubles per matrix at n_off[b].
template <int CL>
__global__ void k_schur_rows(const int32_t* __restrict__ mdim, const int32_t* __restrict__ nodim,
                             const int64_t* __restrict__ a_off, const int64_t* __restrict__ pair_ptr,
                             const int32_t* __restrict__ pair_grp, const int32_t* __restrict__ pair_nz,
                             const int64_t* __restrict__ map_ptr, const int32_t* __restrict__ map,
                             const int64_t* __restrict__ g_ptr, const int64_t* __restrict__ h_off,
                             const int32_t* __restrict__ rank, const double* __restrict__ R,
                             const int32_t* __restrict__ M, const int64_t* __restrict__ y_off,
                             const int32_t* __restrict__ y_rows, double* __restrict__ Ypool,
                             const int64_t* __restrict__ n_off, double* __restrict__ nrm_pool,
                             double* __restrict__ Atpool, int32_t* __restrict__ rank_out) {
  __shared__ double s_best;
  __shared__ int s_bi;
  const Team<CL> tm;
  const int b = blockIdx.x / CL;
  const int m = mdim[b], no = nodim[b];
  const int nr = y_rows[b];
  double* Y = Ypool + y_off[b];
  double* nrm = nrm_pool + n_off[b];
  for (int64_t e = tm.rank; e < (int64_t)nr * m; e += tm.size) Y[e] = 0.0;
  tm.sync();
  int row = 0;
  for (int64_t p = pair_ptr[b]; p < pair_ptr[b + 1]; ++p) {
    if (!pair_nz[p]) continue;
    const int g = pair_grp[p];
    const int s = (int)(g_ptr[g + 1] - g_ptr[g]);
    const int rk = rank[g];
    const double w = 1.0 / sqrt((double)M[g]);
    const double* Rg = R + h_off[g];
    const int32_t* mp = map + map_ptr[p];
    for (int64_t e = tm.rank; e < (int64_t)rk * s; e += tm.size) {
      const int r = (int)(e / s), a = (int)(e % s);
      const int la = mp[a];
      if (la >= 0) Y[(row + r) + (int64_t)la * nr] = Rg[(int64_t)r * s + a] * w;
    }
    row += rk;
  }
  tm.sync();
  const int warp = tm.rank >> 5, lane = (int)threadIdx.x & 31, nw = tm.size >> 5;
  const int ng = m - no;
  const int kmax = min(nr, ng);
  const double tol = (double)max(nr, ng) * DBL_EPSILON;
  double c1 = 0.0;
  int r = 0;
  for (int k = 0; k < kmax; ++k) {
    // squared norms of the live Gamma columns over rows k.., a warp per column
    for (int j = no + k + warp; j < m; j += nw) {
      const double* cj = Y + (int64_t)j * nr;
      double acc = 0.0;
      for (int i = k + lane; i < nr; i += 32) acc += cj[i] * cj[i];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
      if (lane == 0) nrm[j] = acc;
    }
    tm.sync();
    if (threadIdx.x < 32) {  // every CTA picks the same pivot from the same norms
      double best = -1.0;
      int bi = m;
      for (int j = no + k + (int)threadIdx.x; j < m; j += 32) {
        const double d = nrm[j];
        if (d > best || (d == best && j < bi)) {
          best = d;
          bi = j;
        }
      }
      best = warp_max_idx(best, bi);
      if (threadIdx.x == 0) {
        s_best = best;
        s_bi = bi;
      }
    }
    __syncthreads();
    const double nb2 = s_best;
    const int pj = s_bi;
    const double xn = sqrt(fmax(nb2, 0.0));
    if (k == 0) c1 = xn;
    if (!(xn > tol * c1)) break;
    const int c = no + k;
    if (pj != c)
      for (int i = tm.rank; i < nr; i += tm.size) {
        const double t = Y[i + (int64_t)c * nr];
        Y[i + (int64_t)c * nr] = Y[i + (int64_t)pj * nr];
        Y[i + (int64_t)pj * nr] = t;
      }
    tm.sync();
    const double* xk = Y + (int64_t)c * nr;
    const double x0 = xk[k];
    const double alpha = x0 >= 0.0 ? -xn : xn;
    const double v0 = x0 - alpha;
    const double vtv = v0 * v0 + (nb2 - x0 * x0);
    if (vtv > 0.0) {
      // the omega columns and the Gamma columns after c
      const int nupd = no + (m - c - 1);
      for (int jj = warp; jj < nupd; jj += nw) {
        const int j = jj < no ? jj : c + 1 + (jj - no);
        double* cj = Y + (int64_t)j * nr;
        double acc = lane == 0 ? v0 * cj[k] : 0.0;
        for (int i = k + 1 + lane; i < nr; i += 32) acc += xk[i] * cj[i];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        const double f = 2.0 * acc / vtv;
        if (lane == 0) cj[k] -= f * v0;
        for (int i = k + 1 + lane; i < nr; i += 32) cj[i] -= f * xk[i];
      }
    }
    tm.sync();
    r = k + 1;
  }
  if (tm.rank == 0) rank_out[b] = r;
  // S~ = X_2^T X_2 over rows r.. (the same sum order for (a, c) and (c, a))
  double* At = Atpool + a_off[b];
  for (int64_t e = tm.rank; e < (int64_t)no * no; e += tm.size) {
    const int a = (int)(e % no), cc = (int)(e / no);
    const double* ya = Y + (int64_t)a * nr;
    const double* yc = Y + (int64_t)cc * nr;
    double acc = 0.0;
    for (int i = r; i < nr; ++i) acc += ya[i] * yc[i];
    At[a + (int64_t)cc * m] = acc;
  }
}

int threads_for(int64_t work) { return work <= 64 ? 64 : (work <= 1024 ? 128 : 256); }

}  // namespace

// ---------------------------------------------------------------------------
int launch_gram_rows(int64_t ngroups, const int64_t* g_row0, const int64_t* g_row1, const int64_t* g_ptr,
                     const int64_t* h_off, const int64_t* rowptr, const double* val, double* H, cudaStream_t s) {
  const int64_t chunk = 1 << 20;
  for (int64_t f = 0; f < ngroups; f += chunk) {
    const int64_t c = ngroups - f < chunk ? ngroups - f : chunk;
    k_gram_rows<<<(unsigned)c, 64, 0, s>>>(f, g_row0, g_row1, g_ptr, h_off, rowptr, val, H);
    AMGDD_CUDA(cudaGetLastError());
  }
  return AMGDD_OK;
}

int launch_gram_diag(int64_t n, int64_t first_group, const int64_t* h_off, const double* D1, double* H,
                     cudaStream_t s) {
  if (n == 0) return AMGDD_OK;
  k_gram_diag<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, first_group, h_off, D1, H);
  AMGDD_CUDA(cudaGetLastError());
  count_kernels(1);
  return AMGDD_OK;
}

int launch_pchol(int64_t first, int64_t count, int max_s, const int64_t* g_ptr, const int64_t* h_off,
                 const double* H, double* R64, float* R32, int32_t* rank, double* scratch, int64_t scratch_per,
                 cudaStream_t s) {
  if (count == 0) return AMGDD_OK;
  const size_t smem = (size_t)max_s * sizeof(int);
  if (smem > 48 * 1024) AMGDD_CUDA(cudaFuncSetAttribute(k_pchol, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_pchol<<<(unsigned)count, threads_for((int64_t)max_s * max_s), smem, s>>>(first, g_ptr, h_off, H, R64, R32, rank,
                                                                             scratch, scratch_per);
  AMGDD_CUDA(cudaGetLastError());
  count_kernels(1);
  return AMGDD_OK;
}

int launch_assemble(int nb, int max_m, const LocalBatch& b, const int64_t* g_ptr, const int64_t* h_off,
                    const double* H, const int32_t* M, double* Apool, double* Atpool, cudaStream_t s) {
  if (nb == 0) return AMGDD_OK;
  k_assemble<<<nb, threads_for((int64_t)max_m * max_m), 0, s>>>(b.m.p, b.a_off.p, b.pair_ptr.p, b.pair_grp.p,
                                                                b.pair_nz.p, b.map_ptr.p, b.map.p, g_ptr, h_off, H, M,
                                                                Apool, Atpool);
  AMGDD_CUDA(cudaGetLastError());
  count_kernels(1);
  return AMGDD_OK;
}

template <class K, class... Args>
int launch_team(K kern, int CL, int nb, int threads, size_t smem, cudaStream_t s, Args... args) {
  if (smem > 48 * 1024) AMGDD_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(nb * CL));
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = CL > 1 ? 1 : 0;
  AMGDD_CUDA(cudaLaunchKernelEx(&cfg, kern, args...));
  count_kernels(1);
  return AMGDD_OK;
}

constexpr int kBigTeam = 8;   // CTAs per large matrix (portable cluster size)
constexpr int kBigDim = 160;  // matrices at least this large use a cluster team
constexpr int kHugeTeam = 16;  // CTAs per large matrix when a batch has too few to fill the GPU with teams of 8

// A batch of nb large matrices takes teams of 16 (a non-portable cluster
// size) when nb teams of 16 still fit the SMs and the device can place a
// 16-CTA cluster of this kernel; else teams of 8.
template <class K>
bool huge_team(K kern, int nb, int threads, size_t smem) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return false;
  if (nb * kHugeTeam > sms) return false;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)kHugeTeam);
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)kHugeTeam;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int clusters = 0;
  if (cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return clusters >= 1;
}

int launch_chol(int nb, int max_m, const int32_t* m, const int64_t* a_off, double* Apool, int32_t* status,
                cudaStream_t s) {
  if (nb == 0) return AMGDD_OK;
  if (max_m >= kBigDim) {
    if (huge_team(k_chol<kHugeTeam>, nb, 256, 0))
      return launch_team(k_chol<kHugeTeam>, kHugeTeam, nb, 256, 0, s, m, a_off, Apool, status);
    return launch_team(k_chol<kBigTeam>, kBigTeam, nb, 256, 0, s, m, a_off, Apool, status);
  }
  return launch_team(k_chol<1>, 1, nb, threads_for((int64_t)max_m * max_m), 0, s, m, a_off, Apool, status);
}

int launch_schur(int nb, int max_m, const int32_t* m, const int32_t* no, const int64_t* a_off, double* Atpool,
                 double rtol, cudaStream_t s) {
  if (nb == 0) return AMGDD_OK;
  const size_t smem = (size_t)max_m * sizeof(int);
  if (max_m >= kBigDim) {
    if (huge_team(k_schur<kHugeTeam>, nb, 256, smem))
      return launch_team(k_schur<kHugeTeam>, kHugeTeam, nb, 256, smem, s, m, no, a_off, Atpool, rtol);
    return launch_team(k_schur<kBigTeam>, kBigTeam, nb, 256, smem, s, m, no, a_off, Atpool, rtol);
  }
  return launch_team(k_schur<1>, 1, nb, threads_for((int64_t)max_m * max_m), smem, s, m, no, a_off, Atpool, rtol);
}

int launch_inv_rows(int nb, int max_m, const int32_t* m, const int32_t* no, const int64_t* a_off,
                    const double* Lpool, const int64_t* w_off, double* W64, float* W32, double* Wt64, float* Wt32,
                    double* scratch, const int32_t* chunk_b, const int32_t* chunk_c0, int nchunks, int cw,
                    cudaStream_t s) {
  if (nb == 0 || nchunks == 0) return AMGDD_OK;
  k_inv_rows<<<nchunks, threads_for((int64_t)max_m * cw), 0, s>>>(chunk_b, chunk_c0, cw, m, no, a_off, Lpool, w_off,
                                                                  W64, W32, Wt64, Wt32, scratch);
  AMGDD_CUDA(cudaGetLastError());
  count_kernels(1);
  return AMGDD_OK;
}


int launch_gep(int nb, int max_no, const int32_t* m, const int32_t* no, const int64_t* a_off, const double* Lpool,
               const double* Spool, const int32_t* cap, double thresh, const int64_t* mu_off, double* mu,
               const int64_t* z_off_cap, double* Zcap, int32_t* kout, double* scratch, const int64_t* scr_off,
               int32_t* work_out, cudaStream_t s) {
  if (nb == 0) return AMGDD_OK;
  const size_t smem = (size_t)(2 * (max_no + 1)) * sizeof(double) + (size_t)(max_no + 1) * sizeof(int);
  if (gep_uses_ql(max_no)) {
    // QL: shared copies of d, e and one sweep's rotations (4 doubles and an int per row) when they fit
    const size_t smem_q = (size_t)max_no * (4 * sizeof(double) + sizeof(int)) + 64;
    const int shq = smem_q <= (size_t)200 * 1024 ? 1 : 0;
    const size_t sm = shq ? std::max(smem, smem_q) : smem;
    if (huge_team(k_gep<kHugeTeam, true>, nb, 256, sm))
      return launch_team(k_gep<kHugeTeam, true>, kHugeTeam, nb, 256, sm, s, m, no, a_off, Lpool, Spool, cap,
                         thresh, mu_off, mu, z_off_cap, Zcap, kout, scratch, scr_off, work_out, shq);
    return launch_team(k_gep<kBigTeam, true>, kBigTeam, nb, 256, sm, s, m, no, a_off, Lpool, Spool, cap, thresh,
                       mu_off, mu, z_off_cap, Zcap, kout, scratch, scr_off, work_out, shq);
  }
  return launch_team(k_gep<1, false>, 1, nb, threads_for((int64_t)max_no * max_no), smem, s, m, no, a_off, Lpool,
                     Spool, cap, thresh, mu_off, mu, z_off_cap, Zcap, kout, scratch, scr_off, work_out, 0);
}

bool gep_uses_ql(int max_no) { return max_no >= kBigDim; }

namespace {
// Independent FMA chains: 8 per thread, `iters` steps each (2 flops per FMA).
__global__ void k_fp64_rate(double* out, int iters, double a, double b) {
  double v[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) v[k] = (double)(threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = fma(v[k], a, b);
  }
  double t = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) t += v[k];
  if (t == 12345.678) out[0] = t;  // keeps the chains live; never true for these inputs
}
}  // namespace

int measure_fp64_rate(cudaStream_t s, double* gflops) {
  DBuf<double> out;
  AMGDD_TRY(out.alloc(1));
  const int blocks = 152 * 8, threads = 256, iters = 4096;
  cudaEvent_t e[2];
  for (auto& v : e) AMGDD_CUDA(cudaEventCreate(&v));
  float best = 0.f;
  int rc = AMGDD_OK;
  for (int rep = 0; rep < 4 && rc == AMGDD_OK; ++rep) {
    cudaEventRecord(e[0], s);
    k_fp64_rate<<<blocks, threads, 0, s>>>(out.p, iters, 0.999999, 1e-7);
    cudaEventRecord(e[1], s);
    float ms = 0.f;
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e[1]) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e[0], e[1]) != cudaSuccess)
      rc = AMGDD_ERR_CUDA;
    count_kernels(1);
    if (rep > 0 && (best == 0.f || ms < best)) best = ms;
  }
  for (auto& v : e) cudaEventDestroy(v);
  AMGDD_TRY(rc);
  *gflops = 2.0 * 8.0 * (double)iters * blocks * threads / (best * 1e-3) / 1e9;
  return AMGDD_OK;
}

int launch_pack_z(int nb, const int32_t* no, const int32_t* k, const int64_t* z_off_cap, const double* Zcap,
                  const int64_t* z_off, double* Z64, float* Z32, double* Zt64, float* Zt32, cudaStream_t s) {
  if (nb == 0) return AMGDD_OK;
  k_pack_z<<<nb, 128, 0, s>>>(no, k, z_off_cap, Zcap, z_off, Z64, Z32, Zt64, Zt32);
  AMGDD_CUDA(cudaGetLastError());
  count_kernels(1);
  return AMGDD_OK;
}

int launch_next_gram(const NextGramPlan& p, int max_sn, const int64_t* g_ptr, const int64_t* h_off, const double* H,
                     const double* Z64, double* Hn, double* scratch, int64_t first, int64_t count, cudaStream_t s) {
  if (count == 0) return AMGDD_OK;
  k_next_gram<<<(unsigned)count, threads_for((int64_t)max_sn * max_sn), 0, s>>>(
      first, p.new_ptr.p, p.contrib.p, p.new_sptr.p, p.new_hoff.p, p.rowz_ptr.p, p.rowz_zoff.p, p.rowz_k.p,
      p.rowz_col.p, g_ptr, h_off, H, Z64, Hn, scratch, p.scratch_per);
  AMGDD_CUDA(cudaGetLastError());
  count_kernels(1);
  return AMGDD_OK;
}

int launch_next_rows(const NextGramPlan& p, const int64_t* g_ptr, const int64_t* h_off, const int32_t* rank,
                     const double* R, const double* Z64, const int64_t* t_off, double* scratch, double* Rn64,
                     float* Rn32, int32_t* rank_out, int64_t first, int64_t count, bool team, cudaStream_t s) {
  if (count == 0) return AMGDD_OK;
  DBuf<double> red;
  AMGDD_TRY(red.alloc(count * kHugeTeam));
  // cluster teams for large stacked blocks (3D coarse levels), a CTA each otherwise
  if (team && huge_team(k_next_rows<kHugeTeam>, (int)count, 256, 0))
    return launch_team(k_next_rows<kHugeTeam>, kHugeTeam, (int)count, 256, 0, s, first, p.new_ptr.p, p.contrib.p,
                       p.new_sptr.p, p.new_hoff.p, p.rowz_ptr.p, p.rowz_zoff.p, p.rowz_k.p, p.rowz_col.p, g_ptr,
                       h_off, rank, R, Z64, t_off, scratch, Rn64, Rn32, rank_out, red.p);
  if (team)
    return launch_team(k_next_rows<kBigTeam>, kBigTeam, (int)count, 256, 0, s, first, p.new_ptr.p, p.contrib.p,
                       p.new_sptr.p, p.new_hoff.p, p.rowz_ptr.p, p.rowz_zoff.p, p.rowz_k.p, p.rowz_col.p, g_ptr,
                       h_off, rank, R, Z64, t_off, scratch, Rn64, Rn32, rank_out, red.p);
  return launch_team(k_next_rows<1>, 1, (int)count, 256, 0, s, first, p.new_ptr.p, p.contrib.p, p.new_sptr.p,
                     p.new_hoff.p, p.rowz_ptr.p, p.rowz_zoff.p, p.rowz_k.p, p.rowz_col.p, g_ptr, h_off, rank, R, Z64,
                     t_off, scratch, Rn64, Rn32, rank_out, red.p);
}

int launch_schur_rows(int nb, int max_m, const LocalBatch& b, const int64_t* g_ptr, const int64_t* h_off,
                      const int32_t* rank, const double* R, const int32_t* M, const int64_t* y_off,
                      const int32_t* y_rows, double* Ypool, const int64_t* n_off, double* nrm, double* Atpool,
                      int32_t* rank_out, bool team, cudaStream_t s) {
  if (nb == 0) return AMGDD_OK;
  // cluster teams for large row blocks (each reflection streams the whole
  // block; a CTA alone would take seconds on a 3D coarse level) or while the
  // batch leaves SMs idle; with many small matrices a CTA each keeps every
  // SM busy without the team's barriers
  if (max_m >= kBigDim && (team || nb * kBigTeam <= 2 * 152) && huge_team(k_schur_rows<kHugeTeam>, nb, 256, 0))
    return launch_team(k_schur_rows<kHugeTeam>, kHugeTeam, nb, 256, 0, s, b.m.p, b.no.p, b.a_off.p, b.pair_ptr.p,
                       b.pair_grp.p, b.pair_nz.p, b.map_ptr.p, b.map.p, g_ptr, h_off, rank, R, M, y_off, y_rows,
                       Ypool, n_off, nrm, Atpool, rank_out);
  if (max_m >= kBigDim && (team || nb * kBigTeam <= 2 * 152))
    return launch_team(k_schur_rows<kBigTeam>, kBigTeam, nb, 256, 0, s, b.m.p, b.no.p, b.a_off.p, b.pair_ptr.p,
                       b.pair_grp.p, b.pair_nz.p, b.map_ptr.p, b.map.p, g_ptr, h_off, rank, R, M, y_off, y_rows,
                       Ypool, n_off, nrm, Atpool, rank_out);
  return launch_team(k_schur_rows<1>, 1, nb, max_m >= 64 ? 256 : 128, 0, s, b.m.p, b.no.p, b.a_off.p, b.pair_ptr.p,
                     b.pair_grp.p,
                     b.pair_nz.p, b.map_ptr.p, b.map.p, g_ptr, h_off, rank, R, M, y_off, y_rows, Ypool, n_off, nrm,
                     Atpool, rank_out);
}

namespace {
// One CTA per block of consecutive dofs D_b = d0 .. d0+nr_b-1 sharing the
// row support in_b: A(D_b, in_b) = sum over the groups g whose support holds
// D_b of rows p0_g .. p0_g+nr_b-1 of H_g (Eq. 1: A = sum_g G_g^T G_g), each
// group's columns scattered to their positions in in_b.  Groups are summed in
// a fixed order, so the result is deterministic.  Also writes the FP32 copy
// and the block-wise transposes.
__global__ void k_blockrows(const int32_t* __restrict__ nr, const int32_t* __restrict__ nc,
                            const int64_t* __restrict__ m_off, const int64_t* __restrict__ pair_ptr,
                            const int32_t* __restrict__ pair_grp, const int32_t* __restrict__ pair_p0,
                            const int64_t* __restrict__ pair_map, const int32_t* __restrict__ map,
                            const int64_t* __restrict__ g_ptr, const int64_t* __restrict__ h_off,
                            const double* __restrict__ H, double* __restrict__ A64, float* __restrict__ A32,
                            double* __restrict__ At64, float* __restrict__ At32) {
  const int b = blockIdx.x;
  const int kb = nr[b], nin = nc[b];
  const int64_t len = (int64_t)kb * nin;
  double* Ab = A64 + m_off[b];
  for (int64_t e = threadIdx.x; e < len; e += blockDim.x) Ab[e] = 0.0;
  __syncthreads();
  for (int64_t q = pair_ptr[b]; q < pair_ptr[b + 1]; ++q) {
    const int g = pair_grp[q];
    const int sg = (int)(g_ptr[g + 1] - g_ptr[g]);
    const double* Hg = H + h_off[g] + (int64_t)pair_p0[q] * sg;
    const int32_t* mp = map + pair_map[q];
    for (int64_t e = threadIdx.x; e < (int64_t)kb * sg; e += blockDim.x) {
      const int r = (int)(e / sg), c = (int)(e - (int64_t)r * sg);
      Ab[(int64_t)r * nin + mp[c]] += Hg[(int64_t)r * sg + c];
    }
    __syncthreads();
  }
  for (int64_t e = threadIdx.x; e < len; e += blockDim.x) {
    const int r = (int)(e / nin), c = (int)(e - (int64_t)r * nin);
    const double v = Ab[e];
    A32[m_off[b] + e] = (float)v;
    At64[m_off[b] + (int64_t)c * kb + r] = v;
    At32[m_off[b] + (int64_t)c * kb + r] = (float)v;
  }
}
}  // namespace

int launch_blockrows(int nblk, const int32_t* nr, const int32_t* nc, const int64_t* m_off, const int64_t* pair_ptr,
                     const int32_t* pair_grp, const int32_t* pair_p0, const int64_t* pair_map, const int32_t* map,
                     const int64_t* g_ptr, const int64_t* h_off, const double* H, double* A64, float* A32,
                     double* At64, float* At32, cudaStream_t s) {
  if (nblk == 0) return AMGDD_OK;
  k_blockrows<<<nblk, 256, 0, s>>>(nr, nc, m_off, pair_ptr, pair_grp, pair_p0, pair_map, map, g_ptr, h_off, H, A64,
                                   A32, At64, At32);
  AMGDD_CUDA(cudaGetLastError());
  count_kernels(1);
  return AMGDD_OK;
}

namespace {
// Rows omega_i of the assembled A_i = A(Omega_i, Omega_i) (symmetric, so row
// r is contiguous), in the layout of the smoother rows W_i: A(omega_i,
// Omega_i) row-major at w_off and its block transpose.  The residual of
// rows omega_i reads exactly these, since Omega_i holds their support.
__global__ void k_copy_wrows(const int32_t* __restrict__ mdim, const int32_t* __restrict__ nodim,
                             const int64_t* __restrict__ a_off, const double* __restrict__ Apool,
                             const int64_t* __restrict__ w_off, double* __restrict__ Aw64, float* __restrict__ Aw32,
                             double* __restrict__ AwT64, float* __restrict__ AwT32) {
  const int b = blockIdx.x;
  const int m = mdim[b], no = nodim[b];
  const double* A = Apool + a_off[b];
  const int64_t o = w_off[b];
  for (int64_t e = threadIdx.x; e < (int64_t)no * m; e += blockDim.x) {
    const int r = (int)(e / m), c = (int)(e - (int64_t)r * m);
    const double v = A[e];
    Aw64[o + e] = v;
    Aw32[o + e] = (float)v;
    AwT64[o + (int64_t)c * no + r] = v;
    AwT32[o + (int64_t)c * no + r] = (float)v;
  }
}

// ELL values of level 0 from the rows omega_i of A over Omega_i: entry e
// takes Aw64[src[e]] (0 where src[e] < 0, an unused slot).
__global__ void k_ell_fill(int64_t total, const int64_t* __restrict__ src, const double* __restrict__ Aw64,
                           double* __restrict__ v64, float* __restrict__ v32) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = src[e];
    const double v = o >= 0 ? Aw64[o] : 0.0;
    v64[e] = v;
    v32[e] = (float)v;
  }
}

// Dense tail matrices: from C (row j = B e_j, i.e. C = B^T row-major, n x n)
// write B row-major with leading dimension ld >= n (columns n..ld-1 zero) in
// FP64 and FP32.  32 x 32 tiles through shared memory, 32 x 8 threads.
__global__ void k_dense_pack(const double* __restrict__ C, int n, int64_t ld, double* __restrict__ B64,
                             float* __restrict__ B32) {
  __shared__ double t[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += 8) {
    const int r = by + k, c = bx + threadIdx.x;
    t[k][threadIdx.x] = (r < n && c < n) ? C[(int64_t)r * n + c] : 0.0;
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += 8) {
    const int r = bx + k, c = by + threadIdx.x;
    if (r < n && c < ld) {
      const double v = t[threadIdx.x][k];
      B64[(int64_t)r * ld + c] = v;
      B32[(int64_t)r * ld + c] = (float)v;
    }
  }
}
}  // namespace

int launch_ell_fill(int64_t total, const int64_t* src, const double* Aw64, double* v64, float* v32,
                    cudaStream_t s) {
  if (total <= 0) return AMGDD_OK;
  const int grid = (int)std::min<int64_t>((total + 255) / 256, 152 * 16);
  k_ell_fill<<<grid, 256, 0, s>>>(total, src, Aw64, v64, v32);
  AMGDD_CUDA(cudaGetLastError());
  count_kernels(1);
  return AMGDD_OK;
}

int launch_dense_pack(const double* C, int n, int64_t ld, double* B64, float* B32, cudaStream_t s) {
  if (n <= 0) return AMGDD_OK;
  // x: tiles of B's rows (C's columns), y: tiles of B's columns (C's rows)
  const dim3 grid((unsigned)((n + 31) / 32), (unsigned)((ld + 31) / 32)), block(32, 8);
  k_dense_pack<<<grid, block, 0, s>>>(C, n, ld, B64, B32);
  AMGDD_CUDA(cudaGetLastError());
  count_kernels(1);
  return AMGDD_OK;
}

// The derived copies of stored blocks (a loaded hierarchy): block b is
// rows[b] x cols[b], row-major at off[b] in src; dst32 receives its FP32
// rounding, dstT64 / dstT32 its transpose (cols x rows, row-major, same
// offset) in FP64 / FP32.  Null outputs are skipped.
__global__ void k_block_copies(const int32_t* __restrict__ rows, const int32_t* __restrict__ cols,
                               const int64_t* __restrict__ off, const double* __restrict__ src,
                               float* __restrict__ dst32, double* __restrict__ dstT64, float* __restrict__ dstT32) {
  const int b = blockIdx.x;
  const int nr = rows[b], nc = cols[b];
  const int64_t o = off[b];
  for (int64_t e = threadIdx.x; e < (int64_t)nr * nc; e += blockDim.x) {
    const int r = (int)(e / nc), c = (int)(e - (int64_t)r * nc);
    const double v = src[o + e];
    if (dst32) dst32[o + e] = (float)v;
    if (dstT64) dstT64[o + (int64_t)c * nr + r] = v;
    if (dstT32) dstT32[o + (int64_t)c * nr + r] = (float)v;
  }
}

int launch_block_copies(int nb, const int32_t* rows, const int32_t* cols, const int64_t* off, const double* src,
                        float* dst32, double* dstT64, float* dstT32, cudaStream_t s) {
  if (nb == 0) return AMGDD_OK;
  k_block_copies<<<nb, 256, 0, s>>>(rows, cols, off, src, dst32, dstT64, dstT32);
  AMGDD_CUDA(cudaGetLastError());
  count_kernels(1);
  return AMGDD_OK;
}

int launch_copy_wrows(int nb, const int32_t* m, const int32_t* no, const int64_t* a_off, const double* Apool,
                      const int64_t* w_off, double* Aw64, float* Aw32, double* AwT64, float* AwT32, cudaStream_t s) {
  if (nb == 0) return AMGDD_OK;
  k_copy_wrows<<<nb, 256, 0, s>>>(m, no, a_off, Apool, w_off, Aw64, Aw32, AwT64, AwT32);
  AMGDD_CUDA(cudaGetLastError());
  count_kernels(1);
  return AMGDD_OK;
}

}  // namespace amgdd
