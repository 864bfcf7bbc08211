// Standard aggregation on the device (Section 2.1's three passes, every edge
// strong; Section 3.3 repeats them on the aggregates).
//
// The passes visit the vertices in ascending order, yet each is fixed by an
// order-independent rule, so every vertex can decide in parallel rounds:
//
// * Pass 1 makes j a root when none of its neighbours is aggregated at its
//   visit.  A vertex is aggregated only by a root at distance <= 1, so j is a
//   root exactly when no lower-index root lies within distance 2: the roots
//   are the lexicographically first maximal independent set of the
//   distance-2 graph.  A round decides vertex v as OUT once a root lies
//   within distance 2, and as a ROOT once every lower-index vertex within
//   distance 2 is decided (then none of them is a root).  The smallest
//   undecided vertex decides in every round, so the rounds end.  Roots take
//   ids in ascending order and lend them to their neighbours (two roots are
//   at distance >= 3, so no vertex has two).
// * Pass 2 reads only pass 1's result: a vertex left over joins the
//   aggregate of its lowest-index neighbour aggregated in pass 1.
// * Pass 3 makes a leftover j a new root when no lower-index leftover
//   neighbour became one (the first maximal independent set of the graph
//   induced on the leftovers), and a leftover that is not a root joins the
//   lowest-index adjacent pass-3 root (the first to claim it).  With every
//   edge strong there are no leftovers (a vertex that is not a root had a
//   neighbour aggregated at its visit, so pass 2 places it); the pass stays
//   for completeness and costs one count when it has nothing to do.
//
// The graph is given by hyperedges (vertices adjacent when an edge holds
// both: the rows of G, or the aggregates a row touches); neighbourhoods are
// walked through the vertex -> edge incidence, and every test is an "any"
// or a "min", so repeated members and repeated edges change nothing.  The
// ids equal those of the sequential passes, vertex for vertex.
//
// Pass 1 takes one full round over every vertex, then rounds over the
// frontier only (the vertices whose inputs a change of the previous round
// touched), all of them in one cooperative launch with a bounded grid
// barrier between the two phases of a round.  The visiting order makes the
// rounds a dependent chain (about 2N of them on an N x N grid), each short
// and latency-bound.
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>
#include <vector>

#include "device_util.cuh"
#include "internal.h"

namespace amgdd {

namespace {

constexpr int8_t kUnd = 0, kRoot = 1, kOut = 2, kNone = 3;  // kNone: not a pass-3 candidate
constexpr int kThreads = 256;
constexpr int kScan = 1024;

int grid1(int64_t n) {
  const int64_t g = (n + kThreads - 1) / kThreads;
  return (int)std::min<int64_t>(std::max<int64_t>(g, 1), 152 * 32);
}

#define FOR_V(v, n) for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < (n); v += (int64_t)gridDim.x * blockDim.x)

// ---- exclusive scan of int32 counts into int64 offsets (n + 1 entries) ----
__global__ void __launch_bounds__(kScan) k_scan_block(const int32_t* __restrict__ in, int64_t n,
                                                      int64_t* __restrict__ out, int64_t* __restrict__ bsum) {
  __shared__ int64_t wsum[32];
  const int64_t i = (int64_t)blockIdx.x * kScan + threadIdx.x;
  const int64_t x = i < n ? (int64_t)in[i] : 0;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int64_t v = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  if (lane == 31) wsum[w] = v;
  __syncthreads();
  if (w == 0) {
    int64_t s = wsum[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t t = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += t;
    }
    wsum[lane] = s;  // inclusive over warps
  }
  __syncthreads();
  const int64_t before = w > 0 ? wsum[w - 1] : 0;
  if (i < n) out[i] = before + v - x;
  if (threadIdx.x == kScan - 1) bsum[blockIdx.x] = wsum[31];
}

// One CTA: exclusive scan of the block totals in chunks; out[n] = total.
__global__ void __launch_bounds__(kScan) k_scan_totals(int64_t* __restrict__ bsum, int64_t nb, int64_t* __restrict__ out,
                                                       int64_t n) {
  __shared__ int64_t wsum[32];
  __shared__ int64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int64_t c0 = 0; c0 < nb; c0 += kScan) {
    const int64_t i = c0 + threadIdx.x;
    const int64_t x = i < nb ? bsum[i] : 0;
    int64_t v = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t t = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += t;
    }
    if (lane == 31) wsum[w] = v;
    __syncthreads();
    if (w == 0) {
      int64_t s = wsum[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int64_t t = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += t;
      }
      wsum[lane] = s;
    }
    __syncthreads();
    const int64_t before = (w > 0 ? wsum[w - 1] : 0) + carry;
    if (i < nb) bsum[i] = before + v - x;
    __syncthreads();
    if (threadIdx.x == 0) carry += wsum[31];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[n] = carry;
}

__global__ void k_scan_add(int64_t* __restrict__ out, int64_t n, const int64_t* __restrict__ bsum) {
  FOR_V(i, n) out[i] += bsum[i / kScan];
}

// out (n + 1) = exclusive prefix sums of in (n); out[n] = the total.
int scan_counts(const int32_t* in, int64_t n, int64_t* out, cudaStream_t s) {
  const int64_t nb = std::max<int64_t>((n + kScan - 1) / kScan, 1);
  DBuf<int64_t> bsum;
  AMGDD_TRY(bsum.alloc(nb));
  k_scan_block<<<(unsigned)nb, kScan, 0, s>>>(in, n, out, bsum.p);
  k_scan_totals<<<1, kScan, 0, s>>>(bsum.p, nb, out, n);
  k_scan_add<<<grid1(n), kThreads, 0, s>>>(out, n, bsum.p);
  AMGDD_CUDA(cudaGetLastError());
  count_kernels(3);
  AMGDD_CUDA(cudaStreamSynchronize(s));  // bsum is released on return
  return AMGDD_OK;
}

// ---- vertex -> edge incidence ---------------------------------------------
__global__ void k_inc_count(int64_t total, const int32_t* __restrict__ eidx, int32_t* __restrict__ cnt) {
  FOR_V(q, total) atomicAdd(&cnt[eidx[q]], 1);
}

__global__ void k_inc_fill(int64_t ne, const int64_t* __restrict__ eptr, const int32_t* __restrict__ eidx,
                           const int64_t* __restrict__ vptr, int32_t* __restrict__ cursor, int32_t* __restrict__ ve) {
  FOR_V(e, ne) {
    for (int64_t q = eptr[e]; q < eptr[e + 1]; ++q) {
      const int32_t v = eidx[q];
      ve[vptr[v] + atomicAdd(&cursor[v], 1)] = (int32_t)e;
    }
  }
}

// The graph as the kernels walk it: vertex u's closed neighbourhood is u and
// the members of the edges listed in ve[vptr[u] .. vptr[u + 1]).
struct HGraph {
  const int64_t* vptr;
  const int32_t* ve;
  const int64_t* eptr;
  const int32_t* eidx;
};

// ---- pass 1 ----------------------------------------------------------------
// Per vertex u: near[u] = some vertex of u's closed neighbourhood is a root;
// mu[u] = the lowest undecided vertex there (INT_MAX if none).
__device__ __forceinline__ void p1_inputs(int64_t u, const HGraph& g, const int8_t* __restrict__ st, bool& nr,
                                          int32_t& m) {
  const int8_t su = st[u];
  nr = su == kRoot;
  m = su == kUnd ? (int32_t)u : INT_MAX;
  for (int64_t k = g.vptr[u]; k < g.vptr[u + 1]; ++k) {
    const int32_t e = g.ve[k];
    for (int64_t q = g.eptr[e]; q < g.eptr[e + 1]; ++q) {
      const int32_t w = g.eidx[q];
      const int8_t sw = st[w];
      nr = nr || sw == kRoot;
      if (sw == kUnd && w < m) m = w;
    }
  }
}

// Undecided v: OUT if a root lies within distance 2; ROOT if v is the lowest
// undecided vertex of every closed neighbourhood it belongs to (no lower
// undecided vertex within distance 2); else still undecided.
__device__ __forceinline__ int8_t p1_decision(int64_t v, const HGraph& g, const int8_t* __restrict__ near,
                                              const int32_t* __restrict__ mu) {
  bool out = near[v] != 0;
  bool root = !out && mu[v] == (int32_t)v;
  for (int64_t k = g.vptr[v]; k < g.vptr[v + 1] && !out; ++k) {
    const int32_t e = g.ve[k];
    for (int64_t q = g.eptr[e]; q < g.eptr[e + 1]; ++q) {
      const int32_t w = g.eidx[q];
      if (near[w]) {
        out = true;
        break;
      }
      if (mu[w] != (int32_t)v) root = false;
    }
  }
  return out ? kOut : (root ? kRoot : kUnd);
}

// The frontier of the rounds after the first: a vertex's inputs change only
// when a vertex of its closed neighbourhood changed, so each round revisits
// only those.  F1 lists the vertices whose near/mu to recompute, F2 the
// undecided vertices whose decision to redo; both are deduplicated by
// stamps (the round that last pushed the vertex).  Counts by round parity:
// cnt[0..1] for F1, cnt[2..3] for F2; each kernel clears the slot of the
// list that the next kernel fills.
struct Front {
  int32_t* f1[2];
  int32_t* f2[2];
  int* cnt;
  int32_t* s1;
  int32_t* s2;
};

__device__ __forceinline__ void push(int32_t* list, int* cnt, int32_t* stamp, int32_t v, int32_t tag) {
  if (atomicExch(&stamp[v], tag) != tag) list[atomicAdd(cnt, 1)] = v;
}

__device__ __forceinline__ void push_closed(int64_t v, const HGraph& g, int32_t* list, int* cnt, int32_t* stamp,
                                            int32_t tag, const int8_t* __restrict__ st_und) {
  // the closed neighbourhood of v (only its undecided vertices when st_und is given)
  if (!st_und || st_und[v] == kUnd) push(list, cnt, stamp, (int32_t)v, tag);
  for (int64_t k = g.vptr[v]; k < g.vptr[v + 1]; ++k) {
    const int32_t e = g.ve[k];
    for (int64_t q = g.eptr[e]; q < g.eptr[e + 1]; ++q) {
      const int32_t w = g.eidx[q];
      if (w != (int32_t)v && (!st_und || st_und[w] == kUnd)) push(list, cnt, stamp, w, tag);
    }
  }
}

// Round 0, every vertex: near and mu.
__global__ void k_p1_inputs_all(int64_t nv, HGraph g, const int8_t* __restrict__ st, int8_t* __restrict__ near,
                                int32_t* __restrict__ mu) {
  FOR_V(u, nv) {
    bool nr;
    int32_t m;
    p1_inputs(u, g, st, nr, m);
    near[u] = nr ? 1 : 0;
    mu[u] = m;
  }
}

// Round 0, every vertex: the decisions; the closed neighbourhoods of the
// vertices that decided form F1 of round 1.
__global__ void k_p1_decide_all(int64_t nv, HGraph g, const int8_t* __restrict__ near, const int32_t* __restrict__ mu,
                                int8_t* __restrict__ st, Front F) {
  FOR_V(v, nv) {
    if (st[v] != kUnd) continue;
    const int8_t ns = p1_decision(v, g, near, mu);
    if (ns == kUnd) continue;
    st[v] = ns;
    push_closed(v, g, F.f1[1], &F.cnt[1], F.s1, 1, nullptr);
  }
}

// The frontier rounds 1, 2, ... in one cooperative launch: each round is the
// two phases above, each closed by the bounded grid barrier; the launch ends
// once a round decided nothing (every CTA reads the same count after the
// barrier) or after max_rounds.  Data that other CTAs write during the launch
// (states, near/mu, lists, counts) is read through L2 (__ldcg).
__global__ void __launch_bounds__(512) k_p1_frontier(HGraph g, int8_t* st, int8_t* near, int32_t* mu, Front F,
                                                     int max_rounds, unsigned* bar, int* err, int* rounds_out) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
  volatile int* verr = err;
  int r = 1;
  for (; r <= max_rounds; ++r) {
    // near/mu of F1; undecided neighbourhoods of the changed ones into F2
    const int n1 = __ldcg(&F.cnt[r & 1]);
    if (tid == 0) F.cnt[(r + 1) & 1] = 0;
    for (int i = tid; i < n1; i += nth) {
      const int32_t u = __ldcg(&F.f1[r & 1][i]);
      const int8_t su = __ldcg(&st[u]);
      bool nr = su == kRoot;
      int32_t m = su == kUnd ? u : INT_MAX;
      for (int64_t k = g.vptr[u]; k < g.vptr[u + 1]; ++k) {
        const int32_t e = g.ve[k];
        for (int64_t q = g.eptr[e]; q < g.eptr[e + 1]; ++q) {
          const int32_t w = g.eidx[q];
          const int8_t sw = __ldcg(&st[w]);
          nr = nr || sw == kRoot;
          if (sw == kUnd && w < m) m = w;
        }
      }
      if ((nr ? 1 : 0) != __ldcg(&near[u]) || m != __ldcg(&mu[u])) {
        near[u] = nr ? 1 : 0;
        mu[u] = m;
        if (su == kUnd) push(F.f2[r & 1], &F.cnt[2 + (r & 1)], F.s2, u, r);
        for (int64_t k = g.vptr[u]; k < g.vptr[u + 1]; ++k) {
          const int32_t e = g.ve[k];
          for (int64_t q = g.eptr[e]; q < g.eptr[e + 1]; ++q) {
            const int32_t w = g.eidx[q];
            if (w != u && __ldcg(&st[w]) == kUnd) push(F.f2[r & 1], &F.cnt[2 + (r & 1)], F.s2, w, r);
          }
        }
      }
    }
    grid_barrier(bar, err);
    if (*verr) break;
    // decisions of F2; neighbourhoods of the decided ones into F1 of round r + 1
    const int n2 = __ldcg(&F.cnt[2 + (r & 1)]);
    if (tid == 0) F.cnt[2 + ((r + 1) & 1)] = 0;
    for (int i = tid; i < n2; i += nth) {
      const int32_t v = __ldcg(&F.f2[r & 1][i]);
      if (__ldcg(&st[v]) != kUnd) continue;
      bool out = __ldcg(&near[v]) != 0;
      bool root = !out && __ldcg(&mu[v]) == v;
      for (int64_t k = g.vptr[v]; k < g.vptr[v + 1] && !out; ++k) {
        const int32_t e = g.ve[k];
        for (int64_t q = g.eptr[e]; q < g.eptr[e + 1]; ++q) {
          const int32_t w = g.eidx[q];
          if (__ldcg(&near[w])) {
            out = true;
            break;
          }
          if (__ldcg(&mu[w]) != v) root = false;
        }
      }
      const int8_t ns = out ? kOut : (root ? kRoot : kUnd);
      if (ns == kUnd) continue;
      st[v] = ns;
      push_closed(v, g, F.f1[(r + 1) & 1], &F.cnt[(r + 1) & 1], F.s1, r + 1, nullptr);
    }
    grid_barrier(bar, err);
    if (*verr) break;
    if (__ldcg(&F.cnt[(r + 1) & 1]) == 0) break;  // nothing decided: the rounds have settled
  }
  if (tid == 0) *rounds_out = r;
}

__global__ void k_count_state(int64_t nv, const int8_t* __restrict__ st, int8_t which, int* __restrict__ count) {
  FOR_V(v, nv) if (st[v] == which) atomicAdd(count, 1);
}

__global__ void k_flag(int64_t nv, const int8_t* __restrict__ st, int8_t which, int32_t* __restrict__ flag) {
  FOR_V(v, nv) flag[v] = st[v] == which ? 1 : 0;
}

// Pass-1 aggregates: a root's id is its rank among the roots; its
// neighbours take it.
__global__ void k_p1_label(int64_t nv, HGraph g, const int8_t* __restrict__ st, const int64_t* __restrict__ rid,
                           int32_t* __restrict__ agg1) {
  FOR_V(v, nv) {
    int32_t a = -1;
    if (st[v] == kRoot) {
      a = (int32_t)rid[v];
    } else {
      for (int64_t k = g.vptr[v]; k < g.vptr[v + 1] && a < 0; ++k) {
        const int32_t e = g.ve[k];
        for (int64_t q = g.eptr[e]; q < g.eptr[e + 1]; ++q) {
          const int32_t w = g.eidx[q];
          if (st[w] == kRoot) {
            a = (int32_t)rid[w];
            break;
          }
        }
      }
    }
    agg1[v] = a;
  }
}

// ---- pass 2 ----------------------------------------------------------------
__global__ void k_p2(int64_t nv, HGraph g, const int32_t* __restrict__ agg1, int32_t* __restrict__ agg2,
                     int32_t* __restrict__ left) {
  FOR_V(v, nv) {
    int32_t a = agg1[v];
    if (a < 0) {
      int32_t wmin = INT_MAX;
      for (int64_t k = g.vptr[v]; k < g.vptr[v + 1]; ++k) {
        const int32_t e = g.ve[k];
        for (int64_t q = g.eptr[e]; q < g.eptr[e + 1]; ++q) {
          const int32_t w = g.eidx[q];
          if (w != (int32_t)v && w < wmin && agg1[w] >= 0) wmin = w;
        }
      }
      if (wmin != INT_MAX) a = agg1[wmin];
    }
    agg2[v] = a;
    left[v] = a < 0 ? 1 : 0;
  }
}

// ---- pass 3 ----------------------------------------------------------------
__global__ void k_p3_init(int64_t nv, const int32_t* __restrict__ agg2, int8_t* __restrict__ st) {
  FOR_V(v, nv) st[v] = agg2[v] < 0 ? kUnd : kNone;
}

// One round on the leftovers (double-buffered states): ROOT when no
// lower-index leftover neighbour is undecided or a root, OUT when one is a
// root.
__global__ void k_p3_round(int64_t nv, HGraph g, const int8_t* __restrict__ sin, int8_t* __restrict__ sout,
                           int* __restrict__ remaining) {
  FOR_V(v, nv) {
    const int8_t s = sin[v];
    if (s != kUnd) {
      sout[v] = s;
      continue;
    }
    bool anyroot = false, alldone = true;
    for (int64_t k = g.vptr[v]; k < g.vptr[v + 1] && !anyroot; ++k) {
      const int32_t e = g.ve[k];
      for (int64_t q = g.eptr[e]; q < g.eptr[e + 1]; ++q) {
        const int32_t w = g.eidx[q];
        if (w >= (int32_t)v) continue;
        const int8_t t = sin[w];
        if (t == kRoot) {
          anyroot = true;
          break;
        }
        if (t == kUnd) alldone = false;
      }
    }
    const int8_t ns = anyroot ? kOut : (alldone ? kRoot : kUnd);
    sout[v] = ns;
    if (ns == kUnd) *remaining = 1;
  }
}

__global__ void k_p3_label(int64_t nv, HGraph g, const int8_t* __restrict__ st, const int64_t* __restrict__ rid,
                           int64_t base, const int32_t* __restrict__ agg2, int32_t* __restrict__ agg) {
  FOR_V(v, nv) {
    const int8_t s = st[v];
    if (s == kNone) {
      agg[v] = agg2[v];
      continue;
    }
    if (s == kRoot) {
      agg[v] = (int32_t)(base + rid[v]);
      continue;
    }
    int32_t wmin = INT_MAX;
    for (int64_t k = g.vptr[v]; k < g.vptr[v + 1]; ++k) {
      const int32_t e = g.ve[k];
      for (int64_t q = g.eptr[e]; q < g.eptr[e + 1]; ++q) {
        const int32_t w = g.eidx[q];
        if (w != (int32_t)v && w < wmin && st[w] == kRoot) wmin = w;
      }
    }
    // a leftover that is no root has an adjacent lower root (the guard only keeps the read in bounds)
    agg[v] = wmin == INT_MAX ? -1 : (int32_t)(base + rid[wmin]);
  }
}

// ---- repeated passes -------------------------------------------------------
__global__ void k_gather_ids(int64_t total, const int32_t* __restrict__ eidx, const int32_t* __restrict__ agg,
                             int32_t* __restrict__ out) {
  FOR_V(q, total) out[q] = agg[eidx[q]];
}

__global__ void k_count_bad(int64_t n, const int32_t* __restrict__ agg, int64_t nagg, int* __restrict__ bad) {
  FOR_V(v, n) if (agg[v] < 0 || agg[v] >= nagg) atomicAdd(bad, 1);
}

__global__ void k_compose(int64_t n, int32_t* __restrict__ agg, const int32_t* __restrict__ bagg) {
  FOR_V(v, n) agg[v] = bagg[agg[v]];
}

// Rounds until no vertex is undecided: `round(last)` launches one round and,
// when `last`, lets it raise *d_rem.  The flag is read after batches of
// rounds that grow from 4 to 64 (the extra rounds of a batch change
// nothing); more than nv + 2 rounds is an internal error (each round decides
// the lowest undecided vertex).
template <class F>
int run_rounds(F&& round, int* d_rem, int64_t nv, cudaStream_t s, int64_t* rounds_out) {
  int64_t done = 0;
  int batch = 4;
  for (;;) {
    for (int i = 0; i + 1 < batch; ++i) AMGDD_TRY(round(false));
    AMGDD_CUDA(cudaMemsetAsync(d_rem, 0, sizeof(int), s));
    AMGDD_TRY(round(true));
    int rem = 0;
    AMGDD_CUDA(cudaMemcpyAsync(&rem, d_rem, sizeof(int), cudaMemcpyDeviceToHost, s));
    AMGDD_CUDA(cudaStreamSynchronize(s));
    done += batch;
    if (!rem) break;
    if (done > nv + 2) {
      set_error("aggregation: the rounds did not settle after %lld rounds", (long long)done);
      return AMGDD_ERR_INTERNAL;
    }
    batch = std::min(batch * 2, 64);
  }
  if (rounds_out) *rounds_out += done;
  return AMGDD_OK;
}

// Every id in [0, nagg) (the passes leave no vertex out): checked before
// the ids index anything.
int check_ids(const int32_t* d_agg, int64_t nv, int64_t nagg, int* d_bad, cudaStream_t s) {
  AMGDD_CUDA(cudaMemsetAsync(d_bad, 0, sizeof(int), s));
  k_count_bad<<<grid1(nv), kThreads, 0, s>>>(nv, d_agg, nagg, d_bad);
  count_kernels(1);
  AMGDD_CUDA(cudaGetLastError());
  int bad = 0;
  AMGDD_CUDA(cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  AMGDD_CUDA(cudaStreamSynchronize(s));
  if (bad != 0) {
    set_error("aggregation: %d vertices left without a valid aggregate id", bad);
    return AMGDD_ERR_INTERNAL;
  }
  return AMGDD_OK;
}

}  // namespace

int device_hyper_aggregation(int64_t nv, int64_t ne, const int64_t* d_eptr, const int32_t* d_eidx, int32_t* d_agg,
                             int64_t* nagg, cudaStream_t s, int64_t* rounds) {
  *nagg = 0;
  if (nv <= 0) return AMGDD_OK;
  if (nv > INT_MAX || ne > INT_MAX) {
    set_error("aggregation: %lld vertices / %lld edges exceed the 32-bit ids", (long long)nv, (long long)ne);
    return AMGDD_ERR_INVALID_ARG;
  }
  int64_t total = 0;
  if (ne > 0) AMGDD_CUDA(cudaMemcpyAsync(&total, d_eptr + ne, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  AMGDD_CUDA(cudaStreamSynchronize(s));
  // vertex -> edge incidence
  DBuf<int32_t> cnt, ve;
  DBuf<int64_t> vptr;
  AMGDD_TRY(cnt.alloc(nv));
  AMGDD_TRY(cnt.zero(s));
  AMGDD_TRY(vptr.alloc(nv + 1));
  AMGDD_TRY(ve.alloc(std::max<int64_t>(total, 1)));
  if (total > 0) {
    k_inc_count<<<grid1(total), kThreads, 0, s>>>(total, d_eidx, cnt.p);
    count_kernels(1);
  }
  AMGDD_TRY(scan_counts(cnt.p, nv, vptr.p, s));
  AMGDD_TRY(cnt.zero(s));
  if (ne > 0) {
    k_inc_fill<<<grid1(ne), kThreads, 0, s>>>(ne, d_eptr, d_eidx, vptr.p, cnt.p, ve.p);
    count_kernels(1);
  }
  AMGDD_CUDA(cudaGetLastError());
  HGraph g{vptr.p, ve.p, d_eptr, d_eidx};
  const int gr = grid1(nv);
  // pass 1: one full round, then rounds over the frontier
  DBuf<int8_t> st, st2, near;
  DBuf<int32_t> mu, flag, agg1, agg2, lists, stamps;
  DBuf<int64_t> rid;
  DBuf<int> rem, cnt4;
  AMGDD_TRY(st.alloc(nv));
  AMGDD_TRY(st.zero(s));
  AMGDD_TRY(near.alloc(nv));
  AMGDD_TRY(mu.alloc(nv));
  AMGDD_TRY(rem.alloc(1));
  AMGDD_TRY(lists.alloc(4 * nv));
  AMGDD_TRY(stamps.alloc(2 * nv));
  AMGDD_TRY(cnt4.alloc(4));
  AMGDD_TRY(cnt4.zero(s));
  AMGDD_CUDA(cudaMemsetAsync(stamps.p, 0xff, (size_t)2 * nv * sizeof(int32_t), s));  // -1: never pushed
  Front F{{lists.p, lists.p + nv}, {lists.p + 2 * nv, lists.p + 3 * nv}, cnt4.p, stamps.p, stamps.p + nv};
  k_p1_inputs_all<<<gr, kThreads, 0, s>>>(nv, g, st.p, near.p, mu.p);
  k_p1_decide_all<<<gr, kThreads, 0, s>>>(nv, g, near.p, mu.p, st.p, F);
  count_kernels(2);
  AMGDD_CUDA(cudaGetLastError());
  {
    // rounds 1, 2, ...: one cooperative launch (all CTAs resident)
    int dev = 0, sms = 0, per_sm = 0;
    AMGDD_CUDA(cudaGetDevice(&dev));
    AMGDD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    AMGDD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_p1_frontier, 512, 0));
    if (per_sm < 1) {
      set_error("aggregation: the frontier kernel fits no CTA on an SM");
      return AMGDD_ERR_INTERNAL;
    }
    DBuf<unsigned> bar;
    DBuf<int> err, nr;
    AMGDD_TRY(bar.alloc(2));
    AMGDD_TRY(bar.zero(s));
    AMGDD_TRY(err.alloc(1));
    AMGDD_TRY(err.zero(s));
    AMGDD_TRY(nr.alloc(1));
    const int max_rounds = (int)std::min<int64_t>(nv + 2, INT_MAX - 2);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)sms);
    cfg.blockDim = dim3(512);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    AMGDD_CUDA(cudaLaunchKernelEx(&cfg, k_p1_frontier, g, st.p, near.p, mu.p, F, max_rounds, bar.p, err.p, nr.p));
    count_kernels(1);
    int hv[2] = {0, 0};
    AMGDD_CUDA(cudaMemcpyAsync(&hv[0], err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    AMGDD_CUDA(cudaMemcpyAsync(&hv[1], nr.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    AMGDD_CUDA(cudaStreamSynchronize(s));
    if (hv[0] != 0) {
      set_error("aggregation: a grid barrier of the frontier rounds timed out");
      return AMGDD_ERR_TIMEOUT;
    }
    if (rounds) *rounds += hv[1];
    AMGDD_TRY(rem.zero(s));
    k_count_state<<<gr, kThreads, 0, s>>>(nv, st.p, kUnd, rem.p);
    count_kernels(1);
    int und = 0;
    AMGDD_CUDA(cudaMemcpyAsync(&und, rem.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    AMGDD_CUDA(cudaStreamSynchronize(s));
    if (und != 0) {
      set_error("aggregation: %d vertices undecided when the rounds settled", und);
      return AMGDD_ERR_INTERNAL;
    }
  }
  AMGDD_TRY(flag.alloc(nv));
  AMGDD_TRY(rid.alloc(nv + 1));
  k_flag<<<gr, kThreads, 0, s>>>(nv, st.p, kRoot, flag.p);
  count_kernels(1);
  AMGDD_TRY(scan_counts(flag.p, nv, rid.p, s));
  int64_t n1 = 0;
  AMGDD_CUDA(cudaMemcpyAsync(&n1, rid.p + nv, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  AMGDD_TRY(agg1.alloc(nv));
  AMGDD_TRY(agg2.alloc(nv));
  k_p1_label<<<gr, kThreads, 0, s>>>(nv, g, st.p, rid.p, agg1.p);
  // pass 2 (flag: the vertices still left)
  k_p2<<<gr, kThreads, 0, s>>>(nv, g, agg1.p, agg2.p, flag.p);
  count_kernels(2);
  AMGDD_CUDA(cudaGetLastError());
  AMGDD_TRY(scan_counts(flag.p, nv, rid.p, s));
  int64_t nleft = 0;
  AMGDD_CUDA(cudaMemcpyAsync(&nleft, rid.p + nv, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  AMGDD_CUDA(cudaStreamSynchronize(s));
  if (nleft == 0) {
    AMGDD_CUDA(cudaMemcpyAsync(d_agg, agg2.p, nv * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    *nagg = n1;
    return check_ids(d_agg, nv, n1, rem.p, s);
  }
  // pass 3
  AMGDD_TRY(st2.alloc(nv));
  k_p3_init<<<gr, kThreads, 0, s>>>(nv, agg2.p, st.p);
  count_kernels(1);
  int8_t* cur = st.p;
  int8_t* nxt = st2.p;
  AMGDD_TRY(run_rounds(
      [&](bool) -> int {
        k_p3_round<<<gr, kThreads, 0, s>>>(nv, g, cur, nxt, rem.p);
        count_kernels(1);
        AMGDD_CUDA(cudaGetLastError());
        std::swap(cur, nxt);
        return AMGDD_OK;
      },
      rem.p, nv, s, rounds));
  k_flag<<<gr, kThreads, 0, s>>>(nv, cur, kRoot, flag.p);
  count_kernels(1);
  AMGDD_TRY(scan_counts(flag.p, nv, rid.p, s));
  int64_t n3 = 0;
  AMGDD_CUDA(cudaMemcpyAsync(&n3, rid.p + nv, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  k_p3_label<<<gr, kThreads, 0, s>>>(nv, g, cur, rid.p, n1, agg2.p, d_agg);
  count_kernels(1);
  AMGDD_CUDA(cudaGetLastError());
  AMGDD_CUDA(cudaStreamSynchronize(s));
  *nagg = n1 + n3;
  return check_ids(d_agg, nv, *nagg, rem.p, s);
}

int device_standard_aggregation(int64_t n, int64_t ne, const int64_t* d_eptr, const int32_t* d_eidx, int passes,
                                int32_t* d_agg, int64_t* nagg, cudaStream_t s, int64_t* rounds) {
  AMGDD_TRY(device_hyper_aggregation(n, ne, d_eptr, d_eidx, d_agg, nagg, s, rounds));
  if (passes <= 1 || ne == 0) return AMGDD_OK;
  int64_t total = 0;
  AMGDD_CUDA(cudaMemcpyAsync(&total, d_eptr + ne, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  AMGDD_CUDA(cudaStreamSynchronize(s));
  DBuf<int32_t> eid2, bagg;
  AMGDD_TRY(eid2.alloc(std::max<int64_t>(total, 1)));
  for (int p = 1; p < passes; ++p) {
    // the graph of T^T A T: the aggregates each edge touches
    k_gather_ids<<<grid1(total), kThreads, 0, s>>>(total, d_eidx, d_agg, eid2.p);
    count_kernels(1);
    AMGDD_CUDA(cudaGetLastError());
    AMGDD_TRY(bagg.alloc(std::max<int64_t>(*nagg, 1)));
    int64_t nb = 0;
    AMGDD_TRY(device_hyper_aggregation(*nagg, ne, d_eptr, eid2.p, bagg.p, &nb, s, rounds));
    k_compose<<<grid1(n), kThreads, 0, s>>>(n, d_agg, bagg.p);
    count_kernels(1);
    AMGDD_CUDA(cudaGetLastError());
    AMGDD_CUDA(cudaStreamSynchronize(s));
    *nagg = nb;
  }
  return AMGDD_OK;
}

}  // namespace amgdd
