// Internal declarations of libamgdd: device buffers, level layout, kernel
// launch wrappers.  Nothing here is part of the C ABI (include/amgdd.h).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "amgdd.h"

namespace amgdd {

void set_error(const char* fmt, ...);

#define AMGDD_CUDA(call)                                                              \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) {                                                          \
      ::amgdd::set_error("%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e_)); \
      return e_ == cudaErrorMemoryAllocation ? AMGDD_ERR_OOM : AMGDD_ERR_CUDA;        \
    }                                                                                 \
  } while (0)

#define AMGDD_TRY(call)          \
  do {                           \
    int s_ = (call);             \
    if (s_ != AMGDD_OK) return s_; \
  } while (0)

// Net device bytes allocated through DBuf by the calling thread (setup
// measures a hierarchy's footprint as the change over its build).
extern thread_local int64_t g_alloc_bytes;
// Device allocations made through DBuf in this process (all threads); the
// hierarchy's JSON summary reports it, so a caller can check that a call
// allocated nothing.
int64_t device_alloc_count();
void note_device_alloc();

// Solve-phase kernels are launched with programmatic dependent launch while
// set (per thread: each hierarchy call sets it from its parameters).
extern thread_local bool g_pdl;

// Owning device buffer.
template <class T>
struct DBuf {
  T* p = nullptr;
  size_t n = 0;
  DBuf() = default;
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  ~DBuf() { release(); }
  void release() {
    if (p) {
      cudaFree(p);
      g_alloc_bytes -= (int64_t)(n * sizeof(T) + 16);
    }
    p = nullptr;
    n = 0;
  }
  int alloc(size_t count) {
    release();
    if (count == 0) return AMGDD_OK;
    // 16 bytes of tail padding: staged copies round their ranges out to
    // 16-byte boundaries and may touch up to 12 bytes past the last element
    cudaError_t e = cudaMalloc((void**)&p, count * sizeof(T) + 16);
    if (e != cudaSuccess) {
      p = nullptr;
      set_error("cudaMalloc of %zu bytes failed: %s", count * sizeof(T), cudaGetErrorString(e));
      return e == cudaErrorMemoryAllocation ? AMGDD_ERR_OOM : AMGDD_ERR_CUDA;
    }
    n = count;
    g_alloc_bytes += (int64_t)(count * sizeof(T) + 16);
    note_device_alloc();
    return AMGDD_OK;
  }
  int upload(const std::vector<T>& h, cudaStream_t s) {
    AMGDD_TRY(alloc(h.size()));
    if (!h.empty()) AMGDD_CUDA(cudaMemcpyAsync(p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    return AMGDD_OK;
  }
  int zero(cudaStream_t s) {
    if (n) AMGDD_CUDA(cudaMemsetAsync(p, 0, n * sizeof(T), s));
    return AMGDD_OK;
  }
  size_t bytes() const { return n * sizeof(T); }
};

// ---------------------------------------------------------------------------
// Batched gather-GEMV-scatter: for every block b,
//     y[out_idx[out_off[b] + r]] (op)= sum_c M_b[r, c] * x[in_idx[in_off[b] + c]]
// with M_b row-major (nr_b x nc_b, leading dimension nc_b) at m_off[b].
// Used for RAS (W_i), RAS-T (W_i^T), restriction (Z_i^T), prolongation (Z_i)
// and the coarsest solve (A_L^{-1} as a single block).
// SEG_RESID writes y[o] = c[o] - (M x)[o] with c the csrc argument (the
// residual s = r - A x of a level whose A is stored by block rows).
enum SegMode { SEG_STORE = 0, SEG_ADD = 1, SEG_ATOMIC_ADD = 2, SEG_ATOMIC_SUB = 3, SEG_RESID = 4 };

// One item of a staged gather-GEMV plan (see SegPlan).
struct alignas(16) ItemDesc {
  int64_t m_start;  // first stored matrix element
  int m_len;        // stored matrix elements
  int nb;           // blocks (1 for a row slice)
  int tab;          // offset of the item's tables in SegPlan::tabs
  int nin;          // gathered inputs
  int xin;          // offset of its input indices in SegPlan::gidx
  int nrows;        // output rows
  int out;          // offset of its output indices in SegPlan::gout
  int pad;
};

// Everything a gather-GEMV CTA (chunk) or task needs about its block, in one
// record, so that it is read in a single dependent step.
struct SegDesc {
  int64_t m_off, in_off, out_off;
  int32_t r0, r1;  // rows r0 <= r < r1 of the block (task: r1 = r0 + rows)
  int32_t nc, nr;
};

struct SegPlan {
  int nblocks = 0;
  int nchunks = 0;      // CTAs: chunks of at most `rows_per_chunk` rows of one block
  int rows_per_chunk = 0;
  int lanes = 32;       // lanes cooperating on one row (4, 8, 16 or 32)
  bool vec = false;     // every row 16-byte aligned with a whole number of vectors
  bool shift = false;   // 32 lanes, rows at any alignment: aligned vector loads against shifted copies of x
  bool shift64 = false; // the same for the FP64 copies (chosen separately)
  bool unroll = false;  // long rows (32 lanes, >= 512 entries on average): 4-way unrolled loops
  int lanes16 = 0;      // MIXED16: lanes per row of the FP16 kernel; 0 = read the FP32 copy
  // MIXED16: the plan's matrix in FP16, each row padded with zeros to a
  // multiple of 8 entries (16 bytes) so that every row starts aligned; the
  // chunks' descriptors point into it (row stride = nc rounded up to 8)
  DBuf<__half> m16;
  DBuf<SegDesc> chunk_desc16;
  int64_t mat_len16 = 0;
  // MIXED16, row per lane (lanes16 = -kind): the transposed blocks in FP16
  // (nc x nr, each column of rows padded to an even count), two output rows
  // per lane read as one half2; tasks of up to 2 kind rows
  DBuf<__half> mt16;
  DBuf<SegDesc> task_desc16;
  int ntasks16 = 0;
  int max_nc = 0;       // longest row (shared-memory staging of the gathered x)
  int64_t mat_len = 0;  // total stored matrix entries
  int64_t in_len = 0, out_len = 0;
  DBuf<int64_t> m_off, in_off, out_off;
  DBuf<int32_t> nr, nc;
  DBuf<int32_t> chunk_blk, chunk_row0;
  DBuf<SegDesc> chunk_desc;   // per chunk (the single right-hand-side kernel)
  std::vector<int32_t> h_nr;  // rows per block (host), to rebuild the chunks
  std::vector<int32_t> h_nc;
  std::vector<int64_t> h_moff, h_ioff, h_ooff;
  // index arrays owned elsewhere (level Omega lists or the identity)
  const int32_t* in_idx_ext = nullptr;
  const int32_t* out_idx_ext = nullptr;
  // short rows: one lane per output row over the transposed copy; tasks are
  // (block, first row, rows) and kind is the number of lanes per task
  bool rows_mode = false;
  int kind = 0;
  int ntasks = 0;
  DBuf<int32_t> task_blk, task_row0, task_nrow;
  DBuf<SegDesc> task_desc;    // per task (the single right-hand-side kernel)
  // staged form (preferred when built): items of contiguous matrix rows,
  // either up to 32 whole consecutive blocks or a row slice of one block,
  // each moved to shared memory by one bulk copy; per item the host packs
  // the block tables and flat lists of its input and output indices.
  bool staged = false;
  int nitems = 0;
  int item_lanes = 8;     // lanes per row in the staged kernel
  int item_max_in = 0;    // largest gathered input of an item (elements)
  int item_max_m = 0;     // largest staged matrix range (elements, incl. alignment slack)
  int item_max_rows = 0;  // most output rows of an item
  DBuf<ItemDesc> items;
  DBuf<int32_t> tabs;     // per item: rp[nb+1], mp[nb+1], ip[nb+1], ncs[nb]
  DBuf<int32_t> gidx;     // per item: indices of its inputs
  DBuf<int32_t> gout;     // per item: indices of its output rows
};

// Row groups of G_l (rows sharing one support), compressed: R_g has rank_g
// rows over the support S_g (row-major, leading dimension s_g).  A-apply:
//     y[S_g] (+/-)= R_g^T (R_g x[S_g]).
struct ApplyPlan {
  int ntasks = 0;
  int nbuckets = 0;
  int bucket_start[16] = {0};  // first CTA of each bucket
  int bucket_kind[16] = {0};   // kernel variant (lanes, columns per lane)
  int bucket_tasks[16] = {0};
  int64_t r_len = 0;           // stored entries of R (sum rank * s)
  DBuf<int32_t> task_grp, task_row0, task_nrow;  // per task (grouped by bucket)
};

struct Level {
  int64_t n = 0;
  int nagg = 0;
  bool coarsest = false;
  // ---- row groups of G_l --------------------------------------------------
  std::vector<int64_t> g_ptr;   // ngroups+1 offsets into g_idx
  std::vector<int32_t> g_idx;   // supports (sorted)
  std::vector<int32_t> g_rank;  // rows kept after compression
  std::vector<int64_t> h_off;   // offsets of the s x s Grams (and of R capacity)
  DBuf<int64_t> d_g_ptr, d_h_off;
  DBuf<int32_t> d_g_idx, d_rank;
  DBuf<double> d_H;     // Grams H_g = sum_rows g^T g (setup only, freed after use)
  bool rows_ready = false;  // d_R64 already holds rows carried by QR (row route): no pivoted Cholesky
  bool schur_rows = false;  // this level's Schur complements were formed from rows (else from Grams)
  DBuf<double> d_R64;   // compressed rows, capacity s x s per group
  DBuf<float> d_R32;
  ApplyPlan aplan;  // supports of at most 32 nodes
  // supports above 32 nodes: t = R_g x(S_g) (gt1), then y(S_g) -/+= R_g^T t
  // (gt2, one lane per support node reading R_g as the transposed copy)
  SegPlan gt1, gt2;
  int64_t t_len = 0;
  DBuf<double> t64;
  DBuf<float> t32;
  DBuf<int32_t> d_tidx;  // identity over t
  // ---- A_l assembled by block rows (coarse levels) -------------------------
  // A block is a run of consecutive dofs with identical lists of G groups;
  // its rows share one support in_b, so A(D_b, in_b) is stored dense
  // (row-major, plus the block-wise transpose) and applied by k_seg.
  bool has_blk = false;
  SegPlan ablk;
  DBuf<int32_t> d_blk_in;   // concatenated supports in_b
  DBuf<int32_t> d_blk_out;  // identity over the level's dofs
  DBuf<double> A64, At64;
  DBuf<float> A32, At32;
  double blk_mb = 0, mf_mb = 0, blk_us = 0, mf_us = 0;  // setup-time comparison of the two forms
  // ---- A_l by rows in ELL form (level 0) -----------------------------------
  // ell_w slots per row, slot-major (slot k of row i at k n + i); unused
  // slots hold 0 against the row's own index.  Used when setup measured it
  // faster than the row groups (use_ell).
  int ell_w = 0;
  bool use_ell = false;
  DBuf<int32_t> ellc;
  DBuf<double> ell64;
  DBuf<float> ell32;
  double ell_us = 0;
  // ---- aggregates and subdomains ------------------------------------------
  std::vector<int32_t> agg;      // n
  std::vector<int64_t> om_ptr;   // nagg+1
  std::vector<int32_t> om_idx;   // omega_i ascending then Gamma_i ascending
  std::vector<int32_t> nomega;   // |omega_i|
  std::vector<int32_t> k;        // selected eigenvectors per aggregate
  std::vector<int64_t> col0;     // nagg+1 first coarse column of each aggregate
  std::vector<int64_t> z_off;    // nagg+1 offsets of Z_i (|omega_i| x k_i)
  std::vector<int64_t> mu_off;   // nagg+1 offsets of the local spectra
  DBuf<int32_t> d_om_idx;        // Omega lists on the device
  // ---- smoother and transfer operators -------------------------------------
  SegPlan ras, rast, restr, prol;
  // deterministic RAS-T: y_i = W_i^T s(omega_i) stored at the positions of
  // the Omega lists (rast_det), then x_j += the y entries of node j in
  // ascending position order (det_ptr / det_pos: positions p with
  // om_idx[p] = j); no atomics
  // additive Schwarz (cycle = 1, level 0): every row of A_i^{-1} (|Omega_i|^2
  // per aggregate, row-major, and its block transpose), applied by asp as
  // x(Omega_i) += A_i^{-1} r(Omega_i)
  SegPlan asp;
  DBuf<double> Wf64, Wft64;
  DBuf<float> Wf32, Wft32;
  std::vector<int64_t> wf_off;
  SegPlan rast_det;
  DBuf<int32_t> d_pos_iota;  // identity over the positions of the Omega lists
  DBuf<int64_t> det_ptr;
  DBuf<int32_t> det_pos;
  DBuf<double> yd64;
  DBuf<float> yd32;
  DBuf<double> myd64;  // the same for the batched solves' interleaved columns
  DBuf<float> myd32;
  DBuf<double> W64, Wt64, Z64, Zt64, mu;
  DBuf<float> W32, Wt32, Z32, Zt32;
  // MIXED16 storage: the level's gather-GEMV plans hold FP16 copies of their
  // matrices (SegPlan::m16; built on demand, h16 once every FP32 copy of the
  // level is in the FP16 range)
  bool h16 = false;
  // rows omega_i of A over Omega_i (layout of W_i; the residual of the
  // batched solver where A has no block rows), applied with the RAS plan
  DBuf<double> Aw64, AwT64;
  DBuf<float> Aw32, AwT32;
  double inv_err = 0.0;  // coarsest level: measured ||W A v - v|| / ||v||
  double thresh = 0.0;   // eigenvalue threshold used on this level
  int n_color = 0;       // kappa > 0: colours of the subdomain colouring
  int n_mult = 0;        // kappa > 0: largest row multiplicity M(j)
  // dense tail: the V-cycle from this level to the coarsest as one n x n
  // matrix B (B = its action on the unit vectors), row-major with leading
  // dimension dld = n rounded up to 4 (zero columns); dplan applies it as
  // one block (gathered input index n..dld-1 -> 0) for the batched and
  // persistent forms
  DBuf<double> B64;
  DBuf<float> B32;
  DBuf<int32_t> d_didx;
  int64_t dld = 0;
  SegPlan dplan;
  double vc_us[2] = {0.0, 0.0};  // measured V-cycle from this level (graph), FP64 / mixed
  // ---- work vectors of the V-cycle ----------------------------------------
  DBuf<double> r64, x64, s64;
  DBuf<float> r32, x32, s32;
  // the same for the batched solves' columns (interleaved; allocated at the
  // first batched solve for its width, grown for a wider one)
  DBuf<double> mr64, mx64, ms64;
  DBuf<float> mr32, mx32, ms32;
};

// ---------------------------------------------------------------------------
// kernels (cycle_kernels.cu)
// csrc/cdst (optional, same precision): cdst[out] = csrc[out] for every
// output row, fused into the same launch (the residual's copy of r).
// MT: the block-wise transpose of M (needed by row-per-lane plans).
int launch_seg(const SegPlan& p, const void* M, bool m_fp32, const void* x, void* y, bool v_fp32, SegMode mode,
               const int* skip, cudaStream_t s, const void* csrc = nullptr, void* cdst = nullptr,
               const void* MT = nullptr);
// The same with FP16 matrix entries (MIXED16 storage) and FP32 vectors:
// entries are widened to FP32 and summed in FP32.
// Reads the plan's padded FP16 copy (SegPlan::m16) with p.lanes16 lanes per row.
int launch_seg16(const SegPlan& p, const float* x, float* y, SegMode mode, const int* skip, cudaStream_t s,
                 const float* csrc = nullptr, float* cdst = nullptr);
// The padded FP16 copy of a plan's FP32 matrix (row-major blocks at m_off,
// nr x nc): block b goes to m_off16[b] with rows of nc rounded up to 8
// entries, the padding zero; FP16 round to nearest.
int launch_pad16(const float* M32, const int64_t* m_off, const int32_t* nr, const int32_t* nc,
                 const int64_t* m_off16, int nblocks, __half* dst, cudaStream_t s);
// The same for the transposed blocks (nc x nr row-major at m_off): block b
// goes to m_off16[b] as nc rows of nr rounded up to even, the padding zero.
int launch_pad16t(const float* MT32, const int64_t* m_off, const int32_t* nr, const int32_t* nc,
                  const int64_t* m_off16, int nblocks, __half* dst, cudaStream_t s);
int launch_apply(const ApplyPlan& p, const Level& L, bool fp32, const void* x, void* y, int sign, const int* skip,
                 cudaStream_t s);
int launch_cast(const void* src, bool src32, void* dst, bool dst32, int64_t n, const int* skip, cudaStream_t s);
// *d_count += the number of non-finite entries of v[0..n) (setup checks of the stored operators).
int count_nonfinite(const void* v, int64_t n, bool fp32, int* d_count, cudaStream_t s);

// ---------------------------------------------------------------------------
// Standard aggregation on the device (aggregate_kernels.cu): the graph whose
// vertices 0..nv-1 are adjacent when a hyperedge (d_eptr: ne + 1 offsets,
// d_eidx: members, device memory) holds both; d_agg (nv, device) receives
// the ids of the sequential three passes in creation order, *nagg their
// count; *rounds (optional) accumulates the parallel rounds taken.
int device_hyper_aggregation(int64_t nv, int64_t ne, const int64_t* d_eptr, const int32_t* d_eidx, int32_t* d_agg,
                             int64_t* nagg, cudaStream_t s, int64_t* rounds = nullptr);
// The same with `passes` passes, each on the graph of the aggregates so far
// (the aggregates a hyperedge touches): ids of the last pass, composed.
int device_standard_aggregation(int64_t n, int64_t ne, const int64_t* d_eptr, const int32_t* d_eidx, int passes,
                                int32_t* d_agg, int64_t* nagg, cudaStream_t s, int64_t* rounds = nullptr);
int launch_copy_vec(const void* src, void* dst, bool fp32, int64_t n, const int* skip, cudaStream_t s);

// ---------------------------------------------------------------------------
// Persistent V-cycle tail: the levels from some l >= 1 down to the coarsest
// and back, as a list of phases run by one cooperative launch with a grid
// barrier between phases (the small coarse levels are otherwise bound by
// launch latency).  Every phase is a gather-GEMV-scatter over a SegPlan or a
// precision cast.
enum PhaseOp { PH_SEG = 0, PH_CAST = 1 };
struct PhaseDesc {
  int op = PH_SEG;
  int fp32 = 0;  // PH_SEG: operand precision
  int mode = 0;  // SegMode
  int rows_mode = 0, lanes = 32, vec = 0, rows_per_chunk = 0, nwork = 0, max_nc = 0;
  const int32_t *chunk_blk = nullptr, *chunk_row0 = nullptr;
  const int32_t *task_blk = nullptr, *task_row0 = nullptr, *task_nrow = nullptr;
  const int64_t *m_off = nullptr, *in_off = nullptr, *out_off = nullptr;
  const int32_t *nr = nullptr, *nc = nullptr, *in_idx = nullptr, *out_idx = nullptr;
  const void *M = nullptr, *MT = nullptr, *x = nullptr, *csrc = nullptr;
  void *y = nullptr, *cdst = nullptr;
  int src32 = 0, dst32 = 0;  // PH_CAST
  int64_t n = 0;
  // staged form (nwork = items)
  const ItemDesc* items = nullptr;
  const int32_t *tabs = nullptr, *gidx = nullptr, *gout = nullptr;
  int max_in = 0, max_m = 0, max_rows = 0;
};
PhaseDesc seg_phase(const SegPlan& p, const void* M, const void* MT, bool fp32, const void* x, void* y, SegMode mode,
                    const void* csrc = nullptr, void* cdst = nullptr);
PhaseDesc cast_phase(const void* src, bool src32, void* dst, bool dst32, int64_t n);
size_t phase_smem(const PhaseDesc& d);
// shared memory of the staged kernel for items of at most `max_in` gathered
// inputs, `max_rows` output rows and `max_m` staged matrix entries of `esz` bytes
size_t staged_smem(int max_in, int max_rows, int max_m, size_t esz);
// CTAs of the cooperative launch for `smem` bytes of dynamic shared memory
int persistent_grid(size_t smem, int* grid);
// bar: two device words (arrival count, generation), zero before first use;
// err: set to 1 by a barrier wait that timed out (the launch then drains).
int launch_persistent(const PhaseDesc* d_phases, int nphases, size_t smem, int grid, unsigned* bar, int* err,
                      const int* skip, cudaStream_t s);

// Device word that staged and persistent kernels set when a bounded wait
// expires (the vc_err field of the hierarchy's CG state); set for the
// duration of each API call on a hierarchy.  Staged kernels are used only
// while it is set.
extern thread_local int* g_err_word;
struct ErrScope {
  int* prev;
  explicit ErrScope(int* w) : prev(g_err_word) { g_err_word = w; }
  ~ErrScope() { g_err_word = prev; }
};

struct PdlScope {
  bool prev;
  explicit PdlScope(bool on) : prev(g_pdl) { g_pdl = on; }
  ~PdlScope() { g_pdl = prev; }
};

// Kernel-launch accounting (kernels launched directly, plus the kernels of
// each captured CUDA graph every time it is launched).
void count_kernels(int64_t k);
void capture_begin();
int64_t capture_end();
void count_graph_launch(int64_t kernels);

// PCG state kept in device memory
struct PcgState {
  double rz;      // r_k^T z_k
  double pq;      // p_k^T A p_k
  double rr;      // r_k^T r_k
  double rzn;     // r_{k+1}^T z_{k+1}
  double rzo;     // r_{k+1}^T z_k (flexible variant)
  double alpha, beta;
  double bnorm2;
  double tol2;    // tol^2 * ||b||^2
  double relres;
  int iters, max_iter, done, status, flexible;
  int vc_err;  // set by a persistent V-cycle whose grid barrier timed out
  double rr_mark;  // r^T r at the last stall check (flexible CG)
  unsigned ticket;  // CTAs finished in a fused CG kernel (the last one resets it)
};
// Status of a flexible (FP32-cycle) CG that stopped because ||r|| fell by
// less than 10% over 10 iterations; the host redoes the solve in FP64.
constexpr int kStallStatus = -100;

constexpr int kDotBlocks = 608;  // 4 x 152 SMs; partial sums per dot product

int launch_dot_partial(const double* a, const double* b, const double* c, int64_t n, double* partials,
                       const int* skip, cudaStream_t s);
// which == 3 also sets the conditional of an enclosing CUDA-graph WHILE
// node (when use_cond): 1 to run another iteration, 0 once done.
int launch_pcg_scalar(int which, PcgState* st, const double* partials, cudaStream_t s,
                      cudaGraphConditionalHandle cond = 0, int use_cond = 0);
int launch_update_xr(PcgState* st, double* x, double* r, const double* p, const double* q, int64_t n,
                     cudaStream_t s);
int launch_update_p(PcgState* st, double* p, const double* z, double* zold, int64_t n, cudaStream_t s);
// Fused CG steps (single right-hand side, level 0 by ELL rows): each kernel
// also reduces its dot product and, in its last CTA, runs the scalar step.
//   cg_ap:   q = A p; alpha = rz / (p.q)
//   cg_xr:   x += alpha p, r -= alpha q, r32 = r (when given); r.r and the
//            convergence test
//   cg_zdot: z = x32 (when given); beta from r.z (and r.z_old); sets the
//            graph condition
int launch_cg_ap(const Level& L0, PcgState* st, const double* p, double* q, double* partials, cudaStream_t s);
int launch_cg_xr(PcgState* st, double* x, double* r, float* r32, const double* p, const double* q, int64_t n,
                 double* partials, cudaStream_t s);
int launch_cg_zdot(PcgState* st, const float* x32, double* z, const double* r, const double* zold, int64_t n,
                   double* partials, cudaStream_t s, cudaGraphConditionalHandle cond, int use_cond);

// ---------------------------------------------------------------------------
// K right-hand sides at once (multi_kernels.cu): vectors interleaved by node
// (v[i * K + k]), K in {2, 4, 8, 16, 32}.  Modes as launch_seg (SEG_RESID reads c).
int launch_seg_multi(const SegPlan& p, const void* M, const void* MT, bool fp32, const void* x, void* y, SegMode mode,
                     const void* csrc, int K, const int* skip, cudaStream_t s);
// partials: kDotBlocks x 2K (a.b then a.c per column)
int launch_dot_multi(const double* a, const double* b, const double* c, int64_t n, int K, double* partials,
                     const int* skip, cudaStream_t s);
// st: K states; grp[0] set to 1 once every column is done
int launch_pcg_scalar_multi(int which, PcgState* st, int* grp, const double* partials, int K, cudaStream_t s,
                            cudaGraphConditionalHandle cond = 0, int use_cond = 0);
int launch_update_xr_multi(const PcgState* st, const int* grp, double* x, double* r, const double* p, const double* q,
                           int64_t n, int K, cudaStream_t s);
int launch_update_p_multi(const PcgState* st, const int* grp, double* p, const double* z, double* zold, int64_t n,
                          int K, cudaStream_t s);
// column-major (leading dimension ld, ncols <= K columns; the rest zero) <->
// interleaved
int launch_interleave(const double* src, int64_t ld, int ncols, double* dst, int64_t n, int K, cudaStream_t s);
int launch_deinterleave(const double* src, int64_t n, int K, double* dst, int64_t ld, int ncols, cudaStream_t s);


// ---------------------------------------------------------------------------
// setup kernels (setup_kernels.cu); all FP64
struct LocalBatch {
  // one entry per aggregate of the batch
  DBuf<int32_t> m, no;              // |Omega_i|, |omega_i|
  DBuf<int64_t> a_off;              // offset of A_i / A~_i in the work pools (m x m, column-major)
  DBuf<int64_t> pair_ptr;           // groups touching Omega_i
  DBuf<int32_t> pair_grp, pair_nz;  // group id, 1 if the group is in nz_i
  DBuf<int64_t> map_ptr;            // per pair: offsets into map
  DBuf<int32_t> map;                // local index of each support node (-1 outside Omega_i)
};

struct NextGramPlan {
  int64_t nnew = 0;
  DBuf<int64_t> new_ptr;    // new group -> range in contrib
  DBuf<int32_t> contrib;    // level-l group ids
  DBuf<int64_t> new_sptr;   // new group support offsets
  DBuf<int64_t> new_hoff;   // output Gram offsets
  // per support node of each level-l group: the Z row offset, k and the
  // column offset of its aggregate's block inside the new support
  DBuf<int64_t> rowz_ptr;
  DBuf<int64_t> rowz_zoff;
  DBuf<int32_t> rowz_k;
  DBuf<int32_t> rowz_col;
  int64_t scratch_per = 0;
};

int launch_gram_rows(int64_t ngroups, const int64_t* g_row0, const int64_t* g_row1, const int64_t* g_ptr,
                     const int64_t* h_off, const int64_t* rowptr, const double* val, double* H, cudaStream_t s);
int launch_gram_diag(int64_t n, int64_t first_group, const int64_t* h_off, const double* D1, double* H,
                     cudaStream_t s);
int launch_pchol(int64_t first, int64_t count, int max_s, const int64_t* g_ptr, const int64_t* h_off,
                 const double* H, double* R64, float* R32, int32_t* rank, double* scratch, int64_t scratch_per,
                 cudaStream_t s);
int launch_assemble(int nb, int max_m, const LocalBatch& b, const int64_t* g_ptr, const int64_t* h_off,
                    const double* H, const int32_t* M, double* Apool, double* Atpool, cudaStream_t s);
int launch_chol(int nb, int max_m, const int32_t* m, const int64_t* a_off, double* Apool, int32_t* status,
                cudaStream_t s);
int launch_schur(int nb, int max_m, const int32_t* m, const int32_t* no, const int64_t* a_off, double* Atpool,
                 double rtol, cudaStream_t s);
int launch_inv_rows(int nb, int max_m, const int32_t* m, const int32_t* no, const int64_t* a_off,
                    const double* Lpool, const int64_t* w_off, double* W64, float* W32, double* Wt64, float* Wt32,
                    double* scratch, const int32_t* chunk_b, const int32_t* chunk_c0, int nchunks, int cw,
                    cudaStream_t s);
constexpr int kInvChunk = 32;  // RHS columns per CTA of the inverse-row solves

// Wall-clock accounting of setup phases (printed when AMGDD_VERBOSE is set).
struct PhaseTimer {
  bool on = false;
  double acc[16] = {0};
  double flops[16] = {0};  // FP64 flops of each phase (counted from the block sizes)
  const char* name[16] = {nullptr};
  void add(int i, const char* nm, double ms) {
    acc[i] += ms;
    name[i] = nm;
  }
};
// work_out[b]: Jacobi sweeps (blocks below the team size) or implicit-QL
// rotations (team blocks) that block b's eigensolve took.
int launch_gep(int nb, int max_no, const int32_t* m, const int32_t* no, const int64_t* a_off, const double* Lpool,
               const double* Spool, const int32_t* cap, double thresh, const int64_t* mu_off, double* mu,
               const int64_t* z_off_cap, double* Zcap, int32_t* kout, double* scratch, const int64_t* scr_off,
               int32_t* work_out, cudaStream_t s);
// true when launch_gep takes the tridiagonal + implicit QL path for a batch
// whose largest omega block has max_no entries
bool gep_uses_ql(int max_no);
// Measured FP64 FMA rate of the device (GFLOP/s): independent FMA chains on
// every SM, timed with CUDA events.
int measure_fp64_rate(cudaStream_t s, double* gflops);
int launch_pack_z(int nb, const int32_t* no, const int32_t* k, const int64_t* z_off_cap, const double* Zcap,
                  const int64_t* z_off, double* Z64, float* Z32, double* Zt64, float* Zt32, cudaStream_t s);
// Rows omega_i of each assembled A_i (before its Cholesky) in the layout of
// W_i, plus the block transposes, in FP64 and FP32.
// failure-detection probe of the bounded waits (0: grid barrier, 1: mbarrier)
int launch_wait_probe(int which, unsigned* bar, int* err, cudaStream_t s);
// x_j (+)= sum of Y[pos] over the positions of node j, K interleaved columns
int launch_gather_add(const int64_t* ptr, const int32_t* pos, const void* Y, void* x, int64_t n, int K, bool fp32,
                      const int* skip, cudaStream_t s);
int launch_ell_fill(int64_t total, const int64_t* src, const double* Aw64, double* v64, float* v32,
                    cudaStream_t s);
// y = A x (csrc null) or y = csrc - A x over the ELL rows of L
int launch_ell(const Level& L, bool fp32, const void* x, void* y, const void* csrc, const int* skip, cudaStream_t s);
// the same for K in {2, 4, 8, 16, 32} interleaved columns
int launch_ell_multi(const Level& L, bool fp32, const void* x, void* y, const void* c, int K, const int* skip,
                     cudaStream_t s);
int launch_dense_pack(const double* C, int n, int64_t ld, double* B64, float* B32, cudaStream_t s);
// y = B x for the dense tail (B n x n row-major, leading dimension ld a
// multiple of 4; x and y 16-byte aligned)
int launch_dense(const void* B, int64_t ld, int n, bool fp32, const void* x, void* y, const int* skip,
                 cudaStream_t s);
// FP32 rounding and block transposes (FP64, FP32) of row-major blocks
// rows[b] x cols[b] at off[b] of src (the copies a loaded hierarchy derives
// from its stored FP64 matrices); null outputs are skipped.
int launch_block_copies(int nb, const int32_t* rows, const int32_t* cols, const int64_t* off, const double* src,
                        float* dst32, double* dstT64, float* dstT32, cudaStream_t s);
int launch_copy_wrows(int nb, const int32_t* m, const int32_t* no, const int64_t* a_off, const double* Apool,
                      const int64_t* w_off, double* Aw64, float* Aw32, double* AwT64, float* AwT32, cudaStream_t s);
// Block rows of A_l = sum_g H_g: for block b, rows p0 .. p0+nr_b-1 of each
// touching group's Gram, columns mapped into in_b by `map`.
int launch_blockrows(int nblk, const int32_t* nr, const int32_t* nc, const int64_t* m_off, const int64_t* pair_ptr,
                     const int32_t* pair_grp, const int32_t* pair_p0, const int64_t* pair_map, const int32_t* map,
                     const int64_t* g_ptr, const int64_t* h_off, const double* H, double* A64, float* A32,
                     double* At64, float* At32, cudaStream_t s);
int launch_next_gram(const NextGramPlan& p, int max_sn, const int64_t* g_ptr, const int64_t* h_off, const double* H,
                     const double* Z64, double* Hn, double* scratch, int64_t first, int64_t count, cudaStream_t s);
// G_{l+1}'s rows by QR of the stacked R_g P_g (row route); t_off: prefix of
// rows x sn per new group (scratch holds groups first .. first+count-1).
int launch_next_rows(const NextGramPlan& p, const int64_t* g_ptr, const int64_t* h_off, const int32_t* rank,
                     const double* R, const double* Z64, const int64_t* t_off, double* scratch, double* Rn64,
                     float* Rn32, int32_t* rank_out, int64_t first, int64_t count, bool team, cudaStream_t s);
// S~ of Eq. gevp-S from the rows of the splitting (row route) into the omega
// block of Atpool; Ypool holds y_rows[b] x m per matrix, nrm m per matrix.
int launch_schur_rows(int nb, int max_m, const LocalBatch& b, const int64_t* g_ptr, const int64_t* h_off,
                      const int32_t* rank, const double* R, const int32_t* M, const int64_t* y_off,
                      const int32_t* y_rows, double* Ypool, const int64_t* n_off, double* nrm, double* Atpool,
                      int32_t* rank_out, bool team, cudaStream_t s);

}  // namespace amgdd
