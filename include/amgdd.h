/*
 * amgdd.h -- C ABI of the GB300 LS-AMG-DD library (libamgdd.so).
 *
 * Multilevel least-squares AMG with overlapping Schwarz smoothers and local
 * spectral coarse spaces (Southworth, Al Daas, Wimmer, Threlfall, "Algebraic
 * Multigrid with Overlapping Schwarz Smoothers and Local Spectral Coarse
 * Grids for Least Squares Problems").  The system is A x = b with
 *
 *     A = D1 + G^T G,   G sparse m x n                     (Section 1, Eq. 1)
 *
 * (D1 >= 0 diagonal; it is the sqrt(D1) block of G^T = [sqrt(D1), ...]).
 * `amgdd_setup` builds the hierarchy of Algorithm 1 on one GPU; `amgdd_solve`
 * runs conjugate gradients preconditioned by the V-cycle of Section 3.1 (one
 * RAS pre-smoothing, Eq. ras; coarse-grid correction, Eq. cgc; one RAS-T
 * post-smoothing, Eq. ras-t; exact solve on the coarsest level).
 *
 * Conventions shared by every entry point
 *   - Return value: AMGDD_OK (0) or a negative AMGDD_ERR_* code; no call
 *     throws or aborts.  `amgdd_last_error()` gives a one-line description
 *     of the last failure on the calling thread.
 *   - Pointers are plain host or device addresses.  Where an argument may be
 *     either, the library asks the CUDA runtime which it is.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  All device work of a call is ordered on that stream; calls
 *     that return host data synchronise it first.
 *   - Sizes are element counts.  Index arrays are int32 (node and column
 *     ids); offsets are int64.
 *   - Every routine requires a CUDA device; there is no CPU fallback.
 */
#ifndef AMGDD_H
#define AMGDD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define AMGDD_OK 0
#define AMGDD_ERR_INVALID_ARG -1    /* malformed input (CSR, ids, sizes)   */
#define AMGDD_ERR_NOT_SPD -2        /* a local or coarsest block is not SPD */
#define AMGDD_ERR_NONFINITE -3      /* NaN/Inf in G, D1 or b               */
#define AMGDD_ERR_BREAKDOWN -4      /* CG: p^T A p <= 0                    */
#define AMGDD_ERR_NO_CONVERGENCE -5 /* CG reached max_iter                 */
#define AMGDD_ERR_OOM -6            /* device allocation failed            */
#define AMGDD_ERR_CUDA -7           /* any other CUDA runtime error        */
#define AMGDD_ERR_INTERNAL -8       /* violated internal invariant         */
#define AMGDD_ERR_TIMEOUT -9        /* a bounded device-side wait expired  */

/* ---- memory spaces and precisions ------------------------------------ */
#define AMGDD_HOST 0
#define AMGDD_DEVICE 1

/* FP64: every vector, local inverse and basis in double precision.
 * MIXED32: the V-cycle (local Schwarz solves, P/R, level operators, vectors)
 * in FP32 under an FP64 flexible CG whose residual, inner products, updates
 * and fine-level A-apply stay FP64; the coarsest solve stays FP64.         */
#define AMGDD_FP64 0
#define AMGDD_MIXED32 1
/* MIXED16: MIXED32 with the smoother rows, the basis (P and P^T) and the
 * block rows of coarse A read from FP16 copies (round to nearest, widened
 * to FP32 and summed in FP32): half the bytes of those matrices per
 * V-cycle.  A level holding an entry beyond the FP16 range keeps FP32.
 * The flexible FP64 CG wins the accuracy back (the same stall guard as
 * MIXED32).  Batched solves (nrhs > 1) and the persistent V-cycle tail read
 * the FP32 copies.  The FP16 copies are built at setup (precision =
 * MIXED16) or at the first amgdd_set_precision(MIXED16).                  */
#define AMGDD_MIXED16 2

/* ---- inputs ----------------------------------------------------------- */
/* G in CSR form.  rowptr has m+1 entries (rowptr[0] = 0, nondecreasing,
 * rowptr[m] = nnz); col holds strictly increasing column ids in [0, n) per
 * row; val the values.  Every listed entry is structural, zero or not.
 * `mem` says where the three arrays live (AMGDD_HOST or AMGDD_DEVICE).   */
typedef struct {
  int64_t m, n, nnz;
  const int64_t* rowptr;
  const int32_t* col;
  const double* val;
  int mem;
} amgdd_csr;

/* Method parameters (Algorithm 1 inputs and solver options).            */
typedef struct {
  int L_max;           /* maximum number of levels (Algorithm 1)          */
  int64_t n_coarse;    /* coarsen while n_l > n_coarse                    */
  double thresh;       /* keep local eigenpairs with lambda > thresh      */
  int c_min[8];        /* minimum coarsening ratio per level; the last    */
  int n_cmin;          /*   entry repeats for deeper levels (LS_{a,b,..}) */
  int precision;       /* AMGDD_FP64 or AMGDD_MIXED32                     */
  int max_iter;        /* CG iteration limit                              */
  double schur_rtol;   /* pivots of A~_GG below schur_rtol * max diag are */
                       /*   treated as zero (pseudo-inverse reading)      */
  int use_graph;       /* capture the CG iteration in a CUDA graph        */
  int check_every;     /* host reads the convergence flag every k iters   */
  int tune;            /* 1: setup times the alternative kernel forms of  */
                       /*   each step and keeps the fastest; 0: defaults  */
                       /*   (unstaged kernels, row per lane for rows of   */
                       /*   <= 128 entries, block rows, no persistent     */
                       /*   tail); 2, 3, 4: as 0 with, wherever a plan    */
                       /*   allows it, the staged kernel (2), shifted     */
                       /*   vector loads (3) or lanes per row (4) (for    */
                       /*   profiling and testing each form)              */
  const char* tune_cache; /* NULL, or a text file of earlier choices keyed */
                       /*   by problem, GPU, level and step: read before  */
                       /*   timing, rewritten with new choices at the end */
  int coarse_overlap;  /* hops of overlap on levels >= 1; 0: the level-0  */
                       /*   `overlap` on every level (Algorithm 1 builds   */
                       /*   Omega_i from one layer of neighbours in A_l)  */
  int coarse_refine;   /* one step of iterative refinement after the      */
                       /*   explicit-inverse coarsest solve (FP64):       */
                       /*   0 never; 1 (default) when setup measures      */
                       /*   ||W A v - v|| / ||v|| > 1e-13 for a seeded v  */
                       /*   (W the computed inverse); 2 always            */
  int pdl;             /* 1: solve-phase kernels use programmatic         */
                       /*   dependent launch (each starts while the one   */
                       /*   before it drains, then waits for its results);*/
                       /*   0 (default): plain stream order               */
  int dense_tail;      /* the V-cycle from a coarse level l down applied  */
                       /*   as one dense matrix (its action on the unit   */
                       /*   vectors, computed at setup): 0 (default) the  */
                       /*   level chosen by timing when tune = 1, else    */
                       /*   none; -1 none; l >= 1 from level l            */
  int ell;             /* level 0's A by ELL rows (CG product, residuals,  */
                       /*   fused CG steps): 0 (default) when faster by   */
                       /*   setup timing (tune = 1), else the row groups; */
                       /*   1 always (where Omega_i holds the rows); -1   */
                       /*   never                                         */
  int deterministic;   /* 1: no atomics on the solve path, so repeated    */
                       /*   solves on one hierarchy give bitwise equal x: */
                       /*   RAS-T stores W_i^T s(omega_i) per subdomain   */
                       /*   entry and gathers per node in a fixed order   */
                       /*   (Eq. ras-t); level 0 by ELL rows (ell = 1),   */
                       /*   coarse A by block rows, no persistent tail    */
  int cycle;           /* preconditioner: 0 (default) the multiplicative  */
                       /*   V-cycle (Section 3.1); 1 the additive two-    */
                       /*   level method M_2^{-1} = P (P^T A P)^{-1} P^T  */
                       /*   + sum_i R_i^T A_i^{-1} R_i (additive Schwarz, */
                       /*   Section 3.1 after Eq. cgc): needs a two-level */
                       /*   hierarchy (setup fails otherwise), runs FP64  */
  double kappa;        /* target condition number (Section 3.4): > 0      */
                       /*   replaces `thresh` on each level by            */
                       /*   max{0.1, (kappa - n_color) /                  */
                       /*   (n_color n_multiplicity)}, with n_color the   */
                       /*   colours of a greedy colouring of the Omega_i  */
                       /*   (ascending index; two subdomains coupled by A */
                       /*   differ) and n_multiplicity the largest row    */
                       /*   multiplicity M(j) of the level's G; 0         */
                       /*   (default): `thresh` on every level            */
  int agg_passes;      /* amgdd_setup with agg = NULL: level-0 aggregates */
                       /*   by this many passes of standard aggregation   */
                       /*   (see amgdd_aggregate); >= 1, default 1        */
  int schur_gram;      /* Schur complement of Eq. gevp-S.  Row form:      */
                       /*   S~ = X^T (I - Pi) X with Pi the projector     */
                       /*   onto the Gamma rows (pivoted Householder QR,  */
                       /*   cut at the numerical rank), and the rows of   */
                       /*   G_{l+1} = G_l P_l carried by QR.  Gram form:  */
                       /*   from A~_i with diagonally pivoted elimination */
                       /*   (cut at schur_rtol), rows of G_{l+1} from its */
                       /*   Gram.  0 (default): per level, rows unless    */
                       /*   their QR would cost more than 8 times the     */
                       /*   Gram elimination (3D coarse levels); 1: Gram  */
                       /*   on every level; 2: rows on every level        */
  int batch_cols;      /* amgdd_solve with nrhs > 1: columns per batch,   */
                       /*   2, 4, 8, 16 or 32 (default 8).  Wider batches */
                       /*   read the matrices once for more columns but   */
                       /*   move more vector bytes per launch and hold    */
                       /*   more registers; on the 512^2 Q1 workload 8 is */
                       /*   fastest in mixed precision, on 3D 32^3 16     */
} amgdd_params;

typedef struct amgdd_hierarchy amgdd_hierarchy; /* opaque, library-owned */

/* Per right-hand-side result of amgdd_solve.                            */
typedef struct {
  int iters;           /* CG iterations (A-applications)                  */
  int status;          /* AMGDD_OK, _BREAKDOWN or _NO_CONVERGENCE         */
  double relres;       /* ||r_k|| / ||b|| of the recursively updated r    */
  double relres_true;  /* ||b - A x|| / ||b|| recomputed at the end (FP64) */
  double solve_ms;     /* device time of this right-hand side             */
  int fallback;        /* MIXED32 only: 1 when the FP32 cycle stalled      */
                       /*   (||r|| fell by less than 10% over 10          */
                       /*   iterations) and the solve was redone with the */
                       /*   FP64 cycle; iters then counts both attempts.  */
                       /*   After a stall, later MIXED32 solves on the    */
                       /*   hierarchy use the FP64 cycle directly (until  */
                       /*   amgdd_set_precision is called again)          */
  int iters_mixed;     /* iterations of the stalled FP32 attempt (0 if none) */
} amgdd_info;

/* Defaults: L_max 10, n_coarse 2000, thresh 0.1 (kappa 0), c_min = {2,3,4} (LS_{2,3,4}),
 * FP64, max_iter 1000, schur_rtol 1e-12, graphs on, check_every 4, tune 1,
 * no tune cache, agg_passes 1, batch_cols 8.                              */
amgdd_params amgdd_params_default(void);

/* ---- level-0 aggregation (Section 3.3) ------------------------------- */
/* Standard aggregation on the graph of A = D1 + G^T G, read from the matrix
 * pattern itself with no strength-of-connection test (two unknowns are
 * adjacent when a row of G holds both).  Pass 1 visits unknowns in ascending
 * order and makes every unknown whose neighbours are all unaggregated a root
 * of a new aggregate {root} u neighbours; pass 2 puts each remaining unknown
 * in the aggregate of its lowest-index neighbour aggregated in pass 1;
 * pass 3 starts a new aggregate at each unknown still left, with its
 * unaggregated neighbours.  With passes > 1 the same routine aggregates the
 * aggregates, on the graph of T^T A T (T the 0/1 aggregation matrix so far),
 * and the result is the product T_1 T_2 ... (aggregating aggregates).
 *   G      : CSR as above (only the pattern is read); host or device.
 *   passes : >= 1.
 *   agg    : receives n aggregate ids 0..nagg-1 (creation order of the last
 *            pass); host or device buffer owned by the caller.
 *   nagg   : receives the number of aggregates (may be NULL).
 * Runs on the device, on `stream`: the visiting order fixes the result,
 * yet each pass is an order-independent rule (pass 1's roots are the first
 * maximal independent set, in ascending order, of the graph joining
 * unknowns within distance 2; pass 3's that of the graph on the leftovers),
 * so the unknowns decide in parallel rounds and the ids equal those of the
 * sequential passes.  The row supports are grouped on the host.  Errors:
 * INVALID_ARG, OOM, CUDA.                                                 */
int amgdd_aggregate(const amgdd_csr* G, int passes, void* stream, int32_t* agg, int64_t* nagg);

/* ---- setup: Algorithm 1 ---------------------------------------------- */
/* Builds the hierarchy {G_l, P_l, smoothers} for A = D1 + G^T G.
 *   G        : CSR as above (copied; the caller keeps ownership).
 *   D1       : n diagonal entries (>= 0) or NULL for D1 = 0; host or device.
 *   agg      : n level-0 aggregate ids (host or device).  Ids >= 0 name
 *              aggregates; -1 marks an unaggregated node, which joins the
 *              smallest aggregate id among its neighbours in the graph of A
 *              (Section 3.3); ids are relabelled 0..nagg-1 in ascending
 *              order, skipping unused ids.  NULL: the library aggregates
 *              with params->agg_passes passes (amgdd_aggregate).
 *   overlap  : number of graph hops added around each aggregate (>= 1)
 *              to form Omega_i = omega_i u Gamma_i (Section 2.2).
 *   params   : NULL for amgdd_params_default().
 *   out      : receives the hierarchy, freed with amgdd_free.
 * Errors: INVALID_ARG (bad CSR/ids/params, or a level where no local
 * eigenvector passes the threshold: an empty coarse space), NONFINITE,
 * NOT_SPD (a block A(Omega_i, Omega_i) or the coarsest matrix failed
 * Cholesky), OOM, CUDA.                                                   */
int amgdd_setup(const amgdd_csr* G, const double* D1, const int32_t* agg, int overlap,
                const amgdd_params* params, void* stream, amgdd_hierarchy** out);

/* ---- solve: V-cycle preconditioned CG -------------------------------- */
/* Solves A x = b for nrhs independent right-hand sides stored column-major
 * (n x nrhs, leading dimension n).  b and x may be host or device pointers
 * (each is classified on its own); x is overwritten (x_0 = 0).  Stops when
 * ||r_k|| <= tol ||b|| on the recursively updated residual (the check runs
 * every params.check_every iterations; iterations after convergence leave x
 * unchanged).  info (host, nrhs entries) may be NULL.
 * With nrhs > 1 (and CUDA graphs on) the right-hand sides are solved in
 * batches of up to params.batch_cols (<= 32) that share every V-cycle and
 * A-apply launch: each
 * column is its own CG (own scalars and stopping test, x frozen once it has
 * converged), so a batch reads the hierarchy's matrices once per iteration
 * for all of its columns (a gather-GEMV whose staged input would not fit
 * shared memory at the batch's width reads them once per column tile).  A
 * batch runs at 2, 4, 8, 16 or 32 columns, the next at or above its count
 * (padding columns are zero and finish at once); its workspace is allocated
 * at the first batched solve and grown for a wider one.  Per-column results
 * agree with single solves to rounding (the batched kernels sum in another
 * order).
 * Returns the first non-OK per-RHS status, or an error code.             */
int amgdd_solve(amgdd_hierarchy* h, const double* b, int nrhs, double tol, double* x, void* stream,
                amgdd_info* info);

/* Switches the precision used by later solves (the hierarchy stores both). */
int amgdd_set_precision(amgdd_hierarchy* h, int precision);

/* Sets the CG iteration limit of later solves (params.max_iter at setup);
 * with tol = 0 a solve then runs exactly max_iter iterations, which lets a
 * caller compare iterates at a fixed count.  Errors: INVALID_ARG for
 * max_iter < 1.                                                            */
int amgdd_set_max_iter(amgdd_hierarchy* h, int max_iter);

/* ---- single steps of the cycle (device FP64 vectors; for testing) ---- */
#define AMGDD_OP_A 0        /* y = A_l x                    (Eq. 1)       */
#define AMGDD_OP_RAS 1      /* y = M_RAS^{-1} x             (Eq. ras)     */
#define AMGDD_OP_RAST 2     /* y = M_RAS-T^{-1} x           (Eq. ras-t)   */
#define AMGDD_OP_RESTRICT 3 /* y = P_l^T x  (length n_{l+1}) (Eq. mg-p)   */
#define AMGDD_OP_PROLONG 4  /* y = P_l x    (x of length n_{l+1})         */
#define AMGDD_OP_VCYCLE 5   /* y = B_l x: V-cycle from level l, x_0 = 0   */
#define AMGDD_OP_COARSE 6   /* y = A_L^{-1} x on the coarsest level       */
#define AMGDD_OP_M2 7       /* y = M_2^{-1} x, additive two-level method  */
                            /*   (level 0 of a cycle = 1 hierarchy)       */
/* Applies one operator of level `level` in the hierarchy's current
 * precision; x and y are device arrays of FP64 (converted internally in
 * MIXED32).  x and y must not alias.                                     */
int amgdd_apply(amgdd_hierarchy* h, int op, int level, const double* x, double* y, void* stream);

/* Same operators and arguments as amgdd_apply, but the call allocates no
 * device memory: no cudaMalloc, no cudaFree, no allocating library routine.
 * It is meant for callers that must not allocate once setup is done, for
 * example code that runs while another component owns the device memory
 * budget or inside an allocator-free serving loop (amgdd_setup itself still
 * allocates the hierarchy).  The paper has no counterpart: this is an
 * interface convenience, not a step of the method.
 * In MIXED32 the FP64 x and y are staged through FP32 vectors kept in one
 * file-scope device array of 2 x 131072 floats (1 MiB); every GPU that loads
 * the library holds that array until the process exits.  Levels whose
 * input or output vector has more than 131072 entries are rejected with
 * AMGDD_ERR_INVALID_ARG in MIXED32 (FP64 needs no staging and has no limit).
 * The hierarchy's device must be the current device (AMGDD_ERR_INVALID_ARG
 * otherwise).  The first call on a device looks up the array's device
 * address with that device current and keeps it for the process; make that
 * first call before any stream capture (a cudaDeviceReset invalidates the
 * kept address, as it invalidates every hierarchy on that device).  All
 * calls share the array: calls that overlap on the GPU (other streams,
 * other host threads) race on it.  The call synchronises `stream` before
 * returning, as amgdd_apply does.                                          */
int amgdd_apply_noalloc(amgdd_hierarchy* h, int op, int level, const double* x, double* y, void* stream);

/* ---- inspection ------------------------------------------------------ */
typedef struct {
  int64_t n;           /* unknowns on this level                          */
  int64_t nagg;        /* aggregates (0 on the coarsest level)            */
  int64_t n_next;      /* n_{l+1} (0 on the coarsest level)               */
  int64_t omega_len;   /* sum_i |Omega_i|                                 */
  int64_t z_len;       /* sum_i |omega_i| k_i                             */
  int64_t ngroups;     /* row groups of G_l                               */
  int64_t g_rows;      /* sum of compressed row counts of G_l             */
  int64_t g_vals;      /* stored values of G_l (rows x support)           */
  int64_t w_vals;      /* stored values of the smoother, sum |omega||Omega| */
  int is_coarsest;
  int64_t g_sup_len;   /* sum over row groups of |S_g| (AMGDD_ARR_G_IDX)  */
  int64_t a_nnz;       /* structural nonzeros of A_l (AMGDD_ARR_A_IDX)    */
  int64_t p_nnz;       /* structural nonzeros of P_l, sum |omega_i| k_i   */
} amgdd_level_desc;

int amgdd_num_levels(const amgdd_hierarchy* h);
int amgdd_level_describe(const amgdd_hierarchy* h, int level, amgdd_level_desc* out);

/* Copies one array of a level to host memory `dst` of `cap` bytes.
 *   AGG       int32[n]         aggregate id of each dof
 *   OMEGA_PTR int64[nagg+1]    offsets into OMEGA_IDX
 *   OMEGA_IDX int32[omega_len] Omega_i: omega_i ascending, then Gamma_i ascending
 *   NOMEGA    int32[nagg]      |omega_i|
 *   K         int32[nagg]      k_i, selected eigenvectors
 *   Z         double[z_len]    Z_i row-major |omega_i| x k_i, aggregate order;
 *                              columns ordered by ascending mu, normalised so
 *                              Z_i^T A_ww Z_i = I, largest |entry| positive
 *   MU        double[sum |omega_i|] all local eigenvalues mu = 1/lambda, ascending */
#define AMGDD_ARR_AGG 0
#define AMGDD_ARR_OMEGA_PTR 1
#define AMGDD_ARR_OMEGA_IDX 2
#define AMGDD_ARR_NOMEGA 3
#define AMGDD_ARR_K 4
#define AMGDD_ARR_Z 5
#define AMGDD_ARR_MU 6
/* Structural patterns (Section 3.1: G_{l+1} = G_l P_l, A_l = G_l^T G_l;
 * Eq. mg-p for P), every level:
 *   G_PTR int64[ngroups+1], G_IDX int32[g_sup_len]: the support S_g of each
 *              row group of G_l (rows with one structural support; ascending
 *              node ids; groups in the library's order, and rows with
 *              one support may fall in several groups).  Rows that carry
 *              D1 (level 0) are one-node supports.  Compression changes
 *              the rows a group stores, never its support.
 *   A_PTR int64[n+1], A_IDX int32[a_nnz]: CSR pattern of A_l, j ~ k iff a
 *              support holds both (ascending columns).
 *   P_PTR int64[n+1], P_IDX int32[p_nnz]: CSR pattern of P_l (not on the
 *              coarsest level): row j spans the k_a columns of its
 *              aggregate a, numbered by aggregate, then ascending mu.     */
#define AMGDD_ARR_G_PTR 7
#define AMGDD_ARR_G_IDX 8
#define AMGDD_ARR_A_PTR 9
#define AMGDD_ARR_A_IDX 10
#define AMGDD_ARR_P_PTR 11
#define AMGDD_ARR_P_IDX 12
int amgdd_level_export(const amgdd_hierarchy* h, int level, int which, void* dst, size_t cap);

/* JSON summary (levels, n_l, row groups, stored values, operator
 * complexity, algorithmic bytes per V-cycle, setup time) into json[cap].
 * "process_device_allocs" counts the device allocations the library has
 * made in this process so far (all hierarchies and threads).             */
int amgdd_hierarchy_stats(const amgdd_hierarchy* h, char* json, size_t cap);

/* Algorithmic bytes one V-cycle must move in the current precision, and
 * those of one FP64 fine-level A-apply (used by the roofline report).    */
int amgdd_bytes_model(const amgdd_hierarchy* h, double* vcycle_bytes, double* apply_bytes);

/* ---- measurement ----------------------------------------------------- */
/* Times `reps` V-cycles from level 0 in the current precision with CUDA
 * events recorded between the launches on the library's work stream, and
 * reports per level l and step slot the mean device milliseconds per cycle
 * (ms[l*8 + slot]) and the algorithmic bytes that step moves
 * (bytes[l*8 + slot]: stored matrix values, index arrays, and one pass over
 * each input and output vector).  Slots: 0 RAS (or the coarsest solve),
 * 1 residual copies (casts on the coarsest level), 2 residual A-applies,
 * 3 restriction, 4 prolongation, 5 cast back (coarsest level), 6 the
 * persistent tail, 7 RAS-T.  graph = 0: the launches run eagerly, so a step's
 * time includes host launch gaps; graph != 0: the marked cycle is captured
 * once in a CUDA graph (the marks become event record nodes) and replayed,
 * as the solve replays its cycle, and when cap > 8 * levels, ms[8 * levels]
 * receives the mean time of one replay of the same cycle captured without
 * marks.  cap >= 8 * amgdd_num_levels(h).                                 */
int amgdd_profile_vcycle(amgdd_hierarchy* h, int reps, int graph, double* ms, double* bytes, int cap);

/* Kernels this library has launched in the process so far (a replay of a
 * captured CUDA graph counts every kernel in it).                         */
int64_t amgdd_kernel_launches(void);

/* FP64 FMA throughput of the current device in GFLOP/s: independent fused
 * multiply-add chains (8 per thread) on every SM, the best of three timed
 * launches (CUDA events on `stream`).  The denominator of the setup phases'
 * GFLOP/s ("setup_phases_gflop" in amgdd_hierarchy_stats over
 * "setup_phases_ms").  Errors: INVALID_ARG for a null output, CUDA.       */
int amgdd_measure_fp64(void* stream, double* gflops);

/* Device bytes the hierarchy holds: what setup kept, plus the batched-solve
 * workspace once allocated.  with_batched > 0 counts, as an admission
 * estimate, the workspace a batched solve would grow it to: 1 for a batch
 * of params.batch_cols columns, 2..32 for a batch of that many columns
 * (rounded up to 2, 4, 8, 16 or 32).  -1 for NULL.                        */
int64_t amgdd_device_bytes(const amgdd_hierarchy* h, int with_batched);

/* ---- serving: continuous batching over cached hierarchies ------------ */
/* A server keeps hierarchies ("operators") resident on the device within
 * hbm_budget bytes (setup plus batched-solve workspace, amgdd_device_bytes)
 * and solves queued requests with `slots` worker threads, each on its own
 * stream.  A worker takes the oldest request whose operator is idle and
 * merges the other queued requests for that operator and tolerance into one
 * batched amgdd_solve of at most max_batch (<= 32) columns; requests that
 * arrive meanwhile join later batches as slots free, and batches of
 * different operators overlap on the device.  The serving workload of many
 * grid sizes and right-hand-side counts is beyond the paper (which solves
 * one system at a time); each result is the solve of its own right-hand
 * side and agrees with a solve alone to CG rounding.                      */
typedef struct amgdd_server amgdd_server; /* opaque */
typedef struct {
  int64_t hbm_budget;  /* device bytes for resident operators             */
  int slots;           /* concurrent batches (worker threads)             */
  int max_batch;       /* columns per batched solve, 1..32                */
} amgdd_server_params;

#define AMGDD_PENDING 1 /* amgdd_server_poll: not finished yet            */

/* Defaults: 64 GiB budget, 4 slots, batches of 8 columns.                 */
amgdd_server_params amgdd_server_params_default(void);
int amgdd_server_create(const amgdd_server_params* params, amgdd_server** out);
/* Builds the hierarchy of (G, D1, agg, overlap, params) on the calling
 * thread and makes it resident, evicting idle operators with no queued
 * requests (least recently used first) to stay within the budget; OOM if it
 * cannot fit.  `key` names the operator: adding a key that is resident
 * returns its id with *cached = 1 and builds nothing.                     */
int amgdd_server_add_operator(amgdd_server* s, int64_t key, const amgdd_csr* G, const double* D1,
                              const int32_t* agg, int overlap, const amgdd_params* params, int64_t* op,
                              int* cached);
/* Queues a solve of nrhs columns (host buffers, column-major n x nrhs; both
 * must stay valid until the request is polled to completion) and returns at
 * once with the request id.  INVALID_ARG for an unknown operator or device
 * pointers.                                                               */
int amgdd_server_submit(amgdd_server* s, int64_t op, const double* b, int nrhs, double tol, double* x, int64_t* req);
/* Queues a solve whose operator comes with the request (setup on the request
 * path): if `key` is resident (or already queued for setup) the request joins
 * it (*cached = 1); otherwise the operator (G, D1, agg, overlap, params as in
 * amgdd_setup; the caller keeps them valid until the request is polled to
 * completion) is built by a worker once admission allows: its expected
 * device bytes (bytes per unknown of the operators built so far, x 1.25)
 * fit the budget after evicting idle operators and the device's free memory
 * at that moment.  Meanwhile the request waits and other requests proceed;
 * a setup error completes the operator's requests with that error, and an
 * operator that cannot fit even with nothing else resident fails with
 * AMGDD_ERR_OOM.  b and x as in amgdd_server_submit.                       */
int amgdd_server_submit_problem(amgdd_server* s, int64_t key, const amgdd_csr* G, const double* D1,
                                const int32_t* agg, int overlap, const amgdd_params* params, const double* b,
                                int nrhs, double tol, double* x, int64_t* req, int* cached);
/* AMGDD_PENDING while queued or running (waits up to wait_ms first; < 0:
 * until done); else the request's status, with info (nrhs entries, may be
 * NULL) and the latency from submit to completion, and the request is
 * forgotten.                                                              */
int amgdd_server_poll(amgdd_server* s, int64_t req, int wait_ms, amgdd_info* info, double* latency_ms);
/* JSON: completed requests, batches, mean columns per batch, latency
 * p50/p99/max (ms, over every completed request), resident operators and
 * bytes, evictions, cache hits, queue length, operators built on the request
 * path and their total setup ms, admission waits, bytes per unknown, seconds
 * since creation.                                                         */
int amgdd_server_stats(amgdd_server* s, char* json, size_t cap);
/* Stops the workers after their current batches and frees every operator. */
void amgdd_server_destroy(amgdd_server* s);

/* Save a hierarchy to `path` (a binary file of this library version): its
 * setup inputs (G, D1, aggregates, overlap), parameters and setup-time
 * kernel choices, and what Algorithm 1 computed on every level: the
 * compressed rows of G_l's row groups, the aggregates and Omega lists, the
 * rows omega_i of A_i^{-1} (and of A over Omega_i), the local spectra and
 * bases Z_i, the coarse block rows where setup kept them, every row of
 * A_i^{-1} for the additive form, and the coarsest inverse, all in FP64.
 * Load restores them on `stream` without solving any local problem again:
 * it rebuilds the index plans, derives the FP32 and transposed copies (and
 * the FP16 copies under MIXED16), replays the kernel choices instead of
 * timing them, and builds the dense tail and solve graphs; with the
 * deterministic kernels the loaded hierarchy applies the same operator bit
 * for bit.  Every size and index of the file is checked against the others
 * before use.  Files of the earlier format (inputs and choices only) load by
 * running the setup again with the choices replayed.  Errors:
 * AMGDD_ERR_INVALID_ARG for a path that cannot be written or read, a file of
 * another format or version, or one whose levels are inconsistent; OOM,
 * CUDA.  The caller frees the loaded hierarchy with amgdd_free.          */
int amgdd_hierarchy_save(const amgdd_hierarchy* h, const char* path);
int amgdd_hierarchy_load(const char* path, void* stream, amgdd_hierarchy** out);

/* Failure detection of the bounded device-side waits, without a fault:
 * launches a grid barrier (the wait of the persistent V-cycle) whose last
 * CTA never arrives, then an mbarrier wait (the wait of the staged copies)
 * that nothing completes, on `stream`.  Each gives up after its limit
 * (about 2 s and 1 s at 2 GHz) and sets an error word that the host reads;
 * *barrier_status and *mbarrier_status receive AMGDD_ERR_TIMEOUT when the
 * wait reported its expiry (AMGDD_OK otherwise).  The context stays
 * usable.  Returns AMGDD_ERR_INVALID_ARG for null outputs, AMGDD_ERR_CUDA
 * if a launch fails.                                                     */
int amgdd_selftest_wait_timeouts(void* stream, int* barrier_status, int* mbarrier_status);

void amgdd_free(amgdd_hierarchy* h);
const char* amgdd_status_string(int status);
const char* amgdd_last_error(void);

/* sizeof of the structs a binding mirrors, for a layout check at load time:
 * which = 0 amgdd_params, 1 amgdd_info, 2 amgdd_level_desc, 3 amgdd_csr,
 * 4 amgdd_server_params; 0 for any other value.  Host only.              */
size_t amgdd_struct_size(int which);

#ifdef __cplusplus
}
#endif
#endif /* AMGDD_H */
