// C ABI of libamgdd and the host-side drivers: hierarchy construction
// (Algorithm 1), the V-cycle (Section 3.1: RAS pre-smoothing, coarse-grid
// correction, RAS-T post-smoothing, exact coarsest solve) and the
// V-cycle-preconditioned conjugate gradient solver.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "internal.h"
#include "structure.h"

namespace amgdd {
struct Level;
}
static double apply_bytes(const amgdd::Level& L, size_t esz);

namespace amgdd {

static thread_local std::string g_last_error;
thread_local int* g_err_word = nullptr;
thread_local int64_t g_alloc_bytes = 0;
static std::atomic<int64_t> g_alloc_calls{0};
int64_t device_alloc_count() { return g_alloc_calls.load(); }
void note_device_alloc() { g_alloc_calls.fetch_add(1); }
thread_local bool g_pdl = false;

// Setup-time tuning context: whether to time alternatives, the problem/GPU
// signature that keys the cache, and the cached choices (`key\tvalue` lines).
struct TuneCtx {
  bool on = true;
  int prefer_form = -1;  // without timing: force this gather-GEMV form where a plan allows it
  std::string path, sig;
  std::map<std::string, double> kv;
  bool dirty = false;
  bool get(const std::string& k, double& v) const {
    auto it = kv.find(sig + "|" + k);
    if (it == kv.end()) return false;
    v = it->second;
    return true;
  }
  void put(const std::string& k, double v) {
    kv[sig + "|" + k] = v;
    dirty = true;
  }
  void load() {
    if (path.empty()) return;
    FILE* f = std::fopen(path.c_str(), "r");
    if (!f) return;
    char line[1024];
    while (std::fgets(line, sizeof line, f)) {
      char* tab = std::strchr(line, '\t');
      if (!tab) continue;
      *tab = 0;
      kv[line] = std::atof(tab + 1);
    }
    std::fclose(f);
  }
  void save() const {
    if (path.empty() || !dirty) return;
    const std::string tmp = path + ".tmp";
    FILE* f = std::fopen(tmp.c_str(), "w");
    if (!f) return;
    for (const auto& e : kv) std::fprintf(f, "%s\t%.17g\n", e.first.c_str(), e.second);
    std::fclose(f);
    std::rename(tmp.c_str(), path.c_str());
  }
};
static thread_local TuneCtx* g_tune = nullptr;

// Setup times the kernel forms of each plan on a cold L2, as the V-cycle
// meets them (every matrix is read once per cycle): before each timed launch
// a 256 MiB buffer (twice the L2) is overwritten.  One buffer per setup (or
// per build of the FP16 copies), released with it.
struct L2Flush {
  DBuf<char> buf;
  int run(cudaStream_t s) {
    if (buf.p == nullptr) AMGDD_TRY(buf.alloc((size_t)256 << 20));
    AMGDD_CUDA(cudaMemsetAsync(buf.p, 0, buf.n, s));
    return AMGDD_OK;
  }
};
static thread_local L2Flush* g_flush = nullptr;
struct FlushScope {
  L2Flush f;
  L2Flush* prev;
  FlushScope() : prev(g_flush) {
    if (prev == nullptr) g_flush = &f;
  }
  ~FlushScope() {
    if (prev == nullptr) g_flush = nullptr;
  }
};

// Mean device time (ms) of `reps` launches of `launch`, each on a cold L2
// (when a flush scope is active), after two warm-up launches.
template <class F>
static int time_cold(cudaStream_t s, int reps, F&& launch, float* ms_out) {
  cudaEvent_t e[2];
  for (auto& v : e) AMGDD_CUDA(cudaEventCreate(&v));
  int rc = AMGDD_OK;
  float tot = 0.f;
  for (int rep = 0; rep < reps + 2 && rc == AMGDD_OK; ++rep) {
    if (g_flush) rc = g_flush->run(s);
    if (rc == AMGDD_OK) rc = cudaEventRecord(e[0], s) == cudaSuccess ? AMGDD_OK : AMGDD_ERR_CUDA;
    if (rc == AMGDD_OK) rc = launch();
    if (rc == AMGDD_OK) rc = cudaEventRecord(e[1], s) == cudaSuccess ? AMGDD_OK : AMGDD_ERR_CUDA;
    float ms = 0.f;
    if (rc == AMGDD_OK &&
        (cudaEventSynchronize(e[1]) != cudaSuccess || cudaEventElapsedTime(&ms, e[0], e[1]) != cudaSuccess))
      rc = AMGDD_ERR_CUDA;
    if (rep >= 2) tot += ms;
  }
  for (auto& v : e) cudaEventDestroy(v);
  *ms_out = tot;
  return rc;
}

static std::atomic<int64_t> g_kernels{0};
static thread_local bool g_capturing = false;
static thread_local int64_t g_capture_kernels = 0;

void count_kernels(int64_t k) {
  if (g_capturing)
    g_capture_kernels += k;
  else
    g_kernels += k;
}
void capture_begin() {
  g_capturing = true;
  g_capture_kernels = 0;
}
int64_t capture_end() {
  g_capturing = false;
  return g_capture_kernels;
}
void count_graph_launch(int64_t kernels) { g_kernels += kernels; }

void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
}

namespace {

thread_local PhaseTimer g_timer;

// Synchronise and charge the elapsed time to a phase (AMGDD_VERBOSE only).
struct Phase {
  int id;
  const char* nm;
  cudaStream_t s;
  std::chrono::steady_clock::time_point t0;
  Phase(int i, const char* n, cudaStream_t st) : id(i), nm(n), s(st), t0(std::chrono::steady_clock::now()) {}
  ~Phase() {
    cudaStreamSynchronize(s);
    g_timer.add(id, nm, std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count());
  }
};

template <class T>
int upload_vec(DBuf<T>& d, const std::vector<T>& h, cudaStream_t s) {
  return d.upload(h, s);
}

template <class T>
int download(std::vector<T>& h, const T* d, size_t n, cudaStream_t s) {
  h.resize(n);
  if (n) {
    AMGDD_CUDA(cudaMemcpyAsync(h.data(), d, n * sizeof(T), cudaMemcpyDeviceToHost, s));
    AMGDD_CUDA(cudaStreamSynchronize(s));
  }
  return AMGDD_OK;
}

bool is_device_ptr(const void* p) {
  if (p == nullptr) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Copy n elements of a host-or-device array to a host vector.
template <class T>
int fetch_any(std::vector<T>& h, const T* src, size_t n, bool dev, cudaStream_t s) {
  h.resize(n);
  if (n == 0) return AMGDD_OK;
  if (dev) {
    AMGDD_CUDA(cudaMemcpyAsync(h.data(), src, n * sizeof(T), cudaMemcpyDeviceToHost, s));
    AMGDD_CUDA(cudaStreamSynchronize(s));
  } else {
    std::memcpy(h.data(), src, n * sizeof(T));
  }
  return AMGDD_OK;
}

int lanes_for(int max_nc) { return max_nc >= 64 ? 32 : (max_nc >= 24 ? 16 : (max_nc >= 8 ? 8 : 4)); }

// Items of the staged kernel.  An item is a contiguous range of the stored
// matrix: consecutive whole blocks (at most 32) or a slice of rows of one
// large block.  Items hold at most 8 KB of FP32 matrix, fewer on small
// levels so that every SM gets about 16 of them.  Per item the host packs
// the block tables and flat lists of the input and output indices, so that a
// CTA reaches all of its global data in two dependent steps.  Plans with
// rows longer than kItemMaxIn keep the unstaged kernels.
constexpr int64_t kItemElems = 2048;
constexpr int kItemMaxIn = 1024;
constexpr int kItemMaxRows = 256;
constexpr int kItemMaxBlocks = 32;
int build_items(SegPlan& p, const std::vector<int32_t>& nr, const std::vector<int32_t>& nc,
                const std::vector<int64_t>& m_off, const std::vector<int64_t>& in_off,
                const std::vector<int64_t>& out_off, const int32_t* in_ext, const int32_t* out_ext, cudaStream_t s) {
  p.staged = false;
  p.nitems = 0;
  const int nb = (int)nr.size();
  if (nb == 0 || in_ext == nullptr || out_ext == nullptr) return AMGDD_OK;
  int64_t total = 0, in_end = 0, out_end = 0;
  double ncsum = 0.0, rows = 0.0;
  for (int b = 0; b < nb; ++b) {
    if (nc[b] > kItemMaxIn) return AMGDD_OK;
    total += (int64_t)nr[b] * nc[b];
    ncsum += (double)nr[b] * nc[b];
    rows += nr[b];
    in_end = std::max(in_end, in_off[b] + nc[b]);
    out_end = std::max(out_end, out_off[b] + nr[b]);
  }
  std::vector<int32_t> hin, hout;
  AMGDD_TRY(download(hin, in_ext, (size_t)in_end, s));
  AMGDD_TRY(download(hout, out_ext, (size_t)out_end, s));
  const int64_t tgt = std::max<int64_t>(256, std::min<int64_t>(kItemElems, total / (152 * 16)));
  std::vector<ItemDesc> items;
  std::vector<int32_t> tabs, gidx, gout;
  int max_in = 0, max_m = 0, max_rows = 0;
  // one item over blocks [b0, b0 + cnt) (cnt == 1: rows [r0, r1) of b0)
  auto emit = [&](int b0, int cnt, int r0, int r1) {
    ItemDesc d{};
    d.nb = cnt;
    d.tab = (int)tabs.size();
    d.xin = (int)gidx.size();
    d.out = (int)gout.size();
    std::vector<int32_t> rp(cnt + 1, 0), mp(cnt + 1, 0), ip(cnt + 1, 0), ncs(cnt);
    for (int j = 0; j < cnt; ++j) {
      const int b = b0 + j;
      const int rs = cnt == 1 ? r0 : 0, re = cnt == 1 ? r1 : nr[b];
      rp[j + 1] = rp[j] + (re - rs);
      mp[j + 1] = mp[j] + (re - rs) * nc[b];
      ip[j + 1] = ip[j] + nc[b];
      ncs[j] = nc[b];
      gidx.insert(gidx.end(), hin.begin() + in_off[b], hin.begin() + in_off[b] + nc[b]);
      gout.insert(gout.end(), hout.begin() + out_off[b] + rs, hout.begin() + out_off[b] + re);
    }
    tabs.insert(tabs.end(), rp.begin(), rp.end());
    tabs.insert(tabs.end(), mp.begin(), mp.end());
    tabs.insert(tabs.end(), ip.begin(), ip.end());
    tabs.insert(tabs.end(), ncs.begin(), ncs.end());
    d.m_start = m_off[b0] + (int64_t)(cnt == 1 ? r0 : 0) * nc[b0];
    d.m_len = mp[cnt];
    d.nin = ip[cnt];
    d.nrows = rp[cnt];
    items.push_back(d);
    max_in = std::max(max_in, d.nin);
    max_m = std::max(max_m, d.m_len + 8);
    max_rows = std::max(max_rows, d.nrows);
  };
  int cb0 = 0, cnb = 0;
  int64_t cm = 0, cin = 0, crows = 0;
  auto flush = [&]() {
    if (cnb > 0) emit(cb0, cnb, 0, cnb == 1 ? nr[cb0] : 0);
    cnb = 0;
    cm = cin = crows = 0;
  };
  for (int b = 0; b < nb; ++b) {
    const int64_t mb = (int64_t)nr[b] * nc[b];
    if (mb > tgt || nr[b] > kItemMaxRows) {
      flush();
      const int per = (int)std::min<int64_t>(kItemMaxRows, std::max<int64_t>(1, tgt / std::max(nc[b], 1)));
      for (int r = 0; r < nr[b]; r += per) emit(b, 1, r, std::min(nr[b], r + per));
      continue;
    }
    const bool contiguous = cnb > 0 && m_off[b] == m_off[b - 1] + (int64_t)nr[b - 1] * nc[b - 1];
    if (cnb > 0 && (!contiguous || cm + mb > tgt || cin + nc[b] > kItemMaxIn || crows + nr[b] > kItemMaxRows ||
                    cnb == kItemMaxBlocks))
      flush();
    if (cnb == 0) cb0 = b;
    ++cnb;
    cm += mb;
    cin += nc[b];
    crows += nr[b];
  }
  flush();
  if (gidx.size() >= ((size_t)1 << 31) || gout.size() >= ((size_t)1 << 31) || tabs.size() >= ((size_t)1 << 31))
    return AMGDD_OK;
  // lanes per row from the mean row length in 16-byte vectors of FP32
  const double nvec = (rows > 0 ? ncsum / rows : 0.0) / 4.0;
  p.item_lanes = nvec >= 48 ? 32 : (nvec >= 16 ? 16 : (nvec >= 6 ? 8 : 4));
  p.item_max_in = max_in;
  p.item_max_m = max_m;
  p.item_max_rows = max_rows;
  p.nitems = (int)items.size();
  AMGDD_TRY(p.items.upload(items, s));
  AMGDD_TRY(p.tabs.upload(tabs, s));
  AMGDD_TRY(p.gidx.upload(gidx, s));
  AMGDD_TRY(p.gout.upload(gout, s));
  AMGDD_CUDA(cudaStreamSynchronize(s));
  p.staged = true;
  return AMGDD_OK;
}

// force: 0 picks the mode from the row length, 1 lanes-per-row chunks,
// 2 row per lane (the caller then passes the transposed copy).
// Default rows per CTA of the lanes-per-row form: enough CTAs to fill the GPU
// (8 per SM), at least one row per lane group, at most 64.
int default_rpc(int64_t rows, int lanes) {
  const int ngrp = 128 / lanes;
  const int64_t rpc = rows / (152 * 8);
  return (int)std::max<int64_t>(ngrp, std::min<int64_t>(64, (rpc + ngrp - 1) / ngrp * ngrp));
}

// CTA chunks of the lanes-per-row form: `rpc` rows of one block each.
int set_chunks(SegPlan& p, int rpc, cudaStream_t s) {
  std::vector<int32_t> cb, cr;
  std::vector<SegDesc> cd;
  for (int b = 0; b < p.nblocks; ++b)
    for (int r = 0; r < p.h_nr[b]; r += rpc) {
      cb.push_back(b);
      cr.push_back(r);
      cd.push_back(SegDesc{p.h_moff[b], p.h_ioff[b], p.h_ooff[b], r, std::min(p.h_nr[b], r + rpc), p.h_nc[b],
                           p.h_nr[b]});
    }
  p.rows_per_chunk = rpc;
  p.nchunks = (int)cb.size();
  AMGDD_TRY(p.chunk_blk.upload(cb, s));
  AMGDD_TRY(p.chunk_desc.upload(cd, s));
  return p.chunk_row0.upload(cr, s);
}

int build_seg(SegPlan& p, const std::vector<int32_t>& nr, const std::vector<int32_t>& nc,
              const std::vector<int64_t>& m_off, const std::vector<int64_t>& in_off,
              const std::vector<int64_t>& out_off, const int32_t* in_ext, const int32_t* out_ext, cudaStream_t s,
              int force = 0) {
  p.nblocks = (int)nr.size();
  p.max_nc = 0;
  p.mat_len = 0;
  int64_t rows = 0, cols = 0;
  for (int b = 0; b < p.nblocks; ++b) {
    p.max_nc = std::max(p.max_nc, nc[b]);
    p.mat_len += (int64_t)nr[b] * nc[b];
    rows += nr[b];
    cols += nc[b];
  }
  p.in_len = cols;
  p.out_len = rows;
  p.lanes = lanes_for(p.max_nc);
  p.rows_per_chunk = default_rpc(rows, p.lanes);
  // 16-byte vector loads when every row starts aligned (FP32 and FP64 copies
  // share offsets, so 4-element alignment serves both)
  p.vec = p.nblocks > 0;
  for (int b = 0; b < p.nblocks && p.vec; ++b)
    if (nc[b] % 4 != 0 || m_off[b] % 4 != 0) p.vec = false;
  p.in_idx_ext = in_ext;
  p.out_idx_ext = out_ext;
  // short rows: one lane per output row over the transposed copy
  // row per lane needs no reduction but walks columns with a stride, which
  // streams well only for short rows (measured: long rows lose 2x)
  // (short-row plans carry both forms; the tuner may switch to lanes per row)
  p.rows_mode = force == 2 || (force == 0 && p.max_nc <= 128);
  p.unroll = !p.rows_mode && p.lanes == 32 && rows > 0 && (double)p.mat_len / (double)rows >= 512.0;
  if (p.rows_mode) {
    int max_nr = 0;
    for (int b = 0; b < p.nblocks; ++b) max_nr = std::max(max_nr, nr[b]);
    p.kind = max_nr >= 24 ? 32 : (max_nr >= 12 ? 16 : 8);
    std::vector<int32_t> tb, tr, tn;
    std::vector<SegDesc> td;
    for (int b = 0; b < p.nblocks; ++b) {
      for (int r = 0; r < nr[b]; r += p.kind) {
        tb.push_back(b);
        tr.push_back(r);
        tn.push_back(std::min(p.kind, nr[b] - r));
        td.push_back(SegDesc{m_off[b], in_off[b], out_off[b], r, r + std::min(p.kind, nr[b] - r), nc[b], nr[b]});
      }
    }
    p.ntasks = (int)tb.size();
    AMGDD_TRY(p.task_blk.upload(tb, s));
    AMGDD_TRY(p.task_row0.upload(tr, s));
    AMGDD_TRY(p.task_nrow.upload(tn, s));
    AMGDD_TRY(p.task_desc.upload(td, s));
  }
  p.h_nr = nr;
  p.h_nc = nc;
  p.h_moff = m_off;
  p.h_ioff = in_off;
  p.h_ooff = out_off;
  if (force != 2) {
    AMGDD_TRY(set_chunks(p, p.rows_per_chunk, s));
  } else {
    p.nchunks = 0;
  }
  AMGDD_TRY(p.nr.upload(nr, s));
  AMGDD_TRY(p.nc.upload(nc, s));
  AMGDD_TRY(p.m_off.upload(m_off, s));
  AMGDD_TRY(p.in_off.upload(in_off, s));
  AMGDD_TRY(p.out_off.upload(out_off, s));
  return build_items(p, nr, nc, m_off, in_off, out_off, in_ext, out_ext, s);
}

int apply_kind(int sz) {
  if (sz <= 4) return 0;
  if (sz <= 8) return 1;
  if (sz <= 16) return 2;
  if (sz <= 32) return 3;
  if (sz <= 64) return 4;
  if (sz <= 128) return 5;
  if (sz <= 256) return 6;
  return 7;  // up to kApplyMaxS
}
const int kKindLanes[8] = {1, 8, 16, 32, 32, 32, 32, 32};
constexpr int kApplyMaxS = 512;  // wider supports use the two-pass plans
constexpr int kWideRows = 8;     // rows per task of the wide kinds

int build_apply(Level& L, cudaStream_t s) {
  ApplyPlan& p = L.aplan;
  const int64_t ng = (int64_t)L.g_ptr.size() - 1;
  std::vector<std::vector<int32_t>> tg(8), tr(8), tn(8);
  p.r_len = 0;
  // wide supports: t = R_g x(S_g), then y(S_g) -= R_g^T t
  std::vector<int32_t> n1, c1, n2, c2;
  std::vector<int64_t> moff, in1, out1, in2, out2;
  int64_t toff = 0;
  for (int64_t g = 0; g < ng; ++g) {
    const int sz = (int)(L.g_ptr[g + 1] - L.g_ptr[g]);
    const int rk = L.g_rank[g];
    if (rk == 0 || sz == 0) continue;
    if (sz > kApplyMaxS) {
      n1.push_back(rk);
      c1.push_back(sz);
      n2.push_back(sz);
      c2.push_back(rk);
      moff.push_back(L.h_off[g]);
      in1.push_back(L.g_ptr[g]);
      out1.push_back(toff);
      in2.push_back(toff);
      out2.push_back(L.g_ptr[g]);
      toff += rk;
      continue;
    }
    const int kd = apply_kind(sz);
    p.r_len += (int64_t)rk * sz;
    const int chunk = kd >= 4 ? kWideRows : rk;
    for (int r = 0; r < rk; r += chunk) {
      tg[kd].push_back((int32_t)g);
      tr[kd].push_back(r);
      tn[kd].push_back(std::min(chunk, rk - r));
    }
  }
  std::vector<int32_t> ag, ar, an;
  p.nbuckets = 0;
  int cta = 0;
  for (int kd = 0; kd < 8; ++kd) {
    if (tg[kd].empty()) continue;
    const int per = kd == 0 ? 256 : 128 / kKindLanes[kd];  // kind 0: two groups per thread
    p.bucket_kind[p.nbuckets] = kd;
    p.bucket_start[p.nbuckets] = cta;
    p.bucket_tasks[p.nbuckets] = (int)tg[kd].size();
    cta += (int)((tg[kd].size() + per - 1) / per);
    ++p.nbuckets;
    ag.insert(ag.end(), tg[kd].begin(), tg[kd].end());
    ar.insert(ar.end(), tr[kd].begin(), tr[kd].end());
    an.insert(an.end(), tn[kd].begin(), tn[kd].end());
  }
  p.bucket_start[p.nbuckets] = cta;
  p.ntasks = (int)ag.size();
  AMGDD_TRY(p.task_grp.upload(ag, s));
  AMGDD_TRY(p.task_row0.upload(ar, s));
  AMGDD_TRY(p.task_nrow.upload(an, s));
  L.t_len = toff;
  if (toff > 0) {
    std::vector<int32_t> io(toff);
    std::iota(io.begin(), io.end(), 0);
    AMGDD_TRY(L.d_tidx.upload(io, s));
    AMGDD_TRY(L.t64.alloc(toff));
    AMGDD_TRY(L.t32.alloc(toff));
    AMGDD_TRY(build_seg(L.gt1, n1, c1, moff, in1, out1, L.d_g_idx.p, L.d_tidx.p, s, 1));
    AMGDD_TRY(build_seg(L.gt2, n2, c2, moff, in2, out2, L.d_tidx.p, L.d_g_idx.p, s, 2));
  }
  return AMGDD_OK;
}

// A_l by block rows (Eq. 1 summed per row group): blocks are runs of
// consecutive dofs with identical group lists.  On coarse levels every G_l
// row touches whole blocks of coarse dofs (the columns of one Z_i), so a
// block's rows share the support in_b and A(D_b, in_b) is dense.  Used when
// it moves no more bytes than the matrix-free form.
int build_blockrows(Level& L, cudaStream_t s, const std::vector<double>* saved = nullptr) {
  Supports S;
  S.ptr = L.g_ptr;
  S.idx = L.g_idx;
  std::vector<int64_t> nptr;
  std::vector<int32_t> ngrp;
  node_groups(S, L.n, nptr, ngrp);
  const int64_t n = L.n;
  auto same_groups = [&](int64_t u, int64_t v) {
    return nptr[u + 1] - nptr[u] == nptr[v + 1] - nptr[v] &&
           std::equal(ngrp.begin() + nptr[u], ngrp.begin() + nptr[u + 1], ngrp.begin() + nptr[v]);
  };
  std::vector<int32_t> nr, nc, pgrp, pp0, map, blk_in;
  std::vector<int64_t> moff, ioff, ooff, pptr(1, 0), pmap;
  std::vector<int64_t> mark(n, -1);
  std::vector<int32_t> loc(n, -1);
  int64_t mat = 0;
  for (int64_t d0 = 0; d0 < n;) {
    int64_t d1 = d0 + 1;
    while (d1 < n && same_groups(d0, d1)) ++d1;
    const int32_t kb = (int32_t)(d1 - d0);
    const int64_t b = (int64_t)nr.size();
    const int64_t i0 = (int64_t)blk_in.size();
    for (int64_t q = nptr[d0]; q < nptr[d0 + 1]; ++q) {
      const int32_t g = ngrp[q];
      for (int64_t e = L.g_ptr[g]; e < L.g_ptr[g + 1]; ++e) {
        const int32_t v = L.g_idx[e];
        if (mark[v] != b) {
          mark[v] = b;
          blk_in.push_back(v);
        }
      }
    }
    std::sort(blk_in.begin() + i0, blk_in.end());
    const int32_t nin = (int32_t)(blk_in.size() - i0);
    for (int32_t c = 0; c < nin; ++c) loc[blk_in[i0 + c]] = c;
    for (int64_t q = nptr[d0]; q < nptr[d0 + 1]; ++q) {
      const int32_t g = ngrp[q];
      const auto first = L.g_idx.begin() + L.g_ptr[g], last = L.g_idx.begin() + L.g_ptr[g + 1];
      const int64_t p0 = std::lower_bound(first, last, (int32_t)d0) - first;
      if (p0 + kb > last - first || *(first + p0 + kb - 1) != (int32_t)(d1 - 1)) {
        set_error("block rows: dofs %lld..%lld are not contiguous in a group support", (long long)d0,
                  (long long)(d1 - 1));
        return AMGDD_ERR_INTERNAL;
      }
      pgrp.push_back(g);
      pp0.push_back((int32_t)p0);
      pmap.push_back((int64_t)map.size());
      for (auto it = first; it != last; ++it) map.push_back(loc[*it]);
    }
    for (int32_t c = 0; c < nin; ++c) loc[blk_in[i0 + c]] = -1;
    pptr.push_back((int64_t)pgrp.size());
    nr.push_back(kb);
    nc.push_back(nin);
    moff.push_back(mat);
    ioff.push_back(i0);
    ooff.push_back(d0);
    mat += (int64_t)kb * nin;
    d0 = d1;
  }
  const int nblk = (int)nr.size();
  // bytes of one residual in FP32: block rows against the matrix-free form
  const double blk_bytes = (double)mat * 4.0 + (double)blk_in.size() * 4.0 + 3.0 * n * 4.0;
  const double mf_bytes = apply_bytes(L, 4);
  L.blk_mb = blk_bytes / 1e6;
  L.mf_mb = mf_bytes / 1e6;
  if (nblk * 2 > n) {  // (near-)singleton blocks: nothing to gain
    if (saved && !saved->empty()) {
      set_error("saved hierarchy: block rows stored for a level that has none");
      return AMGDD_ERR_INVALID_ARG;
    }
    return AMGDD_OK;
  }
  if (saved) {  // a loaded hierarchy: the stored FP64 block rows, or none (the row groups won at setup)
    if (saved->empty()) return AMGDD_OK;
    if ((int64_t)saved->size() != mat) {
      set_error("saved hierarchy: %zu block-row entries, the structure has %lld", saved->size(), (long long)mat);
      return AMGDD_ERR_INVALID_ARG;
    }
    DBuf<int32_t> dnr, dnc;
    DBuf<int64_t> dmoff;
    AMGDD_TRY(dnr.upload(nr, s));
    AMGDD_TRY(dnc.upload(nc, s));
    AMGDD_TRY(dmoff.upload(moff, s));
    AMGDD_TRY(L.A64.upload(*saved, s));
    AMGDD_TRY(L.At64.alloc(mat));
    AMGDD_TRY(L.A32.alloc(mat));
    AMGDD_TRY(L.At32.alloc(mat));
    AMGDD_TRY(launch_block_copies(nblk, dnr.p, dnc.p, dmoff.p, L.A64.p, L.A32.p, L.At64.p, L.At32.p, s));
    AMGDD_TRY(L.d_blk_in.upload(blk_in, s));
    std::vector<int32_t> io(n);
    std::iota(io.begin(), io.end(), 0);
    AMGDD_TRY(L.d_blk_out.upload(io, s));
    AMGDD_TRY(build_seg(L.ablk, nr, nc, moff, ioff, ooff, L.d_blk_in.p, L.d_blk_out.p, s));
    AMGDD_CUDA(cudaStreamSynchronize(s));
    L.has_blk = true;
    return AMGDD_OK;
  }
  DBuf<int32_t> dnr, dnc, dpgrp, dpp0, dmap;
  DBuf<int64_t> dmoff, dpptr, dpmap;
  AMGDD_TRY(dnr.upload(nr, s));
  AMGDD_TRY(dnc.upload(nc, s));
  AMGDD_TRY(dmoff.upload(moff, s));
  AMGDD_TRY(dpptr.upload(pptr, s));
  AMGDD_TRY(dpgrp.upload(pgrp, s));
  AMGDD_TRY(dpp0.upload(pp0, s));
  AMGDD_TRY(dpmap.upload(pmap, s));
  AMGDD_TRY(dmap.upload(map, s));
  AMGDD_TRY(L.A64.alloc(mat));
  AMGDD_TRY(L.At64.alloc(mat));
  AMGDD_TRY(L.A32.alloc(mat));
  AMGDD_TRY(L.At32.alloc(mat));
  AMGDD_TRY(launch_blockrows(nblk, dnr.p, dnc.p, dmoff.p, dpptr.p, dpgrp.p, dpp0.p, dpmap.p, dmap.p, L.d_g_ptr.p,
                             L.d_h_off.p, L.d_H.p, L.A64.p, L.A32.p, L.At64.p, L.At32.p, s));
  AMGDD_TRY(L.d_blk_in.upload(blk_in, s));
  std::vector<int32_t> io(n);
  std::iota(io.begin(), io.end(), 0);
  AMGDD_TRY(L.d_blk_out.upload(io, s));
  AMGDD_TRY(build_seg(L.ablk, nr, nc, moff, ioff, ooff, L.d_blk_in.p, L.d_blk_out.p, s));
  AMGDD_CUDA(cudaStreamSynchronize(s));
  L.has_blk = true;
  return AMGDD_OK;
}

// Setup-time choice of the gather-GEMV form for one plan: time the unstaged
// scalar, staged and shifted-vector kernels and the row-per-lane kernel that
// apply on scratch vectors (`nin` inputs, `nout` outputs) and keep the
// fastest; the lanes-per-row forms also over lanes per row and rows per CTA.
// The staged form's arrays are freed when it loses.  The choice is made in
// the precision T; `shift_only` then re-times, in the other precision, only
// shifted against scalar loads for a plan that kept a lanes-per-row form
// (the flag of each precision is separate).  Cached choices are coded
// form + 16 rows-per-CTA + 4096 lanes.
template <class T>
int tune_seg(SegPlan& p, const std::string& key, const T* M, const T* MT, int64_t nin, int64_t nout, SegMode mode,
             cudaStream_t s, bool shift_only = false) {
  constexpr bool f32 = sizeof(T) == 4;
  bool& shift = f32 ? p.shift : p.shift64;
  // candidate forms: 0 lanes per row, scalar loads; 1 staged (when built);
  // 2 lanes per row with shifted vector loads (rows at any alignment; the
  // W shifted copies of x take about 16 bytes of shared
  // memory per column); 3 row per lane over the transposed copy (short rows)
  const bool chunk_now = !p.staged && !p.rows_mode;
  const bool can_rows = !shift_only && p.ntasks > 0 && MT != nullptr;
  const bool can_chunk = p.nchunks > 0 && (!shift_only || chunk_now);
  const bool shift_fits = !p.vec && 16.0 * (p.max_nc + 8) <= 160.0 * 1024.0;
  const bool can_shift = can_chunk && shift_fits;
  const bool rows0 = p.rows_mode;
  const int lanes0 = p.lanes, rpc0 = p.rows_per_chunk;
  int64_t nrows = 0;
  for (int v : p.h_nr) nrows += v;
  auto drop_staged = [&p] {
    p.items.release();
    p.tabs.release();
    p.gidx.release();
    p.gout.release();
  };
  shift = false;
  if (shift_only ? !can_shift : (!p.staged && !can_shift && !(can_rows && can_chunk))) return AMGDD_OK;
  if (g_err_word == nullptr || M == nullptr) return AMGDD_OK;
  auto set_form = [&](int form) {
    shift = form == 2;
    if (shift_only) return;
    p.staged = form == 1;
    p.rows_mode = form == 3 || (form == 1 && rows0);
  };
  // lanes-per-row layout (lanes, rows per CTA); restores the built one for
  // the other forms
  auto set_layout = [&](int lanes, int rpc) -> int {
    if (p.lanes == lanes && p.rows_per_chunk == rpc) return AMGDD_OK;
    p.lanes = lanes;
    p.unroll = lanes == 32 && nrows > 0 && (double)p.mat_len / (double)nrows >= 512.0;
    return set_chunks(p, rpc, s);
  };
  double cached = 0.0;
  if (g_tune && (g_tune->get(key, cached) || !g_tune->on)) {
    // without timing: the built form (row per lane for short rows), or the
    // form asked for (tune = 2, 3, 4) where the plan allows it
    const int code = (int)cached;
    int form = g_tune->on ? code % 16 : (g_tune->prefer_form >= 0 ? g_tune->prefer_form : (rows0 ? 3 : 0));
    if (shift_only) {
      set_form(form == 2 ? 2 : 0);
      return AMGDD_OK;
    }
    const int lanes = g_tune->on ? code / 4096 : 0, rpc = g_tune->on ? (code / 16) % 256 : 0;
    const bool lanes_ok = lanes == 4 || lanes == 8 || lanes == 16 || lanes == 32;
    if (lanes_ok && rpc > 0 && can_chunk) AMGDD_TRY(set_layout(lanes, rpc));
    if ((form == 1 && !p.staged) || (form == 2 && !can_shift) || (form == 3 && !can_rows) ||
        ((form == 0 || form == 2) && !can_chunk)) {
      form = rows0 ? 3 : 0;
      if (can_chunk) AMGDD_TRY(set_layout(lanes0, rpc0));
    }
    set_form(form);
    if (!p.staged) drop_staged();
    return AMGDD_OK;
  }
  DBuf<T> xin, yout, cin;
  AMGDD_TRY(xin.alloc(std::max<int64_t>(nin, 1)));
  AMGDD_TRY(yout.alloc(std::max<int64_t>(nout, 1)));
  AMGDD_TRY(cin.alloc(std::max<int64_t>(nout, 1)));
  AMGDD_TRY(xin.zero(s));
  AMGDD_TRY(yout.zero(s));
  AMGDD_TRY(cin.zero(s));
  const bool built = !shift_only && p.staged;
  // candidates (form, lanes, rows per CTA)
  struct Cand {
    int form, lanes, rpc;
  };
  std::vector<Cand> cands;
  if (shift_only) {
    cands.push_back({0, lanes0, rpc0});
    cands.push_back({2, lanes0, rpc0});
  } else {
    if (built) cands.push_back({1, lanes0, rpc0});
    if (can_rows) cands.push_back({3, lanes0, rpc0});
    if (can_chunk)
      for (int form : {0, 2}) {
        if (form == 2 && !can_shift) continue;
        std::vector<int> ls{lanes0};
        for (int l : {4, 8, 16, 32})
          if (l != lanes0) ls.push_back(l);
        for (int l : ls) {
          const int r0 = l == lanes0 ? rpc0 : default_rpc(nrows, l);
          for (int r = r0; r <= std::max(r0, 128); r *= 2) cands.push_back({form, l, r});
        }
      }
  }
  constexpr int kReps = 8;
  int rc = AMGDD_OK;
  float best_t = 0.f;
  int best = -1;
  float tf[4] = {0.f, 0.f, 0.f, 0.f};
  for (size_t ci = 0; ci < cands.size() && rc == AMGDD_OK; ++ci) {
    const Cand& c = cands[ci];
    set_form(c.form);
    if (c.form == 0 || c.form == 2) rc = set_layout(c.lanes, c.rpc);
    float ms = 0.f;
    if (rc == AMGDD_OK)
      rc = time_cold(s, kReps, [&] {
        return launch_seg(p, M, f32, xin.p, yout.p, f32, mode, nullptr, s, mode == SEG_RESID ? cin.p : nullptr,
                          nullptr, MT);
      }, &ms);
    if (tf[c.form] == 0.f || ms < tf[c.form]) tf[c.form] = ms;
    if (best < 0 || ms < best_t) {
      best = (int)ci;
      best_t = ms;
    }
  }
  AMGDD_TRY(rc);
  const Cand& b = cands[best];
  set_form(b.form);
  if (can_chunk) AMGDD_TRY((b.form == 0 || b.form == 2) ? set_layout(b.lanes, b.rpc) : set_layout(lanes0, rpc0));
  if (g_tune) g_tune->put(key, (double)(b.form + (shift_only ? 0 : 16 * p.rows_per_chunk + 4096 * p.lanes)));
  if (g_timer.on)
    fprintf(stderr,
            "[amgdd]   plan %d blocks (%s): lanes/row %.1f us, staged %.1f us, shifted %.1f us, row/lane %.1f us -> "
            "%d (%d lanes, %d rows per CTA)\n",
            p.nblocks, f32 ? "fp32" : "fp64", 1e3 * tf[0] / kReps, 1e3 * tf[1] / kReps, 1e3 * tf[2] / kReps,
            1e3 * tf[3] / kReps, b.form, p.lanes, p.rows_per_chunk);
  if (!shift_only && !p.staged) drop_staged();
  return AMGDD_OK;
}

// Staged/unstaged choice for every gather-GEMV plan of level `lvl`.
int tune_level_plans(Level& L, int lvl, int64_t n_next, cudaStream_t s) {
  const std::string k = "L" + std::to_string(lvl) + "|";
  if (L.coarsest) return tune_seg<double>(L.ras, k + "coarse", L.W64.p, L.Wt64.p, L.n, L.n, SEG_STORE, s);
  AMGDD_TRY(tune_seg<float>(L.ras, k + "ras", L.W32.p, L.Wt32.p, L.n, L.n, SEG_STORE, s));
  AMGDD_TRY(tune_seg<float>(L.rast, k + "rast", L.Wt32.p, L.W32.p, L.n, L.n, SEG_ATOMIC_ADD, s));
  if (L.yd32.p) AMGDD_TRY(tune_seg<float>(L.rast_det, k + "rastd", L.Wt32.p, L.W32.p, L.n, L.om_ptr.back(), SEG_STORE, s));
  if (L.Wf64.p)  // the additive form runs in FP64 only
    AMGDD_TRY(tune_seg<double>(L.asp, k + "as64", L.Wf64.p, L.Wft64.p, L.n, L.n, SEG_ATOMIC_ADD, s));
  AMGDD_TRY(tune_seg<float>(L.restr, k + "restrict", L.Zt32.p, L.Z32.p, L.n, n_next, SEG_STORE, s));
  AMGDD_TRY(tune_seg<float>(L.prol, k + "prolong", L.Z32.p, L.Zt32.p, n_next, L.n, SEG_ADD, s));
  if (L.A32.p) AMGDD_TRY(tune_seg<float>(L.ablk, k + "blockrows", L.A32.p, L.At32.p, L.n, L.n, SEG_RESID, s));
  // FP64 copies: shifted or scalar loads, within the form chosen above
  AMGDD_TRY(tune_seg<double>(L.ras, k + "ras64", L.W64.p, L.Wt64.p, L.n, L.n, SEG_STORE, s, true));
  AMGDD_TRY(tune_seg<double>(L.rast, k + "rast64", L.Wt64.p, L.W64.p, L.n, L.n, SEG_ATOMIC_ADD, s, true));
  if (L.yd64.p)
    AMGDD_TRY(tune_seg<double>(L.rast_det, k + "rastd64", L.Wt64.p, L.W64.p, L.n, L.om_ptr.back(), SEG_STORE, s,
                               true));
  AMGDD_TRY(tune_seg<double>(L.restr, k + "restrict64", L.Zt64.p, L.Z64.p, L.n, n_next, SEG_STORE, s, true));
  AMGDD_TRY(tune_seg<double>(L.prol, k + "prolong64", L.Z64.p, L.Zt64.p, n_next, L.n, SEG_ADD, s, true));
  if (L.A64.p) AMGDD_TRY(tune_seg<double>(L.ablk, k + "blockrows64", L.A64.p, L.At64.p, L.n, L.n, SEG_RESID, s, true));
  return AMGDD_OK;
}

// A of level 0 by rows in ELL form, from the rows omega_i of A over Omega_i
// (Aw, which holds every entry of those rows once Omega_i contains their
// graph neighbours, i.e. with overlap >= 1).  A row's columns are the union
// of the supports of the G row groups that contain its node.  Not built (and
// the row groups serve) where a column falls outside Omega_i.
int build_ell(Level& L, cudaStream_t s) {
  if (L.Aw64.p == nullptr || L.nagg == 0 || L.n <= 0) return AMGDD_OK;
  const int64_t n = L.n;
  const int64_t ng = (int64_t)L.g_ptr.size() - 1;
  std::vector<int64_t> ip(n + 1, 0);
  for (int64_t g = 0; g < ng; ++g)
    for (int64_t q = L.g_ptr[g]; q < L.g_ptr[g + 1]; ++q) ++ip[L.g_idx[q] + 1];
  for (int64_t i = 0; i < n; ++i) ip[i + 1] += ip[i];
  std::vector<int64_t> ig(ip[n]), fill(ip.begin(), ip.end() - 1);
  for (int64_t g = 0; g < ng; ++g)
    for (int64_t q = L.g_ptr[g]; q < L.g_ptr[g + 1]; ++q) ig[fill[L.g_idx[q]]++] = g;
  // row lists
  std::vector<int64_t> rp(n + 1, 0);
  std::vector<int32_t> rc;
  std::vector<int32_t> tmp;
  for (int64_t i = 0; i < n; ++i) {
    tmp.clear();
    for (int64_t q = ip[i]; q < ip[i + 1]; ++q) {
      const int64_t g = ig[q];
      tmp.insert(tmp.end(), L.g_idx.begin() + L.g_ptr[g], L.g_idx.begin() + L.g_ptr[g + 1]);
    }
    std::sort(tmp.begin(), tmp.end());
    tmp.erase(std::unique(tmp.begin(), tmp.end()), tmp.end());
    rc.insert(rc.end(), tmp.begin(), tmp.end());
    rp[i + 1] = (int64_t)rc.size();
  }
  int w = 0;
  for (int64_t i = 0; i < n; ++i) w = std::max<int>(w, (int)(rp[i + 1] - rp[i]));
  if (w == 0 || w > 64) return AMGDD_OK;
  std::vector<int64_t> src((size_t)(n * w), -1);
  std::vector<int32_t> col((size_t)(n * w));
  for (int64_t k = 0; k < w; ++k)
    for (int64_t i = 0; i < n; ++i) col[k * n + i] = (int32_t)i;
  std::vector<int32_t> pos(n, -1);
  int64_t woff = 0;
  for (int a = 0; a < L.nagg; ++a) {
    const int64_t o0 = L.om_ptr[a], no = L.om_ptr[a + 1] - o0;
    for (int64_t c = 0; c < no; ++c) pos[L.om_idx[o0 + c]] = (int32_t)c;
    bool ok = true;
    for (int r = 0; r < L.nomega[a] && ok; ++r) {
      const int32_t i = L.om_idx[o0 + r];
      for (int64_t q = rp[i]; q < rp[i + 1]; ++q) {
        const int32_t j = rc[q];
        if (pos[j] < 0) {
          ok = false;
          break;
        }
        const int64_t k = q - rp[i];
        src[k * n + i] = woff + (int64_t)r * no + pos[j];
        col[k * n + i] = j;
      }
    }
    for (int64_t c = 0; c < no; ++c) pos[L.om_idx[o0 + c]] = -1;
    if (!ok) return AMGDD_OK;  // a row reaches outside its subdomain
    woff += (int64_t)L.nomega[a] * no;
  }
  DBuf<int64_t> dsrc;
  AMGDD_TRY(dsrc.upload(src, s));
  AMGDD_TRY(L.ellc.upload(col, s));
  AMGDD_TRY(L.ell64.alloc((size_t)(n * w)));
  AMGDD_TRY(L.ell32.alloc((size_t)(n * w)));
  AMGDD_TRY(launch_ell_fill(n * w, dsrc.p, L.Aw64.p, L.ell64.p, L.ell32.p, s));
  AMGDD_CUDA(cudaStreamSynchronize(s));
  L.ell_w = w;
  return AMGDD_OK;
}

// Setup-time choice between the ELL rows and the row groups for level 0's A:
// time one FP32 residual in each and keep the faster (row groups without
// timing).
int tune_ell(Level& L, int forced, cudaStream_t s) {
  if (L.ell_w == 0) return AMGDD_OK;
  auto drop = [&L] {
    L.use_ell = false;
    L.ellc.release();
    L.ell64.release();
    L.ell32.release();
    L.ell_w = 0;
  };
  if (forced != 0) {
    if (forced > 0)
      L.use_ell = true;
    else
      drop();
    return AMGDD_OK;
  }
  double cached = 0.0;
  if (g_tune && (g_tune->get("L0|ell", cached) || !g_tune->on)) {
    if (g_tune->on && cached != 0.0)
      L.use_ell = true;
    else
      drop();
    return AMGDD_OK;
  }
  AMGDD_TRY(L.x32.zero(s));
  AMGDD_TRY(L.r32.zero(s));
  cudaEvent_t e[2];
  for (auto& v : e) AMGDD_CUDA(cudaEventCreate(&v));
  float t[2] = {0.f, 0.f};
  constexpr int kReps = 10;
  int rc = AMGDD_OK;
  for (int form = 0; form < 2 && rc == AMGDD_OK; ++form) {
    for (int rep = 0; rep < kReps + 2 && rc == AMGDD_OK; ++rep) {
      if (rep == 2) cudaEventRecord(e[0], s);
      rc = form == 0 ? launch_ell(L, true, L.x32.p, L.s32.p, L.r32.p, nullptr, s)
                     : launch_apply(L.aplan, L, true, L.x32.p, L.s32.p, -1, nullptr, s);
    }
    cudaEventRecord(e[1], s);
    if (rc == AMGDD_OK &&
        (cudaEventSynchronize(e[1]) != cudaSuccess || cudaEventElapsedTime(&t[form], e[0], e[1]) != cudaSuccess))
      rc = AMGDD_ERR_CUDA;
  }
  for (auto& v : e) cudaEventDestroy(v);
  AMGDD_TRY(rc);
  L.ell_us = 1e3 * t[0] / kReps;
  L.mf_us = 1e3 * t[1] / kReps;
  const bool use = L.ell_us < L.mf_us;
  if (g_tune) g_tune->put("L0|ell", use ? 1.0 : 0.0);
  if (g_timer.on)
    fprintf(stderr, "[amgdd] level 0 A-apply: ELL (%d slots) %.1f us, row groups %.1f us\n", L.ell_w, L.ell_us,
            L.mf_us);
  if (use)
    L.use_ell = true;
  else
    drop();
  return AMGDD_OK;
}

// Setup-time tuning of the coarse A-apply: time one FP32 residual of level L
// in both stored forms and keep the faster.  Block rows move more bytes than
// the compressed row groups but need no atomics and stream dense rows.
int tune_level_A(Level& L, int lvl, cudaStream_t s) {
  if (!L.has_blk) return AMGDD_OK;
  const std::string key = "L" + std::to_string(lvl) + "|A";
  double cached = 0.0;
  if (g_tune && (g_tune->get(key, cached) || !g_tune->on)) {
    // default without tuning: block rows (faster on every coarse level measured)
    if (g_tune->on && cached == 0.0) {
      L.has_blk = false;
      L.A64.release();
      L.At64.release();
      L.A32.release();
      L.At32.release();
    }
    return AMGDD_OK;
  }
  AMGDD_TRY(L.x32.zero(s));
  AMGDD_TRY(L.r32.zero(s));
  cudaEvent_t e[3];
  for (auto& v : e) AMGDD_CUDA(cudaEventCreate(&v));
  float t[2] = {0.f, 0.f};
  constexpr int kReps = 10;
  int rc = AMGDD_OK;
  for (int form = 0; form < 2 && rc == AMGDD_OK; ++form) {
    for (int rep = 0; rep < kReps + 2 && rc == AMGDD_OK; ++rep) {
      if (rep == 2) cudaEventRecord(e[0], s);
      rc = form == 0 ? launch_seg(L.ablk, L.A32.p, true, L.x32.p, L.s32.p, true, SEG_RESID, nullptr, s, L.r32.p,
                                  nullptr, L.At32.p)
                     : launch_apply(L.aplan, L, true, L.x32.p, L.s32.p, -1, nullptr, s);
    }
    cudaEventRecord(e[1], s);
    if (cudaEventSynchronize(e[1]) != cudaSuccess || cudaEventElapsedTime(&t[form], e[0], e[1]) != cudaSuccess)
      rc = AMGDD_ERR_CUDA;
  }
  for (auto& v : e) cudaEventDestroy(v);
  AMGDD_TRY(rc);
  L.blk_us = 1e3 * t[0] / kReps;
  L.mf_us = 1e3 * t[1] / kReps;
  if (g_timer.on)
    fprintf(stderr, "[amgdd] n=%lld A-apply: block rows %.1f MB %.1f us, matrix-free %.1f MB %.1f us\n",
            (long long)L.n, L.blk_mb, L.blk_us, L.mf_mb, L.mf_us);
  if (g_tune) g_tune->put(key, L.mf_us <= L.blk_us ? 0.0 : 1.0);
  if (L.mf_us <= L.blk_us) {
    L.has_blk = false;
    L.A64.release();
    L.At64.release();
    L.A32.release();
    L.At32.release();
  }
  return AMGDD_OK;
}

}  // namespace

// What setup computed for one level, as a saved hierarchy stores it: the
// structure (row groups of G_l, aggregates, Omega lists, k_i and offsets)
// and the FP64 matrices (compressed rows R_g, smoother rows W_i, rows of A
// over Omega_i, spectra, bases Z_i, the additive form's A_i^{-1}, coarse
// block rows, the coarsest inverse).  The FP32 and transposed copies are
// derived again on load.
struct LevelSnap {
  int64_t n = 0, nnzA = 0;
  int32_t nagg = 0, coarsest = 0, schur_rows = 0, n_color = 0, n_mult = 0;
  double thresh = 0.0, inv_err = 0.0;
  std::vector<int64_t> g_ptr, h_off, om_ptr, z_off, mu_off, col0, wf_off;
  std::vector<int32_t> g_idx, g_rank, agg, om_idx, nomega, k;
  std::vector<double> R64, W64, Aw64, mu, Z64, Wf64, A64;
};
}  // namespace amgdd

using namespace amgdd;

struct amgdd_hierarchy {
  amgdd_params prm{};
  int overlap = 1;
  int64_t n = 0;
  // the setup inputs and the setup-time kernel choices, kept for
  // amgdd_hierarchy_save (host memory)
  std::vector<int64_t> in_rowptr;
  std::vector<int32_t> in_col, in_agg;
  std::vector<double> in_val, in_d1;
  bool in_has_d1 = false;
  std::vector<std::pair<std::string, double>> tune_kv;
  int precision = AMGDD_FP64;
  int device = 0;
  std::vector<std::unique_ptr<Level>> lv;
  std::vector<int64_t> nnzA;  // structural nnz of A_l
  DBuf<int32_t> iota;
  DBuf<double> x, r, z, zold, p, q, b, partials;
  DBuf<PcgState> st;
  PcgState* st_host = nullptr;
  cudaGraphExec_t ginit[2] = {nullptr, nullptr}, gloop[2] = {nullptr, nullptr};
  int64_t ginit_kernels[2] = {0, 0}, gloop_kernels[2] = {0, 0};
  cudaStream_t work = nullptr;  // solves run here (capturable, unlike the legacy stream)
  cudaEvent_t join[2] = {nullptr, nullptr};
  double setup_ms = 0.0;
  bool mixed_stalled = false;  // an FP32-cycle solve stalled; later MIXED32 solves use the FP64 cycle
  int64_t setup_bytes = 0;  // device bytes held after setup
  double phase_ms[16] = {};  // setup time by phase, summed over levels
  double phase_flops[16] = {};  // FP64 flops by phase (counted from the block sizes), summed over levels
  const char* phase_name[16] = {};
  int64_t multi_bytes = 0;  // device bytes of the batched-solve workspace, once allocated
  // persistent V-cycle tail per precision (index 1 = MIXED32): phase list,
  // launch shape, first level (0 = not used); barrier words
  DBuf<PhaseDesc> d_ph[2];
  int nph[2] = {0, 0};
  size_t ph_smem[2] = {0, 0};
  int ph_grid[2] = {0, 0};
  int persist_from[2] = {0, 0};
  double persist_us[2][16] = {};  // setup-time V-cycle timings by first level (0 = all separate launches)
  // dense tail per precision: the V-cycle from this level down is one
  // GEMV with the matrix B of that level (0 = not used)
  int dense_from[2] = {0, 0};
  double dense_us[2][16] = {};  // setup-time V-cycle timings by dense level (0 = none)
  DBuf<unsigned> bar;
  // batched right-hand sides: CG vectors (n x cap, interleaved), cap
  // states, graphs per precision and K in {2, 4, 8, 16, 32}; allocated at
  // the first batched solve for its width and grown (graphs rebuilt) when a
  // wider batch comes
  struct Multi {
    bool ready = false;
    int cap = 0;
    DBuf<double> x, r, z, zold, p, q, b, stage, partials;
    DBuf<PcgState> st;
    DBuf<int> grp;
    PcgState* st_host = nullptr;
    cudaGraphExec_t ginit[2][5] = {}, gloop[2][5] = {};
    int64_t ginit_kernels[2][5] = {}, gloop_kernels[2][5] = {};
    void drop_graphs() {
      for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 5; ++j) {
          if (ginit[i][j]) cudaGraphExecDestroy(ginit[i][j]);
          if (gloop[i][j]) cudaGraphExecDestroy(gloop[i][j]);
          ginit[i][j] = gloop[i][j] = nullptr;
        }
    }
  } mw;
  ~amgdd_hierarchy() {
    for (int i = 0; i < 2; ++i) {
      if (ginit[i]) cudaGraphExecDestroy(ginit[i]);
      if (gloop[i]) cudaGraphExecDestroy(gloop[i]);
    }
    if (st_host) cudaFreeHost(st_host);
    mw.drop_graphs();
    if (mw.st_host) cudaFreeHost(mw.st_host);
    for (auto& e : join)
      if (e) cudaEventDestroy(e);
    if (work) cudaStreamDestroy(work);
  }
};

namespace {

// MIXED32 and MIXED16 run the V-cycle on FP32 vectors under the flexible FP64
// CG; MIXED16 reads the gather-GEMV matrices in FP16 where a level has them.
bool mixed(const amgdd_hierarchy& h) { return h.precision != AMGDD_FP64; }
bool use16(const amgdd_hierarchy& h, const Level& L, bool f32) {
  return f32 && h.precision == AMGDD_MIXED16 && L.h16;
}

// ---------------------------------------------------------------------------
// Compression of the row groups of one level: pivoted Cholesky of each Gram.
int compress(Level& L, cudaStream_t s) {
  if (L.rows_ready) return build_apply(L, s);  // rows carried by QR from the level above
  const int64_t ng = (int64_t)L.g_ptr.size() - 1;
  const int64_t cap = L.h_off.back();
  AMGDD_TRY(L.d_R64.alloc(cap));
  AMGDD_TRY(L.d_R32.alloc(cap));
  AMGDD_TRY(L.d_rank.alloc(ng));
  int max_s = 1;
  for (int64_t g = 0; g < ng; ++g) max_s = std::max(max_s, (int)(L.g_ptr[g + 1] - L.g_ptr[g]));
  const int64_t per = (int64_t)max_s * max_s;
  int64_t chunk = std::max<int64_t>(1, (int64_t)(32 << 20) / per);
  chunk = std::min<int64_t>(chunk, std::max<int64_t>(ng, 1));
  DBuf<double> scratch;
  AMGDD_TRY(scratch.alloc(chunk * per));
  for (int64_t f = 0; f < ng; f += chunk) {
    const int64_t c = std::min(chunk, ng - f);
    AMGDD_TRY(launch_pchol(f, c, max_s, L.d_g_ptr.p, L.d_h_off.p, L.d_H.p, L.d_R64.p, L.d_R32.p, L.d_rank.p,
                           scratch.p, per, s));
  }
  AMGDD_TRY(download(L.g_rank, L.d_rank.p, ng, s));
  for (int64_t g = 0; g < ng; ++g) {  // pivoted Cholesky: the trailing update per kept pivot
    const double sz = (double)(L.g_ptr[g + 1] - L.g_ptr[g]);
    for (int k = 0; k < L.g_rank[g]; ++k) g_timer.flops[6] += (sz - k - 1) * (sz - k - 1) + (sz - k);
  }
  return build_apply(L, s);
}

int alloc_vectors(Level& L) {
  AMGDD_TRY(L.r64.alloc(L.n));
  AMGDD_TRY(L.x64.alloc(L.n));
  AMGDD_TRY(L.s64.alloc(L.n));
  AMGDD_TRY(L.r32.alloc(L.n));
  AMGDD_TRY(L.x32.alloc(L.n));
  AMGDD_TRY(L.s32.alloc(L.n));
  return AMGDD_OK;
}

int64_t structural_nnz(const Level& L, const std::vector<int64_t>& nptr, const std::vector<int32_t>& ngrp) {
  const int64_t n = L.n;
  std::vector<int64_t> mark(n, -1);
  int64_t tot = 0;
  for (int64_t j = 0; j < n; ++j) {
    for (int64_t q = nptr[j]; q < nptr[j + 1]; ++q) {
      const int32_t g = ngrp[q];
      for (int64_t p = L.g_ptr[g]; p < L.g_ptr[g + 1]; ++p) {
        const int32_t v = L.g_idx[p];
        if (mark[v] != j) {
          mark[v] = j;
          ++tot;
        }
      }
    }
  }
  return tot;
}

// Local problems of one level: smoother, splitting, eigenproblems, Z.
int build_level(amgdd_hierarchy& h, Level& L, int lvl, const int32_t* agg_in, cudaStream_t s) {
  auto ts = std::chrono::steady_clock::now();
  Supports S;
  S.ptr = L.g_ptr;
  S.idx = L.g_idx;
  std::vector<int64_t> nptr;
  std::vector<int32_t> ngrp;
  node_groups(S, L.n, nptr, ngrp);
  h.nnzA.push_back(structural_nnz(L, nptr, ngrp));
  if (lvl == 0) {
    if (!cleanup_aggregates(agg_in, L.n, S, nptr, ngrp, L.agg, L.nagg)) {
      set_error("aggregate ids must be >= -1");
      return AMGDD_ERR_INVALID_ARG;
    }
  }
  const int nagg = L.nagg;
  const int ov = lvl == 0 || h.prm.coarse_overlap <= 0 ? h.overlap : h.prm.coarse_overlap;
  overlap_sets(L.agg, nagg, S, nptr, ngrp, ov, L.om_ptr, L.om_idx, L.nomega);
  std::vector<int64_t> tptr;
  std::vector<int32_t> tids, M;
  touched_aggregates(S, L.agg, tptr, tids, M);
  L.thresh = h.prm.thresh;
  if (h.prm.kappa > 0) {
    L.n_color = colour_subdomains(L.om_ptr, L.om_idx, L.n, S, nptr, ngrp);
    L.n_mult = 1;
    for (int32_t v : M) L.n_mult = std::max(L.n_mult, (int)v);
    L.thresh = kappa_threshold(h.prm.kappa, L.n_color, L.n_mult);
  }
  const int c = h.prm.c_min[std::min(lvl, h.prm.n_cmin - 1)];
  if (g_timer.on)
    g_timer.add(0, "structure", std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - ts).count());
  std::vector<int32_t> cap(nagg), mdim(nagg);
  int max_m = 0, max_no = 0;
  for (int i = 0; i < nagg; ++i) {
    cap[i] = std::max(1, L.nomega[i] / c);
    mdim[i] = (int32_t)(L.om_ptr[i + 1] - L.om_ptr[i]);
    max_m = std::max(max_m, mdim[i]);
    max_no = std::max(max_no, L.nomega[i]);
  }
  // level-wide device arrays
  DBuf<int32_t> dM;
  AMGDD_TRY(dM.upload(M, s));
  std::vector<int64_t> w_off(nagg + 1, 0), mu_off(nagg + 1, 0);
  for (int i = 0; i < nagg; ++i) {
    w_off[i + 1] = w_off[i] + (int64_t)mdim[i] * L.nomega[i];
    mu_off[i + 1] = mu_off[i] + L.nomega[i];
  }
  L.mu_off = mu_off;
  AMGDD_TRY(L.W64.alloc(w_off[nagg]));
  AMGDD_TRY(L.Wt64.alloc(w_off[nagg]));
  AMGDD_TRY(L.W32.alloc(w_off[nagg]));
  AMGDD_TRY(L.Wt32.alloc(w_off[nagg]));
  AMGDD_TRY(L.Aw64.alloc(w_off[nagg]));
  AMGDD_TRY(L.AwT64.alloc(w_off[nagg]));
  AMGDD_TRY(L.Aw32.alloc(w_off[nagg]));
  AMGDD_TRY(L.AwT32.alloc(w_off[nagg]));
  AMGDD_TRY(L.mu.alloc(mu_off[nagg]));
  DBuf<double> inv_scratch;
  AMGDD_TRY(inv_scratch.alloc(w_off[nagg]));
  // additive Schwarz (cycle = 1): every row of A_i^{-1}
  const bool full_inv = h.prm.cycle == 1 && lvl == 0;
  DBuf<double> full_scratch;
  if (full_inv) {
    L.wf_off.assign(nagg + 1, 0);
    for (int i = 0; i < nagg; ++i) L.wf_off[i + 1] = L.wf_off[i] + (int64_t)mdim[i] * mdim[i];
    AMGDD_TRY(L.Wf64.alloc(L.wf_off[nagg]));
    AMGDD_TRY(L.Wft64.alloc(L.wf_off[nagg]));
    AMGDD_TRY(L.Wf32.alloc(L.wf_off[nagg]));
    AMGDD_TRY(L.Wft32.alloc(L.wf_off[nagg]));
    AMGDD_TRY(full_scratch.alloc(L.wf_off[nagg]));
  }
  DBuf<int64_t> d_w_off, d_mu_off;
  AMGDD_TRY(d_w_off.upload(w_off, s));
  AMGDD_TRY(d_mu_off.upload(mu_off, s));
  // Z pools sized for the caps; packed tightly once k is known
  int64_t zcap_tot = 0;
  for (int i = 0; i < nagg; ++i) zcap_tot += (int64_t)L.nomega[i] * cap[i];
  AMGDD_TRY(L.Z64.alloc(zcap_tot));
  AMGDD_TRY(L.Zt64.alloc(zcap_tot));
  AMGDD_TRY(L.Z32.alloc(zcap_tot));
  AMGDD_TRY(L.Zt32.alloc(zcap_tot));
  L.k.assign(nagg, 0);
  L.z_off.assign(nagg + 1, 0);

  std::vector<int32_t> loc(L.n, -1);
  std::vector<int64_t> gstamp((size_t)(L.g_ptr.size() - 1), -1);
  const int64_t budget = (int64_t)384 << 20;  // doubles per batch for A and A~ pools (and the rows of the splitting)
  // rows of the splitting of each aggregate (row route): sum of rank_g over the groups of nz_i
  std::vector<int64_t> yrows(nagg, 0);
  if (h.prm.schur_gram != 1)
    for (int i = 0; i < nagg; ++i) {
      const int64_t o0 = L.om_ptr[i], o1 = L.om_ptr[i + 1];
      for (int64_t q = o0; q < o1; ++q) {
        const int32_t v = L.om_idx[q];
        if (L.agg[v] != i) continue;  // nz_i: the groups touching omega_i
        for (int64_t e = nptr[v]; e < nptr[v + 1]; ++e) {
          const int32_t g = ngrp[e];
          if (gstamp[g] != -2 - (int64_t)i) {
            gstamp[g] = -2 - (int64_t)i;
            yrows[i] += L.g_rank[g];
          }
        }
      }
    }
  std::fill(gstamp.begin(), gstamp.end(), -1);
  // the route of this level (schur_gram = 0): rows unless their Householder
  // QR would cost more than 8 times the Gram elimination (3D coarse levels,
  // whose splitting holds many more rows than columns)
  bool rows_schur = h.prm.schur_gram == 2;
  if (h.prm.schur_gram == 0) {
    double fr = 0.0, fg = 0.0;
    for (int i = 0; i < nagg; ++i) {
      const double m = mdim[i], ng = m - L.nomega[i], nr = (double)yrows[i];
      fr += 4.0 * nr * m * std::min(nr, ng);
      fg += m * m * m;
    }
    rows_schur = fr <= 8.0 * fg;
  }
  L.schur_rows = rows_schur;
  int i0 = 0;
  while (i0 < nagg) {
    int i1 = i0;
    int64_t pool = 0;
    auto need = [&](int i) { return 2 * (int64_t)mdim[i] * mdim[i] + (rows_schur ? yrows[i] * mdim[i] : 0); };
    while (i1 < nagg && (i1 == i0 || pool + need(i1) <= budget)) {
      pool += need(i1);
      ++i1;
    }
    const int nb = i1 - i0;
    // host batch description
    std::vector<int32_t> bm(nb), bno(nb), bcap(nb), pgrp, pnz, mp;
    std::vector<int64_t> aoff(nb + 1, 0), pptr(nb + 1, 0), mptr, zoffcap(nb + 1, 0), scroff(nb + 1, 0),
        bw_off(nb), bmu_off(nb);
    std::vector<int32_t> glist;
    for (int t = 0; t < nb; ++t) {
      const int i = i0 + t;
      bm[t] = mdim[i];
      bno[t] = L.nomega[i];
      bcap[t] = cap[i];
      aoff[t + 1] = aoff[t] + (int64_t)mdim[i] * mdim[i];
      zoffcap[t + 1] = zoffcap[t] + (int64_t)L.nomega[i] * cap[i];
      const int64_t nn = L.nomega[i];
      scroff[t + 1] = scroff[t] + 5 * nn * nn + 4 * (nn + 1) + 8;
      bw_off[t] = w_off[i];
      bmu_off[t] = mu_off[i];
      const int64_t o0 = L.om_ptr[i], o1 = L.om_ptr[i + 1];
      for (int64_t q = o0; q < o1; ++q) loc[L.om_idx[q]] = (int32_t)(q - o0);
      glist.clear();
      for (int64_t q = o0; q < o1; ++q) {
        const int32_t v = L.om_idx[q];
        for (int64_t e = nptr[v]; e < nptr[v + 1]; ++e) {
          const int32_t g = ngrp[e];
          if (gstamp[g] != i) {
            gstamp[g] = i;
            glist.push_back(g);
          }
        }
      }
      std::sort(glist.begin(), glist.end());
      for (int32_t g : glist) {
        pgrp.push_back(g);
        const bool nz = std::binary_search(tids.begin() + tptr[g], tids.begin() + tptr[g + 1], (int32_t)i);
        pnz.push_back(nz ? 1 : 0);
        mptr.push_back((int64_t)mp.size());
        for (int64_t e = L.g_ptr[g]; e < L.g_ptr[g + 1]; ++e) mp.push_back(loc[L.g_idx[e]]);
      }
      pptr[t + 1] = (int64_t)pgrp.size();
      for (int64_t q = o0; q < o1; ++q) loc[L.om_idx[q]] = -1;
    }
    mptr.push_back((int64_t)mp.size());
    LocalBatch B;
    AMGDD_TRY(B.m.upload(bm, s));
    AMGDD_TRY(B.no.upload(bno, s));
    AMGDD_TRY(B.a_off.upload(aoff, s));
    AMGDD_TRY(B.pair_ptr.upload(pptr, s));
    AMGDD_TRY(B.pair_grp.upload(pgrp, s));
    AMGDD_TRY(B.pair_nz.upload(pnz, s));
    AMGDD_TRY(B.map_ptr.upload(mptr, s));
    AMGDD_TRY(B.map.upload(mp, s));
    DBuf<int32_t> dcap, dk, dstat;
    DBuf<int64_t> dzcap, dscr, dwoff, dmuoff;
    AMGDD_TRY(dcap.upload(bcap, s));
    AMGDD_TRY(dzcap.upload(zoffcap, s));
    AMGDD_TRY(dscr.upload(scroff, s));
    AMGDD_TRY(dwoff.upload(bw_off, s));
    AMGDD_TRY(dmuoff.upload(bmu_off, s));
    AMGDD_TRY(dk.alloc(nb));
    AMGDD_TRY(dstat.alloc(nb));
    DBuf<double> Apool, Atpool, Zcap, gscr;
    AMGDD_TRY(Apool.alloc(aoff[nb]));
    AMGDD_TRY(Atpool.alloc(aoff[nb]));
    AMGDD_TRY(Zcap.alloc(std::max<int64_t>(zoffcap[nb], 1)));
    AMGDD_TRY(gscr.alloc(scroff[nb]));
    {
      Phase ph(1, "assemble", s);
      AMGDD_TRY(launch_assemble(nb, max_m, B, L.d_g_ptr.p, L.d_h_off.p, L.d_H.p, dM.p, Apool.p, Atpool.p, s));
    }
    AMGDD_TRY(launch_copy_wrows(nb, B.m.p, B.no.p, B.a_off.p, Apool.p, dwoff.p, L.Aw64.p, L.Aw32.p, L.AwT64.p,
                                L.AwT32.p, s));
    {
      Phase ph(2, "cholesky", s);
      AMGDD_TRY(launch_chol(nb, max_m, B.m.p, B.a_off.p, Apool.p, dstat.p, s));
      for (int t = 0; t < nb; ++t) g_timer.flops[2] += (double)bm[t] * bm[t] * bm[t] / 3.0;
    }
    std::vector<int32_t> stat;
    AMGDD_TRY(download(stat, dstat.p, nb, s));
    for (int t = 0; t < nb; ++t)
      if (stat[t] != 0) {
        set_error("level %d: local block A(Omega_%d, Omega_%d) is not SPD (pivot %d)", lvl, i0 + t, i0 + t,
                  stat[t] - 1);
        return AMGDD_ERR_NOT_SPD;
      }
    {
      Phase ph(3, "schur", s);
      if (rows_schur) {
        std::vector<int64_t> yoff(nb + 1, 0), noff(nb + 1, 0);
        std::vector<int32_t> yr(nb);
        int bmax_m = 0;
        for (int t = 0; t < nb; ++t) {
          yr[t] = (int32_t)yrows[i0 + t];
          yoff[t + 1] = yoff[t] + yrows[i0 + t] * bm[t];
          noff[t + 1] = noff[t] + bm[t];
          bmax_m = std::max(bmax_m, (int)bm[t]);
        }
        DBuf<int64_t> dyoff, dnoff;
        DBuf<int32_t> dyr;
        DBuf<double> Ypool, nrm;
        AMGDD_TRY(dyoff.upload(yoff, s));
        AMGDD_TRY(dnoff.upload(noff, s));
        AMGDD_TRY(dyr.upload(yr, s));
        AMGDD_TRY(Ypool.alloc(std::max<int64_t>(yoff[nb], 1)));
        AMGDD_TRY(nrm.alloc(std::max<int64_t>(noff[nb], 1)));
        DBuf<int32_t> drk;
        AMGDD_TRY(drk.alloc(nb));
        // cluster teams once the mean row block holds a million entries (8 MB)
        const bool team = yoff[nb] >= (int64_t)nb << 20;
        AMGDD_TRY(launch_schur_rows(nb, bmax_m, B, L.d_g_ptr.p, L.d_h_off.p, L.d_rank.p, L.d_R64.p, dM.p, dyoff.p,
                                    dyr.p, Ypool.p, dnoff.p, nrm.p, Atpool.p, drk.p, team, s));
        std::vector<int32_t> rk;
        AMGDD_TRY(download(rk, drk.p, nb, s));
        for (int t = 0; t < nb; ++t) {  // per reflection: norms and update of the remaining columns; then X_2^T X_2
          const double nr = (double)yr[t], m = (double)bm[t], no = (double)bno[t];
          for (int k = 0; k < rk[t]; ++k) g_timer.flops[3] += 6.0 * (nr - k) * (m - k);
          g_timer.flops[3] += 2.0 * (nr - rk[t]) * no * no;
        }
      } else {
        AMGDD_TRY(launch_schur(nb, max_m, B.m.p, B.no.p, B.a_off.p, Atpool.p, h.prm.schur_rtol, s));
        for (int t = 0; t < nb; ++t)
          g_timer.flops[3] += 2.0 * (double)(bm[t] - bno[t]) * bm[t] * bm[t] / 2.0;  // at most |Gamma| pivots
      }
    }
    {
      Phase ph(4, "inverse rows", s);
      std::vector<int32_t> cb, cc;
      for (int t = 0; t < nb; ++t)
        for (int c = 0; c < bno[t]; c += kInvChunk) {
          cb.push_back(t);
          cc.push_back(c);
        }
      DBuf<int32_t> dcb, dcc;
      AMGDD_TRY(dcb.upload(cb, s));
      AMGDD_TRY(dcc.upload(cc, s));
      AMGDD_TRY(launch_inv_rows(nb, max_m, B.m.p, B.no.p, B.a_off.p, Apool.p, dwoff.p, L.W64.p, L.W32.p, L.Wt64.p,
                                L.Wt32.p, inv_scratch.p, dcb.p, dcc.p, (int)cb.size(), kInvChunk, s));
      for (int t = 0; t < nb; ++t) g_timer.flops[4] += 2.0 * (double)bno[t] * bm[t] * bm[t];  // two solves per column
      if (full_inv) {  // the same solves for every column of A_i^{-1} (rows = columns: m per block)
        std::vector<int32_t> fb, fc;
        std::vector<int64_t> fo(nb);
        for (int t = 0; t < nb; ++t) {
          fo[t] = L.wf_off[i0 + t];
          for (int c = 0; c < bm[t]; c += kInvChunk) {
            fb.push_back(t);
            fc.push_back(c);
          }
        }
        DBuf<int32_t> dfb, dfc;
        DBuf<int64_t> dfo;
        AMGDD_TRY(dfb.upload(fb, s));
        AMGDD_TRY(dfc.upload(fc, s));
        AMGDD_TRY(dfo.upload(fo, s));
        AMGDD_TRY(launch_inv_rows(nb, max_m, B.m.p, B.m.p, B.a_off.p, Apool.p, dfo.p, L.Wf64.p, L.Wf32.p, L.Wft64.p,
                                  L.Wft32.p, full_scratch.p, dfb.p, dfc.p, (int)fb.size(), kInvChunk, s));
      }
      AMGDD_CUDA(cudaStreamSynchronize(s));
    }
    {
      Phase ph(5, "eigen", s);
      DBuf<int32_t> dwork;
      AMGDD_TRY(dwork.alloc(nb));
      AMGDD_TRY(launch_gep(nb, max_no, B.m.p, B.no.p, B.a_off.p, Apool.p, Atpool.p, dcap.p, L.thresh, dmuoff.p,
                           L.mu.p, dzcap.p, Zcap.p, dk.p, gscr.p, dscr.p, dwork.p, s));
      std::vector<int32_t> wk, kk;
      AMGDD_TRY(download(wk, dwork.p, nb, s));
      AMGDD_TRY(download(kk, dk.p, nb, s));
      const bool ql = gep_uses_ql(max_no);
      for (int t = 0; t < nb; ++t) {
        // L^{-1} S~ L^{-T}; Jacobi rounds (a full pass over C and V per round, n - 1 rounds a sweep) or the
        // tridiagonal reduction with its Q and the QL rotations applied to V; Z = L^{-T} V (k columns)
        const double n = (double)bno[t];
        double f = 2.0 * n * n * n + 2.0 * n * n * kk[t];
        f += ql ? (8.0 / 3.0) * n * n * n + 6.0 * n * wk[t] : 12.0 * n * n * (n - 1.0) * wk[t];
        g_timer.flops[5] += f;
      }
    }
    std::vector<int32_t> kb;
    AMGDD_TRY(download(kb, dk.p, nb, s));
    std::vector<int64_t> zoff_b(nb);
    for (int t = 0; t < nb; ++t) {
      const int i = i0 + t;
      L.k[i] = kb[t];
      zoff_b[t] = L.z_off[i];
      L.z_off[i + 1] = L.z_off[i] + (int64_t)L.nomega[i] * kb[t];
    }
    DBuf<int64_t> dzoff;
    AMGDD_TRY(dzoff.upload(zoff_b, s));
    AMGDD_TRY(launch_pack_z(nb, B.no.p, dk.p, dzcap.p, Zcap.p, dzoff.p, L.Z64.p, L.Z32.p, L.Zt64.p, L.Zt32.p, s));
    AMGDD_CUDA(cudaStreamSynchronize(s));
    i0 = i1;
  }
  L.col0.assign(nagg + 1, 0);
  for (int i = 0; i < nagg; ++i) L.col0[i + 1] = L.col0[i] + L.k[i];
  // every stored smoother and basis entry is finite: the shifted vector loads
  // of the gather-GEMV multiply a neighbouring row's entries by zero, which
  // only a finite entry survives (an FP32 overflow would otherwise spread NaN)
  {
    DBuf<int> bad;
    AMGDD_TRY(bad.alloc(1));
    AMGDD_TRY(bad.zero(s));
    AMGDD_TRY(count_nonfinite(L.W64.p, (int64_t)L.W64.n, false, bad.p, s));
    AMGDD_TRY(count_nonfinite(L.W32.p, (int64_t)L.W32.n, true, bad.p, s));
    AMGDD_TRY(count_nonfinite(L.Z64.p, L.z_off.back(), false, bad.p, s));
    AMGDD_TRY(count_nonfinite(L.Z32.p, L.z_off.back(), true, bad.p, s));
    std::vector<int> nb;
    AMGDD_TRY(download(nb, bad.p, 1, s));
    if (nb[0] != 0) {
      set_error("level %d: %d stored smoother or basis entries are not finite", lvl, nb[0]);
      return AMGDD_ERR_NONFINITE;
    }
  }
  return AMGDD_OK;
}

int build_plans(amgdd_hierarchy& h, Level& L, DBuf<int32_t>& d_om_idx, cudaStream_t s) {
  const int nagg = L.nagg;
  AMGDD_TRY(d_om_idx.upload(L.om_idx, s));
  std::vector<int32_t> nr(nagg), nc(nagg);
  std::vector<int64_t> moff(nagg), ioff(nagg), ooff(nagg);
  std::vector<int64_t> w_off(nagg + 1, 0);
  for (int i = 0; i < nagg; ++i)
    w_off[i + 1] = w_off[i] + (int64_t)L.nomega[i] * (L.om_ptr[i + 1] - L.om_ptr[i]);
  // RAS: x(omega_i) = W_i r(Omega_i)
  for (int i = 0; i < nagg; ++i) {
    nr[i] = L.nomega[i];
    nc[i] = (int32_t)(L.om_ptr[i + 1] - L.om_ptr[i]);
    moff[i] = w_off[i];
    ioff[i] = L.om_ptr[i];
    ooff[i] = L.om_ptr[i];
  }
  AMGDD_TRY(build_seg(L.ras, nr, nc, moff, ioff, ooff, d_om_idx.p, d_om_idx.p, s));
  if (L.Wf64.p) {  // additive Schwarz: x(Omega_i) += A_i^{-1} r(Omega_i)
    std::vector<int32_t> fr(nagg);
    for (int i = 0; i < nagg; ++i) fr[i] = nc[i];
    std::vector<int64_t> fo(L.wf_off.begin(), L.wf_off.end() - 1);
    AMGDD_TRY(build_seg(L.asp, fr, fr, fo, ioff, ooff, d_om_idx.p, d_om_idx.p, s));
  }
  // RAS-T: x(Omega_i) += W_i^T s(omega_i)
  for (int i = 0; i < nagg; ++i) std::swap(nr[i], nc[i]);
  AMGDD_TRY(build_seg(L.rast, nr, nc, moff, ioff, ooff, d_om_idx.p, d_om_idx.p, s));
  if (h.prm.deterministic) {
    // the same products stored at the Omega-list positions, and per node the
    // positions that hold its entries (ascending)
    const int64_t tot = L.om_ptr[nagg];
    std::vector<int32_t> io(tot);
    std::iota(io.begin(), io.end(), 0);
    AMGDD_TRY(L.d_pos_iota.upload(io, s));
    AMGDD_TRY(build_seg(L.rast_det, nr, nc, moff, ioff, ooff, d_om_idx.p, L.d_pos_iota.p, s));
    std::vector<int64_t> dp(L.n + 1, 0);
    for (int64_t q = 0; q < tot; ++q) ++dp[L.om_idx[q] + 1];
    for (int64_t j = 0; j < L.n; ++j) dp[j + 1] += dp[j];
    std::vector<int32_t> pos(tot);
    std::vector<int64_t> fill(dp.begin(), dp.end() - 1);
    for (int64_t q = 0; q < tot; ++q) pos[fill[L.om_idx[q]]++] = (int32_t)q;
    AMGDD_TRY(L.det_ptr.upload(dp, s));
    AMGDD_TRY(L.det_pos.upload(pos, s));
    AMGDD_TRY(L.yd64.alloc(tot));
    AMGDD_TRY(L.yd32.alloc(tot));
  }
  // restriction: r_c[col0_i + c] = (Z_i^T s(omega_i))_c
  for (int i = 0; i < nagg; ++i) {
    nr[i] = L.k[i];
    nc[i] = L.nomega[i];
    moff[i] = L.z_off[i];
    ioff[i] = L.om_ptr[i];
    ooff[i] = L.col0[i];
  }
  AMGDD_TRY(build_seg(L.restr, nr, nc, moff, ioff, ooff, d_om_idx.p, h.iota.p, s));
  // prolongation: x(omega_i) += Z_i x_c[col0_i ...]
  for (int i = 0; i < nagg; ++i) {
    nr[i] = L.nomega[i];
    nc[i] = L.k[i];
    ioff[i] = L.col0[i];
    ooff[i] = L.om_ptr[i];
  }
  AMGDD_TRY(build_seg(L.prol, nr, nc, moff, ioff, ooff, h.iota.p, d_om_idx.p, s));
  return AMGDD_OK;
}

// Supports and Grams of G_{l+1} = G_l P_l; aggregates of level l+1.
int build_next(amgdd_hierarchy& h, Level& L, Level& N, cudaStream_t s) {
  (void)h;
  Supports S;
  S.ptr = L.g_ptr;
  S.idx = L.g_idx;
  std::vector<int64_t> tptr;
  std::vector<int32_t> tids, M;
  touched_aggregates(S, L.agg, tptr, tids, M);
  const int64_t ng = S.size();
  // a row whose touched aggregates all kept k = 0 columns becomes zero in
  // G_{l+1} = G_l P_l and is dropped
  std::vector<char> live_row(ng, 0);
  for (int64_t g = 0; g < ng; ++g)
    for (int64_t t = tptr[g]; t < tptr[g + 1]; ++t)
      if (L.k[tids[t]] > 0) live_row[g] = 1;
  std::map<std::vector<int32_t>, int64_t> keys;
  for (int64_t g = 0; g < ng; ++g)
    if (live_row[g]) keys.emplace(std::vector<int32_t>(tids.begin() + tptr[g], tids.begin() + tptr[g + 1]), 0);
  int64_t h_id = 0;
  N.g_ptr.assign(1, 0);
  N.g_idx.clear();
  for (auto& kv : keys) {
    kv.second = h_id++;
    for (int32_t a : kv.first)
      for (int64_t c = L.col0[a]; c < L.col0[a + 1]; ++c) N.g_idx.push_back((int32_t)c);
    N.g_ptr.push_back((int64_t)N.g_idx.size());
  }
  const int64_t nnew = h_id;
  N.h_off.assign(nnew + 1, 0);
  int max_sn = 1;
  for (int64_t q = 0; q < nnew; ++q) {
    const int64_t sn = N.g_ptr[q + 1] - N.g_ptr[q];
    max_sn = std::max<int>(max_sn, (int)sn);
    N.h_off[q + 1] = N.h_off[q] + sn * sn;
  }
  // contributions and per-support-node Z rows
  std::vector<int64_t> owner(ng, -1);
  std::vector<int64_t> cnt(nnew + 1, 0);
  for (int64_t g = 0; g < ng; ++g) {
    if (!live_row[g]) continue;
    owner[g] = keys[std::vector<int32_t>(tids.begin() + tptr[g], tids.begin() + tptr[g + 1])];
    cnt[owner[g] + 1]++;
  }
  for (int64_t q = 0; q < nnew; ++q) cnt[q + 1] += cnt[q];
  std::vector<int32_t> contrib(std::max<int64_t>(cnt[nnew], 1));
  {
    std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
    for (int64_t g = 0; g < ng; ++g)
      if (owner[g] >= 0) contrib[fill[owner[g]]++] = (int32_t)g;
  }
  std::vector<int32_t> pos(L.n, 0);
  for (int i = 0; i < L.nagg; ++i)
    for (int t = 0; t < L.nomega[i]; ++t) pos[L.om_idx[L.om_ptr[i] + t]] = t;
  std::vector<int64_t> rz_ptr(ng + 1, 0), rz_zoff;
  std::vector<int32_t> rz_k, rz_col;
  int max_s = 1;
  for (int64_t g = 0; g < ng; ++g) {
    max_s = std::max(max_s, S.len(g));
    for (int64_t e = S.ptr[g]; e < S.ptr[g + 1]; ++e) {
      const int32_t v = S.idx[e];
      const int32_t a = L.agg[v];
      int64_t col = 0;
      for (int64_t t = tptr[g]; t < tptr[g + 1] && tids[t] < a; ++t) col += L.k[tids[t]];
      rz_zoff.push_back(L.z_off[a] + (int64_t)pos[v] * L.k[a]);
      rz_k.push_back(L.k[a]);
      rz_col.push_back((int32_t)col);
    }
    rz_ptr[g + 1] = (int64_t)rz_zoff.size();
  }
  NextGramPlan P;
  P.nnew = nnew;
  AMGDD_TRY(P.new_ptr.upload(cnt, s));
  AMGDD_TRY(P.contrib.upload(contrib, s));
  AMGDD_TRY(P.new_sptr.upload(N.g_ptr, s));
  AMGDD_TRY(P.new_hoff.upload(N.h_off, s));
  AMGDD_TRY(P.rowz_ptr.upload(rz_ptr, s));
  AMGDD_TRY(P.rowz_zoff.upload(rz_zoff, s));
  AMGDD_TRY(P.rowz_k.upload(rz_k, s));
  AMGDD_TRY(P.rowz_col.upload(rz_col, s));
  P.scratch_per = (int64_t)max_s * max_sn;
  AMGDD_TRY(N.d_H.alloc(std::max<int64_t>(N.h_off[nnew], 1)));
  int64_t chunk = std::max<int64_t>(1, (int64_t)(32 << 20) / P.scratch_per);
  chunk = std::min<int64_t>(chunk, std::max<int64_t>(nnew, 1));
  DBuf<double> scratch;
  AMGDD_TRY(scratch.alloc(chunk * P.scratch_per));
  for (int64_t f = 0; f < nnew; f += chunk) {
    const int64_t c = std::min(chunk, nnew - f);
    AMGDD_TRY(launch_next_gram(P, max_sn, L.d_g_ptr.p, L.d_h_off.p, L.d_H.p, L.Z64.p, N.d_H.p, scratch.p, f, c, s));
  }
  for (int64_t q = 0; q < nnew; ++q) {  // T = H_g P_g and P_g^T T: each entry of P_g (sum k) meets s, then sn terms
    const double sn = (double)(N.g_ptr[q + 1] - N.g_ptr[q]);
    for (int64_t e = cnt[q]; e < cnt[q + 1]; ++e) {
      const int32_t g = contrib[e];
      double ksum = 0.0;
      for (int64_t t = rz_ptr[g]; t < rz_ptr[g + 1]; ++t) ksum += rz_k[t];
      g_timer.flops[7] += 2.0 * ksum * ((double)S.len(g) + sn);
    }
  }
  AMGDD_CUDA(cudaStreamSynchronize(s));
  if (L.schur_rows) {
    // row route (this level formed its Schur complements from rows; the next
    // level most likely will too): G_{l+1}'s rows by QR of the stacked R_g P_g, in chunks of
    // new groups whose stacked rows fit a scratch budget
    std::vector<int64_t> t_off(nnew + 1, 0);
    for (int64_t q = 0; q < nnew; ++q) {
      int64_t rows = 0;
      for (int64_t e = cnt[q]; e < cnt[q + 1]; ++e) rows += L.g_rank[contrib[e]];
      t_off[q + 1] = t_off[q] + rows * (N.g_ptr[q + 1] - N.g_ptr[q]);
    }
    DBuf<int64_t> d_toff;
    AMGDD_TRY(d_toff.upload(t_off, s));
    AMGDD_TRY(N.d_R64.alloc(std::max<int64_t>(N.h_off[nnew], 1)));
    AMGDD_TRY(N.d_R32.alloc(std::max<int64_t>(N.h_off[nnew], 1)));
    AMGDD_TRY(N.d_rank.alloc(std::max<int64_t>(nnew, 1)));
    const int64_t budget = (int64_t)64 << 20;  // doubles of stacked rows per launch
    int64_t maxper = 1;
    for (int64_t q = 0; q < nnew; ++q) maxper = std::max(maxper, t_off[q + 1] - t_off[q]);
    DBuf<double> tscr;
    AMGDD_TRY(tscr.alloc(std::max(budget, maxper)));
    for (int64_t f = 0; f < nnew;) {
      int64_t e = f + 1;
      while (e < nnew && t_off[e + 1] - t_off[f] <= std::max(budget, maxper)) ++e;
      // cluster teams once the mean stacked block holds a million entries
      const bool team = t_off[e] - t_off[f] >= (e - f) << 20;
      AMGDD_TRY(launch_next_rows(P, L.d_g_ptr.p, L.d_h_off.p, L.d_rank.p, L.d_R64.p, L.Z64.p, d_toff.p, tscr.p,
                                 N.d_R64.p, N.d_R32.p, N.d_rank.p, f, e - f, team, s));
      f = e;
    }
    AMGDD_TRY(download(N.g_rank, N.d_rank.p, nnew, s));
    N.rows_ready = true;
    for (int64_t q = 0; q < nnew; ++q) {  // the stacked R_g P_g, then a Householder QR of them
      const double sn = (double)(N.g_ptr[q + 1] - N.g_ptr[q]);
      const double nr = (double)(t_off[q + 1] - t_off[q]) / std::max(1.0, sn);
      g_timer.flops[7] += 2.0 * nr * sn * sn;
      for (int k = 0; k < N.g_rank[q]; ++k) g_timer.flops[7] += 4.0 * (nr - k) * (sn - k);
    }
  }
  N.n = L.col0[L.nagg];
  AMGDD_TRY(N.d_g_ptr.upload(N.g_ptr, s));
  AMGDD_TRY(N.d_g_idx.upload(N.g_idx, s));
  AMGDD_TRY(N.d_h_off.upload(N.h_off, s));
  // aggregates of level l+1: whole blocks of coarse dofs, on the graph of the
  // blocks that kept coarse dofs (k > 0), in ascending order
  std::vector<int32_t> live_id(L.nagg, -1), ltids;
  int nlive = 0;
  for (int a = 0; a < L.nagg; ++a)
    if (L.k[a] > 0) live_id[a] = nlive++;
  std::vector<int64_t> ltptr(1, 0);
  for (int64_t g = 0; g < ng; ++g) {
    for (int64_t t = tptr[g]; t < tptr[g + 1]; ++t)
      if (live_id[tids[t]] >= 0) ltids.push_back(live_id[tids[t]]);
    ltptr.push_back((int64_t)ltids.size());
  }
  std::vector<int32_t> bagg;
  int nn = 0;
  {
    DBuf<int64_t> d_lptr;
    DBuf<int32_t> d_lids, d_bagg;
    AMGDD_TRY(d_lptr.upload(ltptr, s));
    AMGDD_TRY(d_lids.upload(ltids, s));
    AMGDD_TRY(d_bagg.alloc(std::max(nlive, 1)));
    int64_t nb = 0;
    AMGDD_TRY(device_hyper_aggregation(nlive, (int64_t)ltptr.size() - 1, d_lptr.p, d_lids.p, d_bagg.p, &nb, s));
    AMGDD_TRY(download(bagg, d_bagg.p, (size_t)nlive, s));
    nn = (int)nb;
  }
  N.agg.assign(N.n, 0);
  for (int a = 0; a < L.nagg; ++a)
    for (int64_t c = L.col0[a]; c < L.col0[a + 1]; ++c) N.agg[c] = bagg[live_id[a]];
  N.nagg = nn;
  AMGDD_CUDA(cudaStreamSynchronize(s));
  return AMGDD_OK;
}

// Coarsest level: dense A_L, Cholesky, explicit inverse (one block).
int build_coarsest(amgdd_hierarchy& h, Level& L, cudaStream_t s) {
  const int64_t m = L.n;
  if (m > 24000) {
    set_error("coarsest level has %lld unknowns; raise L_max or lower n_coarse", (long long)m);
    return AMGDD_ERR_INVALID_ARG;
  }
  L.coarsest = true;
  Supports S;
  S.ptr = L.g_ptr;
  S.idx = L.g_idx;
  std::vector<int64_t> nptr;
  std::vector<int32_t> ngrp;
  node_groups(S, L.n, nptr, ngrp);
  h.nnzA.push_back(structural_nnz(L, nptr, ngrp));
  const int64_t ng = S.size();
  std::vector<int32_t> bm{(int32_t)m}, bno{(int32_t)m}, pgrp(ng), pnz(ng, 0), mp(L.g_idx.begin(), L.g_idx.end());
  std::vector<int64_t> aoff{0, m * m}, pptr{0, ng}, mptr(L.g_ptr.begin(), L.g_ptr.end());
  std::iota(pgrp.begin(), pgrp.end(), 0);
  std::vector<int32_t> Mv(ng, 1);
  LocalBatch B;
  AMGDD_TRY(B.m.upload(bm, s));
  AMGDD_TRY(B.no.upload(bno, s));
  AMGDD_TRY(B.a_off.upload(aoff, s));
  AMGDD_TRY(B.pair_ptr.upload(pptr, s));
  AMGDD_TRY(B.pair_grp.upload(pgrp, s));
  AMGDD_TRY(B.pair_nz.upload(pnz, s));
  AMGDD_TRY(B.map_ptr.upload(mptr, s));
  AMGDD_TRY(B.map.upload(mp, s));
  DBuf<int32_t> dM, dstat;
  AMGDD_TRY(dM.upload(Mv, s));
  AMGDD_TRY(dstat.alloc(1));
  DBuf<double> Apool, Atpool, scratch;
  AMGDD_TRY(Apool.alloc(m * m));
  AMGDD_TRY(Atpool.alloc(m * m));
  AMGDD_TRY(scratch.alloc(m * m));
  AMGDD_TRY(launch_assemble(1, (int)m, B, L.d_g_ptr.p, L.d_h_off.p, L.d_H.p, dM.p, Apool.p, Atpool.p, s));
  // A_L itself (symmetric) for the refinement step of the coarsest solve
  AMGDD_TRY(L.Aw64.alloc(m * m));
  AMGDD_CUDA(cudaMemcpyAsync(L.Aw64.p, Apool.p, m * m * sizeof(double), cudaMemcpyDeviceToDevice, s));
  AMGDD_TRY(launch_chol(1, (int)m, B.m.p, B.a_off.p, Apool.p, dstat.p, s));
  std::vector<int32_t> stat;
  AMGDD_TRY(download(stat, dstat.p, 1, s));
  if (stat[0] != 0) {
    set_error("coarsest matrix (n = %lld) is not SPD (pivot %d)", (long long)m, stat[0] - 1);
    return AMGDD_ERR_NOT_SPD;
  }
  AMGDD_TRY(L.W64.alloc(m * m));
  AMGDD_TRY(L.Wt64.alloc(m * m));
  AMGDD_TRY(L.W32.alloc(m * m));
  AMGDD_TRY(L.Wt32.alloc(m * m));
  std::vector<int64_t> woff{0};
  DBuf<int64_t> dwoff;
  AMGDD_TRY(dwoff.upload(woff, s));
  {
    std::vector<int32_t> cb, cc;
    for (int64_t c = 0; c < m; c += kInvChunk) {
      cb.push_back(0);
      cc.push_back((int32_t)c);
    }
    DBuf<int32_t> dcb, dcc;
    AMGDD_TRY(dcb.upload(cb, s));
    AMGDD_TRY(dcc.upload(cc, s));
    AMGDD_TRY(launch_inv_rows(1, (int)m, B.m.p, B.no.p, B.a_off.p, Apool.p, dwoff.p, L.W64.p, L.W32.p, L.Wt64.p,
                              L.Wt32.p, scratch.p, dcb.p, dcc.p, (int)cb.size(), kInvChunk, s));
  }
  std::vector<int32_t> nr{(int32_t)m}, nc{(int32_t)m};
  std::vector<int64_t> moff{0}, ioff{0}, ooff{0};
  AMGDD_TRY(build_seg(L.ras, nr, nc, moff, ioff, ooff, h.iota.p, h.iota.p, s));
  // A posteriori accuracy of the computed inverse: e = ||W (A_L v) - v|| / ||v||
  // for a fixed pseudo-random v (xorshift64).  e is about kappa(A_L) * eps;
  // refinement is kept only where it can change the solve beyond rounding.
  {
    std::vector<double> v(m), w;
    uint64_t z = 0x9E3779B97F4A7C15ull;
    for (auto& e : v) {
      z ^= z << 13;
      z ^= z >> 7;
      z ^= z << 17;
      e = (double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5;
    }
    DBuf<double> dv, dr, dw;
    AMGDD_TRY(dv.upload(v, s));
    AMGDD_TRY(dr.alloc(m));
    AMGDD_TRY(dw.alloc(m));
    AMGDD_TRY(launch_seg(L.ras, L.Aw64.p, false, dv.p, dr.p, false, SEG_STORE, nullptr, s, nullptr, nullptr, L.Aw64.p));
    AMGDD_TRY(launch_seg(L.ras, L.W64.p, false, dr.p, dw.p, false, SEG_STORE, nullptr, s, nullptr, nullptr, L.Wt64.p));
    AMGDD_TRY(download(w, dw.p, m, s));
    double num = 0.0, den = 0.0;
    for (int64_t i = 0; i < m; ++i) {
      num += (w[i] - v[i]) * (w[i] - v[i]);
      den += v[i] * v[i];
    }
    L.inv_err = std::sqrt(num / den);
    // (a one-level hierarchy keeps A_L: the batched residual applies it)
    const bool keep = h.prm.coarse_refine == 2 || (h.prm.coarse_refine == 1 && L.inv_err > 1e-13);
    if (!keep && &L != h.lv[0].get()) L.Aw64.release();
  }
  AMGDD_CUDA(cudaStreamSynchronize(s));
  return AMGDD_OK;
}

// ---- loaded hierarchies: what setup computed, restored from a snapshot ----
// Uploads the FP64 blocks (rows[b] x cols[b] at off[b]) and derives their
// FP32 rounding and transposes.
int restore_blocks(const std::vector<double>& src, const std::vector<int32_t>& rows, const std::vector<int32_t>& cols,
                   const std::vector<int64_t>& off, DBuf<double>& m64, DBuf<float>& m32, DBuf<double>& t64,
                   DBuf<float>& t32, cudaStream_t s) {
  AMGDD_TRY(m64.upload(src, s));
  AMGDD_TRY(m32.alloc(src.size()));
  AMGDD_TRY(t64.alloc(src.size()));
  AMGDD_TRY(t32.alloc(src.size()));
  DBuf<int32_t> dr, dc;
  DBuf<int64_t> doff;
  AMGDD_TRY(dr.upload(rows, s));
  AMGDD_TRY(dc.upload(cols, s));
  AMGDD_TRY(doff.upload(off, s));
  AMGDD_TRY(launch_block_copies((int)rows.size(), dr.p, dc.p, doff.p, m64.p, m32.p, t64.p, t32.p, s));
  AMGDD_CUDA(cudaStreamSynchronize(s));
  return AMGDD_OK;
}

// The compressed rows of G_l (ranks and FP64 rows; FP32 rows derived).
int restore_rows(Level& L, const LevelSnap& S, cudaStream_t s) {
  if (S.R64.empty()) return AMGDD_OK;  // a coarsest level below level 0 keeps no rows
  L.g_rank = S.g_rank;
  AMGDD_TRY(L.d_rank.upload(L.g_rank, s));
  AMGDD_TRY(L.d_R64.upload(S.R64, s));
  AMGDD_TRY(L.d_R32.alloc(S.R64.size()));
  AMGDD_TRY(launch_cast(L.d_R64.p, false, L.d_R32.p, true, (int64_t)S.R64.size(), nullptr, s));
  L.rows_ready = true;
  return AMGDD_OK;
}

// The local problems of one level (build_level's results).
int restore_level(amgdd_hierarchy& h, Level& L, const LevelSnap& S, cudaStream_t s) {
  h.nnzA.push_back(S.nnzA);
  L.agg = S.agg;
  L.nagg = S.nagg;
  L.om_ptr = S.om_ptr;
  L.om_idx = S.om_idx;
  L.nomega = S.nomega;
  L.thresh = S.thresh;
  L.n_color = S.n_color;
  L.n_mult = S.n_mult;
  L.k = S.k;
  L.col0 = S.col0;
  L.z_off = S.z_off;
  L.mu_off = S.mu_off;
  L.wf_off = S.wf_off;
  L.schur_rows = S.schur_rows != 0;
  const int nagg = L.nagg;
  std::vector<int32_t> rows(nagg), cols(nagg);
  std::vector<int64_t> off(nagg);
  int64_t w = 0;
  for (int i = 0; i < nagg; ++i) {
    rows[i] = L.nomega[i];
    cols[i] = (int32_t)(L.om_ptr[i + 1] - L.om_ptr[i]);
    off[i] = w;
    w += (int64_t)rows[i] * cols[i];
  }
  AMGDD_TRY(restore_blocks(S.W64, rows, cols, off, L.W64, L.W32, L.Wt64, L.Wt32, s));
  if (!S.Aw64.empty()) AMGDD_TRY(restore_blocks(S.Aw64, rows, cols, off, L.Aw64, L.Aw32, L.AwT64, L.AwT32, s));
  AMGDD_TRY(L.mu.upload(S.mu, s));
  for (int i = 0; i < nagg; ++i) {
    cols[i] = L.k[i];
    off[i] = L.z_off[i];
  }
  AMGDD_TRY(restore_blocks(S.Z64, rows, cols, off, L.Z64, L.Z32, L.Zt64, L.Zt32, s));
  if (!S.Wf64.empty()) {
    for (int i = 0; i < nagg; ++i) {
      rows[i] = cols[i] = (int32_t)(L.om_ptr[i + 1] - L.om_ptr[i]);
      off[i] = L.wf_off[i];
    }
    AMGDD_TRY(restore_blocks(S.Wf64, rows, cols, off, L.Wf64, L.Wf32, L.Wft64, L.Wft32, s));
  }
  return AMGDD_OK;
}

// The structure of level l+1 (build_next's results; its rows come with the
// level's own snapshot).
int restore_next(Level& N, const LevelSnap& S, cudaStream_t s) {
  N.n = S.n;
  N.g_ptr = S.g_ptr;
  N.g_idx = S.g_idx;
  N.h_off = S.h_off;
  AMGDD_TRY(N.d_g_ptr.upload(N.g_ptr, s));
  AMGDD_TRY(N.d_g_idx.upload(N.g_idx, s));
  AMGDD_TRY(N.d_h_off.upload(N.h_off, s));
  N.agg = S.agg;
  N.nagg = S.nagg;
  return AMGDD_OK;
}

// The coarsest level (build_coarsest's results).
int restore_coarsest(amgdd_hierarchy& h, Level& L, const LevelSnap& S, cudaStream_t s) {
  const int64_t m = L.n;
  L.coarsest = true;
  h.nnzA.push_back(S.nnzA);
  const std::vector<int32_t> rows{(int32_t)m};
  const std::vector<int64_t> off{0};
  AMGDD_TRY(restore_blocks(S.W64, rows, rows, off, L.W64, L.W32, L.Wt64, L.Wt32, s));
  if (!S.Aw64.empty()) AMGDD_TRY(L.Aw64.upload(S.Aw64, s));
  L.inv_err = S.inv_err;
  std::vector<int32_t> nr{(int32_t)m}, nc{(int32_t)m};
  std::vector<int64_t> moff{0}, ioff{0}, ooff{0};
  AMGDD_TRY(build_seg(L.ras, nr, nc, moff, ioff, ooff, h.iota.p, h.iota.p, s));
  AMGDD_CUDA(cudaStreamSynchronize(s));
  return AMGDD_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// Algorithmic bytes: stored matrix values, index arrays, and one pass over
// each input and output vector (two for read-modify-write outputs).
// esz: bytes of a vector entry; msz: of a stored matrix entry (0: esz; 2
// for the FP16 copies of MIXED16).
static double seg_bytes(const SegPlan& p, int64_t nin, int64_t nout, bool rmw, size_t esz, size_t msz = 0) {
  return (double)p.mat_len * (msz ? msz : esz) + (double)(p.in_len + p.out_len) * 4.0 + (double)nin * esz +
         (double)nout * esz * (rmw ? 2.0 : 1.0);
}

// One RAS-T: the scatter-add form, or the stored products plus the per-node
// gather (positions, pointers, the stored values and x read and written).
static double rast_bytes(const Level& L, size_t esz, size_t msz = 0) {
  if (L.yd64.p == nullptr) return seg_bytes(L.rast, L.n, L.n, true, esz, msz);
  const double tot = (double)L.om_ptr.back();
  return seg_bytes(L.rast_det, L.n, (int64_t)tot, false, esz, msz) + tot * (4.0 + esz) + (L.n + 1) * 8.0 +
         2.0 * L.n * esz;
}

// One A-apply (residual form y -= A x) of level L.
static double apply_bytes(const Level& L, size_t esz) {
  double b = (double)L.aplan.r_len * esz + 3.0 * L.n * esz;
  for (size_t g = 0; g + 1 < L.g_ptr.size() && g < L.g_rank.size(); ++g) {
    const int64_t sz = L.g_ptr[g + 1] - L.g_ptr[g];
    if (L.g_rank[g] > 0 && sz <= 512) b += (double)sz * 4.0;
  }
  if (L.t_len > 0) b += seg_bytes(L.gt1, 0, L.t_len, false, esz) + seg_bytes(L.gt2, L.t_len, 0, false, esz);
  return b;
}

// One residual s = r - A x of a non-coarsest level, with the copy of r that
// the matrix-free form needs.
static double resid_bytes(const Level& L, size_t esz, size_t msz = 0) {
  if (L.use_ell) return (double)L.n * L.ell_w * (esz + 4.0) + 3.0 * L.n * esz;
  if (L.has_blk) return seg_bytes(L.ablk, L.n, L.n, true, esz, msz);
  return apply_bytes(L, esz) + (double)L.n * esz;
}

// y = A_l x (Eq. 1) in the level's working precision: block rows when stored,
// else G then G^T by row groups.
// One gather-GEMV of a level's operator pair (M and its block transpose) in
// the working precision: FP64, FP32, or the FP16 copies under MIXED16.
static int seg_op(bool h16, bool f32, const SegPlan& p, const DBuf<double>& M64, const DBuf<float>& M32,
                  const DBuf<double>& T64, const DBuf<float>& T32, const void* x, void* y, SegMode mode,
                  const int* skip, cudaStream_t s, const void* csrc = nullptr, void* cdst = nullptr) {
  if (h16 && p.lanes16 != 0)  // plans where setup timed an FP16 form faster
    return launch_seg16(p, (const float*)x, (float*)y, mode, skip, s, (const float*)csrc, (float*)cdst);
  return launch_seg(p, f32 ? (const void*)M32.p : (const void*)M64.p, f32, x, y, f32, mode, skip, s, csrc, cdst,
                    f32 ? (const void*)T32.p : (const void*)T64.p);
}

static int level_apply_A(const Level& L, bool f32, const void* x, void* y, cudaStream_t s, bool h16 = false) {
  if (L.use_ell) return launch_ell(L, f32, x, y, nullptr, nullptr, s);
  if (L.has_blk)
    return seg_op(h16, f32, L.ablk, L.A64, L.A32, L.At64, L.At32, x, y, SEG_STORE, nullptr, s);
  AMGDD_CUDA(cudaMemsetAsync(y, 0, L.n * (f32 ? sizeof(float) : sizeof(double)), s));
  return launch_apply(L.aplan, L, f32, x, y, +1, nullptr, s);
}

// s = r - A_l x.  The matrix-free form subtracts A x from s in place, so the
// launch before it must have copied r into s (`rcopy` tells those launches).
static int level_residual(const Level& L, bool f32, const void* x, const void* r, void* sv, const int* skip,
                          cudaStream_t s, bool h16 = false) {
  if (L.use_ell) return launch_ell(L, f32, x, sv, r, skip, s);
  if (L.has_blk)
    return seg_op(h16, f32, L.ablk, L.A64, L.A32, L.At64, L.At32, x, sv, SEG_RESID, skip, s, r);
  return launch_apply(L.aplan, L, f32, x, sv, -1, skip, s);
}
static bool rcopy(const Level& L) { return !L.has_blk && !L.use_ell; }

// x(Omega_i) += W_i^T s(omega_i) for all i (Eq. ras-t): atomic scatter-add,
// or (deterministic hierarchies) stored per Omega-list position and summed
// per node in a fixed order.  K > 1: K interleaved columns.
static int apply_rast(const Level& L, bool f32, const void* sv, void* x, const int* skip, cudaStream_t s, int K = 1,
                      bool h16 = false) {
  const void* Wt = f32 ? (const void*)L.Wt32.p : (const void*)L.Wt64.p;
  const void* W = f32 ? (const void*)L.W32.p : (const void*)L.W64.p;
  h16 = h16 && K == 1;
  if (L.yd64.p == nullptr) {
    if (K == 1)
      return seg_op(h16, f32, L.rast, L.Wt64, L.Wt32, L.W64, L.W32, sv, x, SEG_ATOMIC_ADD, skip, s);
    return launch_seg_multi(L.rast, Wt, W, f32, sv, x, SEG_ATOMIC_ADD, nullptr, K, skip, s);
  }
  void* Y = K == 1 ? (f32 ? (void*)L.yd32.p : (void*)L.yd64.p) : (f32 ? (void*)L.myd32.p : (void*)L.myd64.p);
  if (K == 1)
    AMGDD_TRY(seg_op(h16, f32, L.rast_det, L.Wt64, L.Wt32, L.W64, L.W32, sv, Y, SEG_STORE, skip, s));
  else
    AMGDD_TRY(launch_seg_multi(L.rast_det, Wt, W, f32, sv, Y, SEG_STORE, nullptr, K, skip, s));
  return launch_gather_add(L.det_ptr.p, L.det_pos.p, Y, x, L.n, K, f32, skip, s);
}

// ---------------------------------------------------------------------------
// Event marks between the launches of one V-cycle (profiling only): the time
// from mark i to mark i+1 is charged to (level, slot) of mark i.
struct VProf {
  std::vector<cudaEvent_t> ev;
  std::vector<int> tag;  // level * kSlots + slot, -1 for the final mark
  size_t used = 0;
  bool in_graph = false;  // marks recorded under stream capture
  static constexpr int kSlots = 8;
  int mark(cudaStream_t s, int level, int slot) {
    if (used == ev.size()) {
      cudaEvent_t e;
      AMGDD_CUDA(cudaEventCreate(&e));
      ev.push_back(e);
      tag.push_back(0);
    }
    tag[used] = level < 0 ? -1 : level * kSlots + slot;
    // External (under stream capture only): the mark becomes an event record
    // node of the graph (a plain record would only carry a capture dependency)
    if (in_graph)
      AMGDD_CUDA(cudaEventRecordWithFlags(ev[used], s, cudaEventRecordExternal));
    else
      AMGDD_CUDA(cudaEventRecord(ev[used], s));
    ++used;
    return AMGDD_OK;
  }
  ~VProf() {
    for (auto e : ev) cudaEventDestroy(e);
  }
};
#define AMGDD_MARK(slot) \
  if (prof) AMGDD_TRY(prof->mark(s, l, (slot)))

// Exact coarsest solve x = A_L^{-1} r (FP64) with the explicit inverse W and
// one step of iterative refinement, x += W (r - A_L x): the inverse of an
// ill-conditioned A_L (kappa ~ 1e7 on the closed-field-line workload) is
// accurate to ~kappa * eps only.  `sv` is scratch of the level's length.
static int coarse_solve(const amgdd_hierarchy& h, const Level& L, const void* r, void* x, void* sv, const int* skip,
                        cudaStream_t s) {
  AMGDD_TRY(launch_seg(L.ras, L.W64.p, false, r, x, false, SEG_STORE, skip, s, nullptr, nullptr, L.Wt64.p));
  if (!h.prm.coarse_refine || L.Aw64.p == nullptr) return AMGDD_OK;
  AMGDD_TRY(launch_seg(L.ras, L.Aw64.p, false, x, sv, false, SEG_RESID, skip, s, r, nullptr, L.Aw64.p));
  return launch_seg(L.ras, L.W64.p, false, sv, x, false, SEG_ADD, skip, s, nullptr, nullptr, L.Wt64.p);
}

// V-cycle of Section 3.1 from level l: z = B_l r.
static int vcycle(amgdd_hierarchy& h, int l, bool f32, const void* r, void* x, const int* skip, cudaStream_t s,
                  VProf* prof = nullptr) {
  Level& L = *h.lv[l];
  const int pi = f32 ? 1 : 0;
  if (l > 0 && h.persist_from[pi] == l && r == (f32 ? (const void*)L.r32.p : (const void*)L.r64.p) &&
      x == (f32 ? (void*)L.x32.p : (void*)L.x64.p)) {
    AMGDD_MARK(6);
    return launch_persistent(h.d_ph[pi].p, h.nph[pi], h.ph_smem[pi], h.ph_grid[pi], h.bar.p, &h.st.p->vc_err, skip,
                             s);
  }
  if (l > 0 && h.dense_from[pi] == l) {  // the V-cycle from here down as one GEMV
    AMGDD_MARK(0);
    if ((((uintptr_t)r | (uintptr_t)x) & 15) == 0)
      return launch_dense(f32 ? (const void*)L.B32.p : (const void*)L.B64.p, L.dld, (int)L.n, f32, r, x, skip, s);
    return launch_seg(L.dplan, f32 ? (const void*)L.B32.p : (const void*)L.B64.p, f32, r, x, f32, SEG_STORE, skip, s,
                      nullptr, nullptr, nullptr);
  }
  if (L.coarsest) {
    if (f32) {
      AMGDD_MARK(1);
      AMGDD_TRY(launch_cast(r, true, L.r64.p, false, L.n, skip, s));
      AMGDD_MARK(0);
      AMGDD_TRY(coarse_solve(h, L, L.r64.p, L.x64.p, L.s64.p, skip, s));
      AMGDD_MARK(5);
      return launch_cast(L.x64.p, false, x, true, L.n, skip, s);
    }
    AMGDD_MARK(0);
    return coarse_solve(h, L, r, x, L.s64.p, skip, s);
  }
  Level& N = *h.lv[l + 1];
  const bool h16 = use16(h, L, f32);
  void* sv = f32 ? (void*)L.s32.p : (void*)L.s64.p;
  void* rn = f32 ? (void*)N.r32.p : (void*)N.r64.p;
  void* xn = f32 ? (void*)N.x32.p : (void*)N.x64.p;
  // pre-smoothing from x = 0: x = M_RAS^{-1} r  (Eq. ras); the same launch
  // copies s(omega_i) = r(omega_i) for the residual
  AMGDD_MARK(0);
  AMGDD_TRY(seg_op(h16, f32, L.ras, L.W64, L.W32, L.Wt64, L.Wt32, r, x, SEG_STORE, skip, s,
                   rcopy(L) ? r : nullptr, rcopy(L) ? sv : nullptr));
  // s = r - A x ; r_c = P^T s
  AMGDD_MARK(2);
  AMGDD_TRY(level_residual(L, f32, x, r, sv, skip, s, h16));
  AMGDD_MARK(3);
  AMGDD_TRY(seg_op(h16, f32, L.restr, L.Zt64, L.Zt32, L.Z64, L.Z32, sv, rn, SEG_STORE, skip, s));
  // x_c = B_{l+1} r_c ; x += P x_c  (Eq. cgc)
  AMGDD_TRY(vcycle(h, l + 1, f32, rn, xn, skip, s, prof));
  AMGDD_MARK(4);
  AMGDD_TRY(seg_op(h16, f32, L.prol, L.Z64, L.Z32, L.Zt64, L.Zt32, xn, x, SEG_ADD, skip, s,
                   rcopy(L) ? r : nullptr, rcopy(L) ? sv : nullptr));
  // post-smoothing: x += M_RAS-T^{-1} (r - A x)  (Eq. ras-t)
  AMGDD_MARK(2);
  AMGDD_TRY(level_residual(L, f32, x, r, sv, skip, s, h16));
  AMGDD_MARK(7);
  return apply_rast(L, f32, sv, x, skip, s, 1, h16);
}

// Phases of the V-cycle from level `from` >= 1 to the coarsest and back, in
// the order the separate launches of `vcycle` take (Section 3.1).  Needs A by
// block rows on every non-coarsest level of the tail; returns false if not.
static bool tail_phases(amgdd_hierarchy& h, int from, bool f32, std::vector<PhaseDesc>& ph) {
  const int df = h.dense_from[f32 ? 1 : 0];
  const int nl = df > 0 ? df + 1 : (int)h.lv.size();  // the dense tail ends the descent
  ph.clear();
  if (df > 0 && from >= df) return false;
  for (int l = from; l < nl; ++l)
    if (!h.lv[l]->coarsest && l != df && !h.lv[l]->has_blk) return false;
  for (int l = from; l < nl; ++l) {
    Level& L = *h.lv[l];
    if (l == df) {
      ph.push_back(seg_phase(L.dplan, f32 ? (const void*)L.B32.p : (const void*)L.B64.p, nullptr, f32,
                             f32 ? (const void*)L.r32.p : (const void*)L.r64.p, f32 ? (void*)L.x32.p : (void*)L.x64.p,
                             SEG_STORE));
      break;
    }
    if (L.coarsest) {
      if (f32) ph.push_back(cast_phase(L.r32.p, true, L.r64.p, false, L.n));
      ph.push_back(seg_phase(L.ras, L.W64.p, L.Wt64.p, false, L.r64.p, L.x64.p, SEG_STORE));
      if (h.prm.coarse_refine && L.Aw64.p) {
        ph.push_back(seg_phase(L.ras, L.Aw64.p, L.Aw64.p, false, L.x64.p, L.s64.p, SEG_RESID, L.r64.p));
        ph.push_back(seg_phase(L.ras, L.W64.p, L.Wt64.p, false, L.s64.p, L.x64.p, SEG_ADD));
      }
      if (f32) ph.push_back(cast_phase(L.x64.p, false, L.x32.p, true, L.n));
      break;
    }
    Level& N = *h.lv[l + 1];
    const void* r = f32 ? (const void*)L.r32.p : (const void*)L.r64.p;
    void* x = f32 ? (void*)L.x32.p : (void*)L.x64.p;
    void* sv = f32 ? (void*)L.s32.p : (void*)L.s64.p;
    void* rn = f32 ? (void*)N.r32.p : (void*)N.r64.p;
    ph.push_back(seg_phase(L.ras, f32 ? (const void*)L.W32.p : (const void*)L.W64.p,
                           f32 ? (const void*)L.Wt32.p : (const void*)L.Wt64.p, f32, r, x, SEG_STORE));
    ph.push_back(seg_phase(L.ablk, f32 ? (const void*)L.A32.p : (const void*)L.A64.p,
                           f32 ? (const void*)L.At32.p : (const void*)L.At64.p, f32, x, sv, SEG_RESID, r));
    ph.push_back(seg_phase(L.restr, f32 ? (const void*)L.Zt32.p : (const void*)L.Zt64.p,
                           f32 ? (const void*)L.Z32.p : (const void*)L.Z64.p, f32, sv, rn, SEG_STORE));
  }
  for (int l = nl - 2; l >= from; --l) {
    Level& L = *h.lv[l];
    Level& N = *h.lv[l + 1];
    const void* r = f32 ? (const void*)L.r32.p : (const void*)L.r64.p;
    void* x = f32 ? (void*)L.x32.p : (void*)L.x64.p;
    void* sv = f32 ? (void*)L.s32.p : (void*)L.s64.p;
    const void* xn = f32 ? (const void*)N.x32.p : (const void*)N.x64.p;
    ph.push_back(seg_phase(L.prol, f32 ? (const void*)L.Z32.p : (const void*)L.Z64.p,
                           f32 ? (const void*)L.Zt32.p : (const void*)L.Zt64.p, f32, xn, x, SEG_ADD));
    ph.push_back(seg_phase(L.ablk, f32 ? (const void*)L.A32.p : (const void*)L.A64.p,
                           f32 ? (const void*)L.At32.p : (const void*)L.At64.p, f32, x, sv, SEG_RESID, r));
    ph.push_back(seg_phase(L.rast, f32 ? (const void*)L.Wt32.p : (const void*)L.Wt64.p,
                           f32 ? (const void*)L.W32.p : (const void*)L.W64.p, f32, sv, x, SEG_ATOMIC_ADD));
  }
  return true;
}

static int set_tail(amgdd_hierarchy& h, int pi, int from) {
  h.persist_from[pi] = 0;
  h.nph[pi] = 0;
  if (from <= 0) return AMGDD_OK;
  std::vector<PhaseDesc> ph;
  if (!tail_phases(h, from, pi == 1, ph)) return AMGDD_OK;
  size_t smem = 0;
  for (const auto& d : ph) smem = std::max(smem, phase_smem(d));
  AMGDD_TRY(persistent_grid(smem, &h.ph_grid[pi]));
  AMGDD_TRY(h.d_ph[pi].upload(ph, h.work));
  AMGDD_CUDA(cudaStreamSynchronize(h.work));
  h.nph[pi] = (int)ph.size();
  h.ph_smem[pi] = smem;
  h.persist_from[pi] = from;
  return AMGDD_OK;
}

// Mean device time, in microseconds, of one V-cycle from level l on (r, x),
// captured in a graph as the solve runs it (eager launches would add host
// launch time): 3 warm-up and 10 timed graph launches.
static int time_vcycle_graph(amgdd_hierarchy& h, int l, bool f32, const void* r, void* x, double* us) {
  cudaStream_t s = h.work;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  AMGDD_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  int rc = vcycle(h, l, f32, r, x, nullptr, s);
  const cudaError_t ce = cudaStreamEndCapture(s, &g);
  if (rc == AMGDD_OK && (ce != cudaSuccess || cudaGraphInstantiate(&ge, g, 0) != cudaSuccess)) {
    set_error("V-cycle graph capture failed during setup");
    rc = AMGDD_ERR_CUDA;
  }
  if (g) cudaGraphDestroy(g);
  cudaEvent_t e[2] = {nullptr, nullptr};
  for (auto& v : e)
    if (rc == AMGDD_OK && cudaEventCreate(&v) != cudaSuccess) rc = AMGDD_ERR_CUDA;
  for (int k = 0; k < 13 && rc == AMGDD_OK; ++k) {
    if (k == 3) cudaEventRecord(e[0], s);
    if (cudaGraphLaunch(ge, s) != cudaSuccess) rc = AMGDD_ERR_CUDA;
  }
  float ms = 0.f;
  if (rc == AMGDD_OK) {
    cudaEventRecord(e[1], s);
    if (cudaEventSynchronize(e[1]) != cudaSuccess || cudaEventElapsedTime(&ms, e[0], e[1]) != cudaSuccess)
      rc = AMGDD_ERR_CUDA;
  }
  if (ge) cudaGraphExecDestroy(ge);
  for (auto& v : e)
    if (v) cudaEventDestroy(v);
  *us = 1e3 * ms / 10.0;
  return rc;
}

// Dense tail of level l: B = the FP64 V-cycle from l applied to the unit
// vectors (the cycle is a fixed linear map of r when x starts at 0, Section
// 3.1), so that the cycle from l down becomes one GEMV.  Column j of B is
// computed into row j of a scratch C = B^T; B64 and B32 (row-major, leading
// dimension n rounded up to 4, zero columns) follow by a tiled transpose.
// Any dense tail already chosen below l serves the computation.
static int build_dense(amgdd_hierarchy& h, int l) {
  cudaStream_t s = h.work;
  Level& L = *h.lv[l];
  const int64_t n = L.n;
  DBuf<double> C, rv, xv, one;
  AMGDD_TRY(C.alloc((size_t)(n * n)));
  AMGDD_TRY(rv.alloc(n));
  AMGDD_TRY(xv.alloc(n));
  const std::vector<double> unit{1.0};
  AMGDD_TRY(one.upload(unit, s));
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  AMGDD_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  int rc = vcycle(h, l, false, rv.p, xv.p, nullptr, s);
  const cudaError_t ce = cudaStreamEndCapture(s, &g);
  if (rc == AMGDD_OK && (ce != cudaSuccess || cudaGraphInstantiate(&ge, g, 0) != cudaSuccess)) {
    set_error("dense tail: V-cycle graph capture failed");
    rc = AMGDD_ERR_CUDA;
  }
  if (g) cudaGraphDestroy(g);
  for (int64_t j = 0; j < n && rc == AMGDD_OK; ++j) {
    if (cudaMemsetAsync(rv.p, 0, n * sizeof(double), s) != cudaSuccess ||
        cudaMemcpyAsync(rv.p + j, one.p, sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        cudaGraphLaunch(ge, s) != cudaSuccess ||
        cudaMemcpyAsync(C.p + j * n, xv.p, n * sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      rc = AMGDD_ERR_CUDA;
  }
  if (ge) cudaGraphExecDestroy(ge);
  AMGDD_TRY(rc);
  L.dld = (n + 3) / 4 * 4;
  AMGDD_TRY(L.B64.alloc((size_t)(n * L.dld)));
  AMGDD_TRY(L.B32.alloc((size_t)(n * L.dld)));
  AMGDD_TRY(launch_dense_pack(C.p, (int)n, L.dld, L.B64.p, L.B32.p, s));
  // dplan: one n x dld block; inputs n..dld-1 gather x[0] against zero columns
  std::vector<int32_t> idx(L.dld, 0);
  for (int64_t j = 0; j < n; ++j) idx[j] = (int32_t)j;
  AMGDD_TRY(L.d_didx.upload(idx, s));
  const std::vector<int32_t> nr{(int32_t)n}, nc{(int32_t)L.dld};
  const std::vector<int64_t> zero{0};
  AMGDD_TRY(build_seg(L.dplan, nr, nc, zero, zero, zero, L.d_didx.p, h.iota.p, s, 1));
  AMGDD_CUDA(cudaStreamSynchronize(s));
  return AMGDD_OK;
}

static void drop_dense(Level& L) {
  L.B64.release();
  L.B32.release();
  L.d_didx.release();
}

// Setup-time choice of the dense tail, per precision.  Candidates are the
// levels l >= 1 above the coarsest with n_l <= kDenseMaxN, deepest first;
// a candidate is built only while a GEMV of its FP32 matrix at the measured
// copy bandwidth could beat the measured V-cycle from l.  Every built
// candidate is timed in the V-cycle from level 0 (graph), against none.
constexpr int64_t kDenseMaxN = 12288;
constexpr double kHbmBytesPerUs = 6.8e6;

// MIXED16 storage: FP16 copies (round to nearest) of every level's smoother
// rows W_i and W_i^T, basis Z_i and Z_i^T and block rows of A.  FP16 holds
// magnitudes up to 65504 with 11 significant bits; a level whose FP32 copies
// hold a larger or non-finite entry keeps FP32 (the V-cycle then reads FP32
// there).  Entries below 2^-24 round to 0 or to subnormals: their absolute
// error, at most 2^-25, is far below the rounding of the row's largest
// entries.  Built once; the FP32 copies stay for MIXED32 and batched solves.
// The padded FP16 copy of one plan's FP32 matrix and its chunk descriptors
// (the plan's chunks as setup chose them, pointing into the padded copy).
static int build_pad16(SegPlan& p, const float* M32, cudaStream_t s) {
  p.m16.release();
  p.chunk_desc16.release();
  p.mat_len16 = 0;
  if (p.nchunks == 0 || M32 == nullptr) return AMGDD_OK;
  std::vector<int64_t> off16(p.nblocks + 1, 0);
  for (int b = 0; b < p.nblocks; ++b)
    off16[b + 1] = off16[b] + (int64_t)p.h_nr[b] * (((int64_t)p.h_nc[b] + 7) / 8 * 8);
  p.mat_len16 = off16[p.nblocks];
  DBuf<int64_t> d_off16;
  AMGDD_TRY(d_off16.upload(off16, s));
  AMGDD_TRY(p.m16.alloc(std::max<int64_t>(p.mat_len16, 1)));
  AMGDD_TRY(launch_pad16(M32, p.m_off.p, p.nr.p, p.nc.p, d_off16.p, p.nblocks, p.m16.p, s));
  std::vector<SegDesc> cd;
  cd.reserve(p.nchunks);
  const int rpc = p.rows_per_chunk;
  for (int b = 0; b < p.nblocks; ++b)
    for (int r = 0; r < p.h_nr[b]; r += rpc)
      cd.push_back(SegDesc{off16[b], p.h_ioff[b], p.h_ooff[b], r, std::min(p.h_nr[b], r + rpc), p.h_nc[b],
                           p.h_nr[b]});
  if ((int)cd.size() != p.nchunks) {
    set_error("build_pad16: chunk count mismatch");
    return AMGDD_ERR_INTERNAL;
  }
  AMGDD_TRY(p.chunk_desc16.upload(cd, s));
  return AMGDD_OK;
}

// The transposed FP16 copy of one plan (columns of rows padded to an even
// count) and tasks of up to 2 kind rows for the FP16 row-per-lane kernel.
static int build_pad16t(SegPlan& p, const float* T32, int kind, cudaStream_t s) {
  if (T32 == nullptr || p.nblocks == 0) return AMGDD_OK;
  std::vector<int64_t> off16(p.nblocks + 1, 0);
  for (int b = 0; b < p.nblocks; ++b)
    off16[b + 1] = off16[b] + (int64_t)p.h_nc[b] * (((int64_t)p.h_nr[b] + 1) / 2 * 2);
  if (p.mt16.p == nullptr) {
    DBuf<int64_t> d_off16;
    AMGDD_TRY(d_off16.upload(off16, s));
    AMGDD_TRY(p.mt16.alloc(std::max<int64_t>(off16[p.nblocks], 2)));
    AMGDD_TRY(launch_pad16t(T32, p.m_off.p, p.nr.p, p.nc.p, d_off16.p, p.nblocks, p.mt16.p, s));
  }
  std::vector<SegDesc> td;
  for (int b = 0; b < p.nblocks; ++b)
    for (int r = 0; r < p.h_nr[b]; r += 2 * kind)
      td.push_back(SegDesc{off16[b], p.h_ioff[b], p.h_ooff[b], r, std::min(p.h_nr[b], r + 2 * kind), p.h_nc[b],
                           p.h_nr[b]});
  p.ntasks16 = (int)td.size();
  return p.task_desc16.upload(td, s);
}

// FP16 form of one plan under MIXED16: the FP32 launch as setup chose it,
// against the FP16 kernels over the same blocks: lanes per row (rows padded
// to 16-byte vectors; 4, 8, 16 or 32 lanes, the plan's chunks) and, for rows
// of at most 256 entries, row per lane (two rows per half2 of the transposed
// copy; 8, 16 or 32 lanes per task), on scratch vectors; the fastest is kept
// (lanes16 = 0: the plan reads its FP32 copy and the FP16 copies are
// dropped).  The choice is cached like the others.
static int tune16(SegPlan& p, const std::string& key, const float* M32, const float* T32, int64_t nin, int64_t nout,
                  SegMode mode, cudaStream_t s) {
  p.lanes16 = 0;
  if (p.nblocks == 0 || M32 == nullptr) return AMGDD_OK;
  const bool can_lanes = p.nchunks > 0;
  const bool can_rows = T32 != nullptr && p.max_nc <= 256;
  auto valid = [&](int l) {
    return l == 0 || (l > 0 && can_lanes && (l == 4 || l == 8 || l == 16 || l == 32)) ||
           (l < 0 && can_rows && (l == -8 || l == -16 || l == -32));
  };
  auto realize = [&](int l) -> int {  // build the copies form l reads, drop the others
    if (l <= 0) {
      p.m16.release();
      p.chunk_desc16.release();
    }
    if (l >= 0) {
      p.mt16.release();
      p.task_desc16.release();
      p.ntasks16 = 0;
    }
    if (l > 0 && p.m16.p == nullptr) AMGDD_TRY(build_pad16(p, M32, s));
    if (l < 0) AMGDD_TRY(build_pad16t(p, T32, -l, s));
    p.lanes16 = l;
    return AMGDD_OK;
  };
  double cached = 0.0;
  if (g_tune && g_tune->get(key, cached)) return realize(valid((int)cached) ? (int)cached : 0);
  if (g_tune && !g_tune->on) return realize(can_lanes ? p.lanes : 0);  // no timing
  DBuf<float> xin, yout, cin;
  AMGDD_TRY(xin.alloc(std::max<int64_t>(nin, 1)));
  AMGDD_TRY(yout.alloc(std::max<int64_t>(nout, 1)));
  AMGDD_TRY(cin.alloc(std::max<int64_t>(nout, 1)));
  AMGDD_TRY(xin.zero(s));
  AMGDD_TRY(yout.zero(s));
  AMGDD_TRY(cin.zero(s));
  constexpr int kReps = 8;
  int rc = AMGDD_OK;
  float best_t = 0.f;
  int best = 0;
  for (int l : {0, 4, 8, 16, 32, -8, -16, -32}) {
    if (!valid(l)) continue;
    if (l > 0 && p.m16.p == nullptr) rc = build_pad16(p, M32, s);
    if (l < 0 && rc == AMGDD_OK) rc = build_pad16t(p, T32, -l, s);
    p.lanes16 = l;
    float ms = 0.f;
    if (rc == AMGDD_OK)
      rc = time_cold(s, kReps, [&] {
        return l == 0 ? launch_seg(p, M32, true, xin.p, yout.p, true, mode, nullptr, s,
                                   mode == SEG_RESID ? cin.p : nullptr, nullptr, T32)
                      : launch_seg16(p, xin.p, yout.p, mode, nullptr, s, mode == SEG_RESID ? cin.p : nullptr,
                                     nullptr);
      }, &ms);
    if (rc != AMGDD_OK) break;
    if (l == 0 || ms < best_t) {
      best_t = ms;
      best = l;
    }
  }
  AMGDD_TRY(rc);
  AMGDD_TRY(realize(best));
  if (g_tune) g_tune->put(key, (double)best);
  return AMGDD_OK;
}

// MIXED16 storage: per gather-GEMV plan of every level, an FP16 copy (round
// to nearest) of its FP32 matrix (smoother rows W_i or W_i^T, basis Z_i or
// Z_i^T, coarse block rows), kept where setup times it faster than the FP32
// copy.  FP16 holds magnitudes up to 65504 with 11 significant bits; a level
// whose FP32 copies hold a larger or non-finite entry keeps FP32 throughout.
// Entries below 2^-24 round to 0 or to subnormals: their absolute error, at
// most 2^-25, is far below the rounding of the row's largest entries.  Built
// once; the FP32 copies stay for MIXED32, batched solves and the persistent
// tail.
static int build_half(amgdd_hierarchy& h) {
  cudaStream_t s = h.work;
  FlushScope flush_scope;
  for (size_t lvl = 0; lvl < h.lv.size(); ++lvl) {
    Level& L = *h.lv[lvl];
    if (L.coarsest || L.h16) continue;
    const DBuf<float>* srcs[6] = {&L.W32, &L.Wt32, &L.Z32, &L.Zt32, &L.A32, &L.At32};
    bool ok = true;
    std::vector<float> hv;
    for (const DBuf<float>* src : srcs) {
      if (src->p == nullptr || src->n == 0) continue;
      AMGDD_TRY(download(hv, src->p, src->n, s));
      for (float v : hv)
        if (!(std::fabs(v) <= 65000.0f)) {
          ok = false;
          break;
        }
      if (!ok) break;
    }
    if (!ok) continue;  // this level keeps FP32
    L.h16 = true;
    const std::string k = "L" + std::to_string(lvl) + "|h16|";
    const int64_t nn = L.col0.back();
    AMGDD_TRY(tune16(L.ras, k + "ras", L.W32.p, L.Wt32.p, L.n, L.n, SEG_STORE, s));
    AMGDD_TRY(tune16(L.rast, k + "rast", L.Wt32.p, L.W32.p, L.n, L.n, SEG_ATOMIC_ADD, s));
    if (L.yd32.p)
      AMGDD_TRY(tune16(L.rast_det, k + "rastd", L.Wt32.p, L.W32.p, L.n, L.om_ptr.back(), SEG_STORE, s));
    AMGDD_TRY(tune16(L.restr, k + "restrict", L.Zt32.p, L.Z32.p, L.n, nn, SEG_STORE, s));
    AMGDD_TRY(tune16(L.prol, k + "prolong", L.Z32.p, L.Zt32.p, nn, L.n, SEG_ADD, s));
    if (L.has_blk) AMGDD_TRY(tune16(L.ablk, k + "ablk", L.A32.p, L.At32.p, L.n, L.n, SEG_RESID, s));
  }
  AMGDD_CUDA(cudaStreamSynchronize(s));
  return AMGDD_OK;
}

static int tune_dense(amgdd_hierarchy& h) {
  cudaStream_t s = h.work;
  const int nl = (int)h.lv.size();
  Level& L0 = *h.lv[0];
  h.dense_from[0] = h.dense_from[1] = 0;
  if (h.prm.dense_tail < 0) return AMGDD_OK;
  if (h.prm.dense_tail > 0) {  // forced level
    const int l = h.prm.dense_tail;
    if (l + 1 >= nl || h.lv[l]->n > kDenseMaxN) {
      set_error("dense_tail = %d: level must be above the coarsest with at most %lld unknowns", l,
                (long long)kDenseMaxN);
      return AMGDD_ERR_INVALID_ARG;
    }
    AMGDD_TRY(build_dense(h, l));
    h.dense_from[0] = h.dense_from[1] = l;
    return AMGDD_OK;
  }
  double c64 = 0.0, c32 = 0.0;
  if (g_tune && ((g_tune->get("dense|fp64", c64) && g_tune->get("dense|mixed", c32)) || !g_tune->on)) {
    const int want[2] = {g_tune->on ? (int)c64 : 0, g_tune->on ? (int)c32 : 0};
    // build deepest first, so that a shallower matrix is computed through it
    for (int l = nl - 2; l >= 1; --l) {
      if (want[0] != l && want[1] != l) continue;
      if (h.lv[l]->coarsest || h.lv[l]->n > kDenseMaxN) continue;
      AMGDD_TRY(build_dense(h, l));
      for (int pi = 0; pi < 2; ++pi)
        if (want[pi] == l) h.dense_from[pi] = l;
    }
    return AMGDD_OK;
  }
  AMGDD_TRY(L0.r32.zero(s));
  AMGDD_TRY(h.r.zero(s));
  const void* r[2] = {h.r.p, L0.r32.p};
  void* x[2] = {h.z.p, L0.x32.p};
  double best_us[2];
  int best[2] = {0, 0};
  for (int pi = 0; pi < 2; ++pi) {
    AMGDD_TRY(time_vcycle_graph(h, 0, pi == 1, r[pi], x[pi], &best_us[pi]));
    h.dense_us[pi][0] = best_us[pi];
  }
  for (int l = nl - 2; l >= 1; --l) {
    Level& L = *h.lv[l];
    if (L.coarsest || L.n > kDenseMaxN) break;
    double from_l = 0.0;
    AMGDD_TRY(L.r32.zero(s));
    AMGDD_TRY(time_vcycle_graph(h, l, true, L.r32.p, L.x32.p, &from_l));
    L.vc_us[1] = from_l;
    if ((double)L.n * (double)L.n * 4.0 / kHbmBytesPerUs >= from_l) break;
    AMGDD_TRY(build_dense(h, l));
    bool keep = false;
    for (int pi = 0; pi < 2; ++pi) {
      const int prev = h.dense_from[pi];
      h.dense_from[pi] = l;
      double us = 0.0;
      AMGDD_TRY(time_vcycle_graph(h, 0, pi == 1, r[pi], x[pi], &us));
      h.dense_us[pi][l] = us;
      if (us < best_us[pi]) {
        best_us[pi] = us;
        best[pi] = l;
        keep = true;
      } else {
        h.dense_from[pi] = prev;
      }
    }
    if (!keep) drop_dense(L);
  }
  for (int l = 1; l + 1 < nl; ++l)
    if (l != best[0] && l != best[1]) drop_dense(*h.lv[l]);
  h.dense_from[0] = best[0];
  h.dense_from[1] = best[1];
  if (g_tune) {
    g_tune->put("dense|fp64", (double)best[0]);
    g_tune->put("dense|mixed", (double)best[1]);
  }
  if (g_timer.on)
    fprintf(stderr, "[amgdd] dense tail: fp64 from level %d (%.1f us), mixed from level %d (%.1f us)\n", best[0],
            best_us[0], best[1], best_us[1]);
  return AMGDD_OK;
}

// Setup-time choice of the persistent tail: time V-cycles with the tail
// starting at each level (and with none) and keep the fastest, per precision.
static int tune_tail(amgdd_hierarchy& h) {
  cudaStream_t s = h.work;
  const int nl = (int)h.lv.size();
  AMGDD_TRY(h.bar.alloc(2));
  AMGDD_TRY(h.bar.zero(s));
  AMGDD_TRY(h.st.zero(s));
  Level& L0 = *h.lv[0];
  AMGDD_TRY(L0.r32.zero(s));
  AMGDD_TRY(h.r.zero(s));
  int rc = AMGDD_OK;
  for (int pi = 0; pi < 2 && rc == AMGDD_OK; ++pi) {
    const bool f32 = pi == 1;
    const std::string key = f32 ? "tail|mixed" : "tail|fp64";
    double cached = 0.0;
    if (h.prm.deterministic) {  // the persistent phases scatter RAS-T with atomics
      rc = set_tail(h, pi, 0);
      continue;
    }
    if (g_tune && (g_tune->get(key, cached) || !g_tune->on)) {
      rc = set_tail(h, pi, g_tune->on ? (int)cached : 0);
      continue;
    }
    const void* r = f32 ? (const void*)L0.r32.p : (const void*)h.r.p;
    void* x = f32 ? (void*)L0.x32.p : (void*)h.z.p;
    int best = 0;
    double best_us = 0.0;
    for (int from = 0; from < std::min(nl, 16) && rc == AMGDD_OK; ++from) {
      if ((rc = set_tail(h, pi, from)) != AMGDD_OK) break;
      if (from > 0 && h.persist_from[pi] != from) continue;  // tail not expressible from this level
      double us = 0.0;
      if ((rc = time_vcycle_graph(h, 0, f32, r, x, &us)) != AMGDD_OK) break;
      h.persist_us[pi][from] = us;
      if (from == 0 || us < best_us) {
        best = from;
        best_us = us;
      }
    }
    if (rc == AMGDD_OK) rc = set_tail(h, pi, best);
    if (rc == AMGDD_OK && g_tune) g_tune->put(key, (double)best);
    if (g_timer.on && rc == AMGDD_OK)
      fprintf(stderr, "[amgdd] %s V-cycle: persistent tail from level %d (%.1f us)\n", f32 ? "mixed" : "fp64", best,
              best_us);
  }
  AMGDD_TRY(rc);
  PcgState st{};
  AMGDD_CUDA(cudaMemcpy(&st, h.st.p, sizeof st, cudaMemcpyDeviceToHost));
  if (st.vc_err != 0) {
    set_error("persistent V-cycle: grid barrier timed out during setup");
    return AMGDD_ERR_TIMEOUT;
  }
  return AMGDD_OK;
}

// z = B r on FP64 PCG vectors, in the hierarchy's precision.
// z = M_2^{-1} r, the additive two-level method (FP64): additive Schwarz
// z = sum_i R_i^T A_i^{-1} R_i r (scatter-add), plus P A_1^{-1} P^T r with
// the exact coarsest solve of level 1.
static int precondition_additive(amgdd_hierarchy& h, const double* r, double* z, const int* skip, cudaStream_t s) {
  Level& L0 = *h.lv[0];
  Level& L1 = *h.lv[1];
  AMGDD_CUDA(cudaMemsetAsync(z, 0, L0.n * sizeof(double), s));
  AMGDD_TRY(launch_seg(L0.asp, L0.Wf64.p, false, r, z, false, SEG_ATOMIC_ADD, skip, s, nullptr, nullptr, L0.Wft64.p));
  AMGDD_TRY(launch_seg(L0.restr, L0.Zt64.p, false, r, L1.r64.p, false, SEG_STORE, skip, s, nullptr, nullptr, L0.Z64.p));
  AMGDD_TRY(coarse_solve(h, L1, L1.r64.p, L1.x64.p, L1.s64.p, skip, s));
  return launch_seg(L0.prol, L0.Z64.p, false, L1.x64.p, z, false, SEG_ADD, skip, s, nullptr, nullptr, L0.Zt64.p);
}

static int precondition(amgdd_hierarchy& h, const double* r, double* z, const int* skip, cudaStream_t s) {
  Level& L0 = *h.lv[0];
  if (h.prm.cycle == 1) return precondition_additive(h, r, z, skip, s);
  if (mixed(h)) {
    AMGDD_TRY(launch_cast(r, false, L0.r32.p, true, L0.n, skip, s));
    AMGDD_TRY(vcycle(h, 0, true, L0.r32.p, L0.x32.p, skip, s));
    return launch_cast(L0.x32.p, true, z, false, L0.n, skip, s);
  }
  return vcycle(h, 0, false, r, z, skip, s);
}

// q = A p in FP64 on level 0.
// A one-level hierarchy keeps its dense A (the coarsest level's Aw64, symmetric):
// in deterministic mode its A-apply is that GEMV instead of the row groups'
// scatter with atomics (level 0 has no ELL rows without aggregates).
static bool dense_level0(const amgdd_hierarchy& h) {
  const Level& L0 = *h.lv[0];
  return h.prm.deterministic && L0.coarsest && L0.Aw64.p != nullptr;
}

static int apply_fine64(amgdd_hierarchy& h, const double* p, double* q, const int* skip, cudaStream_t s) {
  Level& L0 = *h.lv[0];
  if (L0.use_ell) return launch_ell(L0, false, p, q, nullptr, skip, s);
  if (dense_level0(h))
    return launch_seg(L0.ras, L0.Aw64.p, false, p, q, false, SEG_STORE, skip, s, nullptr, nullptr, L0.Aw64.p);
  AMGDD_CUDA(cudaMemsetAsync(q, 0, L0.n * sizeof(double), s));
  return launch_apply(L0.aplan, L0, false, p, q, +1, skip, s);
}

static int pcg_iteration(amgdd_hierarchy& h, cudaStream_t s, cudaGraphConditionalHandle cond = 0,
                         int use_cond = 0) {
  const int64_t n = h.n;
  PcgState* st = h.st.p;
  const int* done = &st->done;
  const bool flex = mixed(h);
  Level& L0 = *h.lv[0];
  if (L0.use_ell) {
    // fused: four launches besides the V-cycle, each reducing its own dot
    // product and taking the scalar step in its last CTA
    AMGDD_TRY(launch_cg_ap(L0, st, h.p.p, h.q.p, h.partials.p, s));
    AMGDD_TRY(launch_cg_xr(st, h.x.p, h.r.p, flex ? L0.r32.p : nullptr, h.p.p, h.q.p, n, h.partials.p, s));
    if (h.prm.cycle == 1)
      AMGDD_TRY(precondition_additive(h, h.r.p, h.z.p, done, s));
    else if (flex)
      AMGDD_TRY(vcycle(h, 0, true, L0.r32.p, L0.x32.p, done, s));
    else
      AMGDD_TRY(vcycle(h, 0, false, h.r.p, h.z.p, done, s));
    AMGDD_TRY(launch_cg_zdot(st, flex ? L0.x32.p : nullptr, h.z.p, h.r.p, flex ? h.zold.p : nullptr, n, h.partials.p,
                             s, cond, use_cond));
    return launch_update_p(st, h.p.p, h.z.p, flex ? h.zold.p : nullptr, n, s);
  }
  AMGDD_TRY(apply_fine64(h, h.p.p, h.q.p, done, s));
  AMGDD_TRY(launch_dot_partial(h.p.p, h.q.p, nullptr, n, h.partials.p, done, s));
  AMGDD_TRY(launch_pcg_scalar(1, st, h.partials.p, s));
  AMGDD_TRY(launch_update_xr(st, h.x.p, h.r.p, h.p.p, h.q.p, n, s));
  AMGDD_TRY(launch_dot_partial(h.r.p, h.r.p, nullptr, n, h.partials.p, done, s));
  AMGDD_TRY(launch_pcg_scalar(2, st, h.partials.p, s));
  AMGDD_TRY(precondition(h, h.r.p, h.z.p, done, s));
  AMGDD_TRY(launch_dot_partial(h.r.p, h.z.p, flex ? h.zold.p : nullptr, n, h.partials.p, done, s));
  AMGDD_TRY(launch_pcg_scalar(3, st, h.partials.p, s, cond, use_cond));
  AMGDD_TRY(launch_update_p(st, h.p.p, h.z.p, flex ? h.zold.p : nullptr, n, s));
  return AMGDD_OK;
}

// CG start: r = b, x = 0, ||b||^2, z = B r, p = z, r^T z.
static int pcg_start(amgdd_hierarchy& h, cudaStream_t s) {
  const int64_t n = h.n;
  PcgState* st = h.st.p;
  const int* done = &st->done;
  AMGDD_CUDA(cudaMemcpyAsync(h.r.p, h.b.p, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  AMGDD_CUDA(cudaMemsetAsync(h.x.p, 0, n * sizeof(double), s));
  AMGDD_TRY(launch_dot_partial(h.b.p, h.b.p, nullptr, n, h.partials.p, nullptr, s));
  AMGDD_TRY(launch_pcg_scalar(4, st, h.partials.p, s));
  AMGDD_TRY(precondition(h, h.r.p, h.z.p, done, s));
  AMGDD_TRY(launch_copy_vec(h.z.p, h.p.p, false, n, done, s));
  if (mixed(h)) AMGDD_TRY(launch_copy_vec(h.z.p, h.zold.p, false, n, done, s));
  AMGDD_TRY(launch_dot_partial(h.r.p, h.z.p, nullptr, n, h.partials.p, done, s));
  AMGDD_TRY(launch_pcg_scalar(0, st, h.partials.p, s));
  return AMGDD_OK;
}

// Graphs of one precision: the CG start, and a WHILE node whose body is one
// CG iteration; the iteration's scalar kernel sets the loop condition on the
// device, so a whole solve runs without returning to the host.
static int build_solve_graphs_once(amgdd_hierarchy& h, int pi, cudaStream_t s) {
  for (auto* ge : {&h.ginit[pi], &h.gloop[pi]})
    if (*ge) {
      cudaGraphExecDestroy(*ge);
      *ge = nullptr;
    }
  cudaGraph_t g;
  AMGDD_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  capture_begin();
  int rc = pcg_start(h, s);
  h.ginit_kernels[pi] = capture_end();
  cudaError_t ce = cudaStreamEndCapture(s, &g);
  if (rc != AMGDD_OK) return rc;
  AMGDD_CUDA(ce);
  AMGDD_CUDA(cudaGraphInstantiate(&h.ginit[pi], g, 0));
  cudaGraphDestroy(g);

  cudaGraph_t lg;
  AMGDD_CUDA(cudaGraphCreate(&lg, 0));
  cudaGraphConditionalHandle cond;
  AMGDD_CUDA(cudaGraphConditionalHandleCreate(&cond, lg, 1u, cudaGraphCondAssignDefault));
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = cond;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  AMGDD_CUDA(cudaGraphAddNode(&node, lg, nullptr, nullptr, 0, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  AMGDD_CUDA(cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  capture_begin();
  rc = pcg_iteration(h, s, cond, 1);
  h.gloop_kernels[pi] = capture_end();
  ce = cudaStreamEndCapture(s, &body);
  if (rc != AMGDD_OK) return rc;
  AMGDD_CUDA(ce);
  AMGDD_CUDA(cudaGraphInstantiate(&h.gloop[pi], lg, 0));
  cudaGraphDestroy(lg);
  return AMGDD_OK;
}

// CUDA graphs of the solve.  If the persistent V-cycle tail cannot be
// captured (a cooperative launch inside the conditional loop body), the tail
// is dropped for this precision and the graphs are captured again.
static int build_solve_graphs(amgdd_hierarchy& h, int pi, cudaStream_t s) {
  int rc = build_solve_graphs_once(h, pi, s);
  if (rc == AMGDD_OK || h.persist_from[pi] == 0) return rc;
  (void)cudaGetLastError();
  AMGDD_TRY(set_tail(h, pi, 0));
  return build_solve_graphs_once(h, pi, s);
}

static int solve_once(amgdd_hierarchy& h, const double* bsrc, bool bdev, double tol, double* xdst, bool xdev,
                      cudaStream_t s, amgdd_info* info);

// One right-hand side.  A MIXED32 solve whose FP32 cycle stalls (flexible CG
// with ||r|| falling by less than 10% over 10 iterations) is redone with the
// FP64 cycle; info then reports both attempts.
static int solve_one(amgdd_hierarchy& h, const double* bsrc, bool bdev, double tol, double* xdst, bool xdev,
                     cudaStream_t s, amgdd_info* info) {
  amgdd_info first{};
  int st = AMGDD_OK;
  if (mixed(h) && h.mixed_stalled) {
    // this hierarchy's FP32 cycle stalled before: go straight to FP64
    first = amgdd_info{};
    st = kStallStatus;
  } else {
    st = solve_once(h, bsrc, bdev, tol, xdst, xdev, s, &first);
  }
  if (st != kStallStatus) {
    if (info) *info = first;
    return st;
  }
  h.mixed_stalled = true;
  const int prec = h.precision;
  h.precision = AMGDD_FP64;
  amgdd_info second{};
  st = solve_once(h, bsrc, bdev, tol, xdst, xdev, s, &second);
  h.precision = prec;
  second.fallback = 1;
  second.iters_mixed = first.iters;
  second.iters += first.iters;
  second.solve_ms += first.solve_ms;
  if (info) *info = second;
  return st;
}

static int solve_once(amgdd_hierarchy& h, const double* bsrc, bool bdev, double tol, double* xdst, bool xdev,
                      cudaStream_t s, amgdd_info* info) {
  const int64_t n = h.n;
  cudaEvent_t e0, e1;
  AMGDD_CUDA(cudaEventCreate(&e0));
  AMGDD_CUDA(cudaEventCreate(&e1));
  AMGDD_CUDA(cudaEventRecord(e0, s));
  AMGDD_CUDA(cudaMemcpyAsync(h.b.p, bsrc, n * sizeof(double), bdev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                             s));
  PcgState init{};
  init.tol2 = tol * tol;
  init.max_iter = h.prm.max_iter;
  init.flexible = mixed(h) ? 1 : 0;
  *h.st_host = init;
  AMGDD_CUDA(cudaMemcpyAsync(h.st.p, h.st_host, sizeof(PcgState), cudaMemcpyHostToDevice, s));
  const int pi = mixed(h) ? 1 : 0;
  if (h.prm.use_graph) {
    if (h.gloop[pi] == nullptr) AMGDD_TRY(build_solve_graphs(h, pi, s));
    AMGDD_CUDA(cudaGraphLaunch(h.ginit[pi], s));
    count_graph_launch(h.ginit_kernels[pi]);
    AMGDD_CUDA(cudaGraphLaunch(h.gloop[pi], s));
    AMGDD_CUDA(cudaMemcpyAsync(h.st_host, h.st.p, sizeof(PcgState), cudaMemcpyDeviceToHost, s));
  } else {
    AMGDD_TRY(pcg_start(h, s));
    const int K = std::max(1, h.prm.check_every);
    for (;;) {
      for (int k = 0; k < K; ++k) AMGDD_TRY(pcg_iteration(h, s));
      AMGDD_CUDA(cudaMemcpyAsync(h.st_host, h.st.p, sizeof(PcgState), cudaMemcpyDeviceToHost, s));
      AMGDD_CUDA(cudaStreamSynchronize(s));
      if (h.st_host->done) break;
    }
  }
  // true residual b - A x in FP64; when the recursively updated residual met
  // the tolerance but the true one did not (rounding drift over many
  // iterations), CG restarts from x with r = b - A x (at most twice)
  std::vector<double> part;
  PcgState fin{};
  double qq = 0.0;
  for (int restarts = 0;; ++restarts) {
    if (h.lv[0]->use_ell) {
      AMGDD_TRY(launch_ell(*h.lv[0], false, h.x.p, h.q.p, h.b.p, nullptr, s));
    } else if (dense_level0(h)) {
      AMGDD_TRY(launch_seg(h.lv[0]->ras, h.lv[0]->Aw64.p, false, h.x.p, h.q.p, false, SEG_RESID, nullptr, s, h.b.p,
                           nullptr, h.lv[0]->Aw64.p));
    } else {
      AMGDD_CUDA(cudaMemcpyAsync(h.q.p, h.b.p, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
      AMGDD_TRY(launch_apply(h.lv[0]->aplan, *h.lv[0], false, h.x.p, h.q.p, -1, nullptr, s));
    }
    AMGDD_TRY(launch_dot_partial(h.q.p, h.q.p, nullptr, n, h.partials.p, nullptr, s));
    AMGDD_TRY(download(part, h.partials.p, 2 * kDotBlocks, s));
    fin = *h.st_host;
    if (fin.vc_err != 0) {
      AMGDD_TRY(h.bar.zero(s));
      AMGDD_CUDA(cudaStreamSynchronize(s));
      set_error("persistent V-cycle: grid barrier timed out");
      return AMGDD_ERR_TIMEOUT;
    }
    qq = 0.0;
    for (int i = 0; i < kDotBlocks; ++i) qq += part[2 * i];
    if (fin.status != AMGDD_OK || qq <= fin.tol2 || restarts == 2 || fin.iters >= fin.max_iter) break;
    PcgState re = fin;
    re.done = 0;
    re.rr_mark = fin.bnorm2;  // the stall guard restarts its window
    *h.st_host = re;
    AMGDD_CUDA(cudaMemcpyAsync(h.st.p, h.st_host, sizeof(PcgState), cudaMemcpyHostToDevice, s));
    AMGDD_CUDA(cudaMemcpyAsync(h.r.p, h.q.p, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    const int* done = &h.st.p->done;
    AMGDD_TRY(precondition(h, h.r.p, h.z.p, done, s));
    AMGDD_TRY(launch_copy_vec(h.z.p, h.p.p, false, n, done, s));
    if (mixed(h)) AMGDD_TRY(launch_copy_vec(h.z.p, h.zold.p, false, n, done, s));
    AMGDD_TRY(launch_dot_partial(h.r.p, h.z.p, nullptr, n, h.partials.p, done, s));
    AMGDD_TRY(launch_pcg_scalar(0, h.st.p, h.partials.p, s));
    if (h.prm.use_graph) {
      AMGDD_CUDA(cudaGraphLaunch(h.gloop[pi], s));
    } else {
      const int K = std::max(1, h.prm.check_every);
      for (;;) {
        for (int k = 0; k < K; ++k) AMGDD_TRY(pcg_iteration(h, s));
        AMGDD_CUDA(cudaMemcpyAsync(h.st_host, h.st.p, sizeof(PcgState), cudaMemcpyDeviceToHost, s));
        AMGDD_CUDA(cudaStreamSynchronize(s));
        if (h.st_host->done) break;
      }
    }
    AMGDD_CUDA(cudaMemcpyAsync(h.st_host, h.st.p, sizeof(PcgState), cudaMemcpyDeviceToHost, s));
  }
  AMGDD_CUDA(cudaMemcpyAsync(xdst, h.x.p, n * sizeof(double), xdev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                             s));
  AMGDD_CUDA(cudaEventRecord(e1, s));
  AMGDD_CUDA(cudaEventSynchronize(e1));
  if (h.prm.use_graph) count_graph_launch(h.gloop_kernels[pi] * std::max(fin.iters, 1));
  float ms = 0.f;
  AMGDD_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (info) {
    info->iters = fin.iters;
    info->status = fin.status;
    info->relres = fin.relres;
    info->relres_true = fin.bnorm2 > 0 ? std::sqrt(qq / fin.bnorm2) : 0.0;
    info->solve_ms = ms;
  }
  return fin.status;
}

// ---------------------------------------------------------------------------
// After a call that launched kernels on `s`: report (and clear) an expired
// bounded wait recorded in the hierarchy's error word.
static int take_err_word(amgdd_hierarchy& h, cudaStream_t s) {
  int v = 0;
  AMGDD_CUDA(cudaMemcpyAsync(&v, &h.st.p->vc_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  AMGDD_CUDA(cudaStreamSynchronize(s));
  if (v == 0) return AMGDD_OK;
  AMGDD_CUDA(cudaMemsetAsync(&h.st.p->vc_err, 0, sizeof(int), s));
  if (h.bar.p) AMGDD_TRY(h.bar.zero(s));
  AMGDD_CUDA(cudaStreamSynchronize(s));
  set_error("a bounded device-side wait expired (staged copy or grid barrier)");
  return AMGDD_ERR_TIMEOUT;
}

// ---------------------------------------------------------------------------
// Batched right-hand sides: K in {2, 4, 8, 16, 32} independent CGs that
// share every V-cycle and A-apply launch (multi_kernels.cu).
constexpr int kMaxRhs = 32;
static int kidx(int K) { return K == 2 ? 0 : (K == 4 ? 1 : (K == 8 ? 2 : (K == 16 ? 3 : 4))); }
static int kclass(int g) { return g <= 2 ? 2 : (g <= 4 ? 4 : (g <= 8 ? 8 : (g <= 16 ? 16 : 32))); }

// Device bytes of the batched-solve workspace for `cap` columns (allocated
// or not): the eight CG vectors, the dot partials and states, and per level
// three FP64 and three FP32 vectors (plus the stored RAS-T products of the
// deterministic form).
static int64_t multi_bytes_estimate(const amgdd_hierarchy& h, int cap) {
  int64_t b = (int64_t)8 * h.n * cap * 8 + (int64_t)kDotBlocks * 2 * cap * 8 + (int64_t)cap * sizeof(PcgState) + 16;
  for (const auto& L : h.lv) {
    b += L->n * cap * (3 * 8 + 3 * 4);
    if (L->yd64.p) b += (int64_t)L->om_ptr.back() * cap * (8 + 4);
  }
  return b;
}

static int ensure_multi(amgdd_hierarchy& h, int K) {
  auto& M = h.mw;
  if (M.ready && M.cap >= K) return AMGDD_OK;
  // (re)allocate for K columns: the captured graphs hold the old pointers
  M.drop_graphs();
  M.ready = false;
  if (M.st_host) {
    cudaFreeHost(M.st_host);
    M.st_host = nullptr;
  }
  const int64_t nk = h.n * K;
  for (auto* v : {&M.x, &M.r, &M.z, &M.zold, &M.p, &M.q, &M.b, &M.stage}) AMGDD_TRY(v->alloc(nk));
  AMGDD_TRY(M.partials.alloc((int64_t)kDotBlocks * 2 * K));
  AMGDD_TRY(M.st.alloc(K));
  AMGDD_TRY(M.grp.alloc(4));
  AMGDD_CUDA(cudaMallocHost((void**)&M.st_host, K * sizeof(PcgState)));
  for (auto& Lp : h.lv) {
    Level& L = *Lp;
    const int64_t lk = L.n * K;
    AMGDD_TRY(L.mr64.alloc(lk));
    AMGDD_TRY(L.mx64.alloc(lk));
    AMGDD_TRY(L.ms64.alloc(lk));
    AMGDD_TRY(L.mr32.alloc(lk));
    AMGDD_TRY(L.mx32.alloc(lk));
    AMGDD_TRY(L.ms32.alloc(lk));
    if (L.yd64.p) {
      AMGDD_TRY(L.myd64.alloc((size_t)L.om_ptr.back() * K));
      AMGDD_TRY(L.myd32.alloc((size_t)L.om_ptr.back() * K));
    }
  }
  M.cap = K;
  M.ready = true;
  h.multi_bytes = multi_bytes_estimate(h, K);
  return AMGDD_OK;
}

// s = r - A x for K columns: block rows where stored, else the rows omega_i
// of A over Omega_i (with the RAS plan's index lists).
static int resid_multi(const Level& L, bool f32, int K, const void* x, const void* r, void* sv, const int* skip,
                       cudaStream_t s) {
  if (L.use_ell) return launch_ell_multi(L, f32, x, sv, r, K, skip, s);
  if (L.has_blk)
    return launch_seg_multi(L.ablk, f32 ? (const void*)L.A32.p : (const void*)L.A64.p,
                            f32 ? (const void*)L.At32.p : (const void*)L.At64.p, f32, x, sv, SEG_RESID, r, K, skip, s);
  return launch_seg_multi(L.ras, f32 ? (const void*)L.Aw32.p : (const void*)L.Aw64.p,
                          f32 ? (const void*)L.AwT32.p : (const void*)L.AwT64.p, f32, x, sv, SEG_RESID, r, K, skip, s);
}

// The V-cycle of Section 3.1 for K interleaved columns.
static int vcycle_multi(amgdd_hierarchy& h, int l, bool f32, int K, const void* r, void* x, const int* skip,
                        cudaStream_t s) {
  Level& L = *h.lv[l];
  // the dense tail stages K columns of its whole input in shared memory;
  // beyond that the separate levels below it serve
  if (l > 0 && h.dense_from[f32 ? 1 : 0] == l && L.dld * K * (f32 ? 4 : 8) <= 200 * 1024)
    return launch_seg_multi(L.dplan, f32 ? (const void*)L.B32.p : (const void*)L.B64.p, nullptr, f32, r, x,
                            SEG_STORE, nullptr, K,
                            skip, s);
  if (L.coarsest) {
    const void* r64 = r;
    void* x64 = x;
    if (f32) {
      AMGDD_TRY(launch_cast(r, true, L.mr64.p, false, L.n * K, skip, s));
      r64 = L.mr64.p;
      x64 = L.mx64.p;
    }
    AMGDD_TRY(launch_seg_multi(L.ras, L.W64.p, L.Wt64.p, false, r64, x64, SEG_STORE, nullptr, K, skip, s));
    if (h.prm.coarse_refine && L.Aw64.p) {  // one step of refinement, as coarse_solve
      AMGDD_TRY(launch_seg_multi(L.ras, L.Aw64.p, L.Aw64.p, false, x64, L.ms64.p, SEG_RESID, r64, K, skip, s));
      AMGDD_TRY(launch_seg_multi(L.ras, L.W64.p, L.Wt64.p, false, L.ms64.p, x64, SEG_ADD, nullptr, K, skip, s));
    }
    return f32 ? launch_cast(L.mx64.p, false, x, true, L.n * K, skip, s) : AMGDD_OK;
  }
  Level& N = *h.lv[l + 1];
  const void* W = f32 ? (const void*)L.W32.p : (const void*)L.W64.p;
  const void* Wt = f32 ? (const void*)L.Wt32.p : (const void*)L.Wt64.p;
  const void* Z = f32 ? (const void*)L.Z32.p : (const void*)L.Z64.p;
  const void* Zt = f32 ? (const void*)L.Zt32.p : (const void*)L.Zt64.p;
  void* sv = f32 ? (void*)L.ms32.p : (void*)L.ms64.p;
  void* rn = f32 ? (void*)N.mr32.p : (void*)N.mr64.p;
  void* xn = f32 ? (void*)N.mx32.p : (void*)N.mx64.p;
  AMGDD_TRY(launch_seg_multi(L.ras, W, Wt, f32, r, x, SEG_STORE, nullptr, K, skip, s));
  AMGDD_TRY(resid_multi(L, f32, K, x, r, sv, skip, s));
  AMGDD_TRY(launch_seg_multi(L.restr, Zt, Z, f32, sv, rn, SEG_STORE, nullptr, K, skip, s));
  AMGDD_TRY(vcycle_multi(h, l + 1, f32, K, rn, xn, skip, s));
  AMGDD_TRY(launch_seg_multi(L.prol, Z, Zt, f32, xn, x, SEG_ADD, nullptr, K, skip, s));
  AMGDD_TRY(resid_multi(L, f32, K, x, r, sv, skip, s));
  return apply_rast(L, f32, sv, x, skip, s, K);
}

static int precondition_multi(amgdd_hierarchy& h, int K, const double* r, double* z, const int* skip,
                              cudaStream_t s) {
  Level& L0 = *h.lv[0];
  if (mixed(h)) {
    AMGDD_TRY(launch_cast(r, false, L0.mr32.p, true, h.n * K, skip, s));
    AMGDD_TRY(vcycle_multi(h, 0, true, K, L0.mr32.p, L0.mx32.p, skip, s));
    return launch_cast(L0.mx32.p, true, z, false, h.n * K, skip, s);
  }
  return vcycle_multi(h, 0, false, K, r, z, skip, s);
}

static int pcg_start_multi(amgdd_hierarchy& h, int K, cudaStream_t s) {
  auto& M = h.mw;
  const int64_t n = h.n, nk = h.n * K;
  const int* skip = M.grp.p;
  AMGDD_CUDA(cudaMemcpyAsync(M.r.p, M.b.p, nk * sizeof(double), cudaMemcpyDeviceToDevice, s));
  AMGDD_CUDA(cudaMemsetAsync(M.x.p, 0, nk * sizeof(double), s));
  AMGDD_TRY(launch_dot_multi(M.b.p, M.b.p, nullptr, n, K, M.partials.p, nullptr, s));
  AMGDD_TRY(launch_pcg_scalar_multi(4, M.st.p, M.grp.p, M.partials.p, K, s));
  AMGDD_TRY(precondition_multi(h, K, M.r.p, M.z.p, skip, s));
  AMGDD_TRY(launch_copy_vec(M.z.p, M.p.p, false, nk, skip, s));
  if (mixed(h)) AMGDD_TRY(launch_copy_vec(M.z.p, M.zold.p, false, nk, skip, s));
  AMGDD_TRY(launch_dot_multi(M.r.p, M.z.p, nullptr, n, K, M.partials.p, skip, s));
  return launch_pcg_scalar_multi(0, M.st.p, M.grp.p, M.partials.p, K, s);
}

static int pcg_iteration_multi(amgdd_hierarchy& h, int K, cudaStream_t s, cudaGraphConditionalHandle cond = 0,
                               int use_cond = 0) {
  auto& M = h.mw;
  const int64_t n = h.n;
  const int* skip = M.grp.p;
  Level& L0 = *h.lv[0];
  if (L0.use_ell)
    AMGDD_TRY(launch_ell_multi(L0, false, M.p.p, M.q.p, nullptr, K, skip, s));
  else
    AMGDD_TRY(launch_seg_multi(L0.ras, L0.Aw64.p, L0.AwT64.p ? L0.AwT64.p : L0.Aw64.p, false, M.p.p, M.q.p, SEG_STORE,
                               nullptr, K, skip, s));
  AMGDD_TRY(launch_dot_multi(M.p.p, M.q.p, nullptr, n, K, M.partials.p, skip, s));
  AMGDD_TRY(launch_pcg_scalar_multi(1, M.st.p, M.grp.p, M.partials.p, K, s));
  AMGDD_TRY(launch_update_xr_multi(M.st.p, M.grp.p, M.x.p, M.r.p, M.p.p, M.q.p, n, K, s));
  AMGDD_TRY(launch_dot_multi(M.r.p, M.r.p, nullptr, n, K, M.partials.p, skip, s));
  AMGDD_TRY(launch_pcg_scalar_multi(2, M.st.p, M.grp.p, M.partials.p, K, s));
  AMGDD_TRY(precondition_multi(h, K, M.r.p, M.z.p, skip, s));
  const bool flex = mixed(h);
  AMGDD_TRY(launch_dot_multi(M.r.p, M.z.p, flex ? M.zold.p : nullptr, n, K, M.partials.p, skip, s));
  AMGDD_TRY(launch_pcg_scalar_multi(3, M.st.p, M.grp.p, M.partials.p, K, s, cond, use_cond));
  return launch_update_p_multi(M.st.p, M.grp.p, M.p.p, M.z.p, flex ? M.zold.p : nullptr, n, K, s);
}

// Graphs of the batched solve (start; WHILE loop over iterations), as for
// one right-hand side.
static int build_multi_graphs(amgdd_hierarchy& h, int pi, int K, cudaStream_t s) {
  auto& M = h.mw;
  const int ki = kidx(K);
  cudaGraph_t g;
  AMGDD_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  capture_begin();
  int rc = pcg_start_multi(h, K, s);
  M.ginit_kernels[pi][ki] = capture_end();
  cudaError_t ce = cudaStreamEndCapture(s, &g);
  if (rc != AMGDD_OK) return rc;
  AMGDD_CUDA(ce);
  AMGDD_CUDA(cudaGraphInstantiate(&M.ginit[pi][ki], g, 0));
  cudaGraphDestroy(g);
  cudaGraph_t lg;
  AMGDD_CUDA(cudaGraphCreate(&lg, 0));
  cudaGraphConditionalHandle cond;
  AMGDD_CUDA(cudaGraphConditionalHandleCreate(&cond, lg, 1u, cudaGraphCondAssignDefault));
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = cond;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  AMGDD_CUDA(cudaGraphAddNode(&node, lg, nullptr, nullptr, 0, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  AMGDD_CUDA(cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  capture_begin();
  rc = pcg_iteration_multi(h, K, s, cond, 1);
  M.gloop_kernels[pi][ki] = capture_end();
  ce = cudaStreamEndCapture(s, &body);
  if (rc != AMGDD_OK) return rc;
  AMGDD_CUDA(ce);
  AMGDD_CUDA(cudaGraphInstantiate(&M.gloop[pi][ki], lg, 0));
  cudaGraphDestroy(lg);
  return AMGDD_OK;
}

// Solves `ncols` <= K columns of b (column-major, leading dimension n) as one
// batch of K; the padding columns are zero and finish at once.
static int solve_group(amgdd_hierarchy& h, const double* b, bool bdev, int ncols, int K, double tol, double* x,
                       bool xdev, cudaStream_t s, amgdd_info* info) {
  auto& M = h.mw;
  const int64_t n = h.n;
  AMGDD_TRY(ensure_multi(h, K));
  cudaEvent_t e0, e1;
  AMGDD_CUDA(cudaEventCreate(&e0));
  AMGDD_CUDA(cudaEventCreate(&e1));
  AMGDD_CUDA(cudaEventRecord(e0, s));
  AMGDD_CUDA(cudaMemcpyAsync(M.stage.p, b, n * ncols * sizeof(double),
                             bdev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  AMGDD_TRY(launch_interleave(M.stage.p, n, ncols, M.b.p, n, K, s));
  for (int k = 0; k < K; ++k) {
    PcgState init{};
    init.tol2 = tol * tol;
    init.max_iter = h.prm.max_iter;
    init.flexible = mixed(h) ? 1 : 0;
    M.st_host[k] = init;
  }
  AMGDD_CUDA(cudaMemcpyAsync(M.st.p, M.st_host, K * sizeof(PcgState), cudaMemcpyHostToDevice, s));
  AMGDD_CUDA(cudaMemsetAsync(M.grp.p, 0, sizeof(int), s));
  const int pi = mixed(h) ? 1 : 0, ki = kidx(K);
  if (M.gloop[pi][ki] == nullptr) AMGDD_TRY(build_multi_graphs(h, pi, K, s));
  AMGDD_CUDA(cudaGraphLaunch(M.ginit[pi][ki], s));
  count_graph_launch(M.ginit_kernels[pi][ki]);
  AMGDD_CUDA(cudaGraphLaunch(M.gloop[pi][ki], s));
  AMGDD_CUDA(cudaMemcpyAsync(M.st_host, M.st.p, K * sizeof(PcgState), cudaMemcpyDeviceToHost, s));
  // true residuals b - A x in FP64; columns whose recursively updated
  // residual met the tolerance but whose true residual did not restart from
  // their iterate with r = b - A x (at most twice); the others stay frozen
  Level& L0 = *h.lv[0];
  std::vector<double> part;
  for (int restarts = 0;; ++restarts) {
    if (L0.use_ell)
      AMGDD_TRY(launch_ell_multi(L0, false, M.x.p, M.q.p, M.b.p, K, nullptr, s));
    else
      AMGDD_TRY(launch_seg_multi(L0.ras, L0.Aw64.p, L0.AwT64.p ? L0.AwT64.p : L0.Aw64.p, false, M.x.p, M.q.p, SEG_RESID, M.b.p, K, nullptr,
                                 s));
    AMGDD_TRY(launch_dot_multi(M.q.p, M.q.p, nullptr, n, K, M.partials.p, nullptr, s));
    AMGDD_TRY(download(part, M.partials.p, (size_t)kDotBlocks * 2 * K, s));
    bool any = false;
    for (int k = 0; k < ncols; ++k) {
      PcgState& f = M.st_host[k];
      double qq = 0.0;
      for (int i = 0; i < kDotBlocks; ++i) qq += part[(size_t)i * 2 * K + k];
      if (restarts < 2 && f.status == AMGDD_OK && qq > f.tol2 && f.iters < f.max_iter) {
        f.done = 0;
        f.rr_mark = f.bnorm2;
        any = true;
      }
    }
    if (!any) break;
    AMGDD_CUDA(cudaMemcpyAsync(M.st.p, M.st_host, K * sizeof(PcgState), cudaMemcpyHostToDevice, s));
    AMGDD_CUDA(cudaMemsetAsync(M.grp.p, 0, sizeof(int), s));
    const int64_t nk = n * K;
    AMGDD_CUDA(cudaMemcpyAsync(M.r.p, M.q.p, nk * sizeof(double), cudaMemcpyDeviceToDevice, s));
    AMGDD_TRY(precondition_multi(h, K, M.r.p, M.z.p, M.grp.p, s));
    AMGDD_TRY(launch_copy_vec(M.z.p, M.p.p, false, nk, M.grp.p, s));
    if (mixed(h)) AMGDD_TRY(launch_copy_vec(M.z.p, M.zold.p, false, nk, M.grp.p, s));
    AMGDD_TRY(launch_dot_multi(M.r.p, M.z.p, nullptr, n, K, M.partials.p, M.grp.p, s));
    AMGDD_TRY(launch_pcg_scalar_multi(0, M.st.p, M.grp.p, M.partials.p, K, s));
    AMGDD_CUDA(cudaGraphLaunch(M.gloop[pi][ki], s));
    AMGDD_CUDA(cudaMemcpyAsync(M.st_host, M.st.p, K * sizeof(PcgState), cudaMemcpyDeviceToHost, s));
  }
  AMGDD_TRY(launch_deinterleave(M.x.p, n, K, M.stage.p, n, ncols, s));
  AMGDD_CUDA(cudaMemcpyAsync(x, M.stage.p, n * ncols * sizeof(double),
                             xdev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
  AMGDD_CUDA(cudaEventRecord(e1, s));
  AMGDD_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  AMGDD_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  int maxit = 0;
  for (int k = 0; k < K; ++k) maxit = std::max(maxit, M.st_host[k].iters);
  count_graph_launch(M.gloop_kernels[pi][ki] * std::max(maxit, 1));
  int first_bad = AMGDD_OK;
  std::vector<int> stalled;
  for (int k = 0; k < ncols; ++k) {
    const PcgState& f = M.st_host[k];
    if (f.vc_err != 0) {
      set_error("a bounded device-side wait expired");
      return AMGDD_ERR_TIMEOUT;
    }
    if (f.status == kStallStatus) stalled.push_back(k);
    double qq = 0.0;
    for (int i = 0; i < kDotBlocks; ++i) qq += part[(size_t)i * 2 * K + k];
    if (info) {
      info[k].iters = f.iters;
      info[k].status = f.status;
      info[k].relres = f.relres;
      info[k].relres_true = f.bnorm2 > 0 ? std::sqrt(qq / f.bnorm2) : 0.0;
      info[k].solve_ms = ms;
      info[k].fallback = 0;
      info[k].iters_mixed = 0;
    }
    if (f.status != AMGDD_OK && f.status != kStallStatus && first_bad == AMGDD_OK) first_bad = f.status;
  }
  // columns whose FP32 cycle stalled: redone one at a time with the FP64 cycle
  if (!stalled.empty()) h.mixed_stalled = true;
  for (int k : stalled) {
    const int mixed_iters = M.st_host[k].iters;
    const int prec = h.precision;
    h.precision = AMGDD_FP64;
    amgdd_info one{};
    const int st = solve_once(h, b + (int64_t)k * n, bdev, tol, x + (int64_t)k * n, xdev, s, &one);
    h.precision = prec;
    one.fallback = 1;
    one.iters_mixed = mixed_iters;
    one.iters += mixed_iters;
    one.solve_ms += ms;
    if (info) info[k] = one;
    const bool per_rhs = st == AMGDD_OK || st == AMGDD_ERR_BREAKDOWN || st == AMGDD_ERR_NO_CONVERGENCE ||
                         st == AMGDD_ERR_NONFINITE;
    if (!per_rhs) return st;
    if (st != AMGDD_OK && first_bad == AMGDD_OK) first_bad = st;
  }
  return first_bad;
}

// Binary helpers of the saved-hierarchy format.
namespace {
// v1: setup inputs, parameters and kernel choices; v2 adds the level
// snapshots (what setup computed), so loading skips the local problems.
constexpr char kSaveMagicV1[8] = {'A', 'M', 'G', 'D', 'D', 'H', 'v', '1'};
constexpr char kSaveMagic[8] = {'A', 'M', 'G', 'D', 'D', 'H', 'v', '2'};

template <class T>
bool put_vec(FILE* f, const std::vector<T>& v) {
  const uint64_t c = v.size();
  return std::fwrite(&c, sizeof c, 1, f) == 1 && (c == 0 || std::fwrite(v.data(), sizeof(T), c, f) == c);
}
template <class T>
bool get_vec(FILE* f, std::vector<T>& v, uint64_t max_count) {
  uint64_t c = 0;
  if (std::fread(&c, sizeof c, 1, f) != 1 || c > max_count) return false;
  v.resize(c);
  return c == 0 || std::fread(v.data(), sizeof(T), c, f) == c;
}

struct SnapScalars {
  int64_t n, nnzA;
  int32_t nagg, coarsest, schur_rows, n_color, n_mult, pad;
  double thresh, inv_err;
};

bool put_snap(FILE* f, const LevelSnap& S) {
  const SnapScalars c{S.n, S.nnzA, S.nagg, S.coarsest, S.schur_rows, S.n_color, S.n_mult, 0, S.thresh, S.inv_err};
  return std::fwrite(&c, sizeof c, 1, f) == 1 && put_vec(f, S.g_ptr) && put_vec(f, S.h_off) &&
         put_vec(f, S.om_ptr) && put_vec(f, S.z_off) && put_vec(f, S.mu_off) && put_vec(f, S.col0) &&
         put_vec(f, S.wf_off) && put_vec(f, S.g_idx) && put_vec(f, S.g_rank) && put_vec(f, S.agg) &&
         put_vec(f, S.om_idx) && put_vec(f, S.nomega) && put_vec(f, S.k) && put_vec(f, S.R64) && put_vec(f, S.W64) &&
         put_vec(f, S.Aw64) && put_vec(f, S.mu) && put_vec(f, S.Z64) && put_vec(f, S.Wf64) && put_vec(f, S.A64);
}

bool get_snap(FILE* f, LevelSnap& S, uint64_t mx) {
  SnapScalars c{};
  if (std::fread(&c, sizeof c, 1, f) != 1) return false;
  S.n = c.n;
  S.nnzA = c.nnzA;
  S.nagg = c.nagg;
  S.coarsest = c.coarsest;
  S.schur_rows = c.schur_rows;
  S.n_color = c.n_color;
  S.n_mult = c.n_mult;
  S.thresh = c.thresh;
  S.inv_err = c.inv_err;
  return get_vec(f, S.g_ptr, mx) && get_vec(f, S.h_off, mx) && get_vec(f, S.om_ptr, mx) && get_vec(f, S.z_off, mx) &&
         get_vec(f, S.mu_off, mx) && get_vec(f, S.col0, mx) && get_vec(f, S.wf_off, mx) && get_vec(f, S.g_idx, mx) &&
         get_vec(f, S.g_rank, mx) && get_vec(f, S.agg, mx) && get_vec(f, S.om_idx, mx) && get_vec(f, S.nomega, mx) &&
         get_vec(f, S.k, mx) && get_vec(f, S.R64, mx) && get_vec(f, S.W64, mx) && get_vec(f, S.Aw64, mx) &&
         get_vec(f, S.mu, mx) && get_vec(f, S.Z64, mx) && get_vec(f, S.Wf64, mx) && get_vec(f, S.A64, mx);
}

// Every size and index of the snapshots consistent (they drive the device
// index lists of the loaded hierarchy): level sizes chain through the
// coarse column counts, supports and Omega lists stay inside their level,
// offsets are the prefix sums of the block sizes, and each stored matrix has
// its blocks' size.
bool snaps_valid(const std::vector<LevelSnap>& v, int64_t n0) {
  if (v.empty()) return false;
  for (size_t l = 0; l < v.size(); ++l) {
    const LevelSnap& S = v[l];
    const int64_t n = S.n;
    if (n != (l == 0 ? n0 : v[l - 1].col0.empty() ? -1 : v[l - 1].col0.back()) || n <= 0) return false;
    if (S.coarsest != (l + 1 == v.size() ? 1 : 0)) return false;
    const int64_t ng = (int64_t)S.g_ptr.size() - 1;
    if (ng < 0 || S.g_ptr[0] != 0 || S.h_off.size() != S.g_ptr.size() || S.h_off[0] != 0) return false;
    for (int64_t g = 0; g < ng; ++g) {
      const int64_t len = S.g_ptr[g + 1] - S.g_ptr[g];
      if (len < 0 || S.h_off[g + 1] - S.h_off[g] != len * len) return false;
    }
    if (S.g_ptr.back() != (int64_t)S.g_idx.size()) return false;
    for (int32_t c : S.g_idx)
      if (c < 0 || c >= n) return false;
    if (!S.R64.empty()) {
      if ((int64_t)S.R64.size() != S.h_off.back() || (int64_t)S.g_rank.size() != ng) return false;
      for (int64_t g = 0; g < ng; ++g)
        if (S.g_rank[g] < 0 || S.g_rank[g] > S.g_ptr[g + 1] - S.g_ptr[g]) return false;
    } else if (!S.coarsest || l == 0) {
      return false;  // every level that applies its G keeps the rows
    }
    if (S.coarsest) {
      if ((int64_t)S.W64.size() != n * n || !(S.Aw64.empty() || (int64_t)S.Aw64.size() == n * n)) return false;
      continue;
    }
    const int64_t na = S.nagg;
    if (na < 1 || (int64_t)S.agg.size() != n || (int64_t)S.om_ptr.size() != na + 1 ||
        (int64_t)S.nomega.size() != na || (int64_t)S.k.size() != na || (int64_t)S.col0.size() != na + 1 ||
        (int64_t)S.z_off.size() != na + 1 || (int64_t)S.mu_off.size() != na + 1)
      return false;
    for (int32_t a : S.agg)
      if (a < 0 || a >= na) return false;
    if (S.om_ptr[0] != 0 || S.om_ptr.back() != (int64_t)S.om_idx.size()) return false;
    for (int32_t c : S.om_idx)
      if (c < 0 || c >= n) return false;
    int64_t w = 0, wf = 0;
    if (S.col0[0] != 0 || S.z_off[0] != 0 || S.mu_off[0] != 0) return false;
    for (int64_t i = 0; i < na; ++i) {
      const int64_t m = S.om_ptr[i + 1] - S.om_ptr[i], no = S.nomega[i], k = S.k[i];
      if (m < 1 || no < 1 || no > m || k < 0 || k > no) return false;
      if (S.col0[i + 1] != S.col0[i] + k || S.z_off[i + 1] != S.z_off[i] + no * k ||
          S.mu_off[i + 1] != S.mu_off[i] + no)
        return false;
      w += no * m;
      wf += m * m;
    }
    if ((int64_t)S.W64.size() != w || !(S.Aw64.empty() || (int64_t)S.Aw64.size() == w) ||
        (int64_t)S.mu.size() != S.mu_off.back() || (int64_t)S.Z64.size() != S.z_off.back())
      return false;
    if (!S.Wf64.empty()) {
      if ((int64_t)S.wf_off.size() != na + 1 || S.wf_off[0] != 0 || (int64_t)S.Wf64.size() != wf) return false;
      for (int64_t i = 0; i < na; ++i) {
        const int64_t m = S.om_ptr[i + 1] - S.om_ptr[i];
        if (S.wf_off[i + 1] != S.wf_off[i] + m * m) return false;
      }
    }
  }
  return true;
}
}  // namespace

extern "C" {

amgdd_params amgdd_params_default(void) {
  amgdd_params p;
  std::memset(&p, 0, sizeof(p));
  p.L_max = 10;
  p.n_coarse = 2000;
  p.thresh = 0.1;
  p.c_min[0] = 2;
  p.c_min[1] = 3;
  p.c_min[2] = 4;
  p.n_cmin = 3;
  p.precision = AMGDD_FP64;
  p.max_iter = 1000;
  p.schur_rtol = 1e-12;
  p.use_graph = 1;
  p.check_every = 4;
  p.tune = 1;
  p.tune_cache = nullptr;
  p.coarse_overlap = 0;
  p.coarse_refine = 1;
  p.pdl = 0;
  p.agg_passes = 1;
  p.batch_cols = 8;
  return p;
}

const char* amgdd_status_string(int st) {
  switch (st) {
    case AMGDD_OK: return "ok";
    case AMGDD_ERR_INVALID_ARG: return "invalid argument";
    case AMGDD_ERR_NOT_SPD: return "matrix not SPD";
    case AMGDD_ERR_NONFINITE: return "non-finite value";
    case AMGDD_ERR_BREAKDOWN: return "CG breakdown";
    case AMGDD_ERR_NO_CONVERGENCE: return "no convergence";
    case AMGDD_ERR_OOM: return "out of device memory";
    case AMGDD_ERR_CUDA: return "CUDA error";
    case AMGDD_ERR_INTERNAL: return "internal error";
    default: return "unknown status";
  }
}

const char* amgdd_last_error(void) { return g_last_error.c_str(); }

size_t amgdd_struct_size(int which) {
  switch (which) {
    case 0: return sizeof(amgdd_params);
    case 1: return sizeof(amgdd_info);
    case 2: return sizeof(amgdd_level_desc);
    case 3: return sizeof(amgdd_csr);
    case 4: return sizeof(amgdd_server_params);
    default: return 0;
  }
}

// CSR pattern rules shared by setup and aggregation: rowptr[0] = 0,
// rowptr[m] = nnz, nondecreasing, column ids strictly increasing in [0, n).
static int check_pattern(const char* who, const std::vector<int64_t>& rowptr, const std::vector<int32_t>& col,
                         int64_t m, int64_t n, int64_t nnz) {
  if (rowptr[0] != 0 || rowptr[m] != nnz) {
    set_error("%s: rowptr[0] must be 0 and rowptr[m] = nnz", who);
    return AMGDD_ERR_INVALID_ARG;
  }
  for (int64_t r = 0; r < m; ++r) {
    if (rowptr[r + 1] < rowptr[r]) {
      set_error("%s: rowptr decreases at row %lld", who, (long long)r);
      return AMGDD_ERR_INVALID_ARG;
    }
    for (int64_t e = rowptr[r]; e < rowptr[r + 1]; ++e) {
      if (col[e] < 0 || col[e] >= n || (e > rowptr[r] && col[e] <= col[e - 1])) {
        set_error("%s: row %lld: column ids must increase strictly within [0, n)", who, (long long)r);
        return AMGDD_ERR_INVALID_ARG;
      }
    }
  }
  return AMGDD_OK;
}

static bool bad_header(const amgdd_csr* G) {
  return G->m < 0 || G->n < 1 || G->nnz < 0 || G->n >= (int64_t)1 << 31 || G->rowptr == nullptr ||
         (G->nnz > 0 && (G->col == nullptr || G->val == nullptr));
}

// Level-0 aggregates by `passes` passes of standard aggregation on the graph
// of A (rows of G as hyperedges; consecutive rows with one support counted once).
// Level-0 aggregates of the graph of A = G^T G (rows of G as hyperedges,
// consecutive rows with one support merged) by `passes` passes of standard
// aggregation on the device; d_agg (n, device) receives the ids.
static int aggregate_rows(const std::vector<int64_t>& rowptr, const std::vector<int32_t>& col, int64_t m, int64_t n,
                          int passes, int32_t* d_agg, int64_t& nagg, cudaStream_t s, int64_t* rounds = nullptr) {
  Supports S;
  S.ptr.assign(1, 0);
  S.idx.reserve(col.size());
  int64_t last = -1;
  for (int64_t r = 0; r < m; ++r) {
    const int64_t a = rowptr[r], b = rowptr[r + 1];
    if (b == a) continue;
    if (last >= 0 && rowptr[last + 1] - rowptr[last] == b - a &&
        std::equal(col.begin() + a, col.begin() + b, col.begin() + rowptr[last]))
      continue;
    S.idx.insert(S.idx.end(), col.begin() + a, col.begin() + b);
    S.ptr.push_back((int64_t)S.idx.size());
    last = r;
  }
  DBuf<int64_t> eptr;
  DBuf<int32_t> eidx;
  AMGDD_TRY(eptr.upload(S.ptr, s));
  AMGDD_TRY(eidx.upload(S.idx, s));
  return device_standard_aggregation(n, S.size(), eptr.p, eidx.p, passes, d_agg, &nagg, s, rounds);
}

static int setup_impl(const amgdd_csr* G, const double* D1, const int32_t* agg, int overlap,
                      const amgdd_params* params, void* stream, amgdd_hierarchy** out,
                      const std::vector<std::pair<std::string, double>>* preset = nullptr,
                      const std::vector<LevelSnap>* snap = nullptr) {
  if (out == nullptr || G == nullptr) {
    set_error("amgdd_setup: G and out must not be NULL");
    return AMGDD_ERR_INVALID_ARG;
  }
  *out = nullptr;
  amgdd_params prm = params ? *params : amgdd_params_default();
  if (prm.L_max < 1 || prm.n_cmin < 1 || prm.n_cmin > 8 || prm.max_iter < 1 || overlap < 1 ||
      (prm.precision != AMGDD_FP64 && prm.precision != AMGDD_MIXED32 && prm.precision != AMGDD_MIXED16) ||
      prm.schur_gram < 0 || prm.schur_gram > 2 ||
      (prm.batch_cols != 2 && prm.batch_cols != 4 && prm.batch_cols != 8 && prm.batch_cols != 16 &&
       prm.batch_cols != 32) ||
      prm.check_every < 1 || prm.n_coarse < 1 ||
      prm.coarse_overlap < 0 || prm.cycle < 0 || prm.cycle > 1 || !(prm.kappa >= 0) ||
      (agg == nullptr && prm.agg_passes < 1) ||
      (prm.cycle == 1 && prm.precision != AMGDD_FP64)) {
    set_error("amgdd_setup: invalid parameters");
    return AMGDD_ERR_INVALID_ARG;
  }
  for (int i = 0; i < prm.n_cmin; ++i)
    if (prm.c_min[i] < 1) {
      set_error("amgdd_setup: c_min entries must be >= 1");
      return AMGDD_ERR_INVALID_ARG;
    }
  const int64_t m = G->m, n = G->n, nnz = G->nnz;
  if (bad_header(G)) {
    set_error("amgdd_setup: bad CSR header (m=%lld n=%lld nnz=%lld)", (long long)m, (long long)n, (long long)nnz);
    return AMGDD_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const auto t0 = std::chrono::steady_clock::now();
  g_timer = PhaseTimer();
  g_timer.on = std::getenv("AMGDD_VERBOSE") != nullptr;  // print per-level phase times
  const bool gdev = G->mem == AMGDD_DEVICE;
  std::vector<int64_t> rowptr;
  std::vector<int32_t> col;
  std::vector<double> val, d1;
  std::vector<int32_t> aggh;
  AMGDD_TRY(fetch_any(rowptr, G->rowptr, (size_t)m + 1, gdev, s));
  AMGDD_TRY(fetch_any(col, G->col, (size_t)nnz, gdev, s));
  AMGDD_TRY(fetch_any(val, G->val, (size_t)nnz, gdev, s));
  if (agg) AMGDD_TRY(fetch_any(aggh, agg, (size_t)n, is_device_ptr(agg), s));
  if (D1) AMGDD_TRY(fetch_any(d1, D1, (size_t)n, is_device_ptr(D1), s));
  AMGDD_TRY(check_pattern("amgdd_setup", rowptr, col, m, n, nnz));
  if (!agg) {  // level-0 aggregates from the graph of A (Section 3.3), on the device
    int64_t na = 0;
    DBuf<int32_t> dagg;
    AMGDD_TRY(dagg.alloc(std::max<int64_t>(n, 1)));
    AMGDD_TRY(aggregate_rows(rowptr, col, m, n, prm.agg_passes, dagg.p, na, s));
    AMGDD_TRY(download(aggh, dagg.p, (size_t)n, s));
  }
  for (double v : val)
    if (!std::isfinite(v)) {
      set_error("amgdd_setup: non-finite value in G");
      return AMGDD_ERR_NONFINITE;
    }
  for (double v : d1)
    if (!std::isfinite(v) || v < 0) {
      set_error("amgdd_setup: D1 must be finite and >= 0");
      return AMGDD_ERR_NONFINITE;
    }
  const int64_t bytes0 = g_alloc_bytes;
  std::unique_ptr<amgdd_hierarchy> H(new amgdd_hierarchy());
  H->prm = prm;
  H->prm.tune_cache = nullptr;  // the caller's string is not kept
  H->overlap = overlap;
  H->n = n;
  H->in_rowptr = rowptr;
  H->in_col = col;
  H->in_val = val;
  H->in_agg = aggh;
  H->in_d1 = d1;
  H->in_has_d1 = D1 != nullptr;
  H->precision = prm.precision;
  AMGDD_CUDA(cudaGetDevice(&H->device));
  AMGDD_TRY(H->st.alloc(1));
  AMGDD_TRY(H->st.zero(s));
  ErrScope err_scope(&H->st.p->vc_err);
  PdlScope pdl_scope(prm.pdl != 0);
  TuneCtx tctx;
  tctx.on = prm.tune == 1;
  tctx.prefer_form = prm.tune == 2 ? 1 : (prm.tune == 3 ? 2 : (prm.tune == 4 ? 0 : -1));
  tctx.path = prm.tune_cache ? prm.tune_cache : "";
  {
    cudaDeviceProp prop;
    AMGDD_CUDA(cudaGetDeviceProperties(&prop, H->device));
    // "f8": plan choices code form, rows per CTA and lanes per row; tails timed as graphs
    std::string sig = std::string(prop.name) + "/" + std::to_string(prop.multiProcessorCount) + "|f8|m" +
                      std::to_string(m) + "|n" + std::to_string(n) + "|nnz" + std::to_string(nnz) + "|ov" +
                      std::to_string(overlap) + "/" + std::to_string(prm.coarse_overlap) + "|cr" + std::to_string(prm.coarse_refine) + "|nc" + std::to_string(prm.n_coarse) + "|L" +
                      std::to_string(prm.L_max) + "|c";
    for (int i = 0; i < prm.n_cmin; ++i) sig += std::to_string(prm.c_min[i]) + ",";
    char buf[64];
    std::snprintf(buf, sizeof buf, "|t%.6g|k%.6g|d1%d", prm.thresh, prm.kappa, D1 ? 1 : 0);
    tctx.sig = sig + buf;
  }
  tctx.load();
  if (preset)  // choices saved with a hierarchy: replayed, not re-timed (tune = 0 keeps its fixed defaults)
    for (const auto& kv : *preset) tctx.kv[kv.first] = kv.second;
  struct TuneScope {
    explicit TuneScope(TuneCtx* t) { g_tune = t; }
    ~TuneScope() { g_tune = nullptr; }
  } tune_scope(&tctx);
  FlushScope flush_scope;  // cold-L2 timing of the kernel forms
  // ---- level 0 row groups: consecutive rows with identical supports ----
  std::unique_ptr<Level> L0(new Level());
  L0->n = n;
  std::vector<int64_t> g_row0, g_row1;
  L0->g_ptr.assign(1, 0);
  int64_t prev = -1;
  for (int64_t r = 0; r < m; ++r) {
    const int64_t len = rowptr[r + 1] - rowptr[r];
    if (len == 0) continue;
    bool same = prev >= 0 && (rowptr[prev + 1] - rowptr[prev]) == len &&
                std::equal(col.begin() + rowptr[r], col.begin() + rowptr[r + 1], col.begin() + rowptr[prev]);
    if (same && g_row1.back() == r) {
      g_row1.back() = r + 1;
    } else {
      g_row0.push_back(r);
      g_row1.push_back(r + 1);
      L0->g_idx.insert(L0->g_idx.end(), col.begin() + rowptr[r], col.begin() + rowptr[r + 1]);
      L0->g_ptr.push_back((int64_t)L0->g_idx.size());
    }
    prev = r;
  }
  const int64_t ncsr = (int64_t)g_row0.size();
  std::vector<double> d1vals;
  for (int64_t j = 0; j < (int64_t)d1.size(); ++j)
    if (d1[j] != 0.0) {
      d1vals.push_back(d1[j]);
      L0->g_idx.push_back((int32_t)j);
      L0->g_ptr.push_back((int64_t)L0->g_idx.size());
    }
  const int64_t ng0 = (int64_t)L0->g_ptr.size() - 1;
  L0->h_off.assign(ng0 + 1, 0);
  for (int64_t g = 0; g < ng0; ++g) {
    const int64_t sz = L0->g_ptr[g + 1] - L0->g_ptr[g];
    L0->h_off[g + 1] = L0->h_off[g] + sz * sz;
  }
  AMGDD_TRY(L0->d_g_ptr.upload(L0->g_ptr, s));
  AMGDD_TRY(L0->d_g_idx.upload(L0->g_idx, s));
  AMGDD_TRY(L0->d_h_off.upload(L0->h_off, s));
  if (snap && ((*snap)[0].g_ptr != L0->g_ptr || (*snap)[0].g_idx != L0->g_idx)) {
    set_error("saved hierarchy: level-0 row groups differ from those of the saved G");
    return AMGDD_ERR_INVALID_ARG;
  }
  if (!snap) {  // the Grams of level 0 (a loaded hierarchy has its rows already)
    AMGDD_TRY(L0->d_H.alloc(std::max<int64_t>(L0->h_off[ng0], 1)));
    DBuf<int64_t> d_rowptr, d_r0, d_r1;
    DBuf<double> d_val, d_d1;
    AMGDD_TRY(d_rowptr.upload(rowptr, s));
    AMGDD_TRY(d_val.upload(val, s));
    AMGDD_TRY(d_r0.upload(g_row0, s));
    AMGDD_TRY(d_r1.upload(g_row1, s));
    AMGDD_TRY(launch_gram_rows(ncsr, d_r0.p, d_r1.p, L0->d_g_ptr.p, L0->d_h_off.p, d_rowptr.p, d_val.p, L0->d_H.p, s));
    if (!d1vals.empty()) {
      AMGDD_TRY(d_d1.upload(d1vals, s));
      AMGDD_TRY(launch_gram_diag((int64_t)d1vals.size(), ncsr, L0->d_h_off.p, d_d1.p, L0->d_H.p, s));
    }
    AMGDD_CUDA(cudaStreamSynchronize(s));
  }
  // iota (shared identity index array)
  {
    std::vector<int32_t> io(n);
    std::iota(io.begin(), io.end(), 0);
    AMGDD_TRY(H->iota.upload(io, s));
  }
  H->lv.push_back(std::move(L0));
  // ---- Algorithm 1 -----------------------------------------------------
  int lvl = 0;
  for (;;) {
    Level& L = *H->lv[lvl];
    const bool coarsest = !(lvl < prm.L_max - 1 && L.n > prm.n_coarse);
    if (snap) {
      if (lvl >= (int)snap->size() || ((*snap)[lvl].coarsest != 0) != coarsest) {
        set_error("saved hierarchy: level %d does not match the saved parameters", lvl);
        return AMGDD_ERR_INVALID_ARG;
      }
      AMGDD_TRY(restore_rows(L, (*snap)[lvl], s));
    }
    if (!coarsest || lvl == 0) {
      Phase ph(6, "compress", s);
      AMGDD_TRY(compress(L, s));
    }
    AMGDD_TRY(alloc_vectors(L));
    if (coarsest) {
      Phase ph(8, "coarsest", s);
      AMGDD_TRY(snap ? restore_coarsest(*H, L, (*snap)[lvl], s) : build_coarsest(*H, L, s));
      AMGDD_TRY(tune_level_plans(L, lvl, 0, s));
      break;
    }
    AMGDD_TRY(snap ? restore_level(*H, L, (*snap)[lvl], s)
                   : build_level(*H, L, lvl, lvl == 0 ? aggh.data() : nullptr, s));
    if (L.col0.back() == 0) {  // no local eigenvector passed the threshold anywhere on this level
      set_error("level %d produced an empty coarse space", lvl);
      return AMGDD_ERR_INVALID_ARG;
    }
    AMGDD_TRY(build_plans(*H, L, L.d_om_idx, s));
    if (lvl > 0) {
      Phase ph(9, "block rows", s);
      AMGDD_TRY(build_blockrows(L, s, snap ? &(*snap)[lvl].A64 : nullptr));
    }
    {
      Phase ph(10, "tune", s);
      AMGDD_TRY(tune_level_plans(L, lvl, L.col0.back(), s));
      if (lvl > 0 && !prm.deterministic) AMGDD_TRY(tune_level_A(L, lvl, s));  // deterministic: block rows
      const int ell_mode = prm.deterministic ? 1 : prm.ell;  // the row groups scatter with atomics
      if (lvl == 0 && ell_mode >= 0) {
        AMGDD_TRY(build_ell(L, s));
        AMGDD_TRY(tune_ell(L, ell_mode, s));
      }
      if (L.has_blk) {  // the batched residual uses the block rows
        L.Aw64.release();
        L.AwT64.release();
        L.Aw32.release();
        L.AwT32.release();
      }
    }
    std::unique_ptr<Level> N(new Level());
    {
      Phase ph(7, "next level", s);
      AMGDD_TRY(snap ? restore_next(*N, (*snap)[lvl + 1], s) : build_next(*H, L, *N, s));
    }
    for (int i = 0; i < 16; ++i) {
      H->phase_ms[i] += g_timer.acc[i];
      H->phase_flops[i] += g_timer.flops[i];
      if (g_timer.name[i]) H->phase_name[i] = g_timer.name[i];
    }
    if (g_timer.on) {
      fprintf(stderr, "[amgdd] level %d: n=%lld nagg=%d", lvl, (long long)L.n, L.nagg);
      for (int i = 0; i < 16; ++i)
        if (g_timer.name[i]) fprintf(stderr, " %s=%.1fms", g_timer.name[i], g_timer.acc[i]);
      fprintf(stderr, "\n");
    }
    for (double& a : g_timer.acc) a = 0.0;
    for (double& a : g_timer.flops) a = 0.0;
    L.d_H.release();

    H->lv.push_back(std::move(N));
    ++lvl;
  }
  H->lv.back()->d_H.release();
  if (prm.cycle == 1 && H->lv.size() != 2) {
    set_error("amgdd_setup: the additive two-level method needs exactly two levels (got %zu; raise n_coarse or set "
              "L_max = 2)", H->lv.size());
    return AMGDD_ERR_INVALID_ARG;
  }
  for (int i = 0; i < 16; ++i) {  // the coarsest level's phases
    H->phase_ms[i] += g_timer.acc[i];
    H->phase_flops[i] += g_timer.flops[i];
    if (g_timer.name[i]) H->phase_name[i] = g_timer.name[i];
  }
  // ---- solver workspace --------------------------------------------------
  AMGDD_TRY(H->x.alloc(n));
  AMGDD_TRY(H->r.alloc(n));
  AMGDD_TRY(H->z.alloc(n));
  AMGDD_TRY(H->zold.alloc(n));
  AMGDD_TRY(H->p.alloc(n));
  AMGDD_TRY(H->q.alloc(n));
  AMGDD_TRY(H->b.alloc(n));
  AMGDD_TRY(H->partials.alloc(2 * kDotBlocks));
  AMGDD_CUDA(cudaMallocHost((void**)&H->st_host, sizeof(PcgState)));
  AMGDD_CUDA(cudaStreamCreateWithFlags(&H->work, cudaStreamNonBlocking));
  AMGDD_CUDA(cudaEventCreateWithFlags(&H->join[0], cudaEventDisableTiming));
  AMGDD_CUDA(cudaEventCreateWithFlags(&H->join[1], cudaEventDisableTiming));
  AMGDD_CUDA(cudaStreamSynchronize(s));
  if (H->precision == AMGDD_MIXED16) AMGDD_TRY(build_half(*H));
  AMGDD_TRY(tune_dense(*H));
  AMGDD_TRY(tune_tail(*H));
  tctx.save();
  for (const auto& kv : tctx.kv)
    if (kv.first.compare(0, tctx.sig.size(), tctx.sig) == 0) H->tune_kv.emplace_back(kv.first, kv.second);
  flush_scope.f.buf.release();
  H->setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  H->setup_bytes = g_alloc_bytes - bytes0;
  *out = H.release();
  return AMGDD_OK;
}

int amgdd_setup(const amgdd_csr* G, const double* D1, const int32_t* agg, int overlap, const amgdd_params* params,
                void* stream, amgdd_hierarchy** out) {
  try {
    return setup_impl(G, D1, agg, overlap, params, stream, out);
  } catch (const std::bad_alloc&) {
    set_error("amgdd_setup: host allocation failed");
    return AMGDD_ERR_OOM;
  } catch (...) {
    set_error("amgdd_setup: unexpected exception");
    return AMGDD_ERR_INTERNAL;
  }
}

int amgdd_aggregate(const amgdd_csr* G, int passes, void* stream, int32_t* agg, int64_t* nagg) {
  if (G == nullptr || agg == nullptr || passes < 1 || bad_header(G)) {
    set_error("amgdd_aggregate: invalid argument");
    return AMGDD_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const bool gdev = G->mem == AMGDD_DEVICE;
  std::vector<int64_t> rowptr;
  std::vector<int32_t> col;
  AMGDD_TRY(fetch_any(rowptr, G->rowptr, (size_t)G->m + 1, gdev, s));
  AMGDD_TRY(fetch_any(col, G->col, (size_t)G->nnz, gdev, s));
  AMGDD_TRY(check_pattern("amgdd_aggregate", rowptr, col, G->m, G->n, G->nnz));
  int64_t na = 0;
  DBuf<int32_t> dagg;
  AMGDD_TRY(dagg.alloc(std::max<int64_t>(G->n, 1)));
  AMGDD_TRY(aggregate_rows(rowptr, col, G->m, G->n, passes, dagg.p, na, s));
  AMGDD_CUDA(cudaMemcpyAsync(agg, dagg.p, (size_t)G->n * sizeof(int32_t),
                             is_device_ptr(agg) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
  AMGDD_CUDA(cudaStreamSynchronize(s));
  if (nagg) *nagg = na;
  return AMGDD_OK;
}

int amgdd_solve(amgdd_hierarchy* h, const double* b, int nrhs, double tol, double* x, void* stream,
                amgdd_info* info) {
  if (h == nullptr || b == nullptr || x == nullptr || nrhs < 0 || !(tol >= 0.0)) {
    set_error("amgdd_solve: invalid argument");
    return AMGDD_ERR_INVALID_ARG;
  }
  try {
    ErrScope err_scope(&h->st.p->vc_err);
    PdlScope pdl_scope(h->prm.pdl != 0);
    cudaStream_t us = (cudaStream_t)stream;
    cudaStream_t s = h->work;
    AMGDD_CUDA(cudaEventRecord(h->join[0], us));
    AMGDD_CUDA(cudaStreamWaitEvent(s, h->join[0], 0));
    const bool bdev = is_device_ptr(b), xdev = is_device_ptr(x);
    int first_bad = AMGDD_OK;
    if (nrhs > 1 && h->prm.use_graph && h->lv[0]->Aw64.p != nullptr && h->prm.cycle == 0) {
      const int bc = std::min(h->prm.batch_cols, kMaxRhs);
      for (int j0 = 0; j0 < nrhs; j0 += bc) {
        const int g = std::min(bc, nrhs - j0);
        const int K = kclass(g);
        std::vector<amgdd_info> tmp(g);
        amgdd_info* inf = info ? info + j0 : tmp.data();
        const int prec = h->precision;
        const bool sticky = mixed(*h) && h->mixed_stalled;
        if (sticky) h->precision = AMGDD_FP64;  // the FP32 cycle stalled on this hierarchy before
        const int st = solve_group(*h, b + (int64_t)j0 * h->n, bdev, g, K, tol, x + (int64_t)j0 * h->n, xdev, s, inf);
        if (sticky) {
          h->precision = prec;
          for (int k = 0; k < g; ++k) inf[k].fallback = 1;
        }
        const bool per_rhs = st == AMGDD_OK || st == AMGDD_ERR_BREAKDOWN || st == AMGDD_ERR_NO_CONVERGENCE ||
                             st == AMGDD_ERR_NONFINITE;
        if (!per_rhs) return st;
        if (st != AMGDD_OK && first_bad == AMGDD_OK) first_bad = st;
      }
      AMGDD_CUDA(cudaEventRecord(h->join[1], s));
      AMGDD_CUDA(cudaStreamWaitEvent(us, h->join[1], 0));
      return first_bad;
    }
    for (int j = 0; j < nrhs; ++j) {
      amgdd_info tmp{};
      const int st = solve_one(*h, b + (int64_t)j * h->n, bdev, tol, x + (int64_t)j * h->n, xdev, s,
                               info ? info + j : &tmp);
      const bool per_rhs = st == AMGDD_OK || st == AMGDD_ERR_BREAKDOWN || st == AMGDD_ERR_NO_CONVERGENCE ||
                           st == AMGDD_ERR_NONFINITE;
      if (!per_rhs) return st;
      if (st != AMGDD_OK && first_bad == AMGDD_OK) first_bad = st;
    }
    AMGDD_CUDA(cudaEventRecord(h->join[1], s));
    AMGDD_CUDA(cudaStreamWaitEvent(us, h->join[1], 0));
    return first_bad;
  } catch (...) {
    set_error("amgdd_solve: unexpected exception");
    return AMGDD_ERR_INTERNAL;
  }
}

int amgdd_set_precision(amgdd_hierarchy* h, int precision) {
  if (h == nullptr || (precision != AMGDD_FP64 && precision != AMGDD_MIXED32 && precision != AMGDD_MIXED16)) {
    set_error("amgdd_set_precision: invalid argument");
    return AMGDD_ERR_INVALID_ARG;
  }
  if (h->prm.cycle == 1 && precision != AMGDD_FP64) {
    set_error("amgdd_set_precision: the additive two-level method runs in FP64 only");
    return AMGDD_ERR_INVALID_ARG;
  }
  if (precision == AMGDD_MIXED16) AMGDD_TRY(build_half(*h));
  if ((precision == AMGDD_MIXED16) != (h->precision == AMGDD_MIXED16)) {
    // the FP32-vector solve graphs read the other matrix copies: recapture
    for (auto* ge : {&h->ginit[1], &h->gloop[1]})
      if (*ge) {
        cudaGraphExecDestroy(*ge);
        *ge = nullptr;
      }
  }
  h->precision = precision;
  h->mixed_stalled = false;  // give the FP32 cycle a fresh chance
  return AMGDD_OK;
}

int amgdd_set_max_iter(amgdd_hierarchy* h, int max_iter) {
  if (h == nullptr || max_iter < 1) {
    set_error("amgdd_set_max_iter: invalid argument");
    return AMGDD_ERR_INVALID_ARG;
  }
  h->prm.max_iter = max_iter;
  return AMGDD_OK;
}

int amgdd_apply(amgdd_hierarchy* h, int op, int level, const double* x, double* y, void* stream) {
  if (h == nullptr || x == nullptr || y == nullptr || level < 0 || level >= (int)h->lv.size()) {
    set_error("amgdd_apply: invalid argument");
    return AMGDD_ERR_INVALID_ARG;
  }
  ErrScope err_scope(&h->st.p->vc_err);
  PdlScope pdl_scope(h->prm.pdl != 0);
  cudaStream_t s = (cudaStream_t)stream;
  Level& L = *h->lv[level];
  const bool f32 = mixed(*h);
  if (op == AMGDD_OP_M2) {
    if (h->prm.cycle != 1 || level != 0) {
      set_error("amgdd_apply: M2 needs level 0 of a hierarchy built with cycle = 1");
      return AMGDD_ERR_INVALID_ARG;
    }
    AMGDD_TRY(precondition_additive(*h, x, y, nullptr, s));
    return take_err_word(*h, s);
  }
  const bool coarsest_op = op == AMGDD_OP_COARSE || (op == AMGDD_OP_VCYCLE && L.coarsest);
  if (coarsest_op) {
    if (!L.coarsest) {
      set_error("amgdd_apply: COARSE needs the coarsest level");
      return AMGDD_ERR_INVALID_ARG;
    }
    AMGDD_TRY(coarse_solve(*h, L, x, y, L.s64.p, nullptr, s));
    return take_err_word(*h, s);
  }
  if (L.coarsest && op != AMGDD_OP_A) {
    set_error("amgdd_apply: operator not defined on the coarsest level");
    return AMGDD_ERR_INVALID_ARG;
  }
  if (op == AMGDD_OP_A && L.coarsest && level != 0) {
    set_error("amgdd_apply: A is not stored on the coarsest level");
    return AMGDD_ERR_INVALID_ARG;
  }
  const int64_t nin = op == AMGDD_OP_PROLONG ? h->lv[level + 1]->n : L.n;
  const int64_t nout = op == AMGDD_OP_RESTRICT ? h->lv[level + 1]->n : L.n;
  // staging buffers in the working precision
  DBuf<float> xin32, yout32;
  const void* xin = x;
  void* yout = y;
  if (f32) {
    AMGDD_TRY(xin32.alloc(nin));
    AMGDD_TRY(yout32.alloc(nout));
    AMGDD_TRY(launch_cast(x, false, xin32.p, true, nin, nullptr, s));
    xin = xin32.p;
    yout = yout32.p;
  }
  const size_t esz = f32 ? sizeof(float) : sizeof(double);
  const bool h16 = use16(*h, L, f32);
  switch (op) {
    case AMGDD_OP_A:
      AMGDD_TRY(level_apply_A(L, f32, xin, yout, s, h16));
      break;
    case AMGDD_OP_RAS:
      AMGDD_TRY(seg_op(h16, f32, L.ras, L.W64, L.W32, L.Wt64, L.Wt32, xin, yout, SEG_STORE, nullptr, s));
      break;
    case AMGDD_OP_RAST:
      AMGDD_CUDA(cudaMemsetAsync(yout, 0, nout * esz, s));
      AMGDD_TRY(apply_rast(L, f32, xin, yout, nullptr, s, 1, h16));
      break;
    case AMGDD_OP_RESTRICT:
      AMGDD_TRY(
          seg_op(h16, f32, L.restr, L.Zt64, L.Zt32, L.Z64, L.Z32, xin, yout, SEG_STORE, nullptr, s));
      break;
    case AMGDD_OP_PROLONG:
      AMGDD_CUDA(cudaMemsetAsync(yout, 0, nout * esz, s));
      AMGDD_TRY(seg_op(h16, f32, L.prol, L.Z64, L.Z32, L.Zt64, L.Zt32, xin, yout, SEG_ADD, nullptr, s));
      break;
    case AMGDD_OP_VCYCLE:
      AMGDD_TRY(vcycle(*h, level, f32, xin, yout, nullptr, s));
      break;
    default:
      set_error("amgdd_apply: unknown operator %d", op);
      return AMGDD_ERR_INVALID_ARG;
  }
  if (f32) AMGDD_TRY(launch_cast(yout32.p, true, y, false, nout, nullptr, s));
  return take_err_word(*h, s);
}

// ---------------------------------------------------------------------------
// Allocation-free variant of amgdd_apply.  In MIXED32 amgdd_apply stages the
// FP64 caller vectors through two FP32 work vectors that it allocates on
// every call.  Here the staging lives in one file-scope device array, so
// the call never allocates.  The array holds 2 x kNoAllocMaxN floats (1 MiB)
// on every device that loads the library, until the process exits.
constexpr int64_t kNoAllocMaxN = (int64_t)1 << 17;
static __device__ __align__(256) float g_noalloc_stage[2 * kNoAllocMaxN];

namespace {
constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mutex;
float* g_noalloc_ptr[kNoAllocMaxDevices] = {nullptr};

// Device address of the staging array on device `dev`, which must be the
// current device: the hierarchy's kernels run there, and the array of
// another device is another allocation.  Host code may not use the symbol
// itself: it names a host-side stand-in.  The address is looked up once per
// device, with that device current, and kept for the life of the process
// (a cudaDeviceReset would invalidate it, as it invalidates every
// hierarchy built on that device).
int noalloc_stage(int dev, float** out) {
  int cur = 0;
  AMGDD_CUDA(cudaGetDevice(&cur));
  if (cur != dev) {
    set_error("amgdd_apply_noalloc: the current device is %d but the hierarchy lives on device %d; make the "
              "hierarchy's device current",
              cur, dev);
    return AMGDD_ERR_INVALID_ARG;
  }
  if (dev < 0 || dev >= kNoAllocMaxDevices) {
    set_error("amgdd_apply_noalloc: device id %d out of range", dev);
    return AMGDD_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(g_noalloc_mutex);
  if (g_noalloc_ptr[dev] == nullptr) {
    void* p = nullptr;
    AMGDD_CUDA(cudaGetSymbolAddress(&p, g_noalloc_stage));
    g_noalloc_ptr[dev] = static_cast<float*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return AMGDD_OK;
}
}  // namespace

int amgdd_apply_noalloc(amgdd_hierarchy* h, int op, int level, const double* x, double* y, void* stream) {
  if (h == nullptr || x == nullptr || y == nullptr || level < 0 || level >= (int)h->lv.size()) {
    set_error("amgdd_apply_noalloc: invalid argument");
    return AMGDD_ERR_INVALID_ARG;
  }
  {
    int cur = 0;
    AMGDD_CUDA(cudaGetDevice(&cur));
    if (cur != h->device) {
      set_error("amgdd_apply_noalloc: the current device is %d but the hierarchy lives on device %d", cur,
                h->device);
      return AMGDD_ERR_INVALID_ARG;
    }
  }
  ErrScope err_scope(&h->st.p->vc_err);
  PdlScope pdl_scope(h->prm.pdl != 0);
  cudaStream_t s = (cudaStream_t)stream;
  Level& L = *h->lv[level];
  const bool f32 = mixed(*h);
  if (op == AMGDD_OP_M2) {
    if (h->prm.cycle != 1 || level != 0) {
      set_error("amgdd_apply: M2 needs level 0 of a hierarchy built with cycle = 1");
      return AMGDD_ERR_INVALID_ARG;
    }
    AMGDD_TRY(precondition_additive(*h, x, y, nullptr, s));
    return take_err_word(*h, s);
  }
  const bool coarsest_op = op == AMGDD_OP_COARSE || (op == AMGDD_OP_VCYCLE && L.coarsest);
  if (coarsest_op) {
    if (!L.coarsest) {
      set_error("amgdd_apply_noalloc: COARSE needs the coarsest level");
      return AMGDD_ERR_INVALID_ARG;
    }
    AMGDD_TRY(coarse_solve(*h, L, x, y, L.s64.p, nullptr, s));
    return take_err_word(*h, s);
  }
  if (L.coarsest && op != AMGDD_OP_A) {
    set_error("amgdd_apply_noalloc: operator not defined on the coarsest level");
    return AMGDD_ERR_INVALID_ARG;
  }
  if (op == AMGDD_OP_A && L.coarsest && level != 0) {
    set_error("amgdd_apply_noalloc: A is not stored on the coarsest level");
    return AMGDD_ERR_INVALID_ARG;
  }
  if ((op == AMGDD_OP_RESTRICT || op == AMGDD_OP_PROLONG) && level + 1 >= (int)h->lv.size()) {
    set_error("amgdd_apply_noalloc: no coarser level below level %d", level);
    return AMGDD_ERR_INVALID_ARG;
  }
  const int64_t nin = op == AMGDD_OP_PROLONG ? h->lv[level + 1]->n : L.n;
  const int64_t nout = op == AMGDD_OP_RESTRICT ? h->lv[level + 1]->n : L.n;
  const void* xin = x;
  void* yout = y;
  float* stage = nullptr;
  if (f32) {
    if (nin > kNoAllocMaxN || nout > kNoAllocMaxN) {
      set_error("amgdd_apply_noalloc: vectors of %lld and %lld entries exceed the fixed staging size of %lld "
                "entries per vector (MIXED32); use amgdd_apply",
                (long long)nin, (long long)nout, (long long)kNoAllocMaxN);
      return AMGDD_ERR_INVALID_ARG;
    }
    AMGDD_TRY(noalloc_stage(h->device, &stage));
    AMGDD_TRY(launch_cast(x, false, stage, true, nin, nullptr, s));
    xin = stage;
    yout = stage + kNoAllocMaxN;
  }
  const size_t esz = f32 ? sizeof(float) : sizeof(double);
  const bool h16 = use16(*h, L, f32);
  switch (op) {
    case AMGDD_OP_A:
      AMGDD_TRY(level_apply_A(L, f32, xin, yout, s, h16));
      break;
    case AMGDD_OP_RAS:
      AMGDD_TRY(seg_op(h16, f32, L.ras, L.W64, L.W32, L.Wt64, L.Wt32, xin, yout, SEG_STORE, nullptr, s));
      break;
    case AMGDD_OP_RAST:
      AMGDD_CUDA(cudaMemsetAsync(yout, 0, nout * esz, s));
      AMGDD_TRY(apply_rast(L, f32, xin, yout, nullptr, s, 1, h16));
      break;
    case AMGDD_OP_RESTRICT:
      AMGDD_TRY(
          seg_op(h16, f32, L.restr, L.Zt64, L.Zt32, L.Z64, L.Z32, xin, yout, SEG_STORE, nullptr, s));
      break;
    case AMGDD_OP_PROLONG:
      AMGDD_CUDA(cudaMemsetAsync(yout, 0, nout * esz, s));
      AMGDD_TRY(seg_op(h16, f32, L.prol, L.Z64, L.Z32, L.Zt64, L.Zt32, xin, yout, SEG_ADD, nullptr, s));
      break;
    case AMGDD_OP_VCYCLE:
      AMGDD_TRY(vcycle(*h, level, f32, xin, yout, nullptr, s));
      break;
    default:
      set_error("amgdd_apply_noalloc: unknown operator %d", op);
      return AMGDD_ERR_INVALID_ARG;
  }
  if (f32) AMGDD_TRY(launch_cast(yout, true, y, false, nout, nullptr, s));
  return take_err_word(*h, s);
}

int amgdd_profile_vcycle(amgdd_hierarchy* h, int reps, int graph, double* ms, double* bytes, int cap) {
  if (h == nullptr || ms == nullptr || bytes == nullptr || reps < 1 ||
      cap < (int)h->lv.size() * VProf::kSlots) {
    set_error("amgdd_profile_vcycle: invalid argument (cap must be >= levels * %d)", VProf::kSlots);
    return AMGDD_ERR_INVALID_ARG;
  }
  ErrScope err_scope(&h->st.p->vc_err);
  PdlScope pdl_scope(h->prm.pdl != 0);
  const int nl = (int)h->lv.size();
  for (int i = 0; i < std::min(cap, nl * VProf::kSlots + 1); ++i) ms[i] = bytes[i] = 0.0;
  cudaStream_t s = h->work;
  const bool f32 = mixed(*h);
  Level& L0 = *h->lv[0];
  const void* r = f32 ? (const void*)L0.s32.p : (const void*)L0.s64.p;
  void* x = f32 ? (void*)L0.r32.p : (void*)L0.r64.p;
  // a deterministic nonzero input
  AMGDD_TRY(launch_cast(h->iota.p ? (const void*)L0.x64.p : nullptr, false, (void*)r, f32, 0, nullptr, s));
  AMGDD_CUDA(cudaMemsetAsync((void*)r, 0, L0.n * (f32 ? 4 : 8), s));
  VProf prof;
  std::vector<double> acc(nl * VProf::kSlots, 0.0);
  auto collect = [&]() -> int {
    for (size_t i = 0; i + 1 < prof.used; ++i) {
      float t = 0.f;
      AMGDD_CUDA(cudaEventElapsedTime(&t, prof.ev[i], prof.ev[i + 1]));
      if (prof.tag[i] >= 0) acc[prof.tag[i]] += t;
    }
    return AMGDD_OK;
  };
  if (!graph) {
    for (int rep = 0; rep < reps; ++rep) {
      prof.used = 0;
      AMGDD_TRY(vcycle(*h, 0, f32, r, x, nullptr, s, &prof));
      AMGDD_TRY(prof.mark(s, -1, 0));
      AMGDD_CUDA(cudaStreamSynchronize(s));
      AMGDD_TRY(collect());
    }
  } else {
    // the marked cycle as one CUDA graph (event record nodes between its
    // kernels), replayed: the per-step times then hold the in-graph gaps
    // between dependent kernels and no host launch overhead
    prof.used = 0;
    prof.in_graph = true;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    capture_begin();
    AMGDD_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    int rc = vcycle(*h, 0, f32, r, x, nullptr, s, &prof);
    if (rc == AMGDD_OK) rc = prof.mark(s, -1, 0);
    const cudaError_t ce = cudaStreamEndCapture(s, &g);
    const int64_t nk = capture_end();
    if (rc == AMGDD_OK && (ce != cudaSuccess || cudaGraphInstantiate(&ge, g, 0) != cudaSuccess)) {
      set_error("amgdd_profile_vcycle: capture of the marked V-cycle failed");
      rc = AMGDD_ERR_CUDA;
    }
    if (g) cudaGraphDestroy(g);
    for (int rep = 0; rep < reps + 2 && rc == AMGDD_OK; ++rep) {  // two warm-up replays
      if (cudaGraphLaunch(ge, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
        set_error("amgdd_profile_vcycle: graph replay failed");
        rc = AMGDD_ERR_CUDA;
        break;
      }
      count_graph_launch(nk);
      if (rep >= 2) rc = collect();
    }
    if (ge) cudaGraphExecDestroy(ge);
    AMGDD_TRY(rc);
    if (cap > nl * VProf::kSlots) {  // the same cycle without marks
      double us = 0.0;
      AMGDD_TRY(time_vcycle_graph(*h, 0, f32, r, x, &us));
      ms[nl * VProf::kSlots] = us * 1e-3;
    }
  }
  const size_t esz = f32 ? 4 : 8;
  const int df = h->dense_from[f32 ? 1 : 0];
  for (int l = 0; l < nl; ++l) {
    const Level& L = *h->lv[l];
    double* b = bytes + l * VProf::kSlots;
    if (df > 0 && l >= df) {  // the dense tail: one GEMV at level df, nothing below
      if (l == df) b[0] = ((double)L.n * L.dld + 2.0 * L.n) * esz;
      continue;
    }
    if (L.coarsest) {
      b[0] = seg_bytes(L.ras, L.n, L.n, false, 8) * (h->prm.coarse_refine && L.Aw64.p ? 3.0 : 1.0);
      if (f32) b[1] = b[5] = (double)L.n * 12.0;
    } else {
      const int64_t nn = L.col0.back();
      const int pf1 = h->persist_from[f32 ? 1 : 0];
      // FP16 entries where MIXED16 reads them (per plan; the persistent tail reads FP32)
      const bool h16 = use16(*h, L, f32) && !(pf1 > 0 && l >= pf1);
      auto msz = [&](const SegPlan& p) -> size_t { return h16 && p.lanes16 != 0 ? 2 : esz; };
      const double cp = rcopy(L) ? (double)L.n * esz : 0.0;  // fused copy r -> s
      b[0] = seg_bytes(L.ras, L.n, L.n, false, esz, msz(L.ras)) + cp;
      b[2] = 2.0 * (resid_bytes(L, esz, msz(L.ablk)) - cp);  // two residuals
      b[3] = seg_bytes(L.restr, L.n, nn, false, esz, msz(L.restr));
      b[4] = seg_bytes(L.prol, nn, L.n, true, esz, msz(L.prol)) + cp;
      b[7] = rast_bytes(L, esz, msz(L.yd64.p ? L.rast_det : L.rast));
    }
  }
  const int pf = h->persist_from[f32 ? 1 : 0];
  if (pf > 0) {
    double tail = 0.0;
    for (int i = pf * VProf::kSlots; i < nl * VProf::kSlots; ++i) {
      tail += bytes[i];
      bytes[i] = 0.0;
    }
    bytes[pf * VProf::kSlots + 6] = tail;
  }
  for (int i = 0; i < nl * VProf::kSlots; ++i) ms[i] = acc[i] / reps;
  return take_err_word(*h, s);
}

int64_t amgdd_kernel_launches(void) { return g_kernels.load(); }

int amgdd_measure_fp64(void* stream, double* gflops) {
  if (gflops == nullptr) {
    set_error("amgdd_measure_fp64: null output");
    return AMGDD_ERR_INVALID_ARG;
  }
  return measure_fp64_rate((cudaStream_t)stream, gflops);
}

int64_t amgdd_device_bytes(const amgdd_hierarchy* h, int with_batched) {
  if (h == nullptr) return -1;
  int64_t b = h->setup_bytes + h->multi_bytes;
  if (with_batched > 0) {  // 1: the hierarchy's batch width; 2..32: a batch of that many columns
    const int want = kclass(std::min(with_batched == 1 ? h->prm.batch_cols : with_batched, kMaxRhs));
    if (h->mw.cap < want) b += multi_bytes_estimate(*h, want) - h->multi_bytes;
  }
  return b;
}

int amgdd_num_levels(const amgdd_hierarchy* h) { return h ? (int)h->lv.size() : 0; }

// Structural pattern of A_l = G_l^T G_l (+ D1 on level 0, carried as rows of
// G): j ~ k iff some row group's support holds both (CSR, ascending columns).
static void level_A_pattern(const Level& L, std::vector<int64_t>& ptr, std::vector<int32_t>& idx) {
  std::vector<std::vector<int32_t>> rows((size_t)L.n);
  for (size_t g = 0; g + 1 < L.g_ptr.size(); ++g)
    for (int64_t a = L.g_ptr[g]; a < L.g_ptr[g + 1]; ++a) {
      auto& r = rows[(size_t)L.g_idx[a]];
      r.insert(r.end(), L.g_idx.begin() + L.g_ptr[g], L.g_idx.begin() + L.g_ptr[g + 1]);
    }
  ptr.assign((size_t)L.n + 1, 0);
  idx.clear();
  for (int64_t j = 0; j < L.n; ++j) {
    auto& r = rows[(size_t)j];
    std::sort(r.begin(), r.end());
    r.erase(std::unique(r.begin(), r.end()), r.end());
    idx.insert(idx.end(), r.begin(), r.end());
    ptr[j + 1] = (int64_t)idx.size();
    std::vector<int32_t>().swap(r);
  }
}

int amgdd_level_describe(const amgdd_hierarchy* h, int level, amgdd_level_desc* out) {
  if (h == nullptr || out == nullptr || level < 0 || level >= (int)h->lv.size()) {
    set_error("amgdd_level_describe: invalid argument");
    return AMGDD_ERR_INVALID_ARG;
  }
  const Level& L = *h->lv[level];
  std::memset(out, 0, sizeof(*out));
  out->n = L.n;
  out->is_coarsest = L.coarsest ? 1 : 0;
  out->ngroups = (int64_t)L.g_ptr.size() - 1;
  for (size_t g = 0; g + 1 < L.g_ptr.size() && g < L.g_rank.size(); ++g) {
    out->g_rows += L.g_rank[g];
    out->g_vals += (int64_t)L.g_rank[g] * (L.g_ptr[g + 1] - L.g_ptr[g]);
  }
  out->g_sup_len = L.g_ptr.empty() ? 0 : L.g_ptr.back();
  out->a_nnz = level < (int)h->nnzA.size() ? h->nnzA[level] : 0;
  if (!L.coarsest) {
    for (int i = 0; i < L.nagg; ++i) out->p_nnz += (int64_t)L.nomega[i] * L.k[i];
    out->nagg = L.nagg;
    out->n_next = L.col0.empty() ? 0 : L.col0.back();
    out->omega_len = (int64_t)L.om_idx.size();
    out->z_len = L.z_off.empty() ? 0 : L.z_off.back();
    for (int i = 0; i < L.nagg; ++i) out->w_vals += (int64_t)L.nomega[i] * (L.om_ptr[i + 1] - L.om_ptr[i]);
  } else {
    out->w_vals = L.n * L.n;
  }
  return AMGDD_OK;
}

int amgdd_level_export(const amgdd_hierarchy* h, int level, int which, void* dst, size_t cap) {
  if (h == nullptr || dst == nullptr || level < 0 || level >= (int)h->lv.size()) {
    set_error("amgdd_level_export: invalid argument");
    return AMGDD_ERR_INVALID_ARG;
  }
  const Level& L = *h->lv[level];
  auto put = [&](const void* src, size_t bytes) -> int {
    if (bytes > cap) {
      set_error("amgdd_level_export: destination holds %zu bytes, %zu needed", cap, bytes);
      return AMGDD_ERR_INVALID_ARG;
    }
    std::memcpy(dst, src, bytes);
    return AMGDD_OK;
  };
  switch (which) {
    case AMGDD_ARR_G_PTR: return put(L.g_ptr.data(), L.g_ptr.size() * sizeof(int64_t));
    case AMGDD_ARR_G_IDX: return put(L.g_idx.data(), L.g_idx.size() * sizeof(int32_t));
    case AMGDD_ARR_A_PTR:
    case AMGDD_ARR_A_IDX: {
      std::vector<int64_t> ptr;
      std::vector<int32_t> idx;
      level_A_pattern(L, ptr, idx);
      return which == AMGDD_ARR_A_PTR ? put(ptr.data(), ptr.size() * sizeof(int64_t))
                                      : put(idx.data(), idx.size() * sizeof(int32_t));
    }
    default:
      break;
  }
  if (L.coarsest && which != AMGDD_ARR_AGG) {
    set_error("amgdd_level_export: the coarsest level has no aggregates");
    return AMGDD_ERR_INVALID_ARG;
  }
  switch (which) {
    case AMGDD_ARR_P_PTR:
    case AMGDD_ARR_P_IDX: {
      // row j of P_l spans the k_a columns of its aggregate a (Eq. mg-p);
      // columns are numbered by aggregate, then by ascending mu
      std::vector<int64_t> c0(L.nagg + 1, 0);
      for (int a = 0; a < L.nagg; ++a) c0[a + 1] = c0[a] + L.k[a];
      std::vector<int64_t> ptr(L.n + 1, 0);
      for (int64_t j = 0; j < L.n; ++j) ptr[j + 1] = ptr[j] + L.k[L.agg[j]];
      if (which == AMGDD_ARR_P_PTR) return put(ptr.data(), ptr.size() * sizeof(int64_t));
      std::vector<int32_t> idx((size_t)ptr[L.n]);
      for (int64_t j = 0; j < L.n; ++j)
        for (int64_t c = 0; c < ptr[j + 1] - ptr[j]; ++c) idx[ptr[j] + c] = (int32_t)(c0[L.agg[j]] + c);
      return put(idx.data(), idx.size() * sizeof(int32_t));
    }
    case AMGDD_ARR_AGG:
      if (L.agg.empty()) {
        set_error("amgdd_level_export: no aggregates on this level");
        return AMGDD_ERR_INVALID_ARG;
      }
      return put(L.agg.data(), L.agg.size() * sizeof(int32_t));
    case AMGDD_ARR_OMEGA_PTR: return put(L.om_ptr.data(), L.om_ptr.size() * sizeof(int64_t));
    case AMGDD_ARR_OMEGA_IDX: return put(L.om_idx.data(), L.om_idx.size() * sizeof(int32_t));
    case AMGDD_ARR_NOMEGA: return put(L.nomega.data(), L.nomega.size() * sizeof(int32_t));
    case AMGDD_ARR_K: return put(L.k.data(), L.k.size() * sizeof(int32_t));
    case AMGDD_ARR_Z:
    case AMGDD_ARR_MU: {
      const bool z = which == AMGDD_ARR_Z;
      const size_t cnt = z ? (size_t)L.z_off.back() : (size_t)L.mu_off.back();
      if (cnt * sizeof(double) > cap) {
        set_error("amgdd_level_export: destination too small");
        return AMGDD_ERR_INVALID_ARG;
      }
      if (cudaMemcpy(dst, z ? L.Z64.p : L.mu.p, cnt * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) {
        set_error("amgdd_level_export: copy failed");
        return AMGDD_ERR_CUDA;
      }
      return AMGDD_OK;
    }
    default:
      set_error("amgdd_level_export: unknown array %d", which);
      return AMGDD_ERR_INVALID_ARG;
  }
}

static void level_bytes(const amgdd_hierarchy& h, const Level& L, size_t esz, double& cyc, bool tail = false) {
  if (L.coarsest) {
    cyc += ((double)L.n * L.n * 8.0 + 2.0 * L.n * 8.0) * (h.prm.coarse_refine && L.Aw64.p ? 3.0 : 1.0);
    return;
  }
  const int64_t nn = L.col0.back();
  // FP16 entries where MIXED16 reads them (per plan; the persistent tail reads FP32)
  const bool h16 = use16(h, L, esz == 4) && !tail;
  auto msz = [&](const SegPlan& p) -> size_t { return h16 && p.lanes16 != 0 ? 2 : esz; };
  cyc += seg_bytes(L.ras, L.n, L.n, false, esz, msz(L.ras)) +
         rast_bytes(L, esz, msz(L.yd64.p ? L.rast_det : L.rast)) +
         seg_bytes(L.restr, L.n, nn, false, esz, msz(L.restr)) + seg_bytes(L.prol, nn, L.n, true, esz, msz(L.prol)) +
         2.0 * resid_bytes(L, esz, msz(L.ablk));
}

int amgdd_bytes_model(const amgdd_hierarchy* h, double* vcycle_bytes, double* apply_out) {
  if (h == nullptr) return AMGDD_ERR_INVALID_ARG;
  const size_t esz = mixed(*h) ? 4 : 8;
  const int df = h->dense_from[esz == 4 ? 1 : 0];
  double cyc = 0.0;
  for (size_t l = 0; l < h->lv.size(); ++l) {
    const Level& L = *h->lv[l];
    if (df > 0 && (int)l == df) {
      cyc += ((double)L.n * L.dld + 2.0 * L.n) * esz;
      break;
    }
    const int pf = h->persist_from[esz == 4 ? 1 : 0];
    level_bytes(*h, L, esz, cyc, pf > 0 && (int)l >= pf);
  }
  const Level& L0 = *h->lv[0];
  const double ap = L0.use_ell ? (double)L0.n * L0.ell_w * 12.0 + 2.0 * L0.n * 8.0 : apply_bytes(L0, 8);
  if (vcycle_bytes) *vcycle_bytes = cyc;
  if (apply_out) *apply_out = ap;
  return AMGDD_OK;
}

int amgdd_hierarchy_stats(const amgdd_hierarchy* h, char* json, size_t cap) {
  if (h == nullptr || json == nullptr || cap == 0) return AMGDD_ERR_INVALID_ARG;
  std::string s = "{\"levels\": " + std::to_string(h->lv.size()) + ", \"n\": [";
  for (size_t l = 0; l < h->lv.size(); ++l) s += (l ? ", " : "") + std::to_string(h->lv[l]->n);
  s += "], \"nnzA\": [";
  for (size_t l = 0; l < h->nnzA.size(); ++l) s += (l ? ", " : "") + std::to_string(h->nnzA[l]);
  double oc = 0;
  for (int64_t v : h->nnzA) oc += (double)v;
  oc /= h->nnzA.empty() ? 1.0 : (double)h->nnzA[0];
  s += "], \"op_complexity\": " + std::to_string(oc);
  s += ", \"process_device_allocs\": " + std::to_string(device_alloc_count());
  s += ", \"nagg\": [";
  for (size_t l = 0; l < h->lv.size(); ++l) s += (l ? ", " : "") + std::to_string(h->lv[l]->nagg);
  s += "], \"g_vals\": [";
  for (size_t l = 0; l < h->lv.size(); ++l) {
    int64_t gv = 0;
    const Level& L = *h->lv[l];
    for (size_t g = 0; g + 1 < L.g_ptr.size() && g < L.g_rank.size(); ++g)
      gv += (int64_t)L.g_rank[g] * (L.g_ptr[g + 1] - L.g_ptr[g]);
    s += (l ? ", " : "") + std::to_string(gv);
  }
  s += "], \"w_vals\": [";
  for (size_t l = 0; l < h->lv.size(); ++l) {
    amgdd_level_desc d;
    amgdd_level_describe(h, (int)l, &d);
    s += (l ? ", " : "") + std::to_string(d.w_vals);
  }
  s += "], \"thresh\": [";
  for (size_t l = 0; l + 1 < h->lv.size(); ++l) {
    char buf[40];
    std::snprintf(buf, sizeof buf, "%s%.17g", l ? ", " : "", h->lv[l]->thresh);
    s += buf;
  }
  s += "], \"n_color\": [";
  for (size_t l = 0; l + 1 < h->lv.size(); ++l) s += (l ? ", " : "") + std::to_string(h->lv[l]->n_color);
  s += "], \"n_mult\": [";
  for (size_t l = 0; l + 1 < h->lv.size(); ++l) s += (l ? ", " : "") + std::to_string(h->lv[l]->n_mult);
  s += "], \"schur_route\": [";
  for (size_t l = 0; l + 1 < h->lv.size(); ++l) s += std::string(l ? ", " : "") + (h->lv[l]->schur_rows ? "\"rows\"" : "\"gram\"");
  s += "], \"fp16_levels\": [";
  for (size_t l = 0; l < h->lv.size(); ++l) s += std::string(l ? ", " : "") + (h->lv[l]->h16 ? "true" : "false");
  s += "], \"fp16_lanes\": [";  // per level: ras, rast, restrict, prolong, block rows (0: FP32 copy)
  for (size_t l = 0; l < h->lv.size(); ++l) {
    const Level& L = *h->lv[l];
    s += std::string(l ? ", [" : "[") + std::to_string(L.ras.lanes16) + ", " + std::to_string(L.rast.lanes16) +
         ", " + std::to_string(L.restr.lanes16) + ", " + std::to_string(L.prol.lanes16) + ", " +
         std::to_string(L.ablk.lanes16) + "]";
  }
  s += "], \"coarse_A\": [";
  for (size_t l = 0; l < h->lv.size(); ++l) {
    const Level& L = *h->lv[l];
    char buf[160];
    std::snprintf(buf, sizeof buf, "%s{\"form\": \"%s\", \"block_rows_us\": %.2f, \"matrix_free_us\": %.2f}",
                  l ? ", " : "", L.coarsest ? "none" : (L.use_ell ? "ELL rows" : (L.has_blk ? "block rows" : "matrix-free")),
                  L.use_ell ? L.ell_us : L.blk_us, L.mf_us);
    s += buf;
  }
  {
    const Level& C = *h->lv.back();
    char buf[96];
    std::snprintf(buf, sizeof buf, "], \"coarsest_inv_err\": %.3e, \"coarsest_refined\": %s", C.inv_err,
                  (h->prm.coarse_refine && C.Aw64.p) ? "true" : "false");
    s += buf;
  }
  s += ", \"dense_tail\": {";
  for (int pi = 0; pi < 2; ++pi) {
    s += std::string(pi ? ", " : "") + (pi ? "\"mixed\"" : "\"fp64\"") + ": {\"from\": " +
         std::to_string(h->dense_from[pi]) + ", \"vcycle_us_by_level\": [";
    for (size_t l = 0; l < std::min<size_t>(h->lv.size(), 16); ++l) {
      char buf[32];
      std::snprintf(buf, sizeof buf, "%s%.1f", l ? ", " : "", h->dense_us[pi][l]);
      s += buf;
    }
    s += "]}";
  }
  s += "}, \"tail\": {";
  for (int pi = 0; pi < 2; ++pi) {
    s += std::string(pi ? ", " : "") + (pi ? "\"mixed\"" : "\"fp64\"") + ": {\"from\": " +
         std::to_string(h->persist_from[pi]) + ", \"vcycle_us_by_from\": [";
    for (size_t l = 0; l < std::min<size_t>(h->lv.size(), 16); ++l) {
      char buf[32];
      std::snprintf(buf, sizeof buf, "%s%.1f", l ? ", " : "", h->persist_us[pi][l]);
      s += buf;
    }
    s += "]}";
  }
  s += "}, \"setup_phases_ms\": {";
  bool first = true;
  for (int i = 0; i < 16; ++i)
    if (h->phase_name[i]) {
      char buf[96];
      std::snprintf(buf, sizeof buf, "%s\"%s\": %.3f", first ? "" : ", ", h->phase_name[i], h->phase_ms[i]);
      s += buf;
      first = false;
    }
  s += "}, \"setup_phases_gflop\": {";  // FP64 flops counted from the actual block sizes (a model per phase)
  first = true;
  for (int i = 0; i < 16; ++i)
    if (h->phase_name[i] && h->phase_flops[i] > 0) {
      char buf[96];
      std::snprintf(buf, sizeof buf, "%s\"%s\": %.4f", first ? "" : ", ", h->phase_name[i], h->phase_flops[i] * 1e-9);
      s += buf;
      first = false;
    }
  s += "}";
  double vb = 0, ab = 0;
  amgdd_bytes_model(h, &vb, &ab);
  s += ", \"vcycle_bytes\": " + std::to_string(vb) + ", \"apply64_bytes\": " + std::to_string(ab);
  s += ", \"setup_ms\": " + std::to_string(h->setup_ms) + "}";
  if (s.size() + 1 > cap) return AMGDD_ERR_INVALID_ARG;
  std::memcpy(json, s.c_str(), s.size() + 1);
  return AMGDD_OK;
}

// ---------------------------------------------------------------------------
// Saved hierarchies: the setup inputs (G, D1, aggregates, overlap), the
// parameters and the setup-time kernel choices.  Loading runs the setup
// again with those choices replayed instead of timed, so the loaded
// hierarchy applies the same arithmetic with the same kernels (on a GPU of
// the same model; elsewhere the choices are timed anew).
// What setup computed for level l, downloaded (FP64 matrices only; unused
// entries of the compressed-row capacity are written as zeros).
static int snapshot_level(const amgdd_hierarchy& h, int l, LevelSnap& S) {
  const Level& L = *h.lv[l];
  cudaStream_t s = h.work;
  S.n = L.n;
  S.nnzA = l < (int)h.nnzA.size() ? h.nnzA[l] : 0;
  S.nagg = L.nagg;
  S.coarsest = L.coarsest ? 1 : 0;
  S.schur_rows = L.schur_rows ? 1 : 0;
  S.n_color = L.n_color;
  S.n_mult = L.n_mult;
  S.thresh = L.thresh;
  S.inv_err = L.inv_err;
  S.g_ptr = L.g_ptr;
  S.g_idx = L.g_idx;
  S.h_off = L.h_off;
  if (L.d_R64.p) {
    S.g_rank = L.g_rank;
    AMGDD_TRY(download(S.R64, L.d_R64.p, (size_t)L.h_off.back(), s));
    for (size_t g = 0; g + 1 < L.g_ptr.size(); ++g) {
      const int64_t sz = L.g_ptr[g + 1] - L.g_ptr[g];
      for (int64_t e = L.h_off[g] + (int64_t)L.g_rank[g] * sz; e < L.h_off[g + 1]; ++e) S.R64[e] = 0.0;
    }
  }
  if (L.coarsest) {
    AMGDD_TRY(download(S.W64, L.W64.p, L.W64.n, s));
    if (L.Aw64.p) AMGDD_TRY(download(S.Aw64, L.Aw64.p, L.Aw64.n, s));
    return AMGDD_OK;
  }
  S.agg = L.agg;
  S.om_ptr = L.om_ptr;
  S.om_idx = L.om_idx;
  S.nomega = L.nomega;
  S.k = L.k;
  S.col0 = L.col0;
  S.z_off = L.z_off;
  S.mu_off = L.mu_off;
  S.wf_off = L.wf_off;
  AMGDD_TRY(download(S.W64, L.W64.p, L.W64.n, s));
  if (L.Aw64.p) AMGDD_TRY(download(S.Aw64, L.Aw64.p, L.Aw64.n, s));
  AMGDD_TRY(download(S.mu, L.mu.p, (size_t)L.mu_off.back(), s));
  AMGDD_TRY(download(S.Z64, L.Z64.p, (size_t)L.z_off.back(), s));
  if (L.Wf64.p) AMGDD_TRY(download(S.Wf64, L.Wf64.p, L.Wf64.n, s));
  if (L.has_blk && L.A64.p) AMGDD_TRY(download(S.A64, L.A64.p, L.A64.n, s));
  return AMGDD_OK;
}

int amgdd_hierarchy_save(const amgdd_hierarchy* h, const char* path) {
  if (h == nullptr || path == nullptr) {
    set_error("amgdd_hierarchy_save: invalid argument");
    return AMGDD_ERR_INVALID_ARG;
  }
  FILE* f = std::fopen(path, "wb");
  if (!f) {
    set_error("amgdd_hierarchy_save: cannot open %s", path);
    return AMGDD_ERR_INVALID_ARG;
  }
  const uint32_t psz = sizeof(amgdd_params);
  const int32_t ov = h->overlap, hd = h->in_has_d1 ? 1 : 0;
  const int64_t n = h->n;
  amgdd_params prm = h->prm;
  prm.tune_cache = nullptr;
  bool ok = std::fwrite(kSaveMagic, 1, 8, f) == 8 && std::fwrite(&psz, sizeof psz, 1, f) == 1 &&
            std::fwrite(&prm, psz, 1, f) == 1 && std::fwrite(&ov, sizeof ov, 1, f) == 1 &&
            std::fwrite(&hd, sizeof hd, 1, f) == 1 && std::fwrite(&n, sizeof n, 1, f) == 1 &&
            put_vec(f, h->in_rowptr) && put_vec(f, h->in_col) && put_vec(f, h->in_val) && put_vec(f, h->in_agg) &&
            put_vec(f, h->in_d1);
  const uint64_t nkv = h->tune_kv.size();
  ok = ok && std::fwrite(&nkv, sizeof nkv, 1, f) == 1;
  for (const auto& kv : h->tune_kv) {
    const uint32_t len = (uint32_t)kv.first.size();
    ok = ok && std::fwrite(&len, sizeof len, 1, f) == 1 && std::fwrite(kv.first.data(), 1, len, f) == len &&
         std::fwrite(&kv.second, sizeof(double), 1, f) == 1;
  }
  // the level snapshots, one at a time
  const uint64_t nl = h->lv.size();
  ok = ok && std::fwrite(&nl, sizeof nl, 1, f) == 1;
  for (size_t l = 0; ok && l < h->lv.size(); ++l) {
    LevelSnap S;
    const int rc = snapshot_level(*h, (int)l, S);
    if (rc != AMGDD_OK) {
      std::fclose(f);
      return rc;
    }
    ok = put_snap(f, S);
  }
  ok = (std::fclose(f) == 0) && ok;
  if (!ok) {
    set_error("amgdd_hierarchy_save: write to %s failed", path);
    return AMGDD_ERR_INVALID_ARG;
  }
  return AMGDD_OK;
}

int amgdd_hierarchy_load(const char* path, void* stream, amgdd_hierarchy** out) {
  if (path == nullptr || out == nullptr) {
    set_error("amgdd_hierarchy_load: invalid argument");
    return AMGDD_ERR_INVALID_ARG;
  }
  *out = nullptr;
  FILE* f = std::fopen(path, "rb");
  if (!f) {
    set_error("amgdd_hierarchy_load: cannot open %s", path);
    return AMGDD_ERR_INVALID_ARG;
  }
  char magic[8];
  uint32_t psz = 0;
  amgdd_params prm;
  int32_t ov = 0, hd = 0;
  int64_t n = 0;
  std::vector<int64_t> rowptr;
  std::vector<int32_t> col, agg;
  std::vector<double> val, d1;
  std::vector<std::pair<std::string, double>> kv;
  constexpr uint64_t kMax = (uint64_t)1 << 40;
  bool ok = std::fread(magic, 1, 8, f) == 8 &&
            (std::memcmp(magic, kSaveMagic, 8) == 0 || std::memcmp(magic, kSaveMagicV1, 8) == 0) &&
            std::fread(&psz, sizeof psz, 1, f) == 1 && psz == sizeof(amgdd_params) &&
            std::fread(&prm, psz, 1, f) == 1 && std::fread(&ov, sizeof ov, 1, f) == 1 &&
            std::fread(&hd, sizeof hd, 1, f) == 1 && std::fread(&n, sizeof n, 1, f) == 1 && get_vec(f, rowptr, kMax) &&
            get_vec(f, col, kMax) && get_vec(f, val, kMax) && get_vec(f, agg, kMax) && get_vec(f, d1, kMax);
  uint64_t nkv = 0;
  ok = ok && std::fread(&nkv, sizeof nkv, 1, f) == 1 && nkv < (1u << 20);
  for (uint64_t i = 0; ok && i < nkv; ++i) {
    uint32_t len = 0;
    double v = 0.0;
    ok = std::fread(&len, sizeof len, 1, f) == 1 && len < 4096;
    std::string k(ok ? len : 0, '\0');
    ok = ok && std::fread(&k[0], 1, len, f) == len && std::fread(&v, sizeof v, 1, f) == 1;
    if (ok) kv.emplace_back(std::move(k), v);
  }
  std::vector<LevelSnap> snaps;
  const bool v2 = ok && std::memcmp(magic, kSaveMagic, 8) == 0;
  if (v2) {
    uint64_t nl = 0;
    ok = std::fread(&nl, sizeof nl, 1, f) == 1 && nl >= 1 && nl <= 64;
    snaps.resize(ok ? nl : 0);
    for (auto& S : snaps) ok = ok && get_snap(f, S, kMax);
    ok = ok && snaps_valid(snaps, n);
  }
  std::fclose(f);
  if (!ok || rowptr.empty() || col.size() != val.size() || (int64_t)agg.size() != n ||
      (hd && (int64_t)d1.size() != n)) {
    set_error("amgdd_hierarchy_load: %s is not a saved hierarchy of this library version", path);
    return AMGDD_ERR_INVALID_ARG;
  }
  prm.tune_cache = nullptr;
  amgdd_csr G;
  G.m = (int64_t)rowptr.size() - 1;
  G.n = n;
  G.nnz = (int64_t)val.size();
  G.rowptr = rowptr.data();
  G.col = col.data();
  G.val = val.data();
  G.mem = AMGDD_HOST;
  try {
    return setup_impl(&G, hd ? d1.data() : nullptr, agg.data(), ov, &prm, stream, out, &kv, v2 ? &snaps : nullptr);
  } catch (const std::bad_alloc&) {
    set_error("amgdd_hierarchy_load: host allocation failed");
    return AMGDD_ERR_OOM;
  } catch (...) {
    set_error("amgdd_hierarchy_load: unexpected exception");
    return AMGDD_ERR_INTERNAL;
  }
}

int amgdd_selftest_wait_timeouts(void* stream, int* barrier_status, int* mbarrier_status) {
  if (barrier_status == nullptr || mbarrier_status == nullptr) {
    set_error("amgdd_selftest_wait_timeouts: invalid argument");
    return AMGDD_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  DBuf<unsigned> bar;
  DBuf<int> err;
  AMGDD_TRY(bar.alloc(2));
  AMGDD_TRY(err.alloc(1));
  int* out[2] = {barrier_status, mbarrier_status};
  for (int which = 0; which < 2; ++which) {
    AMGDD_TRY(bar.zero(s));
    AMGDD_TRY(err.zero(s));
    AMGDD_TRY(launch_wait_probe(which, bar.p, err.p, s));
    int e = 0;
    AMGDD_CUDA(cudaMemcpyAsync(&e, err.p, sizeof e, cudaMemcpyDeviceToHost, s));
    AMGDD_CUDA(cudaStreamSynchronize(s));
    *out[which] = e != 0 ? AMGDD_ERR_TIMEOUT : AMGDD_OK;
  }
  return AMGDD_OK;
}

void amgdd_free(amgdd_hierarchy* h) {
  if (h == nullptr) return;
  delete h;
}

}  // extern "C"
