// Serving: continuous batching of solve requests over cached hierarchies.
//
// Operators (hierarchies) are built once and stay resident on the device
// within a byte budget; when adding one would exceed it, idle operators are
// evicted least recently used first.  Requests (an operator, host right-hand
// sides, a tolerance) enter one FIFO.  Each of `slots` worker threads takes
// the oldest request whose operator is not being solved, merges the other
// queued requests for that operator and tolerance into the same batched
// solve (up to max_batch columns: the K independent CGs of amgdd_solve that
// share every V-cycle launch), runs it on its own stream and completes the
// requests.  Requests that arrive while batches are on the device join the
// next batch as a slot frees; batches of different operators overlap on the
// device (each hierarchy solves on its own stream).
// A request may also carry its operator (amgdd_server_submit_problem): an
// operator whose key is not resident is queued for setup, which a worker runs
// on its own stream once admission allows it: the bytes the hierarchy is
// expected to hold (bytes per unknown of the operators built so far, a fixed
// guess before the first) must fit both the budget, after evicting idle
// operators least recently used first, and the device's free memory at that
// moment.  Until then the request waits, and other work proceeds.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "amgdd.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Req {
  int64_t id = 0, op = 0;
  const double* b = nullptr;
  double* x = nullptr;
  int nrhs = 0;
  double tol = 0.0;
  Clock::time_point t_submit, t_start, t_done;
  int status = AMGDD_PENDING;
  int batch_cols = 0;
  std::vector<amgdd_info> info;
};

struct Op {
  int64_t id = 0, key = 0, n = 0;
  amgdd_hierarchy* h = nullptr;
  int64_t bytes = 0;
  bool busy = false;
  int queued = 0;  // requests waiting in the FIFO
  uint64_t last_use = 0;
  // operators submitted with a request: built by a worker (setup on the
  // request path); the caller keeps the inputs valid until the request is
  // polled to completion
  bool ready = true;
  int status = AMGDD_OK;  // a failed setup fails the operator's requests
  amgdd_csr G{};
  const double* D1 = nullptr;
  const int32_t* agg = nullptr;
  int overlap = 1;
  amgdd_params prm{};
  double setup_ms = 0.0;
};

struct Staging {
  double* b = nullptr;
  double* x = nullptr;
  size_t cap = 0;  // doubles each
  ~Staging() {
    if (b) cudaFreeHost(b);
    if (x) cudaFreeHost(x);
  }
  bool reserve(size_t n) {
    if (n <= cap) return true;
    if (b) cudaFreeHost(b);
    if (x) cudaFreeHost(x);
    b = x = nullptr;
    cap = 0;
    if (cudaMallocHost((void**)&b, n * sizeof(double)) != cudaSuccess) return false;
    if (cudaMallocHost((void**)&x, n * sizeof(double)) != cudaSuccess) return false;
    cap = n;
    return true;
  }
};

}  // namespace

struct amgdd_server {
  amgdd_server_params prm{};
  int device = 0;
  std::mutex mu;
  std::condition_variable work_cv, done_cv;
  std::map<int64_t, Op> ops;
  std::map<int64_t, std::shared_ptr<Req>> reqs;
  std::deque<std::shared_ptr<Req>> fifo;
  std::vector<std::thread> workers;
  bool stop = false;
  int64_t next_req = 1, next_op = 1;
  int64_t used = 0;
  uint64_t tick = 0;
  // statistics
  int64_t completed = 0, batches = 0, batch_cols = 0, evictions = 0, cache_hits = 0;
  int64_t builds = 0, building = 0, waits_for_memory = 0;
  double build_ms = 0.0;
  double bytes_per_unknown = 0.0;  // of the operators built so far (admission estimate)
  std::vector<double> latencies_ms;
  Clock::time_point t0 = Clock::now();

  void worker_loop();
  int64_t evict_for(int64_t need);  // returns freed bytes; caller holds mu
  bool admit(int64_t need);         // budget and free device memory; caller holds mu
  void fail_op(Op& op, int status); // complete the operator's queued requests with an error; caller holds mu
};

bool amgdd_server::admit(int64_t need) {
  evict_for(need);
  if (used + need > prm.hbm_budget) return false;
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  if ((int64_t)free_b >= need) return true;
  // the device is short although the budget is not: evict idle operators
  // until it fits or nothing idle is left
  while ((int64_t)free_b < need) {
    const int64_t before = used;
    evict_for(prm.hbm_budget - used + 1);  // evicts one idle operator at least, when there is one
    if (used == before) return false;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return false;
  }
  return true;
}

void amgdd_server::fail_op(Op& op, int status) {
  for (auto it = fifo.begin(); it != fifo.end();) {
    if ((*it)->op == op.id) {
      auto& r = *it;
      r->status = status;
      r->t_start = r->t_done = Clock::now();
      r->info.assign(r->nrhs, amgdd_info{});
      ++completed;
      it = fifo.erase(it);
    } else {
      ++it;
    }
  }
  op.queued = 0;
}

int64_t amgdd_server::evict_for(int64_t need) {
  int64_t freed = 0;
  while (used + need > prm.hbm_budget) {
    Op* lru = nullptr;
    for (auto& e : ops)
      if (e.second.ready && e.second.h && !e.second.busy && e.second.queued == 0 &&
          (!lru || e.second.last_use < lru->last_use))
        lru = &e.second;
    if (!lru) break;
    amgdd_free(lru->h);
    used -= lru->bytes;
    freed += lru->bytes;
    ++evictions;
    ops.erase(lru->id);
  }
  return freed;
}

void amgdd_server::worker_loop() {
  cudaSetDevice(device);
  cudaStream_t stream;
  cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking);
  Staging st;
  for (;;) {
    std::vector<std::shared_ptr<Req>> batch;
    Op* op = nullptr;
    {
      std::unique_lock<std::mutex> lock(mu);
      for (;;) {
        if (stop) {
          cudaStreamDestroy(stream);
          return;
        }
        // oldest request whose operator is idle: built and not being solved,
        // or still to be built (setup on the request path) and admitted
        auto it = fifo.begin();
        Op* build = nullptr;
        int64_t reserve = 0;  // the admitted estimate, held in `used` while the build runs
        for (; it != fifo.end(); ++it) {
          auto o = ops.find((*it)->op);
          if (o == ops.end() || o->second.busy) continue;
          if (o->second.ready) break;
          const double bpu = bytes_per_unknown > 0.0 ? bytes_per_unknown : 16384.0;
          const int64_t need = (int64_t)(bpu * (double)o->second.n * 1.25);
          // with nothing resident or being built the estimate is not trusted: build and check the real bytes
          if (admit(need) || (used == 0 && building == 0)) {
            build = &o->second;
            reserve = std::min(need, std::max<int64_t>(prm.hbm_budget - used, 0));
            used += reserve;
            break;
          }
          ++waits_for_memory;
        }
        if (build) {
          build->busy = true;
          ++building;
          Op* b = build;
          lock.unlock();
          const auto t0b = Clock::now();
          amgdd_hierarchy* h = nullptr;
          const int rc = amgdd_setup(&b->G, b->D1, b->agg, b->overlap, &b->prm, stream, &h);
          const double ms = std::chrono::duration<double, std::milli>(Clock::now() - t0b).count();
          lock.lock();
          --building;
          b->busy = false;
          used -= reserve;
          if (rc != AMGDD_OK) {
            b->status = rc;
            fail_op(*b, rc);
            const int64_t id = b->id;
            ops.erase(id);
            done_cv.notify_all();
            continue;
          }
          const int64_t bytes = amgdd_device_bytes(h, 1);
          evict_for(bytes);
          if (used + bytes > prm.hbm_budget) {  // larger than the budget even with every idle operator evicted
            amgdd_free(h);
            fail_op(*b, AMGDD_ERR_OOM);
            const int64_t id = b->id;
            ops.erase(id);
            done_cv.notify_all();
            continue;
          }
          b->h = h;
          b->bytes = bytes;
          b->ready = true;
          b->setup_ms = ms;
          b->last_use = ++tick;
          used += b->bytes;
          ++builds;
          build_ms += ms;
          bytes_per_unknown = std::max(bytes_per_unknown, (double)b->bytes / (double)std::max<int64_t>(b->n, 1));
          continue;  // its requests are now solvable: pick again
        }
        if (it != fifo.end()) {
          op = &ops[(*it)->op];
          const double tol = (*it)->tol;
          int cols = 0;
          for (auto jt = it; jt != fifo.end();) {
            const auto& r = *jt;
            if (r->op == op->id && r->tol == tol && (cols == 0 || cols + r->nrhs <= prm.max_batch)) {
              cols += r->nrhs;
              batch.push_back(r);
              jt = fifo.erase(jt);
              if (cols >= prm.max_batch) break;
            } else {
              ++jt;
            }
          }
          op->busy = true;
          op->queued -= (int)batch.size();
          break;
        }
        work_cv.wait(lock);
      }
    }
    // one batched solve over the merged columns (host staging, pinned)
    const int64_t n = op->n;
    int cols = 0;
    for (auto& r : batch) cols += r->nrhs;
    const auto t_start = Clock::now();
    int rc = st.reserve((size_t)n * cols) ? AMGDD_OK : AMGDD_ERR_OOM;
    std::vector<amgdd_info> info(cols);
    if (rc == AMGDD_OK) {
      int c = 0;
      for (auto& r : batch) {
        std::memcpy(st.b + (size_t)c * n, r->b, sizeof(double) * n * r->nrhs);
        c += r->nrhs;
      }
      rc = amgdd_solve(op->h, st.b, cols, batch.front()->tol, st.x, stream, info.data());
      cudaStreamSynchronize(stream);
    }
    const bool per_rhs = rc == AMGDD_OK || rc == AMGDD_ERR_BREAKDOWN || rc == AMGDD_ERR_NO_CONVERGENCE ||
                         rc == AMGDD_ERR_NONFINITE;
    const auto t_done = Clock::now();
    {
      std::lock_guard<std::mutex> lock(mu);
      int c = 0;
      for (auto& r : batch) {
        if (per_rhs) std::memcpy(r->x, st.x + (size_t)c * n, sizeof(double) * n * r->nrhs);
        r->info.assign(info.begin() + c, info.begin() + c + r->nrhs);
        c += r->nrhs;
        int s = per_rhs ? AMGDD_OK : rc;
        if (per_rhs)
          for (const auto& i : r->info)
            if (i.status != AMGDD_OK && s == AMGDD_OK) s = i.status;
        r->status = s;
        r->t_start = t_start;
        r->t_done = t_done;
        r->batch_cols = cols;
        latencies_ms.push_back(std::chrono::duration<double, std::milli>(t_done - r->t_submit).count());
        ++completed;
      }
      ++batches;
      batch_cols += cols;
      op->busy = false;
      op->last_use = ++tick;
    }
    done_cv.notify_all();
    work_cv.notify_all();
  }
}

extern "C" {

amgdd_server_params amgdd_server_params_default(void) {
  amgdd_server_params p;
  p.hbm_budget = (int64_t)64 << 30;
  p.slots = 4;
  p.max_batch = 8;
  return p;
}

int amgdd_server_create(const amgdd_server_params* params, amgdd_server** out) {
  if (out == nullptr) return AMGDD_ERR_INVALID_ARG;
  *out = nullptr;
  amgdd_server_params p = params ? *params : amgdd_server_params_default();
  if (p.slots < 1 || p.slots > 64 || p.max_batch < 1 || p.hbm_budget <= 0) return AMGDD_ERR_INVALID_ARG;
  p.max_batch = std::min(p.max_batch, 32);
  std::unique_ptr<amgdd_server> s(new amgdd_server());
  s->prm = p;
  if (cudaGetDevice(&s->device) != cudaSuccess) return AMGDD_ERR_CUDA;
  for (int i = 0; i < p.slots; ++i) s->workers.emplace_back([srv = s.get()] { srv->worker_loop(); });
  *out = s.release();
  return AMGDD_OK;
}

int amgdd_server_add_operator(amgdd_server* s, int64_t key, const amgdd_csr* G, const double* D1,
                              const int32_t* agg, int overlap, const amgdd_params* params, int64_t* op,
                              int* cached) {
  if (s == nullptr || op == nullptr) return AMGDD_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    for (auto& e : s->ops)
      if (e.second.key == key) {
        *op = e.first;
        e.second.last_use = ++s->tick;
        ++s->cache_hits;
        if (cached) *cached = 1;
        return AMGDD_OK;
      }
  }
  if (cached) *cached = 0;
  amgdd_hierarchy* h = nullptr;
  int rc = amgdd_setup(G, D1, agg, overlap, params, nullptr, &h);
  if (rc != AMGDD_OK) return rc;
  const int64_t bytes = amgdd_device_bytes(h, 1);
  std::lock_guard<std::mutex> lock(s->mu);
  s->evict_for(bytes);
  if (s->used + bytes > s->prm.hbm_budget) {
    amgdd_free(h);
    return AMGDD_ERR_OOM;
  }
  Op o;
  o.id = s->next_op++;
  o.key = key;
  o.n = G->n;
  o.h = h;
  o.bytes = bytes;
  o.last_use = ++s->tick;
  s->used += bytes;
  s->ops[o.id] = o;
  *op = o.id;
  return AMGDD_OK;
}

int amgdd_server_submit(amgdd_server* s, int64_t op, const double* b, int nrhs, double tol, double* x, int64_t* req) {
  if (s == nullptr || b == nullptr || x == nullptr || req == nullptr || nrhs < 1 || !(tol >= 0.0))
    return AMGDD_ERR_INVALID_ARG;
  cudaPointerAttributes a;
  for (const void* ptr : {(const void*)b, (const void*)x})
    if (cudaPointerGetAttributes(&a, ptr) == cudaSuccess && a.type == cudaMemoryTypeDevice)
      return AMGDD_ERR_INVALID_ARG;  // host buffers only
  (void)cudaGetLastError();
  auto r = std::make_shared<Req>();
  r->op = op;
  r->b = b;
  r->x = x;
  r->nrhs = nrhs;
  r->tol = tol;
  r->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lock(s->mu);
    auto o = s->ops.find(op);
    if (o == s->ops.end()) return AMGDD_ERR_INVALID_ARG;
    r->id = s->next_req++;
    ++o->second.queued;
    s->reqs[r->id] = r;
    s->fifo.push_back(r);
    *req = r->id;
  }
  s->work_cv.notify_one();
  return AMGDD_OK;
}

int amgdd_server_submit_problem(amgdd_server* s, int64_t key, const amgdd_csr* G, const double* D1,
                                const int32_t* agg, int overlap, const amgdd_params* params, const double* b,
                                int nrhs, double tol, double* x, int64_t* req, int* cached) {
  if (s == nullptr || G == nullptr || b == nullptr || x == nullptr || req == nullptr || nrhs < 1 || !(tol >= 0.0) ||
      G->n < 1)
    return AMGDD_ERR_INVALID_ARG;
  int64_t op = -1;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    for (auto& e : s->ops)
      if (e.second.key == key) {
        op = e.first;
        e.second.last_use = ++s->tick;
        ++s->cache_hits;
        break;
      }
    if (cached) *cached = op >= 0 ? 1 : 0;
    if (op < 0) {
      Op o;
      o.id = s->next_op++;
      o.key = key;
      o.n = G->n;
      o.ready = false;
      o.G = *G;
      o.D1 = D1;
      o.agg = agg;
      o.overlap = overlap;
      o.prm = params ? *params : amgdd_params_default();
      o.last_use = ++s->tick;
      s->ops[o.id] = o;
      op = o.id;
    }
  }
  return amgdd_server_submit(s, op, b, nrhs, tol, x, req);
}

int amgdd_server_poll(amgdd_server* s, int64_t req, int wait_ms, amgdd_info* info, double* latency_ms) {
  if (s == nullptr) return AMGDD_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lock(s->mu);
  auto it = s->reqs.find(req);
  if (it == s->reqs.end()) return AMGDD_ERR_INVALID_ARG;
  auto r = it->second;
  if (r->status == AMGDD_PENDING && wait_ms != 0) {
    auto pred = [&] { return r->status != AMGDD_PENDING; };
    if (wait_ms < 0)
      s->done_cv.wait(lock, pred);
    else
      s->done_cv.wait_for(lock, std::chrono::milliseconds(wait_ms), pred);
  }
  if (r->status == AMGDD_PENDING) return AMGDD_PENDING;
  if (info)
    for (int i = 0; i < r->nrhs && i < (int)r->info.size(); ++i) info[i] = r->info[i];
  if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
  const int st = r->status;
  s->reqs.erase(it);
  return st;
}

int amgdd_server_stats(amgdd_server* s, char* json, size_t cap) {
  if (s == nullptr || json == nullptr || cap == 0) return AMGDD_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(s->mu);
  std::vector<double> lat = s->latencies_ms;
  std::sort(lat.begin(), lat.end());
  auto pct = [&](double q) { return lat.empty() ? 0.0 : lat[std::min(lat.size() - 1, (size_t)(q * lat.size()))]; };
  const double el = std::chrono::duration<double>(Clock::now() - s->t0).count();
  char buf[1024];
  std::snprintf(buf, sizeof buf,
                "{\"completed\": %lld, \"batches\": %lld, \"mean_batch_columns\": %.3f, \"p50_ms\": %.4f, "
                "\"p99_ms\": %.4f, \"max_ms\": %.4f, \"operators\": %zu, \"device_bytes\": %lld, "
                "\"budget_bytes\": %lld, \"evictions\": %lld, \"cache_hits\": %lld, \"queued\": %zu, "
                "\"builds\": %lld, \"build_ms_total\": %.1f, \"waits_for_memory\": %lld, "
                "\"bytes_per_unknown\": %.1f, \"elapsed_s\": %.4f}",
                (long long)s->completed, (long long)s->batches,
                s->batches ? (double)s->batch_cols / (double)s->batches : 0.0, pct(0.5), pct(0.99),
                lat.empty() ? 0.0 : lat.back(), s->ops.size(), (long long)s->used, (long long)s->prm.hbm_budget,
                (long long)s->evictions, (long long)s->cache_hits, s->fifo.size(), (long long)s->builds, s->build_ms,
                (long long)s->waits_for_memory, s->bytes_per_unknown, el);
  if (std::strlen(buf) + 1 > cap) return AMGDD_ERR_INVALID_ARG;
  std::memcpy(json, buf, std::strlen(buf) + 1);
  return AMGDD_OK;
}

void amgdd_server_destroy(amgdd_server* s) {
  if (s == nullptr) return;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop = true;
  }
  s->work_cv.notify_all();
  for (auto& t : s->workers) t.join();
  for (auto& e : s->ops)
    if (e.second.h) amgdd_free(e.second.h);
  delete s;
}

}  // extern "C"
