// Serving loop (tc_serve_*): count requests of mixed size, answered as they
// arrive, with continuous batching on one GPU.
//
//  * Registered graphs stay resident: CSR, BFS levels and cover edges are
//    computed once (tc_graph cache) and reused by every request on them.
//  * Admission: a scheduler thread admits queued requests in arrival order
//    while fewer than `slots` are in flight and the device bytes they are
//    estimated to need fit the HBM budget next to the resident graphs.
//  * Continuous batching: admitted small one-shot requests wait in a group;
//    whenever the batch worker is idle it takes the whole group (per mode)
//    and counts it with one tc_count_batch launch.  Large and resident
//    requests go to worker threads, each with its own CUDA stream, so work
//    from different requests overlaps on the device.
//  * Every internal wait is bounded (wait_limit_ms): a request that cannot be
//    admitted in time finishes with TC_ERR_TIMEOUT instead of waiting forever.
//  * Host-side fault injection for tests: fail_admitted = k > 0 makes the k-th
//    admitted request fail with TC_ERR_OOM as if its allocation had failed.
//  * Tracing: with TC_SERVE_TRACE=<path> in the environment the server writes
//    one line per device job (kind B/L/R = batch / large / resident, start
//    and end seconds since creation, requests in the job) when destroyed.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.cuh"

namespace tc {

namespace {

using Clock = std::chrono::steady_clock;

constexpr uint32_t kServeSmallN = 1u << 16;      // one-shot graphs this small are batched
constexpr int64_t kServeSmallNnz = 1ll << 20;
constexpr size_t kServeMaxGroup = 4096;           // requests per batched launch
constexpr int kLargeWorkers = 3;

struct Request {
  uint64_t ticket = 0;
  int mode = TC_MODE_COVER;
  uint64_t graph_id = 0;  // resident graph, or 0 for a one-shot CSR
  std::vector<int64_t> off;   // the request's own copy of a one-shot CSR
  std::vector<uint32_t> cols;  // (empty when the server borrows views)
  tc_csr_view view{};          // what the workers count: the copy or the caller's arrays
  uint32_t n = 0;
  size_t est_bytes = 0;
  bool small = false;
  int status = TC_OK;
  uint64_t count = 0;
  bool done = false;
  Clock::time_point t_submit;
};

struct Resident {
  tc_graph* g = nullptr;
  cudaStream_t stream = nullptr;
  std::mutex mu;  // one request at a time per graph
  size_t bytes = 0;
  int64_t num_cover = 0;
};

size_t csr_bytes(uint32_t n, int64_t nnz) {
  return sizeof(int64_t) * ((size_t)n + 1) + sizeof(uint32_t) * (size_t)nnz;
}

// Device bytes a one-shot count needs (an upper bound for either mode): the
// CSR, its COO rows (built only by a plain count), levels, the segmented rows
// and cover edges, and the bucketing scratch (descriptor, cursor, split and
// list entries per edge).
size_t one_shot_bytes(uint32_t n, int64_t nnz) {
  return csr_bytes(n, nnz) + (size_t)nnz * (4 + 4 + 4 + 22) + (size_t)n * 80;
}

}  // namespace
}  // namespace tc

using namespace tc;

struct tc_server {
  tc_serve_config cfg{};
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_sched, cv_work;
  // submitted, not yet admitted: small one-shot requests and the others
  // (large one-shot and resident), each in arrival order
  std::deque<std::shared_ptr<Request>> queue_small, queue_large;
  std::deque<std::shared_ptr<Request>> ready_large;
  std::deque<std::shared_ptr<Request>> ready_small;
  std::unordered_map<uint64_t, std::shared_ptr<Request>> tickets;
  std::unordered_map<uint64_t, std::unique_ptr<Resident>> residents;
  size_t resident_bytes = 0;
  size_t inflight_bytes = 0;
  int inflight = 0;        // admitted requests not yet finished
  int inflight_large = 0;  // of which large one-shot or resident (these take slots)
  uint64_t next_ticket = 1;
  uint64_t next_graph = 1;
  uint64_t admitted = 0;
  // optional trace (TC_SERVE_TRACE=<path>): one record per device job
  struct TraceRec { char kind; double t0, t1; size_t nreq; };
  std::vector<TraceRec> trace;
  Clock::time_point t_create = Clock::now();
  bool tracing = false;
  void record(char kind, Clock::time_point a, Clock::time_point b, size_t nreq) {
    if (!tracing) return;
    std::lock_guard<std::mutex> lk(mu);
    trace.push_back({kind, std::chrono::duration<double>(a - t_create).count(),
                     std::chrono::duration<double>(b - t_create).count(), nreq});
  }
  bool stopping = false;
  std::thread scheduler;
  std::vector<std::thread> workers;

  std::chrono::milliseconds wait_limit() const {
    return std::chrono::milliseconds(cfg.wait_limit_ms > 0 ? cfg.wait_limit_ms : 10000);
  }

  void finish(const std::shared_ptr<Request>& r, int status, uint64_t count) {
    std::lock_guard<std::mutex> lk(mu);
    r->status = status;
    r->count = count;
    r->done = true;
    inflight_bytes -= r->est_bytes;
    --inflight;
    if (!r->small) --inflight_large;
    cv_sched.notify_all();
  }

  // ---------------------------------------------------------------- scheduler
  // Admit the head of q while `fits` holds; a head that does not fit
  // blocks its queue (arrival order) and times out after wait_limit.
  template <class Fits>
  void admit_from(std::deque<std::shared_ptr<Request>>& q, Fits fits) {
    while (!q.empty()) {
      auto r = q.front();
      if (!fits(*r)) {
        if (Clock::now() - r->t_submit > wait_limit()) {  // bounded wait for admission
          q.pop_front();
          r->status = TC_ERR_TIMEOUT;
          r->done = true;
          continue;
        }
        return;
      }
      q.pop_front();
      ++inflight;
      if (!r->small) ++inflight_large;
      inflight_bytes += r->est_bytes;
      ++admitted;
      if (cfg.fail_admitted > 0 && admitted == (uint64_t)cfg.fail_admitted) {
        // injected allocation failure (host side)
        --inflight;
        if (!r->small) --inflight_large;
        inflight_bytes -= r->est_bytes;
        r->status = TC_ERR_OOM;
        r->done = true;
        continue;
      }
      (r->small ? ready_small : ready_large).push_back(r);
      cv_work.notify_all();
    }
  }

  // Small one-shot requests are admitted whenever their bytes fit (they are
  // batched, and a large request waiting for a slot does not hold them
  // back); large and resident requests also need one of the `slots`.
  void schedule_loop() {
    std::unique_lock<std::mutex> lk(mu);
    while (true) {
      cv_sched.wait_for(lk, std::chrono::milliseconds(50));
      if (stopping) return;
      auto bytes_fit = [&](const Request& r) {
        return resident_bytes + inflight_bytes + r.est_bytes <= cfg.hbm_budget_bytes;
      };
      admit_from(queue_small, bytes_fit);
      admit_from(queue_large,
                 [&](const Request& r) { return inflight_large < cfg.slots && bytes_fit(r); });
    }
  }

  // ---------------------------------------------------------------- workers
  // Stream priorities: the batch worker's launches (many small requests)
  // are scheduled ahead of the large ones' CTAs whenever SMs free up.
  static cudaStream_t make_stream(bool high) {
    int least = 0, greatest = 0;
    cudaDeviceGetStreamPriorityRange(&least, &greatest);
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, high ? greatest : least) !=
        cudaSuccess) {
      cudaGetLastError();
      cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    }
    return s;
  }

  void large_worker() {
    cudaSetDevice(device);
    cudaStream_t s = make_stream(false);
    while (true) {
      std::shared_ptr<Request> r;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv_work.wait_for(lk, std::chrono::milliseconds(50),
                         [&] { return stopping || !ready_large.empty(); });
        if (stopping) break;
        if (ready_large.empty()) continue;
        r = ready_large.front();
        ready_large.pop_front();
      }
      uint64_t c = 0;
      int st = TC_OK;
      const auto ta = Clock::now();
      if (r->graph_id) {
        Resident* res = nullptr;
        {
          std::lock_guard<std::mutex> lk(mu);
          auto it = residents.find(r->graph_id);
          if (it != residents.end()) res = it->second.get();
        }
        if (!res) {
          st = TC_ERR_NOT_FOUND;
        } else {
          std::lock_guard<std::mutex> g(res->mu);
          st = tc_count(res->g, r->mode, &c);
        }
      } else {
        tc_graph* g = nullptr;
        st = tc_graph_create(&r->view, TC_GRAPH_VALIDATE, s, &g);
        if (st == TC_OK) st = tc_count(g, r->mode, &c);
        tc_graph_destroy(g);
        std::vector<int64_t>().swap(r->off);
        std::vector<uint32_t>().swap(r->cols);
      }
      record(r->graph_id ? 'R' : 'L', ta, Clock::now(), 1);
      finish(r, st, st == TC_OK ? c : 0);
    }
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  }

  void batch_worker() {
    cudaSetDevice(device);
    cudaStream_t s = make_stream(true);
    while (true) {
      std::vector<std::shared_ptr<Request>> group;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv_work.wait_for(lk, std::chrono::milliseconds(50),
                         [&] { return stopping || !ready_small.empty(); });
        if (stopping) break;
        // everything admitted so far joins this launch (one mode per launch)
        const int mode = ready_small.empty() ? 0 : ready_small.front()->mode;
        for (auto it = ready_small.begin(); it != ready_small.end() && group.size() < kServeMaxGroup;) {
          if ((*it)->mode == mode) {
            group.push_back(*it);
            it = ready_small.erase(it);
          } else {
            ++it;
          }
        }
      }
      if (group.empty()) continue;
      const auto ta = Clock::now();
      std::vector<tc_csr_view> views(group.size());
      for (size_t i = 0; i < group.size(); ++i)
        views[i] = group[i]->view;
      std::vector<uint64_t> counts(group.size(), 0);
      std::vector<int> status(group.size(), TC_OK);
      const int rc = tc_count_batch(views.data(), (int32_t)views.size(), group[0]->mode, nullptr,
                                    s, counts.data(), status.data());
      record('B', ta, Clock::now(), group.size());
      for (size_t i = 0; i < group.size(); ++i) {
        std::vector<int64_t>().swap(group[i]->off);
        std::vector<uint32_t>().swap(group[i]->cols);
        finish(group[i], rc != TC_OK ? rc : status[i], rc != TC_OK ? 0 : counts[i]);
      }
    }
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  }
};

extern "C" {

int tc_serve_create(const tc_serve_config* cfg, tc_server** out) {
  if (!cfg || !out) return fail(TC_ERR_INVALID_ARG, "tc_serve_create: NULL argument");
  if (cfg->hbm_budget_bytes == 0 || cfg->slots <= 0)
    return fail(TC_ERR_INVALID_ARG, "tc_serve_create: budget and slots must be positive");
  tc_server* s = new (std::nothrow) tc_server();
  if (!s) return fail(TC_ERR_OOM, "host allocation failed");
  s->cfg = *cfg;
  if (s->cfg.queue_capacity <= 0) s->cfg.queue_capacity = 4096;
  cudaGetDevice(&s->device);
  s->tracing = getenv("TC_SERVE_TRACE") != nullptr;
  s->scheduler = std::thread([s] { s->schedule_loop(); });
  for (int i = 0; i < kLargeWorkers; ++i) s->workers.emplace_back([s] { s->large_worker(); });
  s->workers.emplace_back([s] { s->batch_worker(); });
  *out = s;
  return TC_OK;
}

int tc_serve_register(tc_server* s, const tc_csr_view* csr, uint64_t* graph_id) {
  if (!s || !csr || !graph_id) return fail(TC_ERR_INVALID_ARG, "tc_serve_register: NULL argument");
  auto res = std::make_unique<Resident>();
  TC_CUDA(cudaStreamCreateWithFlags(&res->stream, cudaStreamNonBlocking));
  int st = tc_graph_create(csr, TC_GRAPH_VALIDATE, res->stream, &res->g);
  // levels and cover edges are computed now and stay cached
  int64_t h = 0;
  if (st == TC_OK) st = tc_cover_edges(res->g, nullptr, 0, &h);
  if (st != TC_OK) {
    tc_graph_destroy(res->g);
    cudaStreamDestroy(res->stream);
    return st;
  }
  res->num_cover = h;
  res->bytes = csr_bytes(csr->n, csr->nnz) + (size_t)csr->nnz * 8 + (size_t)csr->n * 40 +
               (size_t)h * 8;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->resident_bytes + res->bytes > s->cfg.hbm_budget_bytes) {
    tc_graph_destroy(res->g);
    cudaStreamDestroy(res->stream);
    return fail(TC_ERR_OOM, "tc_serve_register: graph needs %zu bytes, budget left %zu",
                res->bytes, s->cfg.hbm_budget_bytes - s->resident_bytes);
  }
  s->resident_bytes += res->bytes;
  *graph_id = s->next_graph++;
  s->residents[*graph_id] = std::move(res);
  return TC_OK;
}

int tc_serve_submit(tc_server* s, const tc_csr_view* csr_or_null, uint64_t graph_id, int mode,
                    uint64_t* ticket) {
  if (!s || !ticket) return fail(TC_ERR_INVALID_ARG, "tc_serve_submit: NULL argument");
  if (mode != TC_MODE_COVER && mode != TC_MODE_PLAIN)
    return fail(TC_ERR_INVALID_ARG, "tc_serve_submit: unknown mode %d", mode);
  auto r = std::make_shared<Request>();
  r->mode = mode;
  if (csr_or_null) {
    const tc_csr_view& v = *csr_or_null;
    if (!v.offsets || v.nnz < 0 || (v.nnz > 0 && !v.cols))
      return fail(TC_ERR_INVALID_ARG, "tc_serve_submit: NULL arrays or nnz < 0");
    if (s->cfg.borrow_views) {
      r->view = v;  // the caller keeps the arrays until the request is done
    } else {
      // the request keeps its own host copy, so the caller's buffers are free
      // as soon as this returns
      r->off.resize((size_t)v.n + 1);
      r->cols.resize((size_t)v.nnz);
      if (is_device_ptr(v.offsets)) {
        TC_CUDA(cudaMemcpy(r->off.data(), v.offsets, sizeof(int64_t) * r->off.size(),
                           cudaMemcpyDeviceToHost));
      } else {
        memcpy(r->off.data(), v.offsets, sizeof(int64_t) * r->off.size());
      }
      if (v.nnz > 0) {
        if (is_device_ptr(v.cols)) {
          TC_CUDA(cudaMemcpy(r->cols.data(), v.cols, sizeof(uint32_t) * r->cols.size(),
                             cudaMemcpyDeviceToHost));
        } else {
          memcpy(r->cols.data(), v.cols, sizeof(uint32_t) * r->cols.size());
        }
      }
      r->view = tc_csr_view{r->off.data(), r->cols.data(), v.n, v.nnz, 0};
    }
    r->n = v.n;
    r->small = v.n <= kServeSmallN && v.nnz <= kServeSmallNnz;
    r->est_bytes = r->small ? 2 * csr_bytes(v.n, v.nnz) + (size_t)v.n * 16
                            : one_shot_bytes(v.n, v.nnz);
  } else {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->residents.find(graph_id);
    if (it == s->residents.end())
      return fail(TC_ERR_NOT_FOUND, "tc_serve_submit: unknown graph id %llu",
                  (unsigned long long)graph_id);
    r->graph_id = graph_id;
    r->est_bytes = (size_t)it->second->num_cover * 48 + (size_t)it->second->g->n * 40;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stopping) return fail(TC_ERR_CANCELLED, "tc_serve_submit: server is shutting down");
  if (r->est_bytes + s->resident_bytes > s->cfg.hbm_budget_bytes)
    return fail(TC_ERR_OOM, "tc_serve_submit: request needs ~%zu bytes, above the budget",
                r->est_bytes);
  if ((int32_t)(s->queue_small.size() + s->queue_large.size()) >= s->cfg.queue_capacity)
    return fail(TC_ERR_AGAIN, "tc_serve_submit: queue full");
  r->ticket = s->next_ticket++;
  r->t_submit = Clock::now();
  s->tickets[r->ticket] = r;
  (r->small ? s->queue_small : s->queue_large).push_back(r);
  *ticket = r->ticket;
  s->cv_sched.notify_all();
  return TC_OK;
}

int tc_serve_poll(tc_server* s, uint64_t ticket, int* done, uint64_t* count, int* status) {
  if (!s || !done) return fail(TC_ERR_INVALID_ARG, "tc_serve_poll: NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->tickets.find(ticket);
  if (it == s->tickets.end())
    return fail(TC_ERR_NOT_FOUND, "tc_serve_poll: unknown ticket %llu", (unsigned long long)ticket);
  const Request& r = *it->second;
  *done = r.done ? 1 : 0;
  if (r.done) {
    if (count) *count = r.count;
    if (status) *status = r.status;
    s->tickets.erase(it);  // a finished ticket is reported once
  }
  return TC_OK;
}

int tc_serve_destroy(tc_server* s) {
  if (!s) return TC_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stopping = true;
    for (auto* q : {&s->queue_small, &s->queue_large, &s->ready_small, &s->ready_large})
      for (auto& r : *q) {
        r->status = TC_ERR_CANCELLED;
        r->done = true;
      }
  }
  s->cv_sched.notify_all();
  s->cv_work.notify_all();
  if (s->scheduler.joinable()) s->scheduler.join();
  for (auto& t : s->workers)
    if (t.joinable()) t.join();
  if (s->tracing) {
    if (FILE* f = fopen(getenv("TC_SERVE_TRACE"), "w")) {
      for (const auto& r : s->trace) fprintf(f, "%c %.6f %.6f %zu\n", r.kind, r.t0, r.t1, r.nreq);
      fclose(f);
    }
  }
  for (auto& kv : s->residents) {
    tc_graph_destroy(kv.second->g);
    cudaStreamDestroy(kv.second->stream);
  }
  delete s;
  return TC_OK;
}

}  // extern "C"
