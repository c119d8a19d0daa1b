// serve.cu -- a continuous-batching solve server.
//
// Requests (a registered graph + one right-hand side) arrive at any time.
// `max_active` worker threads (slots) take requests from a FIFO queue as soon
// as a slot and device memory are free: a request whose graph's hierarchy is
// resident starts at once; otherwise the hierarchy is set up first, after
// evicting least-recently-used idle hierarchies until the estimated bytes fit
// under the memory cap.  Hierarchies stay resident between requests.  Every
// resident graph owns a CUDA stream, so solves of different graphs overlap
// on the device; requests for one graph take turns on its hierarchy (a
// handle is not shared by two solves at once).  All kernels are
// deterministic, so a request's result does not depend on what else runs.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "common.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct GraphEntry {
  int64_t n = 0;
  std::vector<int64_t> rowptr;
  std::vector<int32_t> col;
  std::vector<double> w, d;
  bool has_d = false;
  amg_handle h = nullptr;      // resident hierarchy or null
  cudaStream_t stream = nullptr;
  size_t bytes = 0;            // device bytes of the resident hierarchy (estimate before setup)
  size_t measured = 0;         // arena bytes of this graph's last hierarchy (0: never set up)
  bool busy = false;           // a solve is using the hierarchy
  int64_t last_used = 0;
};

struct Request {
  int64_t ticket = 0;
  int64_t graph = 0;
  std::vector<double> rhs, x;
  double tol = 1e-8;
  Clock::time_point submitted, finished;
  bool done = false;
  amg_status status = AMG_OK;
  amg_info info{};
  std::string err;
};

// device bytes to reserve for a graph's hierarchy: the measured size once it
// has been set up, else an estimate (all levels ~1.2x the fine level: CSR and
// SELL copies of the matrix, ~25 work vectors per level, ~20 outer vectors)
size_t reserve_bytes(const GraphEntry &g) {
  if (g.measured) return g.measured;
  const double nnz = (double)g.rowptr.back(), n = (double)g.n;
  return (size_t)(1.2 * (nnz * 28.0 + n * 200.0) + n * 160.0) + ((size_t)1 << 20);
}

}  // namespace

struct amg_server_s {
  amg_server_config cfg{};
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::map<int64_t, GraphEntry> graphs;
  std::deque<int64_t> queue;                 // tickets waiting for a slot
  std::map<int64_t, Request> requests;
  std::vector<std::thread> workers;
  int64_t next_graph = 1, next_ticket = 1, clock = 0;
  size_t resident_bytes = 0, peak_bytes = 0;
  int active = 0, peak_active = 0;
  int64_t setups = 0, evictions = 0, completed = 0;
  bool stop = false;
  int device = 0;
};

namespace {

// evict idle resident hierarchies (least recently used first) until `need`
// more bytes fit under the cap; returns false if that is impossible now
bool make_room(amg_server_s *s, size_t need) {
  while (s->resident_bytes + need > s->cfg.mem_cap_bytes) {
    GraphEntry *victim = nullptr;
    for (auto &kv : s->graphs) {
      GraphEntry &g = kv.second;
      if (g.h && !g.busy && (!victim || g.last_used < victim->last_used)) victim = &g;
    }
    if (!victim) return false;
    amg_free(victim->h);
    victim->h = nullptr;
    s->resident_bytes -= victim->bytes;
    ++s->evictions;
  }
  return true;
}

void worker(amg_server_s *s) {
  cudaSetDevice(s->device);
  for (;;) {
    int64_t ticket = 0;
    GraphEntry *g = nullptr;
    bool need_setup = false;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      for (;;) {
        if (s->stop) return;
        // first queued request whose graph is idle and fits
        for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
          Request &r = s->requests[*it];
          GraphEntry &ge = s->graphs[r.graph];
          if (ge.busy) continue;
          if (!ge.h) {
            ge.bytes = reserve_bytes(ge);
            // With no other solve running and every idle hierarchy evicted,
            // a graph that still does not fit is set up anyway: the check of
            // its real size after the setup decides (an estimate may be high).
            if (!make_room(s, ge.bytes) && s->active > 0) continue;
            s->resident_bytes += ge.bytes;  // reserved before the setup
            need_setup = true;
          }
          ge.busy = true;
          ge.last_used = ++s->clock;
          ticket = *it;
          g = &ge;
          s->queue.erase(it);
          break;
        }
        if (ticket) break;
        s->cv_work.wait(lk);
      }
      ++s->active;
      s->peak_active = std::max(s->peak_active, s->active);
    }
    Request *r;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      r = &s->requests[ticket];
    }
    amg_status st = AMG_OK;
    std::string err;
    if (need_setup) {
      if (!g->stream) cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking);
      amg_handle h = nullptr;
      st = amg_setup(g->n, g->rowptr.data(), g->col.data(), g->w.data(), g->has_d ? g->d.data() : nullptr,
                     &s->cfg.opt, AMG_MEM_HOST, g->stream, &h);
      if (st != AMG_OK) err = amg_last_error(nullptr);
      std::lock_guard<std::mutex> lk(s->mu);
      s->resident_bytes -= g->bytes;
      if (st == AMG_OK) {
        g->measured = h->arena.bytes;
        ++s->setups;
        if (g->measured > s->cfg.mem_cap_bytes) {
          // this hierarchy alone exceeds the cap: the request fails
          amg_free(h);
          g->bytes = 0;
          st = AMG_ERR_OOM;
          err = "the hierarchy needs " + std::to_string(g->measured) + " device bytes, more than mem_cap_bytes = " +
                std::to_string(s->cfg.mem_cap_bytes);
        } else {
          g->h = h;
          g->bytes = g->measured;
          s->resident_bytes += g->bytes;
          s->peak_bytes = std::max(s->peak_bytes, s->resident_bytes);
        }
      } else {
        g->bytes = 0;
      }
    }
    if (st == AMG_OK) {
      r->x.assign((size_t)g->n, 0.0);
      memset(&r->info, 0, sizeof(r->info));
      st = amg_solve(g->h, r->rhs.data(), r->x.data(), 1, g->n, r->tol, &r->info);
      if (st != AMG_OK) err = amg_last_error(g->h);
    }
    {
      std::lock_guard<std::mutex> lk(s->mu);
      r->status = st;
      r->err = err;
      r->finished = Clock::now();
      r->done = true;
      g->busy = false;
      g->last_used = ++s->clock;
      --s->active;
      ++s->completed;
    }
    s->cv_done.notify_all();
    s->cv_work.notify_all();
  }
}

}  // namespace

using amg::fail;

extern "C" {

amg_status amg_server_create(const amg_server_config *cfg, amg_server *out) {
  if (!cfg || !out) return fail(AMG_ERR_INVALID_ARG, "cfg or out is NULL");
  *out = nullptr;
  if (cfg->max_active < 1 || cfg->max_active > 64 || cfg->mem_cap_bytes < ((size_t)1 << 20))
    return fail(AMG_ERR_INVALID_ARG, "max_active must be in [1, 64] and mem_cap_bytes >= 1 MiB");
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || count == 0) {
    cudaGetLastError();
    return fail(AMG_ERR_CUDA, "no usable CUDA device");
  }
  amg_server_s *s = new amg_server_s();
  s->cfg = *cfg;
  cudaGetDevice(&s->device);
  for (int i = 0; i < cfg->max_active; ++i) s->workers.emplace_back(worker, s);
  *out = s;
  return AMG_OK;
}

amg_status amg_server_add_graph(amg_server s, int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                                const double *w, const double *d, int64_t *graph_id) {
  if (!s || !graph_id || n < 1 || !row_ptr) return fail(AMG_ERR_INVALID_ARG, "server, n, row_ptr or graph_id invalid");
  const int64_t nnz = row_ptr[n];
  if (row_ptr[0] != 0 || nnz < 0 || (nnz > 0 && (!col_idx || !w)))
    return fail(AMG_ERR_INVALID_ARG, "row_ptr/col_idx/w invalid");
  GraphEntry g;
  g.n = n;
  g.rowptr.assign(row_ptr, row_ptr + n + 1);
  g.col.assign(col_idx, col_idx + nnz);
  g.w.assign(w, w + nnz);
  if (d) {
    g.d.assign(d, d + n);
    g.has_d = true;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  *graph_id = s->next_graph++;
  s->graphs[*graph_id] = std::move(g);
  return AMG_OK;
}

amg_status amg_server_submit(amg_server s, int64_t graph_id, const double *rhs, double tol, int64_t *ticket) {
  if (!s || !rhs || !ticket || !(tol >= 0.0)) return fail(AMG_ERR_INVALID_ARG, "server, rhs, tol or ticket invalid");
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->graphs.find(graph_id);
    if (it == s->graphs.end()) return fail(AMG_ERR_INVALID_ARG, "unknown graph id");
    Request r;
    r.ticket = s->next_ticket++;
    r.graph = graph_id;
    r.rhs.assign(rhs, rhs + it->second.n);
    r.tol = tol;
    r.submitted = Clock::now();
    *ticket = r.ticket;
    s->requests[r.ticket] = std::move(r);
    s->queue.push_back(*ticket);
  }
  s->cv_work.notify_all();
  return AMG_OK;
}

static amg_status take(amg_server s, Request &r, double *x, amg_info *info, double *latency_ms) {
  if (x) memcpy(x, r.x.data(), sizeof(double) * r.x.size());
  if (info) {
    double *hist = info->history;
    const int cap = info->history_cap;
    *info = r.info;
    info->history = hist;
    info->history_cap = cap;
    info->history_len = 0;
  }
  if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r.finished - r.submitted).count();
  const amg_status st = r.status;
  if (st != AMG_OK) fail(st, r.err);
  s->requests.erase(r.ticket);
  s->cv_done.notify_all();  // other waiters on this ticket see it released
  return st;
}

amg_status amg_server_poll(amg_server s, int64_t ticket, double *x, amg_info *info, int *done, double *latency_ms) {
  if (!s || !done) return fail(AMG_ERR_INVALID_ARG, "server or done is NULL");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->requests.find(ticket);
  if (it == s->requests.end()) return fail(AMG_ERR_INVALID_ARG, "unknown ticket");
  *done = it->second.done ? 1 : 0;
  if (!*done) return AMG_OK;
  return take(s, it->second, x, info, latency_ms);
}

amg_status amg_server_wait(amg_server s, int64_t ticket, double *x, amg_info *info, double *latency_ms) {
  if (!s) return fail(AMG_ERR_INVALID_ARG, "server is NULL");
  std::unique_lock<std::mutex> lk(s->mu);
  if (s->requests.find(ticket) == s->requests.end()) return fail(AMG_ERR_INVALID_ARG, "unknown ticket");
  // looked up again after every wake-up: another caller may have taken the
  // ticket (and erased the request) in the meantime
  s->cv_done.wait(lk, [&] {
    auto f = s->requests.find(ticket);
    return f == s->requests.end() || f->second.done;
  });
  auto it = s->requests.find(ticket);
  if (it == s->requests.end()) return fail(AMG_ERR_INVALID_ARG, "the ticket was taken by another caller");
  return take(s, it->second, x, info, latency_ms);
}

amg_status amg_server_stats(amg_server s, amg_server_stats_t *out) {
  if (!s || !out) return fail(AMG_ERR_INVALID_ARG, "server or out is NULL");
  std::lock_guard<std::mutex> lk(s->mu);
  out->resident_bytes = s->resident_bytes;
  out->peak_resident_bytes = s->peak_bytes;
  out->active = s->active;
  out->peak_active = s->peak_active;
  out->queued = (int64_t)s->queue.size();
  out->completed = s->completed;
  out->setups = s->setups;
  out->evictions = s->evictions;
  return AMG_OK;
}

void amg_server_destroy(amg_server s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto &t : s->workers) t.join();
  cudaSetDevice(s->device);
  for (auto &kv : s->graphs) {
    if (kv.second.h) amg_free(kv.second.h);
    if (kv.second.stream) cudaStreamDestroy(kv.second.stream);
  }
  delete s;
}

}  // extern "C"
