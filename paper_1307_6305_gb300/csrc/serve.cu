// serve.cu -- a continuous-batching solve server.
//
// Requests (a registered graph + one right-hand side) arrive at any time.
// `max_active` worker threads (slots) take work from a FIFO queue as soon as
// a slot and device memory are free.  A worker takes the oldest request whose
// graph is idle together with every other queued request for that graph with
// the same tolerance, up to `batch_max`, and solves them as one
// multi-right-hand-side solve on the graph's resident hierarchy: requests
// that arrived while the graph was busy share the next sweep over its levels
// instead of taking turns.  A graph without a resident hierarchy is set up
// first, after evicting least-recently-used idle hierarchies until its bytes
// fit under the memory cap.  Every resident graph owns a CUDA stream, so
// solves of different graphs overlap on the device.  A lone request runs the
// single-right-hand-side path; a batch runs the block kernels at the
// smallest power-of-two width that holds it (a captured graph per width),
// with per-column Krylov scalars, so each result meets its own tolerance
// whatever shares its block.  With batch_max <= 1 requests for one graph
// take turns on the single-right-hand-side path.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <cmath>
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
  int width = 0;                             // block width of batched solves (0: no batching)
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
  int64_t solves = 0, setup_retries = 0;     // solve calls (a batch is one); setups redone to stay under the cap
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

// finish every request of a batch (under the lock)
void complete(amg_server_s *s, Request *const *rs, int nr, amg_status st, const std::string &err) {
  const Clock::time_point now = Clock::now();
  for (int c = 0; c < nr; ++c) {
    Request *r = rs[c];
    if (r->status == AMG_OK) r->status = st;
    if (r->err.empty()) r->err = err;
    r->finished = now;
    r->done = true;
  }
  s->completed += nr;
}

void worker(amg_server_s *s) {
  cudaSetDevice(s->device);
  const int bmax = std::max(1, std::min(s->cfg.batch_max, amg::kMaxBatchServe));
  for (;;) {
    std::vector<int64_t> batch;
    GraphEntry *g = nullptr;
    bool need_setup = false;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      for (;;) {
        if (s->stop) return;
        // the oldest queued request whose graph is idle and fits ...
        int64_t gid = 0;
        double tol = 0.0;
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
          g = &ge;
          gid = r.graph;
          tol = r.tol;
          break;
        }
        if (g) {
          // ... with the other queued requests of its graph and tolerance
          for (auto it = s->queue.begin(); it != s->queue.end() && (int)batch.size() < bmax;) {
            const Request &r = s->requests[*it];
            if (r.graph == gid && r.tol == tol) {
              batch.push_back(*it);
              it = s->queue.erase(it);
            } else {
              ++it;
            }
          }
          break;
        }
        s->cv_work.wait(lk);
      }
      ++s->active;
      s->peak_active = std::max(s->peak_active, s->active);
    }
    const int nr = (int)batch.size();
    std::vector<Request *> rs(nr);
    {
      std::lock_guard<std::mutex> lk(s->mu);
      for (int c = 0; c < nr; ++c) rs[c] = &s->requests[batch[c]];
    }
    amg_status st = AMG_OK;
    std::string err;
    bool retry = false;
    if (need_setup) {
      if (!g->stream) cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking);
      amg_handle h = nullptr;
      st = amg_setup(g->n, g->rowptr.data(), g->col.data(), g->w.data(), g->has_d ? g->d.data() : nullptr,
                     &s->cfg.opt, AMG_MEM_HOST, g->stream, &h);
      if (st != AMG_OK) err = amg_last_error(nullptr);
      // the block buffers (for the widest batch) are part of the
      // hierarchy's size: made now, before it is measured
      if (st == AMG_OK && s->width > 0) {
        st = amg::prepare_batched(h, s->width);
        if (st == AMG_OK && cudaStreamSynchronize(g->stream) != cudaSuccess) st = amg::fail(AMG_ERR_CUDA, "setup");
        if (st != AMG_OK) {
          err = amg::thread_error();
          amg_free(h);
          h = nullptr;
        }
      }
      std::lock_guard<std::mutex> lk(s->mu);
      s->resident_bytes -= g->bytes;  // the reservation
      if (st == AMG_OK) {
        g->measured = h->arena.bytes;
        ++s->setups;
        if (g->measured > s->cfg.mem_cap_bytes) {
          // this hierarchy alone exceeds the cap: the requests fail
          amg_free(h);
          g->bytes = 0;
          st = AMG_ERR_OOM;
          err = "the hierarchy needs " + std::to_string(g->measured) + " device bytes, more than mem_cap_bytes = " +
                std::to_string(s->cfg.mem_cap_bytes);
        } else if (!make_room(s, g->measured)) {
          // larger than its reservation and the difference cannot be freed
          // now (the other resident hierarchies are busy): give the memory
          // back and queue the requests again at the front; the next attempt
          // reserves the measured size
          amg_free(h);
          g->bytes = 0;
          retry = true;
          ++s->setup_retries;
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
    if (retry) {
      std::lock_guard<std::mutex> lk(s->mu);
      for (int c = nr - 1; c >= 0; --c) s->queue.push_front(batch[c]);
      g->busy = false;
      --s->active;
      s->cv_work.notify_all();
      continue;
    }
    if (st == AMG_OK) {
      for (Request *r : rs) {
        r->x.assign((size_t)g->n, 0.0);
        memset(&r->info, 0, sizeof(r->info));
      }
      const auto t0 = Clock::now();
      if (nr == 1) {
        // one request: the single-right-hand-side path (its own kernels,
        // the fastest for one vector)
        st = amg_solve(g->h, rs[0]->rhs.data(), rs[0]->x.data(), 1, g->n, rs[0]->tol, &rs[0]->info);
        if (st != AMG_OK && st != AMG_ERR_NOT_CONVERGED && st != AMG_ERR_BREAKDOWN) {
          err = amg_last_error(g->h);
        } else if (st != AMG_OK) {
          rs[0]->status = st;
          rs[0]->err = amg_last_error(g->h);
          st = AMG_OK;
        }
      } else {
        // a batch: the block path at the smallest power-of-two width that
        // holds it
        std::vector<const double *> bp(nr);
        std::vector<double *> xp(nr);
        std::vector<amg::ColumnReport> cols(nr);
        for (int c = 0; c < nr; ++c) {
          bp[c] = rs[c]->rhs.data();
          xp[c] = rs[c]->x.data();
        }
        int width = 1;
        while (width < nr) width <<= 1;
        st = amg::solve_host_columns(g->h, bp.data(), xp.data(), nr, rs[0]->tol, width, cols.data());
        if (st != AMG_OK) err = amg::thread_error();
        const double ms = std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
        for (int c = 0; c < nr && st == AMG_OK; ++c) {
          amg_info &inf = rs[c]->info;
          inf.iterations = cols[c].iterations;
          inf.converged = cols[c].converged ? 1 : 0;
          inf.rel_residual = cols[c].rel_residual;
          inf.true_rel_residual = cols[c].true_rel_residual;
          inf.n_levels = g->h->L;
          inf.grid_complexity = g->h->grid_complexity;
          inf.op_complexity = g->h->op_complexity;
          inf.setup_ms = g->h->setup_ms;
          inf.solve_ms = ms;
          if (cols[c].breakdown) {
            rs[c]->status = AMG_ERR_BREAKDOWN;
            rs[c]->err = "flexible CG breakdown";
          } else if (!cols[c].converged) {
            rs[c]->status = AMG_ERR_NOT_CONVERGED;
            rs[c]->err = "max_iters reached before tol";
          }
        }
      }
    }
    {
      std::lock_guard<std::mutex> lk(s->mu);
      ++s->solves;
      complete(s, rs.data(), nr, st, err);
      g->busy = false;
      g->last_used = ++s->clock;
      --s->active;
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
  if (cfg->batch_max < 0 || cfg->batch_max > amg::kMaxBatchServe)
    return fail(AMG_ERR_INVALID_ARG, "batch_max must be in [0, 32]");
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || count == 0) {
    cudaGetLastError();
    return fail(AMG_ERR_CUDA, "no usable CUDA device");
  }
  amg_server_s *s = new amg_server_s();
  s->cfg = *cfg;
  if (cfg->batch_max >= 2) {  // block width: the smallest power of two >= batch_max
    s->width = 1;
    while (s->width < cfg->batch_max) s->width <<= 1;
  }
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
    // refused here rather than in the solve, where it would fail the other
    // requests sharing its block
    double ss = 0.0;
    for (int64_t i = 0; i < it->second.n; ++i) ss += rhs[i] * rhs[i];
    if (!std::isfinite(ss))
      return fail(AMG_ERR_INVALID_ARG, "right-hand side has a non-finite entry or a norm beyond the fp64 range");
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
  out->solves = s->solves;
  out->setup_retries = s->setup_retries;
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
