// Request server (truss_serve_*): continuous batching of truss decompositions.
//
// Worker threads, each owning a context (device workspace) and a CUDA stream,
// take requests from one FIFO.  A worker admits the request at the head of
// the queue when the projected device footprint of everything admitted and
// unfinished, plus this request, stays within the budget and the in-flight
// cap allows it; if the head is small (<= batch_rows rows) the worker also
// takes the small requests queued behind it (up to max_batch, same budget
// rule) and decomposes them together as a disjoint union in one batched run.
// Requests that arrive while others are on the GPU are admitted as soon as
// workers and memory free up, and runs of different workers overlap on the
// device through their separate streams.  Each request's result is exactly
// that of a decomposition of the request alone (truss numbers of a disjoint
// union are those of its components, Definition 2).
//
// The projection behind admission cannot know a graph's triangle count, so
// each run's workspace is capped at twice the projected footprint of its
// requests (the context's arena refuses to hand out more; the pipeline
// first falls back to its lower-memory list layouts).  A run that still
// needs more fails with TRUSS_ENOMEM without taking memory from the others;
// its requests are then queued again at the head, once each, with the whole
// budget as their footprint, so each runs alone with the whole budget as its
// cap and either completes or fails alone.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "engine.h"

namespace tr {
int decompose_batch_counts(truss_ctx *ctx, int32_t G, const int64_t *n, const int64_t *row_off,
                           const int32_t *src, const int32_t *dst, int32_t *support_out,
                           int32_t *truss_out, int32_t *kmax_out, cudaStream_t s,
                           int64_t *graph_m, int64_t *graph_tri);
int ctx_device(truss_ctx *ctx);
const truss_opts *ctx_opts(truss_ctx *ctx);
void ctx_trim(truss_ctx *ctx, size_t max_bytes);
void ctx_set_limit(truss_ctx *ctx, size_t bytes);
}  // namespace tr

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Request {
  uint64_t id = 0;
  int64_t n = 0, rows = 0;
  const int32_t *src = nullptr, *dst = nullptr;
  int64_t fp = 0;
  Clock::time_point t_submit, t_start, t_done;
  bool done = false;
  bool retried = false;  // queued again after a run that ran out of its cap
  int rc = TRUSS_OK;
  std::vector<int32_t> sup, tr;
  truss_req_stats st{};
};

}  // namespace

struct truss_server {
  int device = 0;
  truss_opts copts{};
  truss_serve_opts o{};
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request *> pending;
  std::unordered_map<uint64_t, Request *> reqs;
  std::vector<std::thread> workers;
  int64_t inflight_fp = 0;
  int inflight = 0;
  bool stopping = false;
  uint64_t next_id = 1;
  // statistics
  int64_t submitted = 0, admitted = 0, rejected = 0, completed = 0, failed = 0, edges = 0;
  int64_t retried = 0;
  int64_t launches = 0;
  std::vector<double> lat_ms;
  Clock::time_point first_submit, last_done;
  bool have_first = false;
  int start_error = TRUSS_OK;
};

namespace {

// Run one job (one request alone, or a batch of small ones) on the worker's
// context; fills each request's results and per-request statistics.
void run_job(truss_ctx *ctx, cudaStream_t st, std::vector<Request *> &job, int32_t **dsrc,
             int32_t **ddst, int64_t *dcap) {
  const Clock::time_point t0 = Clock::now();
  for (Request *r : job) {
    r->t_start = t0;
    r->sup.resize((size_t)std::max<int64_t>(r->rows, 1));
    r->tr.resize((size_t)std::max<int64_t>(r->rows, 1));
  }
  if (job.size() == 1) {
    Request *r = job[0];
    int32_t kmax = 0;
    r->rc = truss_decompose(ctx, r->n, r->rows, r->src, r->dst, r->sup.data(), r->tr.data(),
                            &kmax, st);
    truss_run_stats rs{};
    truss_last_stats(ctx, &rs);
    r->st.m = rs.m;
    r->st.triangles = rs.triangles;
    r->st.kmax = kmax;
    r->st.batched = 1;
  } else {
    const int32_t G = (int32_t)job.size();
    std::vector<int64_t> ns(G), off(G + 1, 0), gm(G), gt(G);
    std::vector<int32_t> kmax(G);
    for (int32_t g = 0; g < G; g++) {
      ns[g] = job[g]->n;
      off[g + 1] = off[g] + job[g]->rows;
    }
    const int64_t R = off[G];
    int rc = TRUSS_OK;
    if (R > *dcap) {
      cudaFree(*dsrc);
      cudaFree(*ddst);
      *dsrc = *ddst = nullptr;
      *dcap = 0;
      if (cudaMalloc(dsrc, sizeof(int32_t) * R) != cudaSuccess ||
          cudaMalloc(ddst, sizeof(int32_t) * R) != cudaSuccess) {
        cudaGetLastError();
        rc = TRUSS_ENOMEM;
      } else {
        *dcap = R;
      }
    }
    for (int32_t g = 0; g < G && rc == TRUSS_OK; g++) {
      const int64_t rw = job[g]->rows;
      if (rw == 0) continue;
      if (cudaMemcpyAsync(*dsrc + off[g], job[g]->src, sizeof(int32_t) * rw, cudaMemcpyDefault,
                          st) != cudaSuccess ||
          cudaMemcpyAsync(*ddst + off[g], job[g]->dst, sizeof(int32_t) * rw, cudaMemcpyDefault,
                          st) != cudaSuccess)
        rc = TRUSS_ECUDA;
    }
    std::vector<int32_t> hs((size_t)std::max<int64_t>(R, 1)), ht((size_t)std::max<int64_t>(R, 1));
    if (rc == TRUSS_OK)
      rc = tr::decompose_batch_counts(ctx, G, ns.data(), off.data(), *dsrc, *ddst, hs.data(),
                                      ht.data(), kmax.data(), st, gm.data(), gt.data());
    for (int32_t g = 0; g < G; g++) {
      Request *r = job[g];
      r->rc = rc;
      if (rc == TRUSS_OK && r->rows > 0) {
        memcpy(r->sup.data(), hs.data() + off[g], sizeof(int32_t) * r->rows);
        memcpy(r->tr.data(), ht.data() + off[g], sizeof(int32_t) * r->rows);
      }
      r->st.m = rc == TRUSS_OK ? gm[g] : 0;
      r->st.triangles = rc == TRUSS_OK ? gt[g] : 0;
      r->st.kmax = rc == TRUSS_OK ? kmax[g] : 0;
      r->st.batched = G;
    }
  }
  const Clock::time_point t1 = Clock::now();
  for (Request *r : job) {
    r->t_done = t1;
    r->st.queue_ms = ms_between(r->t_submit, r->t_start);
    r->st.run_ms = ms_between(r->t_start, t1);
    r->st.total_ms = ms_between(r->t_submit, t1);
  }
}

// True if request r can be admitted now.
bool fits(const truss_server *S, const Request *r, int extra_count, int64_t extra_fp) {
  if (S->inflight + extra_count + 1 > S->o.max_inflight) return false;
  return S->inflight_fp + extra_fp + r->fp <= S->o.hbm_budget_bytes;
}

void worker_main(truss_server *S) {
  truss_ctx *ctx = nullptr;
  cudaStream_t st = nullptr;
  int rc = truss_ctx_create(&ctx, S->device, &S->copts);
  if (rc == TRUSS_OK && cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess)
    rc = TRUSS_ECUDA;
  int32_t *dsrc = nullptr, *ddst = nullptr;
  int64_t dcap = 0;
  for (;;) {
    std::vector<Request *> job;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_work.wait(lk, [&] {
        if (S->pending.empty()) return S->stopping;
        return fits(S, S->pending.front(), 0, 0);
      });
      if (S->pending.empty()) break;  // stopping and drained
      Request *h = S->pending.front();
      S->pending.pop_front();
      job.push_back(h);
      int64_t fp = h->fp;
      if (h->rows <= S->o.batch_rows) {
        while (!S->pending.empty() && (int)job.size() < S->o.max_batch) {
          Request *r = S->pending.front();
          if (r->rows > S->o.batch_rows || !fits(S, r, (int)job.size(), fp)) break;
          S->pending.pop_front();
          job.push_back(r);
          fp += r->fp;
        }
      }
      S->inflight += (int)job.size();
      S->inflight_fp += fp;
      S->admitted += (int64_t)job.size();
      S->launches++;
    }
    if (rc == TRUSS_OK) {
      // workspace cap of this run: twice the projection, or the whole budget
      // for a request queued again after running out of its cap
      size_t cap = 0;
      for (Request *r : job) cap += (size_t)(r->retried ? r->fp : 2 * r->fp);
      tr::ctx_set_limit(ctx, cap);
      run_job(ctx, st, job, &dsrc, &ddst, &dcap);
      // keep the cached workspace within this worker's share of the budget
      tr::ctx_trim(ctx, (size_t)(S->o.hbm_budget_bytes / S->o.streams));
    } else {
      const Clock::time_point t = Clock::now();
      for (Request *r : job) {
        r->rc = rc;
        r->t_start = r->t_done = t;
      }
    }
    {
      std::lock_guard<std::mutex> lk(S->mu);
      for (Request *r : job) {
        S->inflight--;
        S->inflight_fp -= r->fp;
        if (r->rc == TRUSS_ENOMEM && !r->retried) {
          r->retried = true;
          r->fp = S->o.hbm_budget_bytes;  // admitted only when nothing else runs
          r->rc = TRUSS_OK;
          S->retried++;
          S->admitted--;  // counted again when it is admitted alone
          S->pending.push_front(r);
          continue;
        }
        r->done = true;
        if (r->rc == TRUSS_OK) {
          S->completed++;
          S->edges += r->st.m;
          S->lat_ms.push_back(r->st.total_ms);
        } else {
          S->failed++;
        }
        if (r->t_done > S->last_done) S->last_done = r->t_done;
      }
    }
    S->cv_done.notify_all();
    S->cv_work.notify_all();
  }
  cudaFree(dsrc);
  cudaFree(ddst);
  if (st) cudaStreamDestroy(st);
  truss_ctx_destroy(ctx);
}

int take_result(truss_server *S, Request *r, int32_t *support_out, int32_t *truss_out,
                truss_req_stats *st) {
  // called with S->mu held and r->done
  const int rc = r->rc;
  if (rc == TRUSS_OK && r->rows > 0) {
    if (support_out) memcpy(support_out, r->sup.data(), sizeof(int32_t) * r->rows);
    if (truss_out) memcpy(truss_out, r->tr.data(), sizeof(int32_t) * r->rows);
  }
  if (st) *st = r->st;
  S->reqs.erase(r->id);
  delete r;
  return rc;
}

}  // namespace

extern "C" {

int64_t truss_serve_footprint(int64_t n, int64_t rows) {
  if (n < 0 || rows < 0) return 0;
  return 96 * rows + 16 * n + 8 * 96 * rows;
}

int truss_serve_start(truss_ctx *ctx, const truss_serve_opts *opts, truss_server **out) {
  if (!ctx || !out) return TRUSS_EINVAL;
  *out = nullptr;
  truss_server *S = new (std::nothrow) truss_server();
  if (!S) return TRUSS_ENOMEM;
  S->device = tr::ctx_device(ctx);
  S->copts = *tr::ctx_opts(ctx);
  S->copts.profile = 0;
  S->copts.count_bytes = 0;
  if (opts) S->o = *opts;
  if (S->o.max_inflight <= 0) S->o.max_inflight = 256;
  if (S->o.streams <= 0) S->o.streams = 4;
  if (S->o.batch_rows <= 0) S->o.batch_rows = 65536;
  if (S->o.max_batch <= 0) S->o.max_batch = 512;
  if (S->o.max_queue <= 0) S->o.max_queue = 1 << 20;
  if (S->o.hbm_budget_bytes <= 0) {
    size_t fr = 0, tot = 0;
    if (cudaSetDevice(S->device) != cudaSuccess || cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      cudaGetLastError();
      delete S;
      return TRUSS_ECUDA;
    }
    // runs use at most twice their projection, plus the workspace each
    // worker keeps cached between runs (at most budget / streams)
    S->o.hbm_budget_bytes = (int64_t)(fr / 3);
  }
  try {
    for (int i = 0; i < S->o.streams; i++) S->workers.emplace_back(worker_main, S);
  } catch (...) {
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->stopping = true;
    }
    S->cv_work.notify_all();
    for (auto &t : S->workers) t.join();
    delete S;
    return TRUSS_ENOMEM;
  }
  *out = S;
  return TRUSS_OK;
}

int truss_serve_submit(truss_server *S, int64_t n, int64_t rows, const int32_t *src,
                       const int32_t *dst, uint64_t *ticket) {
  if (!S || !ticket || n < 0 || n >= ((int64_t)1 << 31) || rows < 0 ||
      rows >= ((int64_t)1 << 31) || (rows > 0 && (!src || !dst)) || (rows > 0 && n == 0))
    return TRUSS_EINVAL;
  Request *r = new (std::nothrow) Request();
  if (!r) return TRUSS_ENOMEM;
  r->n = n;
  r->rows = rows;
  r->src = src;
  r->dst = dst;
  r->fp = truss_serve_footprint(n, rows);
  r->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->submitted++;
    if (!S->have_first) {
      S->first_submit = r->t_submit;
      S->last_done = r->t_submit;
      S->have_first = true;
    }
    if (S->stopping) {
      delete r;
      return TRUSS_ESHUTDOWN;
    }
    if (r->fp > S->o.hbm_budget_bytes || (int64_t)S->pending.size() >= S->o.max_queue) {
      S->rejected++;
      delete r;
      return TRUSS_EBUSY;
    }
    r->id = S->next_id++;
    S->reqs[r->id] = r;
    S->pending.push_back(r);
    *ticket = r->id;
  }
  S->cv_work.notify_one();
  return TRUSS_OK;
}

int truss_serve_poll(truss_server *S, uint64_t ticket, int32_t *support_out, int32_t *truss_out,
                     truss_req_stats *st) {
  if (!S) return TRUSS_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return TRUSS_EINVAL;
  if (!it->second->done) return TRUSS_EAGAIN;
  return take_result(S, it->second, support_out, truss_out, st);
}

int truss_serve_wait(truss_server *S, uint64_t ticket, int64_t timeout_ns, int32_t *support_out,
                     int32_t *truss_out, truss_req_stats *st) {
  if (!S) return TRUSS_EINVAL;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return TRUSS_EINVAL;
  Request *r = it->second;
  auto ready = [&] { return r->done; };
  if (timeout_ns < 0) {
    S->cv_done.wait(lk, ready);
  } else if (!S->cv_done.wait_for(lk, std::chrono::nanoseconds(timeout_ns), ready)) {
    return TRUSS_EAGAIN;
  }
  return take_result(S, r, support_out, truss_out, st);
}

int truss_serve_stop(truss_server *S, truss_serve_stats *st) {
  if (!S) return TRUSS_OK;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stopping = true;
  }
  S->cv_work.notify_all();
  for (auto &t : S->workers) t.join();
  if (st) {
    truss_serve_stats o{};
    o.submitted = S->submitted;
    o.admitted = S->admitted;
    o.rejected = S->rejected;
    o.completed = S->completed;
    o.failed = S->failed;
    o.edges = S->edges;
    o.launches = S->launches;
    o.retried = S->retried;
    std::vector<double> l = S->lat_ms;
    std::sort(l.begin(), l.end());
    if (!l.empty()) {
      auto pct = [&](double p) {
        size_t i = (size_t)(p * (double)(l.size() - 1) + 0.5);
        return l[std::min(i, l.size() - 1)];
      };
      o.p50_ms = pct(0.50);
      o.p99_ms = pct(0.99);
      double sum = 0;
      for (double x : l) sum += x;
      o.mean_ms = sum / (double)l.size();
      o.max_ms = l.back();
    }
    o.wall_s = S->have_first ? ms_between(S->first_submit, S->last_done) / 1e3 : 0.0;
    o.edges_per_s = o.wall_s > 0 ? (double)o.edges / o.wall_s : 0.0;
    *st = o;
  }
  for (auto &kv : S->reqs) delete kv.second;
  delete S;
  return TRUSS_OK;
}

}  // extern "C"
