// Serving: a continuous-batching request loop over device-resident graphs.
//
// Requests enter per-kind FIFO queues and are admitted while their estimated
// device working set fits in the memory budget beside the requests in flight.
// Score requests (cheap, batched) are admitted first; a maximise request is
// admitted only when a worker is free to run it, so queued maximisations never
// hold memory that waiting score requests could use.
// Admitted score requests wait in their graph's lane; whenever the lane is
// free it takes every waiting request with the same (alpha, L) (up to
// max_batch) and scores them as the columns of one batched SpMM on the lane's
// own stream. Maximize requests run on a small pool of workers, each with its
// own stream and workspace, so their sweeps overlap with the scoring lanes.
// A column's arithmetic never depends on the other columns of its batch, so a
// result is bitwise the same alone and in a mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <thread>
#include <unordered_map>

#include "internal.h"

namespace gw {
namespace {

using Clock = std::chrono::steady_clock;
constexpr int kMaxWorkers = 8;
constexpr size_t kMaxQueue = size_t(1) << 20;

struct Request {
  uint64_t ticket = 0;
  int32_t graph = 0;
  int32_t kind = 0;
  std::vector<int32_t> S;  // internal ids, sorted, unique
  int32_t k = 0;
  int32_t flags = 0;
  Resolved r{};
  int64_t mem = 0;
  Clock::time_point t_submit, t_done;
  bool done = false;
  gedwalk_status status = GEDWALK_OK;
  std::string error;
  double score = 0.0;
  std::vector<int32_t> group;
  std::vector<double> gains;
};
using ReqPtr = std::shared_ptr<Request>;

struct Lane {  // one per graph: batched scoring
  std::deque<ReqPtr> queue;
  bool busy = false;
  cudaStream_t stream = nullptr;
  Workspace ws;
  std::thread th;
};

struct Worker {  // maximize pool
  cudaStream_t stream = nullptr;
  Workspace ws;
  std::thread th;
};

}  // namespace

struct Server {
  std::vector<Graph*> graphs;
  int64_t budget = 0;
  int32_t max_batch = 256;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work;  // lanes / workers wait here
  std::condition_variable cv_done;  // pollers wait here
  std::deque<ReqPtr> pending;       // score requests not yet admitted
  std::deque<ReqPtr> pending_max;   // maximise requests not yet admitted
  std::deque<ReqPtr> max_queue;     // admitted maximize requests
  int32_t max_running = 0;          // admitted maximise requests (queued or running)
  std::unordered_map<uint64_t, ReqPtr> table;
  std::vector<std::unique_ptr<Lane>> lanes;
  std::vector<std::unique_ptr<Worker>> workers;
  uint64_t next_ticket = 1;
  int64_t in_flight = 0, peak = 0;
  int64_t completed = 0, batches = 0, batched_requests = 0;
  bool stop = false;

  // working-set estimates in bytes (accounting for admission)
  int64_t estimate(const Request& q) const {
    const Graph& g = *graphs[q.graph];
    if (q.kind == GEDWALK_REQ_SCORE) return int64_t(g.n) * 8 + int64_t(q.S.size()) * 16 + 64;
    const int64_t es = q.r.fp64 ? 8 : 4;
    return int64_t(g.n) * (es * (q.r.L + 1 + 16) + 8) + 4096;
  }

  void admit_locked() {
    while (!pending.empty()) {  // score requests first (FIFO)
      ReqPtr q = pending.front();
      if (in_flight > 0 && in_flight + q->mem > budget) break;
      pending.pop_front();
      in_flight += q->mem;
      peak = std::max(peak, in_flight);
      lanes[q->graph]->queue.push_back(q);
    }
    while (!pending_max.empty() && max_running < kMaxWorkers) {  // then maximise requests, one per free worker
      ReqPtr q = pending_max.front();
      if (in_flight > 0 && in_flight + q->mem > budget) break;
      pending_max.pop_front();
      in_flight += q->mem;
      peak = std::max(peak, in_flight);
      ++max_running;
      max_queue.push_back(q);
    }
    cv_work.notify_all();
  }

  void finish_locked(const ReqPtr& q) {
    if (q->kind == GEDWALK_REQ_MAXIMIZE) --max_running;
    q->done = true;
    q->t_done = Clock::now();
    in_flight -= q->mem;
    ++completed;
    admit_locked();
    cv_done.notify_all();
  }

  void lane_loop(int gi) {
    cudaSetDevice(device);
    Lane& lane = *lanes[gi];
    Graph& g = *graphs[gi];
    for (;;) {
      std::vector<ReqPtr> batch;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv_work.wait(lk, [&] { return stop || !lane.queue.empty(); });
        if (lane.queue.empty()) return;  // stopping and idle
        const ReqPtr first = lane.queue.front();
        for (auto it = lane.queue.begin(); it != lane.queue.end() && int(batch.size()) < max_batch;) {
          if ((*it)->r.alpha == first->r.alpha && (*it)->r.L == first->r.L) {
            batch.push_back(*it);
            it = lane.queue.erase(it);
          } else {
            ++it;
          }
        }
        lane.busy = true;
      }
      std::vector<int32_t> off(1, 0), mem;
      for (const ReqPtr& q : batch) {
        mem.insert(mem.end(), q->S.begin(), q->S.end());
        off.push_back(static_cast<int32_t>(mem.size()));
      }
      std::vector<double> scores(batch.size());
      Resolved r = batch[0]->r;
      r.fp64 = false;
      r.stream = lane.stream;
      const gedwalk_status st =
          score_batch_impl(g, lane.ws, off.data(), mem.data(), static_cast<int32_t>(batch.size()), r, scores.data());
      const std::string err = st == GEDWALK_OK ? "" : gedwalk_last_error();
      std::lock_guard<std::mutex> lk(mu);
      ++batches;
      batched_requests += static_cast<int64_t>(batch.size());
      for (size_t i = 0; i < batch.size(); ++i) {
        batch[i]->status = st;
        batch[i]->error = err;
        batch[i]->score = scores[i];
        finish_locked(batch[i]);
      }
      lane.busy = false;
    }
  }

  void worker_loop(int wi) {
    cudaSetDevice(device);
    Worker& w = *workers[wi];
    for (;;) {
      ReqPtr q;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv_work.wait(lk, [&] { return stop || !max_queue.empty(); });
        if (max_queue.empty()) return;
        q = max_queue.front();
        max_queue.pop_front();
      }
      Graph& g = *graphs[q->graph];
      Resolved r = q->r;
      r.stream = w.stream;
      std::vector<int32_t> grp(std::max(q->k, 1));
      std::vector<double> gn(std::max(q->k, 1));
      double sc = 0;
      const gedwalk_status st = maximize_impl(g, w.ws, q->k, r, q->flags, {}, grp.data(), gn.data(), &sc);
      const std::string err = st == GEDWALK_OK ? "" : gedwalk_last_error();
      std::lock_guard<std::mutex> lk(mu);
      q->status = st;
      q->error = err;
      q->score = sc;
      grp.resize(q->k);
      gn.resize(q->k);
      q->group = std::move(grp);
      q->gains = std::move(gn);
      finish_locked(q);
    }
  }
};

}  // namespace gw

using namespace gw;

extern "C" {

gedwalk_status gedwalk_serve_create(const gedwalk_graph_t* graphs, int32_t n_graphs, int64_t mem_budget,
                                    int32_t max_batch, gedwalk_server_t* out) {
  if (!graphs || n_graphs < 1 || !out) return fail(GEDWALK_ERR_INVALID, "graphs/out NULL or n_graphs < 1");
  if (mem_budget < 0 || max_batch < 0) return fail(GEDWALK_ERR_INVALID, "negative budget or batch");
  std::unique_ptr<Server> srv(new Server());
  srv->budget = mem_budget > 0 ? mem_budget : (int64_t(1) << 30);
  srv->max_batch = max_batch > 0 ? max_batch : 256;
  GW_CUDA(cudaGetDevice(&srv->device));
  for (int32_t i = 0; i < n_graphs; ++i) {
    if (!graphs[i]) return fail(GEDWALK_ERR_INVALID, "graph %d is NULL", i);
    srv->graphs.push_back(G(graphs[i]));
  }
  for (int32_t i = 0; i < n_graphs; ++i) {
    std::unique_ptr<Lane> lane(new Lane());
    GW_CUDA(cudaStreamCreateWithFlags(&lane->stream, cudaStreamNonBlocking));
    srv->lanes.push_back(std::move(lane));
  }
  for (int i = 0; i < kMaxWorkers; ++i) {
    std::unique_ptr<Worker> w(new Worker());
    GW_CUDA(cudaStreamCreateWithFlags(&w->stream, cudaStreamNonBlocking));
    srv->workers.push_back(std::move(w));
  }
  // the batched path needs each graph's column width tuned and its walk-total table ready
  for (int32_t i = 0; i < n_graphs; ++i) {
    Graph& g = *srv->graphs[i];
    std::lock_guard<std::mutex> lk(g.mu);
    Resolved r;
    GW_TRY(resolve(g, nullptr, 0.0, &r));
    GW_TRY(ensure_totals(g, r.alpha, r.L + 1, nullptr));
    GW_TRY(autotune_batch(g, g.ws, r));
  }
  Server* s = srv.get();
  for (int32_t i = 0; i < n_graphs; ++i) s->lanes[i]->th = std::thread([s, i] { s->lane_loop(i); });
  for (int i = 0; i < kMaxWorkers; ++i) s->workers[i]->th = std::thread([s, i] { s->worker_loop(i); });
  *out = reinterpret_cast<gedwalk_server_t>(srv.release());
  return GEDWALK_OK;
}

gedwalk_status gedwalk_serve_submit(gedwalk_server_t h, int32_t graph, int32_t kind, const int32_t* S,
                                    int32_t s_len_or_k, const gedwalk_params* params, uint64_t* ticket) {
  Server* srv = reinterpret_cast<Server*>(h);
  if (!srv || !ticket) return fail(GEDWALK_ERR_INVALID, "server or ticket is NULL");
  if (graph < 0 || graph >= static_cast<int32_t>(srv->graphs.size()))
    return fail(GEDWALK_ERR_INVALID, "graph index %d out of range", graph);
  if (kind != GEDWALK_REQ_SCORE && kind != GEDWALK_REQ_MAXIMIZE) return fail(GEDWALK_ERR_INVALID, "bad kind");
  Graph& g = *srv->graphs[graph];
  ReqPtr q = std::make_shared<Request>();
  q->graph = graph;
  q->kind = kind;
  gedwalk_params p;
  gedwalk_params_default(&p);
  if (params) p = *params;
  p.stream = 0;
  {
    // resolving may extend the graph's walk-total table: serialise with its other users
    std::lock_guard<std::mutex> lk(g.mu);
    // The walk-total table holds one alpha, the one the server prepared at creation; scoring
    // lanes read it while other requests are submitted, so a request with another alpha is
    // rejected before anything could replace the table under them.
    if (p.alpha < 0.0 || std::isnan(p.alpha)) return fail(GEDWALK_ERR_INVALID, "alpha must be positive (0 = default)");
    const double alpha = p.alpha > 0.0 ? p.alpha : g.alpha_default;
    {
      std::shared_lock<std::shared_mutex> rl(g.tt_lock);
      if (g.tt_rows > 0 && alpha != g.tt_alpha)
        return fail(GEDWALK_ERR_INVALID, "served requests use one alpha per graph (%.17g), not %.17g", g.tt_alpha,
                    alpha);
    }
    if (kind == GEDWALK_REQ_SCORE) {
      GW_TRY(map_group(g, S, s_len_or_k, &q->S));
      GW_TRY(resolve(g, &p, 0.0, &q->r));
      GW_TRY(ensure_totals(g, q->r.alpha, q->r.L + 1, nullptr));
    } else {
      if (s_len_or_k < 0 || s_len_or_k > g.n) return fail(GEDWALK_ERR_INVALID, "k out of range");
      q->k = s_len_or_k;
      q->flags = p.flags;
      const double eps = (p.greedy_eps_rule == GEDWALK_EPS_OVER_K && q->k > 0) ? p.epsilon / q->k : p.epsilon;
      GW_TRY(resolve(g, &p, eps, &q->r));
    }
  }
  std::lock_guard<std::mutex> lk(srv->mu);
  if (srv->stop) return fail(GEDWALK_ERR_BUSY, "server is stopping");
  if (srv->pending.size() + srv->pending_max.size() >= kMaxQueue)
    return fail(GEDWALK_ERR_BUSY, "request queue is full");
  q->mem = srv->estimate(*q);
  q->ticket = srv->next_ticket++;
  q->t_submit = Clock::now();
  srv->table[q->ticket] = q;
  (kind == GEDWALK_REQ_SCORE ? srv->pending : srv->pending_max).push_back(q);
  srv->admit_locked();
  *ticket = q->ticket;
  return GEDWALK_OK;
}

gedwalk_status gedwalk_serve_poll(gedwalk_server_t h, uint64_t ticket, int32_t wait_us, double* score,
                                  int32_t* group, double* gains, double* latency_us, int32_t* done) {
  Server* srv = reinterpret_cast<Server*>(h);
  if (!srv || !done) return fail(GEDWALK_ERR_INVALID, "server or done is NULL");
  std::unique_lock<std::mutex> lk(srv->mu);
  auto it = srv->table.find(ticket);
  if (it == srv->table.end()) return fail(GEDWALK_ERR_NOT_FOUND, "unknown ticket %llu", (unsigned long long)ticket);
  ReqPtr q = it->second;
  if (!q->done && wait_us != 0) {
    if (wait_us < 0)
      srv->cv_done.wait(lk, [&] { return q->done; });
    else
      srv->cv_done.wait_for(lk, std::chrono::microseconds(wait_us), [&] { return q->done; });
  }
  if (!q->done) {
    *done = 0;
    return GEDWALK_OK;
  }
  *done = 1;
  srv->table.erase(ticket);
  if (latency_us)
    *latency_us = std::chrono::duration<double, std::micro>(q->t_done - q->t_submit).count();
  if (q->status != GEDWALK_OK) return fail(q->status, "%s", q->error.c_str());
  if (score) *score = q->score;
  if (q->kind == GEDWALK_REQ_MAXIMIZE) {
    Graph& g = *srv->graphs[q->graph];
    (void)g;
    if (group)
      for (int32_t j = 0; j < q->k; ++j) group[j] = q->group[j];
    if (gains)
      for (int32_t j = 0; j < q->k; ++j) gains[j] = q->gains[j];
  }
  return GEDWALK_OK;
}

gedwalk_status gedwalk_serve_stats(gedwalk_server_t h, int64_t* completed, int64_t* batches, int64_t* batched_requests,
                                   int64_t* peak_bytes) {
  Server* srv = reinterpret_cast<Server*>(h);
  if (!srv) return fail(GEDWALK_ERR_INVALID, "server is NULL");
  std::lock_guard<std::mutex> lk(srv->mu);
  if (completed) *completed = srv->completed;
  if (batches) *batches = srv->batches;
  if (batched_requests) *batched_requests = srv->batched_requests;
  if (peak_bytes) *peak_bytes = srv->peak;
  return GEDWALK_OK;
}

gedwalk_status gedwalk_serve_destroy(gedwalk_server_t h) {
  Server* srv = reinterpret_cast<Server*>(h);
  if (!srv) return GEDWALK_OK;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->stop = true;
    srv->pending.clear();
    srv->pending_max.clear();
    srv->cv_work.notify_all();
  }
  for (auto& l : srv->lanes)
    if (l->th.joinable()) l->th.join();
  for (auto& w : srv->workers)
    if (w->th.joinable()) w->th.join();
  for (auto& l : srv->lanes) {
    cudaStreamSynchronize(l->stream);
    cudaStreamDestroy(l->stream);
  }
  for (auto& w : srv->workers) {
    cudaStreamSynchronize(w->stream);
    cudaStreamDestroy(w->stream);
  }
  delete srv;
  return GEDWALK_OK;
}

}  // extern "C"
