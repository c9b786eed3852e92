// Serving: a continuous-batching request loop over device-resident graphs.
//
// Threads: one scoring lane per graph and kMaxWorkers maximise workers, each with its own CUDA
// stream and workspace; admission runs on the threads that submit and complete requests.
//
// Admission is by the device memory the server's workspaces hold. Every lane and worker has a
// workspace whose buffers grow to the largest request it has run and stay allocated, so the
// server charges each workspace its held bytes, or, while it has work, the larger of those and the
// exact footprint of that work (the same sizes the algorithms allocate). A request is admitted when
// the total charge stays within the budget; if it does not, idle workspaces are released (largest
// first) to make room, and otherwise the request waits in its FIFO queue. A request larger than the
// budget runs when nothing else holds memory. Score requests are admitted before maximise requests,
// and a maximise request only to a free worker, preferring one whose buffers already fit it.
//
// Admitted score requests wait in their graph's lane; whenever the lane is free it takes every
// waiting request with the same (alpha, L) (up to max_batch) and scores them as the columns of one
// batched SpMM on the lane's own stream, while maximise requests run on the workers' streams, so
// their sweeps overlap on the device. A column's arithmetic never depends on the other columns of
// its batch, so a result is bitwise the same alone and in a mix.
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
  int64_t need = 0;  // maximise: the footprint of its run
  bool admitted = false;
  bool waited = false;  // not admitted by the call that submitted it
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
  int32_t graph = 0;
  std::deque<ReqPtr> queue;
  int64_t q_members = 0;     // members of the queued requests
  int32_t q_groups = 0;      // queued requests
  bool busy = false;
  int64_t need_running = 0;  // footprint of the batch being scored
  int64_t held = 0;          // device bytes of the workspace when it was last idle
  cudaStream_t stream = nullptr;
  Workspace ws;
  std::thread th;
};

struct Worker {  // maximize pool
  ReqPtr job;
  int64_t held = 0;
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
  std::unordered_map<uint64_t, ReqPtr> table;
  std::vector<std::unique_ptr<Lane>> lanes;
  std::vector<std::unique_ptr<Worker>> workers;
  uint64_t next_ticket = 1;
  gedwalk_serve_counters st{};
  bool stop = false;
  int32_t pollers = 0;  // gedwalk_serve_poll calls inside the server (destroy waits for them)

  // A lane's charge: what its workspace holds, or more while it has work (the batch it scores now,
  // or the next batch its queue forms).
  int64_t lane_charge(const Lane& l) const {
    int64_t c = l.held;
    if (l.busy) c = std::max(c, l.need_running);
    if (l.q_groups > 0)
      c = std::max(c, score_batch_footprint(*graphs[l.graph], l.q_members, std::min(l.q_groups, max_batch)));
    return c;
  }
  static int64_t worker_charge(const Worker& w) { return w.job ? std::max(w.held, w.job->need) : w.held; }
  int64_t total() const {
    int64_t t = 0;
    for (const auto& l : lanes) t += lane_charge(*l);
    for (const auto& w : workers) t += worker_charge(*w);
    return t;
  }
  void note_peak() {
    const int64_t t = total();
    st.peak_bytes = std::max(st.peak_bytes, t);
    int64_t running = 0;
    for (const auto& w : workers) running += w->job ? 1 : 0;
    st.peak_maximize_running = std::max(st.peak_maximize_running, running);
  }

  // Releases idle workspaces other than `keep_lane` / `keep_worker`, largest first, until the total
  // charge plus `delta` fits the budget. Returns whether it fits.
  bool make_room(int64_t delta, const Lane* keep_lane, const Worker* keep_worker) {
    for (;;) {
      if (total() + delta <= budget) return true;
      Workspace* best = nullptr;
      int64_t* best_held = nullptr;
      for (auto& l : lanes)
        if (l.get() != keep_lane && !l->busy && l->q_groups == 0 && l->held > 0 && (!best_held || l->held > *best_held)) {
          best = &l->ws;
          best_held = &l->held;
        }
      for (auto& w : workers)
        if (w.get() != keep_worker && !w->job && w->held > 0 && (!best_held || w->held > *best_held)) {
          best = &w->ws;
          best_held = &w->held;
        }
      if (!best) return false;
      // the idle workspace's stream has nothing in flight (its owner synchronised before going idle)
      best->release_device();
      st.released_bytes += *best_held;
      ++st.releases;
      *best_held = 0;
    }
  }

  void mark_admitted(const ReqPtr& q, bool at_submit) {
    q->admitted = true;
    if (at_submit) ++st.admitted_at_submit;
    else ++st.admitted_after_wait;
  }

  // Admits what fits; `submitting` is the request whose submit call runs this (if any).
  void admit_locked(const Request* submitting) {
    while (!pending.empty()) {  // score requests first (FIFO)
      ReqPtr q = pending.front();
      Lane& l = *lanes[q->graph];
      const int64_t members = static_cast<int64_t>(q->S.size());
      const int64_t before = lane_charge(l);
      l.q_members += members;  // the lane's charge with q queued
      ++l.q_groups;
      const int64_t delta = lane_charge(l) - before;
      l.q_members -= members;
      --l.q_groups;
      if (!make_room(delta, &l, nullptr) && total() - lane_charge(l) > 0) break;  // wait
      l.q_members += members;
      ++l.q_groups;
      pending.pop_front();
      mark_admitted(q, q.get() == submitting);
      l.queue.push_back(q);
      note_peak();
    }
    while (!pending_max.empty()) {  // then maximise requests, one per free worker
      ReqPtr q = pending_max.front();
      Worker* pick = nullptr;  // a free worker: the smallest held bytes that fit q, else the largest
      for (auto& w : workers) {
        if (w->job) continue;
        if (!pick) {
          pick = w.get();
          continue;
        }
        const bool fits = w->held >= q->need, pfits = pick->held >= q->need;
        if ((fits && (!pfits || w->held < pick->held)) || (!fits && !pfits && w->held > pick->held)) pick = w.get();
      }
      if (!pick) break;
      const int64_t delta = std::max(pick->held, q->need) - pick->held;
      if (!make_room(delta, nullptr, pick) && total() - pick->held > 0) break;
      pending_max.pop_front();
      mark_admitted(q, q.get() == submitting);
      pick->job = q;
      note_peak();
    }
    cv_work.notify_all();
  }

  void finish_locked(const ReqPtr& q) {
    q->done = true;
    q->t_done = Clock::now();
    ++st.completed;
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
        int64_t members = 0;
        for (auto it = lane.queue.begin(); it != lane.queue.end() && int(batch.size()) < max_batch;) {
          if ((*it)->r.alpha == first->r.alpha && (*it)->r.L == first->r.L) {
            members += static_cast<int64_t>((*it)->S.size());
            batch.push_back(*it);
            it = lane.queue.erase(it);
          } else {
            ++it;
          }
        }
        lane.q_members -= members;
        lane.q_groups -= static_cast<int32_t>(batch.size());
        lane.need_running = score_batch_footprint(g, members, static_cast<int32_t>(batch.size()));
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
      const gedwalk_status stt =
          score_batch_impl(g, lane.ws, off.data(), mem.data(), static_cast<int32_t>(batch.size()), r, scores.data());
      const std::string err = stt == GEDWALK_OK ? "" : gedwalk_last_error();
      cudaStreamSynchronize(lane.stream);
      std::lock_guard<std::mutex> lk(mu);
      ++st.batches;
      st.batched_requests += static_cast<int64_t>(batch.size());
      for (size_t i = 0; i < batch.size(); ++i) {
        batch[i]->status = stt;
        batch[i]->error = err;
        batch[i]->score = scores[i];
        finish_locked(batch[i]);
      }
      lane.held = lane.ws.device_bytes();
      lane.need_running = 0;
      lane.busy = false;
      admit_locked(nullptr);
    }
  }

  void worker_loop(int wi) {
    cudaSetDevice(device);
    Worker& w = *workers[wi];
    for (;;) {
      ReqPtr q;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv_work.wait(lk, [&] { return stop || w.job; });
        if (!w.job) return;
        q = w.job;
      }
      Graph& g = *graphs[q->graph];
      Resolved r = q->r;
      r.stream = w.stream;
      std::vector<int32_t> grp(std::max(q->k, 1));
      std::vector<double> gn(std::max(q->k, 1));
      double sc = 0;
      const gedwalk_status stt = maximize_impl(g, w.ws, q->k, r, q->flags, {}, grp.data(), gn.data(), &sc);
      const std::string err = stt == GEDWALK_OK ? "" : gedwalk_last_error();
      cudaStreamSynchronize(w.stream);
      std::lock_guard<std::mutex> lk(mu);
      q->status = stt;
      q->error = err;
      q->score = sc;
      grp.resize(q->k);
      gn.resize(q->k);
      q->group = std::move(grp);
      q->gains = std::move(gn);
      finish_locked(q);
      w.held = w.ws.device_bytes();
      w.job = nullptr;
      admit_locked(nullptr);
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
  srv->st.budget = srv->budget;
  GW_CUDA(cudaGetDevice(&srv->device));
  for (int32_t i = 0; i < n_graphs; ++i) {
    if (!graphs[i]) return fail(GEDWALK_ERR_INVALID, "graph %d is NULL", i);
    srv->graphs.push_back(G(graphs[i]));
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
  // one stream per lane and worker; on a failure the ones already made are destroyed
  cudaError_t ce = cudaSuccess;
  for (int32_t i = 0; i < n_graphs && ce == cudaSuccess; ++i) {
    std::unique_ptr<Lane> lane(new Lane());
    lane->graph = i;
    ce = cudaStreamCreateWithFlags(&lane->stream, cudaStreamNonBlocking);
    srv->lanes.push_back(std::move(lane));
  }
  for (int i = 0; i < kMaxWorkers && ce == cudaSuccess; ++i) {
    std::unique_ptr<Worker> w(new Worker());
    ce = cudaStreamCreateWithFlags(&w->stream, cudaStreamNonBlocking);
    srv->workers.push_back(std::move(w));
  }
  if (ce != cudaSuccess) {
    for (auto& l : srv->lanes)
      if (l->stream) cudaStreamDestroy(l->stream);
    for (auto& w : srv->workers)
      if (w->stream) cudaStreamDestroy(w->stream);
    return fail(GEDWALK_ERR_DEVICE, "cudaStreamCreateWithFlags failed: %s", cudaGetErrorString(ce));
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
      GreedyShape sh{};
      GW_TRY(greedy_shape(g, q->r, q->flags, &sh));  // rejects bad lookahead / spec_cols now
      q->need = maximize_footprint(g, q->r, q->flags, q->k);
    }
  }
  std::lock_guard<std::mutex> lk(srv->mu);
  if (srv->stop) return fail(GEDWALK_ERR_BUSY, "server is stopping");
  if (srv->pending.size() + srv->pending_max.size() >= kMaxQueue)
    return fail(GEDWALK_ERR_BUSY, "request queue is full");
  q->ticket = srv->next_ticket++;
  q->t_submit = Clock::now();
  srv->table[q->ticket] = q;
  (kind == GEDWALK_REQ_SCORE ? srv->pending : srv->pending_max).push_back(q);
  srv->admit_locked(q.get());
  if (!q->admitted) q->waited = true;
  *ticket = q->ticket;
  return GEDWALK_OK;
}

gedwalk_status gedwalk_serve_poll(gedwalk_server_t h, uint64_t ticket, int32_t wait_us, double* score,
                                  int32_t* group, double* gains, double* latency_us, int32_t* done) {
  Server* srv = reinterpret_cast<Server*>(h);
  if (!srv || !done) return fail(GEDWALK_ERR_INVALID, "server or done is NULL");
  std::unique_lock<std::mutex> lk(srv->mu);
  // counted while inside (the mutex is held again whenever it changes): destroy frees the server
  // only once no poll is left in it
  struct Inside {
    Server* s;
    explicit Inside(Server* v) : s(v) { ++s->pollers; }
    ~Inside() {
      if (--s->pollers == 0 && s->stop) s->cv_done.notify_all();
    }
  } inside(srv);
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
  if (completed) *completed = srv->st.completed;
  if (batches) *batches = srv->st.batches;
  if (batched_requests) *batched_requests = srv->st.batched_requests;
  if (peak_bytes) *peak_bytes = srv->st.peak_bytes;
  return GEDWALK_OK;
}

gedwalk_status gedwalk_serve_counters_read(gedwalk_server_t h, gedwalk_serve_counters* out) {
  Server* srv = reinterpret_cast<Server*>(h);
  if (!srv || !out) return fail(GEDWALK_ERR_INVALID, "server or out is NULL");
  std::lock_guard<std::mutex> lk(srv->mu);
  *out = srv->st;
  out->charged_bytes = srv->total();
  int64_t held = 0;
  for (const auto& l : srv->lanes) held += l->busy ? 0 : l->ws.device_bytes();
  for (const auto& w : srv->workers) held += w->job ? 0 : w->ws.device_bytes();
  out->idle_held_bytes = held;
  out->pending = static_cast<int64_t>(srv->pending.size() + srv->pending_max.size());
  return GEDWALK_OK;
}

gedwalk_status gedwalk_serve_destroy(gedwalk_server_t h) {
  Server* srv = reinterpret_cast<Server*>(h);
  if (!srv) return GEDWALK_OK;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->stop = true;
    // requests still waiting for admission end here, with BUSY, so that their pollers return
    for (std::deque<ReqPtr>* dq : {&srv->pending, &srv->pending_max}) {
      for (const ReqPtr& q : *dq) {
        q->status = GEDWALK_ERR_BUSY;
        q->error = "the server was destroyed before the request was admitted";
        q->done = true;
        q->t_done = Clock::now();
      }
      dq->clear();
    }
    srv->cv_done.notify_all();
    srv->cv_work.notify_all();
  }
  // admitted requests finish: the lanes drain their queues and the workers their jobs
  for (auto& l : srv->lanes)
    if (l->th.joinable()) l->th.join();
  for (auto& w : srv->workers)
    if (w->th.joinable()) w->th.join();
  {
    // every request is done now; polls blocked on one of them wake up and leave
    std::unique_lock<std::mutex> lk(srv->mu);
    srv->cv_done.notify_all();
    srv->cv_done.wait(lk, [&] { return srv->pollers == 0; });
  }
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
