// Scoring a given group (problem (i) of Section 2.1, Algorithm 1): one group by the
// paper's two-state hit/miss recurrences, many groups as columns of one SpMM.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "internal.h"

namespace gw {
namespace {

// X0[v] = (h_0(v), m_0(v)) = (1_S(v), 1_{V\S}(v))
template <typename T>
__global__ void init_two_state(T* __restrict__ X, const uint32_t* __restrict__ mask, int32_t n,
                               const T* __restrict__ rs) {
  for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const bool inS = (mask[v >> 5] >> (v & 31)) & 1u;
    const T sv = rs ? rs[v] : T(1);  // weighted graph: the gathered vectors are scaled by s_v
    X[2 * static_cast<size_t>(v)] = inS ? sv : T(0);
    X[2 * static_cast<size_t>(v) + 1] = inS ? T(0) : sv;
  }
}

// Batched scoring, first-visit form. Column j of a block is m_0 = 1_{V \ S_j}.
// Isolated rows (r >= n_active) hold 0: the sweeps never write them and nothing gathers them,
// so they read as the (zero) first-visit counts of such vertices.
__global__ void init_batch(float* __restrict__ X, int32_t n, int32_t n_active, int32_t cols, int32_t active,
                           const float* __restrict__ rs) {
  const size_t total = static_cast<size_t>(n) * cols;
  const size_t live = static_cast<size_t>(n_active) * cols;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < total; i += size_t(gridDim.x) * blockDim.x)
    X[i] = (i < live && static_cast<int32_t>(i % cols) < active) ? (rs ? rs[i / cols] : 1.0f) : 0.0f;
}

__global__ void zero_members(float* __restrict__ X, int32_t cols, const int32_t* __restrict__ mrow,
                             const int32_t* __restrict__ mcol, int32_t count) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) X[static_cast<size_t>(mrow[i]) * cols + mcol[i]] = 0.0f;
}

// After sweep p: Y_p(s, j) = alpha (A m_{p-1})(s) is alpha^p F_p(s), the weighted p-walks whose
// first visit to S_j is their last vertex s. It meets every walk continuing from s:
// acc += alpha^p F_p(s) * K_{L-p}(s), K_q(s) = sum_{r<=q} t_r(s). Then m_p(s) = 0.
// On a weighted graph (rs = the vertex scales) Y and the table hold s times the true values.
__global__ void batch_member_epilogue(float* __restrict__ Y, int32_t cols, const int32_t* __restrict__ mrow,
                                      const int32_t* __restrict__ mcol, double* __restrict__ acc, int32_t count,
                                      const double* __restrict__ ttab, int32_t n, int32_t q,
                                      const double* __restrict__ rs) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const int32_t s = mrow[i];
  float* y = Y + static_cast<size_t>(s) * cols + mcol[i];
  const double f = static_cast<double>(*y);
  double K = 0.0;
  for (int32_t r = 0; r <= q; ++r) K += ttab[static_cast<size_t>(r) * n + s];
  if (rs) {
    const double sv = rs[s];
    K = sv > 0.0 ? K / (sv * sv) : 0.0;  // a vertex without edges starts and ends no walk
  }
  acc[i] += f * K;
  *y = 0.0f;
}

// acc starts with the p = 0 term: every walk that starts at s (length 1..L) hits S_j at s.
__global__ void batch_member_init(const int32_t* __restrict__ mrow, double* __restrict__ acc, int32_t count,
                                  const double* __restrict__ ttab, int32_t n, int32_t L,
                                  const double* __restrict__ rs) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const int32_t s = mrow[i];
  double K = 0.0;
  for (int32_t r = 1; r <= L; ++r) K += ttab[static_cast<size_t>(r) * n + s];
  if (rs) K = rs[s] > 0.0 ? K / rs[s] : 0.0;
  acc[i] = K;
}

// score_j = sum over the members of group j, in member order.
__global__ void batch_group_sum(const double* __restrict__ acc, const int32_t* __restrict__ goff, int32_t groups,
                                double* __restrict__ out) {
  const int32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= groups) return;
  double s = 0.0;
  for (int32_t i = goff[j]; i < goff[j + 1]; ++i) s += acc[i];
  out[j] = s;
}

int blocks_for(int64_t n, int per = 256) { return static_cast<int>(std::min<int64_t>((n + per - 1) / per, 152 * 32)); }

}  // namespace

namespace {
// Waits for a stream when a call leaves early with an error, so that nothing it launched still
// runs when its buffers are reused or freed.
struct StreamGuard {
  cudaStream_t s;
  bool ok = false;
  ~StreamGuard() {
    if (!ok) {
      cudaStreamSynchronize(s);
      cudaGetLastError();
    }
  }
};
}  // namespace

gedwalk_status score_one(Graph& g, Workspace& ws, const std::vector<int32_t>& S_int, const Resolved& r,
                         double* score) {
  cudaStream_t s = r.stream;
  if (S_int.empty()) {
    *score = 0.0;
    return GEDWALK_OK;
  }
  StreamGuard guard{s};
  const size_t es = r.fp64 ? 8 : 4;
  const size_t vbytes = static_cast<size_t>(g.n) * 2 * es;
  GW_TRY(ws.x0.ensure(vbytes, s));
  GW_TRY(ws.x1.ensure(vbytes, s));
  GW_TRY(ensure_sweep_scratch(g, ws, 2, r.fp64, s));
  GW_TRY(ws.small.ensure(64, s));
  GW_TRY(upload_mask(g, ws, S_int, s));
  if (r.fp64)
    init_two_state<double><<<blocks_for(g.n), 256, 0, s>>>(ws.x0.as<double>(), ws.mask.as<uint32_t>(), g.n,
                                                            g.weighted ? g.rs_d.as<double>() : nullptr);
  else
    init_two_state<float><<<blocks_for(g.n), 256, 0, s>>>(ws.x0.as<float>(), ws.mask.as<uint32_t>(), g.n,
                                                           g.weighted ? g.rs_f.as<float>() : nullptr);
  GW_KCHECK();
  SweepArgs a = base_args(g, ws);
  a.alpha = r.alpha;
  void* cur = ws.x0.p;
  void* nxt = ws.x1.p;
  for (int32_t i = 1; i <= r.L; ++i) {
    a.X = cur;
    a.Y = nxt;
    a.accumulate = i > 1;
    GW_TRY(launch_sweep(MODE_SCORE, r.fp64, 2, a, s));
    std::swap(cur, nxt);
  }
  GW_TRY(reduce_slots(g, ws, 1, ws.small.as<double>(), s));
  double h = 0;
  GW_CUDA(cudaMemcpyAsync(&h, ws.small.p, sizeof h, cudaMemcpyDeviceToHost, s));
  GW_CUDA(cudaStreamSynchronize(s));
  *score = h;
  guard.ok = true;
  return GEDWALK_OK;
}

// Picks the column-block width with the lowest sweep time per column (timed on this graph). A
// gather fetches whole 32-byte sectors, so widths below 8 FP32 columns waste part of each; above
// 32 the walk vectors of a 10^6-vertex graph (n * C * 4 bytes, twice) outgrow the L2 and the
// per-column time rises (the tuning log records it).
gedwalk_status autotune_batch(Graph& g, Workspace& ws, const Resolved& r) {
  if (g.batch_cols > 0) return GEDWALK_OK;
  cudaStream_t s = r.stream;
  static const int kCand[] = {8, 16, 32, 64};
  double best = INFINITY;
  int best_c = 16;
  cudaEvent_t e0, e1;
  GW_CUDA(cudaEventCreate(&e0));
  GW_CUDA(cudaEventCreate(&e1));
  g.tune_log.clear();
  for (int c : kCand) {
    const size_t vbytes = static_cast<size_t>(g.n) * c * 4;
    if (ws.x0.ensure(vbytes, s) != GEDWALK_OK || ws.x1.ensure(vbytes, s) != GEDWALK_OK) break;
    GW_TRY(ensure_sweep_scratch(g, ws, c, false, s));
    init_batch<<<blocks_for(static_cast<int64_t>(g.n) * c), 256, 0, s>>>(ws.x0.as<float>(), g.n, g.n, c, c,
                                                                          nullptr);
    GW_KCHECK();
    SweepArgs a = base_args(g, ws);
    a.alpha = r.alpha;
    a.X = ws.x0.p;
    a.Y = ws.x1.p;
    for (int w = 0; w < 2; ++w) GW_TRY(launch_sweep(MODE_PLAIN, false, c, a, s));
    const int reps = 5;
    GW_CUDA(cudaEventRecord(e0, s));
    for (int w = 0; w < reps; ++w) GW_TRY(launch_sweep(MODE_PLAIN, false, c, a, s));
    GW_CUDA(cudaEventRecord(e1, s));
    GW_CUDA(cudaEventSynchronize(e1));
    float ms = 0;
    GW_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    const double per_col = ms / reps / c;
    g.tune_log.emplace_back(c, per_col);
    if (per_col < best) {
      best = per_col;
      best_c = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  g.batch_cols = best_c;
  return GEDWALK_OK;
}

int64_t score_batch_footprint(const Graph& g, int64_t members, int32_t groups) {
  const int64_t C = g.batch_cols > 0 ? g.batch_cols : 32;  // before tuning: the widest width tried
  const int64_t n = g.n;
  int64_t b = 2 * n * C * 4;                                      // walk vectors x0, x1
  b += members * (4 + 4 + 8) + static_cast<int64_t>(groups + 1) * 4 + 256;  // members, columns, sums
  b += static_cast<int64_t>(std::max(g.plan.num_slices, 1)) * C * 4 + std::max(g.plan.num_heavy, 1) * 4;
  b += static_cast<int64_t>(std::max(g.plan.num_slots, 1)) * C * 8 + C * kReduceParts * 8;
  b += static_cast<int64_t>(groups) * 8 + 64;
  return b;
}

gedwalk_status score_batch_impl(Graph& g, Workspace& ws, const int32_t* offsets, const int32_t* members_int,
                                int32_t G, const Resolved& r, double* scores) {
  cudaStream_t s = r.stream;
  if (G == 0) return GEDWALK_OK;
  StreamGuard guard{s};
  // the caller has made the walk-total table hold rows 0..L for alpha and tuned the width
  std::shared_lock<std::shared_mutex> rl(g.tt_lock);
  if (g.tt_alpha != r.alpha || g.tt_rows < r.L + 1 || g.batch_cols <= 0)
    return fail(GEDWALK_ERR_INVALID, "walk-total table or column width not prepared for this batch");
  const int C = g.batch_cols;
  const int64_t total = offsets[G];
  // members: row (internal id), column within its block, accumulator; group offsets
  const size_t mbytes = static_cast<size_t>(total) * (4 + 4 + 8) + static_cast<size_t>(G + 1) * 4 + 256;
  GW_TRY(ws.members.ensure(mbytes, s));
  char* base = ws.members.as<char>();
  double* acc = reinterpret_cast<double*>(base);
  int32_t* mrow = reinterpret_cast<int32_t*>(acc + total);
  int32_t* mcol = mrow + total;
  int32_t* goff = mcol + total;
  // members, their columns and the group offsets go up in one copy from pinned staging
  const size_t up = sizeof(int32_t) * (2 * static_cast<size_t>(total) + G + 1);
  GW_TRY(ws.ensure_pinned(std::max(up, sizeof(double) * static_cast<size_t>(G)) + 64));
  int32_t* hst = static_cast<int32_t*>(ws.pinned);
  if (total > 0) memcpy(hst, members_int, sizeof(int32_t) * total);
  for (int32_t j = 0; j < G; ++j)
    for (int32_t i = offsets[j]; i < offsets[j + 1]; ++i) hst[total + i] = j % C;
  memcpy(hst + 2 * total, offsets, sizeof(int32_t) * (G + 1));
  GW_CUDA(cudaMemcpyAsync(mrow, hst, up, cudaMemcpyHostToDevice, s));
  const size_t vbytes = static_cast<size_t>(g.n) * C * 4;
  GW_TRY(ws.x0.ensure(vbytes, s));
  GW_TRY(ws.x1.ensure(vbytes, s));
  GW_TRY(ensure_sweep_scratch(g, ws, C, false, s));
  GW_TRY(ws.small.ensure(static_cast<size_t>(G) * sizeof(double) + 64, s));
  const double* T = g.ttab.as<double>();
  const double* rsd = g.weighted ? g.rs_d.as<double>() : nullptr;
  SweepArgs a = base_args(g, ws);
  a.alpha = r.alpha;
  if (g.n_active < g.n)
    GW_CUDA(cudaMemsetAsync(ws.x1.as<float>() + static_cast<size_t>(g.n_active) * C, 0,
                            sizeof(float) * C * (static_cast<size_t>(g.n) - g.n_active), s));
  if (total > 0) {
    batch_member_init<<<blocks_for(total), 256, 0, s>>>(mrow, acc, static_cast<int32_t>(total), T, g.n, r.L, rsd);
    GW_KCHECK();
  }
  for (int32_t g0 = 0; g0 < G; g0 += C) {
    const int32_t g1 = std::min(G, g0 + C);
    const int32_t m0 = offsets[g0], m1 = offsets[g1];
    const int32_t cnt = m1 - m0;
    init_batch<<<blocks_for(static_cast<int64_t>(g.n) * C), 256, 0, s>>>(ws.x0.as<float>(), g.n, g.n_active, C,
                                                                          g1 - g0,
                                                                          g.weighted ? g.rs_f.as<float>() : nullptr);
    GW_KCHECK();
    if (cnt > 0) {
      zero_members<<<blocks_for(cnt), 256, 0, s>>>(ws.x0.as<float>(), C, mrow + m0, mcol + m0, cnt);
      GW_KCHECK();
    }
    void* cur = ws.x0.p;
    void* nxt = ws.x1.p;
    for (int32_t p = 1; p <= r.L; ++p) {
      a.X = cur;
      a.Y = nxt;
      GW_TRY(launch_sweep(MODE_PLAIN, false, C, a, s));
      if (cnt > 0) {
        batch_member_epilogue<<<blocks_for(cnt), 256, 0, s>>>(static_cast<float*>(nxt), C, mrow + m0, mcol + m0,
                                                               acc + m0, cnt, T, g.n, r.L - p, rsd);
        GW_KCHECK();
      }
      std::swap(cur, nxt);
    }
  }
  batch_group_sum<<<blocks_for(G), 256, 0, s>>>(acc, goff, G, ws.small.as<double>());
  GW_KCHECK();
  GW_CUDA(cudaMemcpyAsync(ws.pinned, ws.small.p, sizeof(double) * G, cudaMemcpyDeviceToHost, s));
  GW_CUDA(cudaStreamSynchronize(s));
  memcpy(scores, ws.pinned, sizeof(double) * G);
  guard.ok = true;
  return GEDWALK_OK;
}

}  // namespace gw

using namespace gw;

extern "C" {

gedwalk_status gedwalk_score(gedwalk_graph_t h, const int32_t* S, int32_t s_len, const gedwalk_params* params,
                             double* score, int32_t* L_used, double* tail_bound) {
  if (!h || !score) return fail(GEDWALK_ERR_INVALID, "graph or score is NULL");
  Graph* g = G(h);
  std::lock_guard<std::mutex> lk(g->mu);
  GW_CUDA(cudaSetDevice(g->device));
  std::vector<int32_t> S_int;
  GW_TRY(map_group(*g, S, s_len, &S_int));
  Resolved r;
  GW_TRY(resolve(*g, params, 0.0, &r));
  double v = 0;
  GW_TRY(score_one(*g, g->ws, S_int, r, &v));
  *score = v;
  if (L_used) *L_used = r.L;
  if (tail_bound) *tail_bound = r.bound;
  return GEDWALK_OK;
}

gedwalk_status gedwalk_batch_tuning(gedwalk_graph_t h, int32_t* cols, double* us_per_col, int32_t cap, int32_t* count,
                                    int32_t* chosen) {
  if (!h) return fail(GEDWALK_ERR_INVALID, "graph is NULL");
  if (cap < 0 || (cap > 0 && (!cols || !us_per_col))) return fail(GEDWALK_ERR_INVALID, "NULL output or cap < 0");
  Graph* g = gw::G(h);
  std::lock_guard<std::mutex> lk(g->mu);
  const int32_t m = static_cast<int32_t>(g->tune_log.size());
  for (int32_t j = 0; j < std::min(m, cap); ++j) {
    cols[j] = g->tune_log[j].first;
    us_per_col[j] = g->tune_log[j].second * 1e3;
  }
  if (count) *count = m;
  if (chosen) *chosen = g->batch_cols;
  return GEDWALK_OK;
}

gedwalk_status gedwalk_batch_set_width(gedwalk_graph_t h, int32_t cols) {
  if (!h) return fail(GEDWALK_ERR_INVALID, "graph is NULL");
  if (!(cols == 0 || cols == 8 || cols == 16 || cols == 32 || cols == 64))
    return fail(GEDWALK_ERR_INVALID, "column-block width must be 0 (tune), 8, 16, 32 or 64");
  Graph* g = gw::G(h);
  std::lock_guard<std::mutex> lk(g->mu);
  g->batch_cols = cols;
  return GEDWALK_OK;
}

gedwalk_status gedwalk_score_batch(gedwalk_graph_t h, const int32_t* offsets, const int32_t* members, int32_t G,
                                   const gedwalk_params* params, double* scores, int32_t* L_used) {
  if (!h || (G > 0 && (!offsets || !scores))) return fail(GEDWALK_ERR_INVALID, "NULL argument");
  if (G < 0) return fail(GEDWALK_ERR_INVALID, "G must be >= 0");
  Graph* g = gw::G(h);
  std::lock_guard<std::mutex> lk(g->mu);
  GW_CUDA(cudaSetDevice(g->device));
  if (G > 0 && offsets[0] != 0) return fail(GEDWALK_ERR_INVALID, "offsets[0] must be 0");
  // map and deduplicate each group (set semantics), rebuilding the offsets
  std::vector<int32_t> off(static_cast<size_t>(G) + 1, 0), mem, tmp;
  for (int32_t j = 0; j < G; ++j) {
    if (offsets[j + 1] < offsets[j]) return fail(GEDWALK_ERR_INVALID, "offsets decrease at group %d", j);
    GW_TRY(map_group(*g, members + offsets[j], offsets[j + 1] - offsets[j], &tmp));
    mem.insert(mem.end(), tmp.begin(), tmp.end());
    off[j + 1] = static_cast<int32_t>(mem.size());
  }
  Resolved r;
  GW_TRY(resolve(*g, params, 0.0, &r));
  r.fp64 = false;
  GW_TRY(ensure_totals(*g, r.alpha, r.L + 1, r.stream));
  GW_TRY(autotune_batch(*g, g->ws, r));
  GW_TRY(score_batch_impl(*g, g->ws, off.data(), mem.data(), G, r, scores));
  if (L_used) *L_used = r.L;
  return GEDWALK_OK;
}

}  // extern "C"
