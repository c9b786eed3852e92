// Graph upload, validation, degree relabelling, the sweep plan, the FP64 walk-total
// table behind the combinatorial bound, and the small shared helpers of the C ABI.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <thread>

#include "internal.h"

namespace gw {

// ---------------------------------------------------------------- errors
static thread_local std::string t_last_error;

void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  t_last_error = buf;
}

gedwalk_status fail(gedwalk_status st, const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  t_last_error = buf;
  return st;
}

// ---------------------------------------------------------------- profiling
namespace {
struct Profiler {
  std::mutex mu;
  std::atomic<bool> enabled{false};
  std::atomic<int64_t> launches{0};
  struct Rec {
    cudaEvent_t a, b;
    double bytes;
    int key;  // (mode * 1000 + cols) * 2 + fp64
  };
  std::vector<Rec> recs;
  struct Done {
    double ms, bytes;
    int key;
  };
  std::vector<Done> done;  // timings read directly (graph replays)
  std::vector<cudaEvent_t> pool;
  cudaEvent_t take() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return e;
  }
};
Profiler& prof() {
  static Profiler* p = new Profiler();  // lives until exit; never destroyed after the CUDA runtime
  return *p;
}
}  // namespace

void count_launch() { prof().launches.fetch_add(1, std::memory_order_relaxed); }
void count_launches(int n) { prof().launches.fetch_add(n, std::memory_order_relaxed); }

void profile_add(double ms, double bytes, int key) {
  Profiler& p = prof();
  std::lock_guard<std::mutex> lk(p.mu);
  if (p.enabled.load()) p.done.push_back({ms, bytes, key});
}
bool profiling() { return prof().enabled.load(std::memory_order_relaxed); }

void profile_begin(cudaStream_t s, cudaEvent_t* a) {
  Profiler& p = prof();
  std::lock_guard<std::mutex> lk(p.mu);
  *a = p.take();
  if (*a) cudaEventRecord(*a, s);
}

void profile_end(cudaStream_t s, cudaEvent_t a, double bytes, int key) {
  Profiler& p = prof();
  std::lock_guard<std::mutex> lk(p.mu);
  if (!a) return;
  cudaEvent_t b = p.take();
  if (!b) {
    p.pool.push_back(a);
    return;
  }
  cudaEventRecord(b, s);
  p.recs.push_back({a, b, bytes, key});
}

double sweep_bytes(int mode, bool fp64, int cols, int32_t n, int64_t nnz) {
  const double es = mode == MODE_TOTALS ? 8.0 : (fp64 ? 8.0 : 4.0);
  double b = 4.0 * double(nnz) + 4.0 * (double(n) + 1.0) + 2.0 * cols * es * double(n);
  if (mode == MODE_SCORE || mode == MODE_FUSED || mode == MODE_CAND) b += double(n) / 8.0;
  if (mode == MODE_FUSED) b += es * double(n);
  return b;
}

// ---------------------------------------------------------------- device memory
static gedwalk_alloc_fn g_alloc = nullptr;
static gedwalk_free_fn g_free = nullptr;
static void* g_alloc_ctx = nullptr;

void* dalloc(size_t bytes, cudaStream_t s) {
  if (bytes == 0) bytes = 16;
  if (g_alloc) return g_alloc(bytes, reinterpret_cast<int64_t>(s), g_alloc_ctx);
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();  // clear the sticky-free error state of a failed allocation
    return nullptr;
  }
  return p;
}

void dfree(void* p, size_t bytes, cudaStream_t s) {
  if (!p) return;
  if (g_free) {
    g_free(p, bytes, reinterpret_cast<int64_t>(s), g_alloc_ctx);
    return;
  }
  cudaFree(p);
}

gedwalk_status DevBuf::ensure(size_t need, cudaStream_t s, bool zero) {
  if (need == 0) need = 16;
  if (p && bytes >= need) return GEDWALK_OK;
  release();
  p = dalloc(need, s);
  if (!p) return fail(GEDWALK_ERR_OOM, "device allocation of %zu bytes failed", need);
  bytes = need;
  if (zero) GW_CUDA(cudaMemsetAsync(p, 0, need, s));
  return GEDWALK_OK;
}

void SweepGraph::reset() {
  if (exec) cudaGraphExecDestroy(exec);
  exec = nullptr;
  for (cudaEvent_t e : ev) cudaEventDestroy(e);
  ev.clear();
  key = 0;
  uses = 0;
  timing_pending = false;
}

Workspace::~Workspace() {
  for (SweepGraph& sg : graphs) sg.reset();
  if (order_ev) cudaEventDestroy(order_ev);
  if (own_stream) cudaStreamDestroy(own_stream);
  if (pinned) cudaFreeHost(pinned);
}

gedwalk_status Workspace::ensure_pinned(size_t need) {
  if (pinned && pinned_bytes >= need) return GEDWALK_OK;
  if (pinned) cudaFreeHost(pinned);
  pinned = nullptr;
  pinned_bytes = 0;
  if (cudaMallocHost(&pinned, need) != cudaSuccess) {
    cudaGetLastError();
    pinned = nullptr;
    return fail(GEDWALK_ERR_OOM, "pinned host allocation of %zu bytes failed", need);
  }
  pinned_bytes = need;
  return GEDWALK_OK;
}

// ---------------------------------------------------------------- host parallel helpers
template <class F>
static void parallel_rows(int64_t n, F&& f) {
  unsigned hw = std::thread::hardware_concurrency();
  unsigned T = std::max(1u, std::min(hw == 0 ? 1u : hw, 64u));
  if (n < (1 << 15) || T == 1) {
    f(int64_t(0), n);
    return;
  }
  // dynamic chunks: heavy rows sit at the front after relabelling
  const int64_t chunk = 4096;
  std::atomic<int64_t> next(0);
  std::vector<std::thread> th;
  for (unsigned t = 0; t < T; ++t)
    th.emplace_back([&]() {
      for (;;) {
        const int64_t b = next.fetch_add(chunk);
        if (b >= n) break;
        f(b, std::min(n, b + chunk));
      }
    });
  for (auto& x : th) x.join();
}

// First malformed row (or -1) and a reason.
static int64_t validate_csr(const int32_t* rp, const int32_t* ci, int32_t n, int64_t nnz, bool full,
                            std::string* why) {
  if (rp[0] != 0) {
    *why = "row_ptr[0] != 0";
    return 0;
  }
  if (static_cast<int64_t>(rp[n]) != nnz) {
    *why = "row_ptr[n] != nnz";
    return n;
  }
  for (int32_t v = 0; v < n; ++v)
    if (rp[v + 1] < rp[v]) {
      *why = "row_ptr decreases";
      return v;
    }
  std::atomic<int64_t> bad(INT64_MAX);
  std::atomic<int> kind(0);
  parallel_rows(n, [&](int64_t b, int64_t e) {
    for (int64_t v = b; v < e; ++v) {
      if (v >= bad.load(std::memory_order_relaxed)) return;
      int k = 0;
      for (int32_t j = rp[v]; j < rp[v + 1] && !k; ++j) {
        const int32_t u = ci[j];
        if (u < 0 || u >= n) k = 1;
        else if (!full) continue;
        else if (u == v) k = 2;
        else if (j > rp[v] && ci[j - 1] >= u) k = 3;
        else if (full && !std::binary_search(ci + rp[u], ci + rp[u + 1], static_cast<int32_t>(v))) k = 4;
      }
      if (k) {
        int64_t cur = bad.load();
        while (v < cur && !bad.compare_exchange_weak(cur, v)) {
        }
        if (v <= bad.load()) kind.store(k);
        return;
      }
    }
  });
  static const char* reasons[] = {"", "column index out of range", "self-loop", "row not strictly increasing",
                                  "graph is not symmetric (undirected graphs only)"};
  if (bad.load() != INT64_MAX) {
    *why = reasons[kind.load()];
    return bad.load();
  }
  return -1;
}

// Degree class of a light row: 2^cls lanes with at most two entries each (cls <= 5), or a
// whole warp looping over the row (cls 6).
static int row_class(int32_t d) {
  int cls = 0;
  while (cls < 6 && d > (2 << cls)) ++cls;
  return cls;
}

static gedwalk_status build_plan(Graph& g, const std::vector<int32_t>& rp) {
  std::vector<int4> units, heavy;
  int32_t nh = 0;
  while (nh < g.n && g.deg[nh] > kHeavyDeg) ++nh;
  int32_t slice = 0;
  for (int32_t h = 0; h < nh; ++h) {
    const int32_t d = g.deg[h];
    const int32_t ns = (d + kSliceEdges - 1) / kSliceEdges;
    heavy.push_back(make_int4(h, slice, ns, 0));
    for (int32_t k = 0; k < ns; ++k) {
      const int32_t e0 = rp[h] + static_cast<int32_t>(static_cast<int64_t>(d) * k / ns);
      const int32_t e1 = rp[h] + static_cast<int32_t>(static_cast<int64_t>(d) * (k + 1) / ns);
      units.push_back(make_int4(h, e0, e1, slice + k));
    }
    slice += ns;
  }
  g.plan.num_slices = slice;
  g.plan.num_heavy = nh;
  // isolated rows (degree 0, sorted last) get no units: their sums are 0, nothing gathers
  // their x, and the few outputs read back at such rows are zeroed by the callers
  g.n_active = g.n;
  while (g.n_active > 0 && g.deg[g.n_active - 1] == 0) --g.n_active;
  int32_t r = nh;
  while (r < g.n_active) {
    const int cls = row_class(g.deg[r]);
    // a short-row unit takes up to kUnitRowsMax rows; on small graphs fewer, down to one
    // iteration of its warp (2 rows per lane group), so that every SM gets work
    const int32_t iter_rows = cls == 6 ? 1 : 2 * (32 >> cls);
    const int32_t small_cap = std::max<int32_t>(iter_rows, g.n_active / kTargetUnits);
    const int32_t max_rows = std::min<int32_t>(cls == 6 ? 32 : kUnitRowsMax, small_cap);
    const int64_t max_edges = cls == 6 ? kLongUnitEdges : kUnitEdges;
    int32_t r1 = r;
    int64_t edges = 0;
    while (r1 < g.n_active && row_class(g.deg[r1]) == cls && r1 - r < max_rows &&
           (r1 == r || edges + g.deg[r1] <= max_edges)) {
      edges += g.deg[r1];
      ++r1;
    }
    units.push_back(make_int4(r, r1, cls, -1));
    r = r1;
  }
  g.plan.num_units = static_cast<int32_t>(units.size());
  g.plan.num_slots = g.plan.num_units + nh;
  GW_TRY(g.plan.units.ensure(units.size() * sizeof(int4) + 16, 0));
  GW_TRY(g.plan.heavy.ensure(heavy.size() * sizeof(int4) + 16, 0));
  if (!units.empty()) GW_CUDA(cudaMemcpy(g.plan.units.p, units.data(), units.size() * sizeof(int4), cudaMemcpyHostToDevice));
  if (!heavy.empty()) GW_CUDA(cudaMemcpy(g.plan.heavy.p, heavy.data(), heavy.size() * sizeof(int4), cudaMemcpyHostToDevice));
  return GEDWALK_OK;
}

// ---------------------------------------------------------------- small kernels
__global__ void fill_f64_kernel(double* p, int64_t n, double v) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) p[i] = v;
}

// Device-side truncation test (Algorithm 1's stop test with Eq. comb-bound): the first
// l in [lo, rows) with coef * Wa[l] < eps, where coef = alpha dmax / (1 - alpha dmax).
__global__ void first_crossing_kernel(const double* Wa, int32_t lo, int32_t rows, double coef, double eps,
                                      int32_t* out_l, double* out_b) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int32_t l = -1;
  double b = 0.0;
  for (int32_t i = lo; i < rows; ++i) {
    b = coef * Wa[i];
    if (b < eps) {
      l = i;
      break;
    }
  }
  *out_l = l;
  *out_b = b;
}

static int grid_for(int64_t n) { return static_cast<int>(std::min<int64_t>((n + 255) / 256, 152 * 16)); }

SweepArgs base_args(Graph& g, Workspace& ws) {
  SweepArgs a{};
  a.rp = g.rp.as<int32_t>();
  a.ci = g.ci.as<int32_t>();
  a.units = g.plan.units.as<int4>();
  a.heavy = g.plan.heavy.as<int4>();
  a.num_units = g.plan.num_units;
  a.n = g.n;
  a.nnz = g.nnz;
  a.mask = ws.mask.as<uint32_t>();
  a.partial = ws.partial.p;
  a.counters = ws.counters.as<unsigned>();
  a.slots = ws.slots.as<double>();
  a.accumulate = 0;
  a.cand = nullptr;
  return a;
}

gedwalk_status ensure_sweep_scratch(Graph& g, Workspace& ws, int cols, bool fp64, cudaStream_t s) {
  const size_t es = fp64 ? 8 : 4;
  GW_TRY(ws.partial.ensure(static_cast<size_t>(std::max(g.plan.num_slices, 1)) * cols * es, s));
  const size_t cbytes = static_cast<size_t>(std::max(g.plan.num_heavy, 1)) * sizeof(unsigned);
  if (ws.counters.bytes < cbytes || !ws.counters.p) GW_TRY(ws.counters.ensure(cbytes, s, /*zero=*/true));
  GW_TRY(ws.slots.ensure(static_cast<size_t>(std::max(g.plan.num_slots, 1)) * cols * sizeof(double), s));
  GW_TRY(ws.parts.ensure(static_cast<size_t>(cols) * kReduceParts * sizeof(double), s));
  return GEDWALK_OK;
}

gedwalk_status reduce_slots(Graph& g, Workspace& ws, int nsum, double* out, cudaStream_t s) {
  return launch_reduce_slots(ws.slots.as<double>(), g.plan.num_slots, nsum, out, ws.parts.as<double>(), s);
}

// ---------------------------------------------------------------- walk totals
gedwalk_status ensure_totals(Graph& g, double alpha, int32_t rows, cudaStream_t s) {
  if (g.tt_alpha == alpha && rows <= g.tt_rows) return GEDWALK_OK;
  std::unique_lock<std::shared_mutex> wl(g.tt_lock);
  if (g.tt_alpha != alpha) {
    g.tt_alpha = alpha;
    g.tt_rows = 0;
    g.Wa.clear();
  }
  if (rows <= g.tt_rows) return GEDWALK_OK;
  const size_t n = static_cast<size_t>(g.n);
  const size_t need = static_cast<size_t>(rows) * n * sizeof(double);
  if (need > (size_t(24) << 30)) return fail(GEDWALK_ERR_OOM, "walk-total table of %d rows does not fit", rows);
  if (g.ttab.bytes < need) {
    // grow, keeping the rows already computed
    DevBuf fresh;
    GW_TRY(fresh.ensure(need + need / 2, s));
    if (g.tt_rows > 0)
      GW_CUDA(cudaMemcpyAsync(fresh.p, g.ttab.p, static_cast<size_t>(g.tt_rows) * n * sizeof(double),
                              cudaMemcpyDeviceToDevice, s));
    std::swap(g.ttab.p, fresh.p);
    std::swap(g.ttab.bytes, fresh.bytes);
    GW_CUDA(cudaStreamSynchronize(s));
  }
  Workspace& ws = g.ws;
  GW_TRY(ensure_sweep_scratch(g, ws, 1, true, s));
  GW_TRY(ws.small.ensure(static_cast<size_t>(rows) * sizeof(double) + 64, s));
  double* T = g.ttab.as<double>();
  double* dWa = ws.small.as<double>();
  int32_t r0 = g.tt_rows;
  if (r0 == 0) {
    fill_f64_kernel<<<grid_for(g.n), 256, 0, s>>>(T, g.n, 1.0);
    GW_KCHECK();
    g.Wa.assign(1, static_cast<double>(g.n));
    r0 = 1;
  }
  SweepArgs a = base_args(g, ws);
  a.alpha = alpha;
  a.accumulate = 0;
  for (int32_t r = r0; r < rows; ++r) {
    a.X = T + static_cast<size_t>(r - 1) * n;
    a.Y = T + static_cast<size_t>(r) * n;
    if (g.n_active < g.n)  // isolated vertices start no walk of length >= 1
      GW_CUDA(cudaMemsetAsync(T + static_cast<size_t>(r) * n + g.n_active, 0,
                              sizeof(double) * (n - static_cast<size_t>(g.n_active)), s));
    GW_TRY(launch_sweep(MODE_TOTALS, true, 1, a, s));
    GW_TRY(reduce_slots(g, ws, 1, dWa + r, s));
  }
  std::vector<double> tmp(rows);
  GW_CUDA(cudaMemcpyAsync(tmp.data() + r0, dWa + r0, sizeof(double) * (rows - r0), cudaMemcpyDeviceToHost, s));
  GW_CUDA(cudaStreamSynchronize(s));
  g.Wa.resize(rows);
  for (int32_t r = r0; r < rows; ++r) g.Wa[r] = tmp[r];
  g.tt_rows = rows;
  return GEDWALK_OK;
}

gedwalk_status truncation_length(Graph& g, double alpha, double eps, int32_t* L, double* bound, cudaStream_t s) {
  if (!(alpha > 0.0) || !std::isfinite(alpha)) return fail(GEDWALK_ERR_INVALID, "alpha must be positive");
  if (!(eps > 0.0)) return fail(GEDWALK_ERR_INVALID, "epsilon must be positive");
  if (!(alpha * g.dmax < 1.0))
    return fail(GEDWALK_ERR_NOT_CONVERGENT,
                "alpha * d_max = %g >= 1: the combinatorial bound needs alpha < 1/d_max (force L instead)",
                alpha * g.dmax);
  for (const Graph::Trunc& t : g.trunc_cache)  // L depends only on (graph, alpha, epsilon)
    if (t.alpha == alpha && t.eps == eps) {
      *L = t.L;
      if (bound) *bound = t.bound;
      return GEDWALK_OK;
    }
  const double coef = alpha * g.dmax / (1.0 - alpha * g.dmax);
  const int32_t kCap = 4096;
  int32_t rows = std::max(g.tt_alpha == alpha ? g.tt_rows : 0, 4);
  Workspace& ws = g.ws;
  for (;;) {
    GW_TRY(ensure_totals(g, alpha, rows, s));
    GW_TRY(ws.small.ensure(static_cast<size_t>(rows) * sizeof(double) + 64, s));
    // the Wa row sums are re-staged on the device so that the stop test runs there
    double* dWa = ws.small.as<double>();
    GW_CUDA(cudaMemcpyAsync(dWa, g.Wa.data(), sizeof(double) * rows, cudaMemcpyHostToDevice, s));
    int32_t* dl = reinterpret_cast<int32_t*>(dWa + rows);
    double* db = dWa + rows + 1;
    first_crossing_kernel<<<1, 32, 0, s>>>(dWa, 1, rows, coef, eps, dl, db);
    GW_KCHECK();
    int32_t hl = -1;
    double hb = 0;
    GW_CUDA(cudaMemcpyAsync(&hl, dl, sizeof hl, cudaMemcpyDeviceToHost, s));
    GW_CUDA(cudaMemcpyAsync(&hb, db, sizeof hb, cudaMemcpyDeviceToHost, s));
    GW_CUDA(cudaStreamSynchronize(s));
    if (hl > 0) {
      *L = hl;
      if (bound) *bound = hb;
      if (g.trunc_cache.size() >= 64) g.trunc_cache.erase(g.trunc_cache.begin());
      g.trunc_cache.push_back({alpha, eps, hl, hb});
      return GEDWALK_OK;
    }
    if (rows >= kCap) return fail(GEDWALK_ERR_INVALID, "no truncation length <= %d reaches epsilon %g", kCap, eps);
    rows = std::min(rows * 2, kCap);
  }
}

gedwalk_status resolve(Graph& g, const gedwalk_params* p, double eps_override, Resolved* r) {
  gedwalk_params d;
  gedwalk_params_default(&d);
  if (!p) p = &d;
  if (p->alpha < 0.0 || std::isnan(p->alpha)) return fail(GEDWALK_ERR_INVALID, "alpha must be positive (0 = default)");
  r->alpha = p->alpha > 0.0 ? p->alpha : g.alpha_default;
  if (!(r->alpha > 0.0) || !std::isfinite(r->alpha)) return fail(GEDWALK_ERR_INVALID, "alpha must be positive");
  if (p->precision != GEDWALK_FP64 && p->precision != GEDWALK_FP32)
    return fail(GEDWALK_ERR_INVALID, "precision must be GEDWALK_FP64 or GEDWALK_FP32");
  r->fp64 = p->precision == GEDWALK_FP64;
  r->stream = reinterpret_cast<cudaStream_t>(p->stream);
  r->eta = p->eta;
  r->seed = p->seed;
  if (p->L < 0) return fail(GEDWALK_ERR_INVALID, "L must be >= 0");
  if (p->L > 0) {
    if (p->L > 4096) return fail(GEDWALK_ERR_INVALID, "L must be <= 4096");
    r->L = p->L;
    r->bound = NAN;
    if (r->alpha * g.dmax < 1.0) {
      GW_TRY(ensure_totals(g, r->alpha, p->L + 1, r->stream));
      r->bound = r->alpha * g.dmax / (1.0 - r->alpha * g.dmax) * g.Wa[p->L];
    }
    return GEDWALK_OK;
  }
  const double eps = eps_override > 0.0 ? eps_override : p->epsilon;
  return truncation_length(g, r->alpha, eps, &r->L, &r->bound, r->stream);
}

gedwalk_status map_group(const Graph& g, const int32_t* S, int32_t s_len, std::vector<int32_t>* out) {
  out->clear();
  if (s_len < 0) return fail(GEDWALK_ERR_INVALID, "negative group size");
  if (s_len > 0 && !S) return fail(GEDWALK_ERR_INVALID, "group pointer is NULL");
  out->reserve(s_len);
  for (int32_t j = 0; j < s_len; ++j) {
    if (S[j] < 0 || S[j] >= g.n) return fail(GEDWALK_ERR_INVALID, "vertex id %d out of range [0, %d)", S[j], g.n);
    out->push_back(g.inv[S[j]]);
  }
  std::sort(out->begin(), out->end());
  out->erase(std::unique(out->begin(), out->end()), out->end());
  return GEDWALK_OK;
}

gedwalk_status upload_mask(Graph& g, Workspace& ws, const std::vector<int32_t>& S_int, cudaStream_t s) {
  const size_t words = (static_cast<size_t>(g.n) + 31) / 32;
  GW_TRY(ws.mask.ensure(words * 4, s));
  std::vector<uint32_t> m(words, 0u);
  for (int32_t v : S_int) m[v >> 5] |= 1u << (v & 31);
  GW_CUDA(cudaMemcpyAsync(ws.mask.p, m.data(), words * 4, cudaMemcpyHostToDevice, s));
  GW_CUDA(cudaStreamSynchronize(s));
  return GEDWALK_OK;
}

}  // namespace gw

using namespace gw;

// ================================================================ C ABI
extern "C" {

void gedwalk_params_default(gedwalk_params* p) {
  if (!p) return;
  p->alpha = 0.0;
  p->epsilon = 1e-4;
  p->L = 0;
  p->precision = GEDWALK_FP32;
  p->greedy_eps_rule = GEDWALK_EPS_OVER_K;
  p->flags = 0;
  p->stream = 0;
  p->eta = 0.1;
  p->seed = 0;
}

const char* gedwalk_last_error(void) { return t_last_error.c_str(); }

gedwalk_status gedwalk_profile(int32_t enable) {
  Profiler& p = prof();
  std::lock_guard<std::mutex> lk(p.mu);
  for (auto& r : p.recs) {
    cudaEventSynchronize(r.b);
    p.pool.push_back(r.a);
    p.pool.push_back(r.b);
  }
  p.recs.clear();
  p.done.clear();
  p.launches.store(0);
  p.enabled.store(enable != 0);
  return GEDWALK_OK;
}

gedwalk_status gedwalk_profile_read(gedwalk_profile_stats* out) {
  if (!out) return fail(GEDWALK_ERR_INVALID, "out is NULL");
  Profiler& p = prof();
  std::lock_guard<std::mutex> lk(p.mu);
  double ms = 0.0, bytes = 0.0;
  struct Agg {
    int64_t n = 0;
    double ms = 0.0, bytes = 0.0;
  };
  std::vector<std::pair<int, Agg>> per;
  auto add = [&](double t, double b, int key) {
    ms += t;
    bytes += b;
    auto it = std::find_if(per.begin(), per.end(), [&](const std::pair<int, Agg>& e) { return e.first == key; });
    if (it == per.end()) {
      per.push_back({key, Agg()});
      it = per.end() - 1;
    }
    it->second.n++;
    it->second.ms += t;
    it->second.bytes += b;
  };
  for (auto& r : p.recs) {
    GW_CUDA(cudaEventSynchronize(r.b));
    float t = 0.0f;
    GW_CUDA(cudaEventElapsedTime(&t, r.a, r.b));
    add(t, r.bytes, r.key);
  }
  for (auto& d : p.done) add(d.ms, d.bytes, d.key);
  *out = gedwalk_profile_stats{};
  out->launches = p.launches.load();
  out->sweep_launches = static_cast<int64_t>(p.recs.size() + p.done.size());
  out->sweep_ms = ms;
  out->sweep_bytes = bytes;
  const std::pair<int, Agg>* top = nullptr;
  for (const auto& e : per)
    if (!top || e.second.ms > top->second.ms) top = &e;
  if (top) {
    out->top_fp64 = top->first % 2;
    out->top_cols = (top->first / 2) % 1000;
    out->top_mode = (top->first / 2) / 1000;
    out->top_launches = top->second.n;
    out->top_ms = top->second.ms;
    out->top_bytes = top->second.bytes;
  }
  return GEDWALK_OK;
}

gedwalk_status gedwalk_set_allocator(gedwalk_alloc_fn alloc, gedwalk_free_fn release, void* ctx) {
  if ((alloc == nullptr) != (release == nullptr))
    return fail(GEDWALK_ERR_INVALID, "allocator and release must both be set or both be NULL");
  g_alloc = alloc;
  g_free = release;
  g_alloc_ctx = ctx;
  return GEDWALK_OK;
}

gedwalk_status gedwalk_graph_upload(const int32_t* row_ptr, const int32_t* col_idx, int32_t n, int64_t nnz,
                                    int32_t flags, gedwalk_graph_t* out) {
  if (!out) return fail(GEDWALK_ERR_INVALID, "out is NULL");
  if (n < 1) return fail(GEDWALK_ERR_INVALID, "n must be >= 1");
  if (nnz < 0 || nnz >= (int64_t(1) << 31) - 8) return fail(GEDWALK_ERR_INVALID, "nnz must be in [0, 2^31 - 8)");
  if (!row_ptr || (nnz > 0 && !col_idx)) return fail(GEDWALK_ERR_INVALID, "row_ptr/col_idx is NULL");
  std::string why;
  const bool trusted = (flags & GEDWALK_UPLOAD_TRUSTED) != 0;
  {
    // row_ptr and index ranges are always checked (the plan and the kernels index with
    // them); TRUSTED skips the sortedness, self-loop and symmetry checks
    const int64_t bad = validate_csr(row_ptr, col_idx, n, nnz, !trusted, &why);
    if (bad >= 0)
      return fail(GEDWALK_ERR_INVALID, "malformed graph at row %lld: %s", static_cast<long long>(bad), why.c_str());
  }
  std::unique_ptr<Graph> g(new Graph());
  GW_CUDA(cudaGetDevice(&g->device));
  g->n = n;
  g->nnz = nnz;
  std::vector<int32_t> deg_old(n);
  int32_t dmax = 0;
  for (int32_t v = 0; v < n; ++v) {
    deg_old[v] = row_ptr[v + 1] - row_ptr[v];
    dmax = std::max(dmax, deg_old[v]);
  }
  g->dmax = dmax;
  g->alpha_default = 1.0 / (1.0 + dmax);
  // relabel: decreasing degree, ties by caller id (stable counting sort)
  std::vector<int64_t> start(static_cast<size_t>(dmax) + 2, 0);
  for (int32_t v = 0; v < n; ++v) start[dmax - deg_old[v] + 1]++;
  for (size_t i = 1; i < start.size(); ++i) start[i] += start[i - 1];
  g->perm.resize(n);
  g->inv.resize(n);
  for (int32_t v = 0; v < n; ++v) {
    const int64_t pos = start[dmax - deg_old[v]]++;
    g->perm[pos] = v;
    g->inv[v] = static_cast<int32_t>(pos);
  }
  g->deg.resize(n);
  std::vector<int32_t> rp(static_cast<size_t>(n) + 1);
  rp[0] = 0;
  for (int32_t i = 0; i < n; ++i) {
    g->deg[i] = deg_old[g->perm[i]];
    rp[i + 1] = rp[i] + g->deg[i];
  }
  std::vector<int32_t> ci(static_cast<size_t>(nnz) + 4, 0);
  const Graph* gp = g.get();
  parallel_rows(n, [&](int64_t b, int64_t e) {
    for (int64_t i = b; i < e; ++i) {
      const int32_t v = gp->perm[i];
      int32_t* dst = ci.data() + rp[i];
      const int32_t len = rp[i + 1] - rp[i];
      for (int32_t j = 0; j < len; ++j) dst[j] = gp->inv[col_idx[row_ptr[v] + j]];
      std::sort(dst, dst + len);
    }
  });
  GW_TRY(g->rp.ensure(rp.size() * sizeof(int32_t), 0));
  GW_TRY(g->ci.ensure(ci.size() * sizeof(int32_t), 0));
  GW_TRY(g->perm_d.ensure(static_cast<size_t>(n) * sizeof(int32_t), 0));
  GW_CUDA(cudaMemcpy(g->rp.p, rp.data(), rp.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  GW_CUDA(cudaMemcpy(g->ci.p, ci.data(), ci.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  GW_CUDA(cudaMemcpy(g->perm_d.p, g->perm.data(), static_cast<size_t>(n) * sizeof(int32_t), cudaMemcpyHostToDevice));
  GW_TRY(build_plan(*g, rp));
  *out = reinterpret_cast<gedwalk_graph_t>(g.release());
  return GEDWALK_OK;
}

gedwalk_status gedwalk_graph_free(gedwalk_graph_t h) {
  if (!h) return GEDWALK_OK;
  Graph* g = G(h);
  cudaDeviceSynchronize();
  delete g;
  return GEDWALK_OK;
}

gedwalk_status gedwalk_graph_info(gedwalk_graph_t h, int32_t* n, int64_t* nnz, int32_t* dmax, double* alpha_default) {
  if (!h) return fail(GEDWALK_ERR_INVALID, "graph is NULL");
  Graph* g = G(h);
  if (n) *n = g->n;
  if (nnz) *nnz = g->nnz;
  if (dmax) *dmax = g->dmax;
  if (alpha_default) *alpha_default = g->alpha_default;
  return GEDWALK_OK;
}

gedwalk_status gedwalk_truncation(gedwalk_graph_t h, double alpha, double epsilon, int32_t* L, double* bound) {
  if (!h || !L) return fail(GEDWALK_ERR_INVALID, "graph or L is NULL");
  Graph* g = G(h);
  std::lock_guard<std::mutex> lk(g->mu);
  if (alpha < 0.0 || std::isnan(alpha)) return fail(GEDWALK_ERR_INVALID, "alpha must be positive (0 = default)");
  if (alpha == 0.0) alpha = g->alpha_default;
  double b = 0;
  int32_t l = 0;
  GW_TRY(truncation_length(*g, alpha, epsilon, &l, &b, 0));
  *L = l;
  if (bound) *bound = b;
  return GEDWALK_OK;
}

}  // extern "C"
