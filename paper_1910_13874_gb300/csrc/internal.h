// Internal declarations shared by the library's translation units (not installed).
#pragma once

#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdint>
#include <cstring>
#include <memory>
#include <mutex>
#include <shared_mutex>
#include <string>
#include <utility>
#include <vector>

#include "gedwalk.h"

namespace gw {

// ---------------------------------------------------------------- errors
void set_error(const char* fmt, ...);
gedwalk_status fail(gedwalk_status st, const char* fmt, ...);

#define GW_CUDA(call)                                                                                 \
  do {                                                                                                \
    cudaError_t e_ = (call);                                                                          \
    if (e_ != cudaSuccess)                                                                            \
      return ::gw::fail(GEDWALK_ERR_DEVICE, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                        __FILE__, __LINE__);                                                          \
  } while (0)

#define GW_TRY(expr)                 \
  do {                               \
    gedwalk_status s_ = (expr);      \
    if (s_ != GEDWALK_OK) return s_; \
  } while (0)

// Counts a kernel launch and checks that it was accepted.
void count_launch();
#define GW_KCHECK()               \
  do {                            \
    GW_CUDA(cudaGetLastError());  \
    ::gw::count_launch();         \
  } while (0)

// ---------------------------------------------------------------- device memory
// The allocator a block came from: the caller's hook (gedwalk_set_allocator) or cudaMalloc
// (release == nullptr). Every block is freed through the allocator that made it, whatever the
// hook is when it is freed.
struct Allocator {
  gedwalk_free_fn release = nullptr;
  void* ctx = nullptr;
};
void* dalloc(size_t bytes, cudaStream_t s, Allocator* from);
void dfree(void* p, size_t bytes, cudaStream_t s, const Allocator& from);

// A device buffer that grows on demand and is released with its owner.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  Allocator from;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { release(); }
  void release() {
    if (p) dfree(p, bytes, 0, from);
    p = nullptr;
    bytes = 0;
  }
  // Exchanges two buffers (storage, size and the allocator that made the storage).
  void swap(DevBuf& o) {
    std::swap(p, o.p);
    std::swap(bytes, o.bytes);
    std::swap(from, o.from);
  }
  // Ensures capacity >= need bytes; contents are not preserved. zero: memset new storage to 0.
  gedwalk_status ensure(size_t need, cudaStream_t s, bool zero = false);
  template <typename T>
  T* as() const {
    return static_cast<T*>(p);
  }
};

// ---------------------------------------------------------------- sweep plan
// The masked SpMV/SpMM "sweep" y = alpha * A x runs one warp per work unit (int4):
//  - light unit {r0, r1, cls, -1}: rows [r0, r1) of one degree class; classes 0..5 give
//    2^cls lanes to a row of degree <= 2^(cls+1), class 6 a whole warp to a row of degree
//    <= kHeavyDeg;
//  - heavy slice {h, e0, e1, slice >= 0}: entries [e0, e1) of heavy row h (degree >
//    kHeavyDeg); the slices of a row are combined by the last warp to finish, in order.
constexpr int kThreads = 256;
constexpr int kHeavyDeg = 1024;
constexpr int kSliceEdges = 1024;
constexpr int kUnitEdges = 1024;      // entries per short-row unit (at least one row)
constexpr int kLongUnitEdges = 2048;  // entries per long-row unit (at least one row)
constexpr int kUnitRowsMax = 128;     // rows per unit (short classes); long units take <= 32
constexpr int kTargetUnits = 4096;    // small graphs get units of fewer rows, aiming at this many
constexpr int kReduceParts = 64;      // first-stage parts of the deterministic slot reduction
constexpr int64_t kL1HubBytes = 160 * 1024;  // x rows per SM kept in L1 with high priority

struct Plan {
  int32_t num_units = 0;   // grid size: heavy slices first, then light units
  int32_t num_slices = 0;  // heavy slices (units [0, num_slices))
  int32_t num_heavy = 0;   // heavy rows (degree > kHeavyDeg)
  int32_t num_slots = 0;   // num_units + num_heavy column-sum slots
  DevBuf units;            // int4[num_units]
  DevBuf heavy;            // int4[num_heavy]: {row, first slice, slice count, 0}
};

// ---------------------------------------------------------------- captured sweep sequences
// A greedy sweep sequence (initialisation, L sweeps, column-sum reduction) captured as a CUDA
// graph and replayed while its configuration is unchanged. Two external event nodes bracket the
// run of sweeps, so the profiler still sees their device time.
struct SweepGraph {
  cudaGraphExec_t exec = nullptr;
  std::vector<cudaEvent_t> ev;  // start and end of the run of sweeps
  uint64_t key = 0;             // configuration of the captured sequence
  int uses = 0;                 // direct runs of this configuration before it is captured
  int kernels = 0;              // kernel nodes per replay
  int sweeps = 0;               // sweep kernels per replay
  double bytes = 0.0;           // algorithmic bytes per sweep
  int prof_key = 0;
  bool timing_pending = false;  // replayed while profiling; events not read yet
  uint64_t last_use = 0;        // recency, for eviction from a workspace's cache
  void reset();
  SweepGraph() = default;
  SweepGraph(const SweepGraph&) = delete;
  SweepGraph& operator=(const SweepGraph&) = delete;
  ~SweepGraph() { reset(); }
};

// ---------------------------------------------------------------- workspaces
// Per-request scratch. The graph owns one for the synchronous API; the server
// creates one per concurrent request slot.
struct Workspace {
  DevBuf x0, x1;     // walk vectors, [n][C]
  DevBuf mtab;       // phi^miss table, [(L+1)][n]
  DevBuf ztab;       // directed graphs: psi^miss table (walks in the other orientation), [(L+1)][n]
  DevBuf pvec;       // power iteration: three FP64 vectors and the statistics
  DevBuf partial;    // heavy-slice partial sums, [num_slices][C]
  DevBuf counters;   // heavy-row arrival counters, [num_heavy] (kept at 0 between launches)
  DevBuf slots;      // column-sum slots, [num_slots][C] doubles
  DevBuf parts;      // slot-reduction partials, [C][kReduceParts] doubles
  DevBuf mask;       // S bitmask, [ceil(n/32)]
  DevBuf stale;      // greedy: {float upper bound, int step} per vertex
  DevBuf sel;        // greedy: per-block candidate lists
  DevBuf small;      // small device-side results
  DevBuf members;    // batched scoring: member ids / group ids / accumulators
  DevBuf pinned_dummy;
  int64_t st_evals = 0, st_batches = 0, st_sweeps = 0, st_spec_miss = 0;  // last maximize
  std::vector<int32_t> st_ell;  // last maximize: the walk length of each step
  int64_t st_sep_fail = 0;      // last maximize: failed separation tests (l doublings)
  // captured greedy sequences, one per configuration (mode, width, graph, L, alpha, buffers); a
  // serving worker that alternates between graphs keeps each graph's sequences
  static constexpr int kGraphCache = 16;
  SweepGraph graphs[kGraphCache];
  uint64_t graph_clock = 0;
  SweepGraph greedy_loop;  // the device-resident greedy loop of the last configuration
  DevBuf ctl;              // its controller state and outputs
  cudaStream_t own_stream = nullptr;  // capturable stream used when the caller passes stream 0
  cudaEvent_t order_ev = nullptr;     // orders own_stream after the caller's stream
  std::vector<uint8_t> host_small;  // staging
  void* pinned = nullptr;           // pinned host staging buffer
  size_t pinned_bytes = 0;
  ~Workspace();
  gedwalk_status ensure_pinned(size_t bytes);
  // Device bytes the workspace holds now (its buffers only; the captured graphs hold none).
  int64_t device_bytes() const;
  // Releases every device buffer and the captured sequences that refer to them (the workspace
  // must be idle: no call is using it and nothing of it is in flight on the device).
  void release_device();
};

// ---------------------------------------------------------------- graph
struct Graph {
  int device = 0;
  int32_t n = 0;
  int64_t nnz = 0;
  int32_t dmax = 0;
  int32_t n_active = 0;     // rows with at least one entry; isolated rows are [n_active, n)
  double alpha_default = 0;
  // Weighted walks (Section 5.4) with vertex-separable weights w(v,u) = s_v s_u: rs_* hold s by
  // new id (empty for an unweighted graph). delta is the degree of the combinatorial bound:
  // d_max, or the largest weighted degree max_v s_v sum_u s_u.
  bool weighted = false;
  double delta = 0;
  DevBuf rs_f, rs_d;
  // Directed graphs (Section 2): rp/ci/plan hold the successor lists; the reverse CSR (row v: the
  // u with an arc u -> v) serves the sweeps that count walks in the other orientation (psi of
  // Lemma initialize, the walk-total table of batched scoring).
  bool directed = false;
  DevBuf rp_r, ci_r;
  Plan plan_r;
  std::vector<int32_t> deg_r;
  // certified upper bound of sigma_max (0: not computed) and the last Rayleigh estimate
  double sigma_up = 0.0, sigma_lo = 0.0;
  DevBuf rp, ci;            // relabelled CSR (new ids), ci padded by 4 entries
  DevBuf perm_d;            // int32[n]: new -> caller id
  std::vector<int32_t> perm;  // new -> caller id
  std::vector<int32_t> inv;   // caller id -> new
  std::vector<int32_t> deg;   // degree by new id (directed graphs only; else the row pointers give it)
  Plan plan;

  // alpha-scaled walk totals t_r = alpha A t_{r-1}, t_0 = 1 (FP64, [rows][n]; on a weighted graph
  // the rows hold s * t_r, the form the sweeps gather) and their sums Wa[r] = 1^T t_r
  double tt_alpha = -1.0;
  int32_t tt_rows = 0;
  DevBuf ttab;
  std::vector<double> Wa;
  DevBuf Wa_d;  // the same sums on the device, where the truncation test reads them
  // readers of ttab hold it shared; growing or replacing the table holds it exclusively
  std::shared_mutex tt_lock;
  // truncation lengths already found: {alpha, epsilon, L, B_L}
  struct Trunc {
    double alpha, eps;
    int32_t L;
    double bound;
    int32_t kind;  // the tail bound used
  };
  std::vector<Trunc> trunc_cache;

  // batched-scoring autotuner result: column-block width per graph (0 = not tuned)
  int32_t batch_cols = 0;
  std::vector<std::pair<int32_t, double>> tune_log;

  // statistics of the last maximize
  int64_t st_evals = 0, st_batches = 0, st_sweeps = 0, st_spec_miss = 0;
  std::vector<int32_t> st_ell;
  int64_t st_sep_fail = 0;

  Workspace ws;    // workspace of the synchronous API
  std::mutex mu;   // serialises calls on this handle
};

// ---------------------------------------------------------------- launchers
enum SweepMode : int {
  MODE_TOTALS = 0,  // y = alpha A x, FP64, stores the column sum
  MODE_SCORE = 1,   // two-state hit/miss step, sums h
  MODE_FUSED = 2,   // greedy: column 0 = phi^miss under S, columns 1.. candidate columns
  MODE_CAND = 3,    // greedy: candidate columns only; candidate rows read phi^miss from a table
  MODE_PLAIN = 4,   // batched scoring: y = alpha A x, no mask
  MODE_LOOK = 5     // greedy lookahead: phi^miss under S, then the walks through c_j avoiding S + {c_1..c_{j-1}}
};

struct SweepArgs {
  const int32_t* rp;
  const int32_t* ci;
  const int4* units;
  const int4* heavy;
  int32_t num_units;
  int32_t n;
  int64_t nnz;
  const void* X;
  void* Y;
  double alpha;
  const uint32_t* mask;
  void* partial;
  unsigned* counters;
  double* slots;
  int32_t accumulate;
  void* Mout;
  int64_t mout_stride;  // MODE_LOOK: elements between the phi^miss tables of consecutive levels
  const void* Min;
  const int32_t* cand;
  int32_t hub;  // rows [0, hub) of x are gathered with L1 retention priority (set by the launcher)
  // Vertex scales s of a weighted graph (nullptr: unweighted). Vectors are then gathered in the
  // scaled form x~ = s * x: (N x)(v) = s_v (A x~)(v) for N = diag(s) A diag(s), so the epilogue
  // computes the true value alpha s_v (A x~)(v), sums it, and stores it times s_v.
  const float* rs_f;
  const double* rs_d;
  // MODE_CAND with the table chosen on the device: candidate rows read Min + level * level_stride
  // (level read from level_ptr once per launch; nullptr: Min as given)
  const int32_t* level_ptr;
  int64_t level_stride;
};

// Profiling hooks around sweep launches (no-ops unless gedwalk_profile(1) was called).
bool profiling();
void profile_begin(cudaStream_t s, cudaEvent_t* a);
void profile_end(cudaStream_t s, cudaEvent_t a, double bytes, int key);
// Adds one timed sweep launch measured outside the event list (graph replays).
void profile_add(double ms, double bytes, int key);
// Counts n kernel launches (graph replays).
void count_launches(int n);
// Marks the calling thread as capturing a graph (its launches are counted when the graph runs).
void set_capturing(bool on);
// Algorithmic bytes of one sweep launch: CSR once, x read once, y written once, plus the mask
// and the phi^miss row where the mode reads or writes them.
double sweep_bytes(int mode, bool fp64, int cols, int32_t n, int64_t nnz, bool weighted = false);

// Sets a sweep instantiation's launch attributes on the current device (before a stream capture
// that launches it; launch_sweep does it on first use otherwise).
gedwalk_status configure_sweep(int mode, bool fp64, int cols);
// Launches one sweep (instantiated for the supported (type, columns, mode) triples).
gedwalk_status launch_sweep(int mode, bool fp64, int cols, const SweepArgs& a, cudaStream_t s, bool profile = true);
// Column-sum count of a mode at width cols.
int sweep_sums(int mode, int cols);
// out[c] = sum over slots of slots[slot][c], c < nsum, in a fixed order (parts: nsum*kReduceParts).
gedwalk_status launch_reduce_slots(const double* slots, int32_t num_slots, int32_t nsum, double* out,
                                   double* parts, cudaStream_t s);
// The same over a workspace's slots after sweeps of width cols.
gedwalk_status reduce_slots(Graph& g, Workspace& ws, int nsum, double* out, cudaStream_t s, bool rev = false);

// Ensures workspace scratch for sweeps of width cols (partials, counters, slots).
gedwalk_status ensure_sweep_scratch(Graph& g, Workspace& ws, int cols, bool fp64, cudaStream_t s);
// Fills a SweepArgs with the graph/plan/scratch fields.
SweepArgs base_args(Graph& g, Workspace& ws);
// The same over the reverse CSR of a directed graph.
SweepArgs base_args_rev(Graph& g, Workspace& ws);

// ---------------------------------------------------------------- shared algorithm helpers
struct Resolved {
  double alpha;
  int32_t L;
  double bound;  // B_L, NaN when L was forced without a valid bound
  bool fp64;
  cudaStream_t stream;
  double eta = 0.1;    // stochastic greedy sample parameter
  uint64_t seed = 0;   // stochastic greedy seed
  double eps = 0.0;    // the epsilon L was selected for (0 when L was forced)
  int32_t bound_kind = 0;  // GEDWALK_BOUND_COMBINATORIAL or GEDWALK_BOUND_SPECTRAL
  int32_t lookahead = 0;   // gedwalk_params.lookahead (0 = default)
  int32_t spec_cols = 0;   // gedwalk_params.spec_cols (0 = default)
};

// The configuration of one greedy maximisation (sweep widths, lookahead levels, table rows),
// fixed before it starts; maximize_impl runs it and maximize_footprint sizes it.
struct GreedyShape {
  int32_t levels;     // lookahead levels per run of sweeps (1 = no lookahead)
  int32_t cols_fused; // columns of the fused sweep (phi^miss + speculative candidates)
  int32_t cols_cand;  // columns of a candidate batch
  int32_t cols_all;   // columns per batch of GEDWALK_GAINS_ALL
  int32_t tab_L;      // rows 0..tab_L of every phi^miss table
  int32_t ell_max;    // adaptive: the largest walk length it may reach (else L)
  int32_t cols_max;   // widest sweep of the run (walk vectors are sized for it)
};
gedwalk_status greedy_shape(const Graph& g, const Resolved& r, int32_t flags, GreedyShape* out);
// Device bytes a maximisation of k vertices with this configuration needs in its workspace.
int64_t maximize_footprint(const Graph& g, const Resolved& r, int32_t flags, int32_t k);
// Device bytes a batched scoring of `groups` groups with `members` members needs in its workspace.
int64_t score_batch_footprint(const Graph& g, int64_t members, int32_t groups);
// Resolves alpha (0 -> default), L (from epsilon unless forced) for a given epsilon.
gedwalk_status resolve(Graph& g, const gedwalk_params* p, double eps_override, Resolved* r);
// Ensures the FP64 walk-total table holds rows 0..rows-1 for alpha.
gedwalk_status ensure_totals(Graph& g, double alpha, int32_t rows, cudaStream_t s);
// Truncation length from the chosen tail bound (device-side test).
gedwalk_status truncation_length(Graph& g, double alpha, double eps, int32_t* L, double* bound, cudaStream_t s,
                                 int32_t kind = 0);
// Coefficient c of the tail bound B_l = c * Wa_l for (alpha, kind); NOT_CONVERGENT when it does not apply.
gedwalk_status bound_coef(Graph& g, double alpha, int32_t kind, cudaStream_t s, double* coef);
// Maps caller ids to internal ids with set semantics; INVALID on out-of-range ids.
gedwalk_status map_group(const Graph& g, const int32_t* S, int32_t s_len, std::vector<int32_t>* out);
// Uploads the S bitmask (internal ids) into ws.mask.
gedwalk_status upload_mask(Graph& g, Workspace& ws, const std::vector<int32_t>& S_int, cudaStream_t s);

gedwalk_status score_one(Graph& g, Workspace& ws, const std::vector<int32_t>& S_int, const Resolved& r,
                         double* score);
// Picks the batched-scoring column width for this graph (timed once, then cached).
gedwalk_status autotune_batch(Graph& g, Workspace& ws, const Resolved& r);
gedwalk_status score_batch_impl(Graph& g, Workspace& ws, const int32_t* offsets, const int32_t* members_int,
                                int32_t G, const Resolved& r, double* scores);
gedwalk_status maximize_impl(Graph& g, Workspace& ws, int32_t k, const Resolved& r, int32_t flags,
                             const std::vector<int32_t>& init_int, int32_t* group, double* gains, double* score);
gedwalk_status gains_impl(Graph& g, Workspace& ws, const std::vector<int32_t>& S_int, const Resolved& r,
                          double* gains_caller);

inline Graph* G(gedwalk_graph_t h) { return reinterpret_cast<Graph*>(h); }

}  // namespace gw
