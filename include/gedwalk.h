/*
 * gedwalk.h - C ABI of the GB300 GED-Walk library (libgedwalk.so).
 *
 * GED-Walk group centrality (Angriman, van der Grinten, Bojchevski, Zuegner,
 * Guennemann, Meyerhenke, "Group Centrality Maximization for Large-scale
 * Graphs", ALENEX 2020):
 *
 *   GED(S) = sum_{i>=1} alpha^i * phi_i(S)              (Def. ged-walk, Eq. ged_def)
 *
 * where phi_i(S) is the number of length-i walks that contain at least one
 * vertex of S (Def. ed-walk). The library evaluates the truncated sum
 * GED_{<=L}(S) (Section 3.1) and maximises it greedily (Def. ged-max,
 * Section 3.2) on an NVIDIA GB300 (sm_103a).
 *
 * Conventions shared by every entry point
 *  - Every call returns a gedwalk_status. Output buffers are caller-owned host
 *    memory and are written only when the call returns GEDWALK_OK.
 *  - Host inputs are copied; the caller keeps ownership of them. Device memory
 *    belongs to the library (see gedwalk_set_allocator).
 *  - Graphs are undirected and unweighted (Section 2): a CSR with int32
 *    row_ptr[n+1] and col_idx[nnz], every row strictly increasing, no
 *    self-loops, and (u,v) present iff (v,u) is. Each undirected edge is two
 *    entries, so it yields two 1-walks.
 *  - Vertex ids in S, groups and results are the caller's ids in [0, n).
 *    Groups have set semantics: repeated ids count once. An id outside
 *    [0, n) returns GEDWALK_ERR_INVALID.
 *  - Ties in the greedy argmax go to the lowest vertex id.
 *  - gedwalk_last_error() returns a message for the last failing call made by
 *    the calling thread.
 *  - One graph handle may be used from several threads; calls on the same
 *    handle are serialised inside the library.
 */
#ifndef GEDWALK_H
#define GEDWALK_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define GEDWALK_API __attribute__((visibility("default")))
#else
#define GEDWALK_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gedwalk_graph* gedwalk_graph_t; /* opaque, device-resident, owned by the library */
typedef struct gedwalk_server* gedwalk_server_t;

typedef enum {
  GEDWALK_OK = 0,
  GEDWALK_ERR_INVALID = 1,        /* bad argument or malformed graph */
  GEDWALK_ERR_OOM = 2,            /* a device or host allocation failed; state is unchanged */
  GEDWALK_ERR_NOT_CONVERGENT = 3, /* alpha >= 1/d_max and no forced L: the bound does not apply */
  GEDWALK_ERR_DEVICE = 4,         /* a CUDA call failed (message in gedwalk_last_error) */
  GEDWALK_ERR_TIMEOUT = 5,        /* a bounded wait expired */
  GEDWALK_ERR_BUSY = 6,           /* serving: no admission slot or memory left */
  GEDWALK_ERR_NOT_FOUND = 7       /* serving: unknown ticket */
} gedwalk_status;

/* precision of the walk vectors; sums of alpha^i-weighted counts are always FP64 */
enum { GEDWALK_FP64 = 0, GEDWALK_FP32 = 1 };

/* gedwalk_params.greedy_eps_rule: how epsilon sets L for maximisation */
enum {
  GEDWALK_EPS_OVER_K = 0, /* L from the bound at epsilon/k (Algorithm 2 separates at epsilon/k) */
  GEDWALK_EPS_PLAIN = 1   /* L from the bound at epsilon */
};

/* gedwalk_params.flags */
enum {
  GEDWALK_GAINS_ALL = 1,  /* maximize: evaluate every vertex's exact gain at every step (no pruning) */
  GEDWALK_STOCHASTIC = 2, /* maximize: stochastic greedy (Appendix D), see gedwalk_maximize */
  GEDWALK_ADAPTIVE_L = 4, /* maximize: lazy greedy with l-doubling (Algorithm 2), see gedwalk_maximize */
  GEDWALK_DEVICE_LOOP = 8 /* maximize: with the lookahead on, run the k steps as one device-resident
                           * CUDA graph instead of the host loop; same kernels, same result */
};

/* gedwalk_graph_upload flags */
enum {
  GEDWALK_UPLOAD_TRUSTED = 1, /* skip the sortedness / symmetry / self-loop validation */
  GEDWALK_UPLOAD_DIRECTED = 2 /* the rows are successor lists of a directed graph (no symmetry) */
};

typedef struct {
  double alpha;            /* walk damping; 0 selects 1/(1+d_max). Must be > 0. */
  double epsilon;          /* additive error for the truncation bound; > 0 unless L > 0 */
  int32_t L;               /* 0: smallest l with B_l < epsilon (Algorithm 1); > 0: forced length */
  int32_t precision;       /* GEDWALK_FP64 or GEDWALK_FP32 */
  int32_t greedy_eps_rule; /* GEDWALK_EPS_OVER_K (default) or GEDWALK_EPS_PLAIN */
  int32_t flags;           /* GEDWALK_GAINS_ALL, GEDWALK_STOCHASTIC, GEDWALK_ADAPTIVE_L, GEDWALK_DEVICE_LOOP */
  int64_t stream;          /* cudaStream_t to run on (e.g. torch.cuda.current_stream().cuda_stream); 0 = default */
  double eta;              /* stochastic greedy: sample (n/k) ln(1/eta) vertices per step, 0 < eta < 1 */
  uint64_t seed;           /* stochastic greedy: seed of the counter-based sample draws */
  int32_t bound;           /* GEDWALK_BOUND_COMBINATORIAL (default) or GEDWALK_BOUND_SPECTRAL */
  int32_t lookahead;       /* maximize: greedy steps carried by one run of sweeps (see gedwalk_maximize):
                              0 = default (7 in FP32, 3 in FP64), 1 = off, 3 or (FP32) 7 */
  int32_t spec_cols;       /* maximize without lookahead: columns of the fused sweep (phi^miss plus
                              speculative candidates): 0 = default (2; 4 with GEDWALK_ADAPTIVE_L), 2, 4
                              or (FP32) 8 */
  int32_t reserved;        /* 0 */
} gedwalk_params;

/* gedwalk_params.bound: the tail bound behind every truncation length */
enum {
  GEDWALK_BOUND_COMBINATORIAL = 0, /* Eq. comb-bound: needs alpha < 1/d_max (1/delta) */
  GEDWALK_BOUND_SPECTRAL = 1       /* Lemma spectral-bound: needs alpha < 1/sigma_max, see gedwalk_sigma_max */
};

/* Fills *p with the defaults: alpha 0, epsilon 1e-4, L 0, FP32, EPS_OVER_K, no flags, stream 0,
 * eta 0.1, seed 0, the combinatorial bound, lookahead 0, spec_cols 0. (alpha, epsilon and the
 * epsilon/k rule are those of Section 3.1.2 and Algorithm 2; the rest has no counterpart in the
 * paper.) */
GEDWALK_API void gedwalk_params_default(gedwalk_params* p);

/*
 * Device memory hook (no counterpart in the paper). alloc(bytes, stream, ctx) returns device
 * memory or NULL;
 * release(ptr, bytes, stream, ctx) frees it. Passing NULL restores the
 * built-in cudaMalloc/cudaFree. The Python binding installs PyTorch's caching
 * allocator here when it loads the library. The hook applies to every later
 * allocation of the process; each block is freed through the allocator that
 * allocated it, so the functions of a replaced hook must stay callable while
 * blocks they allocated are alive. Before calling a hook's release the library
 * waits for the device (as cudaFree does), since a caching allocator may hand
 * the block to another stream at once. Set it while no other call is running.
 */
typedef void* (*gedwalk_alloc_fn)(size_t bytes, int64_t stream, void* ctx);
typedef void (*gedwalk_free_fn)(void* ptr, size_t bytes, int64_t stream, void* ctx);
GEDWALK_API gedwalk_status gedwalk_set_allocator(gedwalk_alloc_fn alloc, gedwalk_free_fn release, void* ctx);

/*
 * Uploads a graph to the current CUDA device (Section 2: an undirected,
 * unweighted graph G = (V, E); each edge {u, v} is stored as the two entries
 * (u, v) and (v, u), the two 1-walks it carries).
 *  row_ptr: host int32[n+1], row_ptr[0] = 0, non-decreasing, row_ptr[n] = nnz.
 *  col_idx: host int32[nnz], see the conventions above.
 *  n >= 1; nnz >= 0 and < 2^31.
 *  flags: GEDWALK_UPLOAD_TRUSTED skips validation (a malformed graph then gives
 *  unspecified results, never a device fault: indices are still range-checked).
 * The library relabels vertices by decreasing degree internally (ties by id) for
 * gather locality; results are always reported in the caller's ids. The arrays
 * are copied to the device once; the checks, the relabelling and the sorting of
 * every row run there (the upload briefly holds a second copy of col_idx on the
 * device). The call returns after the device work is done.
 * GEDWALK_UPLOAD_DIRECTED: the rows are successor lists of a directed graph (see
 * the flag); no symmetry is required.
 * On success *out receives a handle to release with gedwalk_graph_free.
 * Errors: INVALID (malformed input, with the first offending row named in
 * gedwalk_last_error), OOM, DEVICE.
 */
GEDWALK_API gedwalk_status gedwalk_graph_upload(const int32_t* row_ptr, const int32_t* col_idx, int32_t n, int64_t nnz,
                                    int32_t flags, gedwalk_graph_t* out);

/*
 * Weighted GED-Walk (Section 5.4): a walk of length i contributes alpha^i times
 * the product of its edge weights, the weights entering the recurrences as
 * coefficients. This upload takes vertex-separable weights
 *   w(v, u) = vertex_scale[v] * vertex_scale[u]
 * on the edges of the same undirected CSR as gedwalk_graph_upload. With
 * vertex_scale NULL the weights are those of the symmetrically normalised
 * adjacency D^{-1/2} A D^{-1/2} (vertex_scale[v] = deg(v)^{-1/2}), the weighting
 * the paper's applications use. No per-entry value array is stored: sweeps
 * gather the scaled vectors s * x and scale each row once.
 *  vertex_scale: host double[n] (copied; positive and finite) or NULL.
 * The combinatorial bound then uses delta = max_v s_v sum_{u ~ v} s_u (the
 * largest weighted degree, which bounds W_{l+1}/W_l) in place of d_max, and
 * the default alpha is 1/(1 + delta). Every other entry point works on the
 * weighted graph unchanged. Errors as gedwalk_graph_upload.
 */
GEDWALK_API gedwalk_status gedwalk_graph_upload_weighted(const int32_t* row_ptr, const int32_t* col_idx, int32_t n,
                                             int64_t nnz, const double* vertex_scale, int32_t flags,
                                             gedwalk_graph_t* out);

/* *weighted = 1 for a graph from gedwalk_graph_upload_weighted; *delta the degree of the
 * combinatorial bound (Eq. comb-bound: d_max, or for the weighted walks of Section 5.4 the
 * largest weighted degree). Either pointer may be NULL. */
GEDWALK_API gedwalk_status gedwalk_graph_info_weighted(gedwalk_graph_t g, int32_t* weighted, double* delta);

/* Releases a graph and all device memory tied to it. NULL is accepted. (Resource management: no
 * counterpart in the paper.) */
GEDWALK_API gedwalk_status gedwalk_graph_free(gedwalk_graph_t g);

/* n, nnz (directed entries), d_max and the default alpha 1/(1+d_max), which lies below 1/d_max as
 * the combinatorial bound requires (Section 3.1.2, Eq. comb-bound). Any pointer may be NULL. */
GEDWALK_API gedwalk_status gedwalk_graph_info(gedwalk_graph_t g, int32_t* n, int64_t* nnz, int32_t* dmax, double* alpha_default);

/*
 * Truncation length for (alpha, epsilon) (Algorithm 1 with the combinatorial
 * bound, Eq. comb-bound): the smallest l >= 1 with
 *   B_l = alpha^{l+1} d_max / (1 - alpha d_max) * W_l < epsilon,
 * W_l the number of l-walks of G. The walk totals come from FP64 sweeps on the
 * device and the test B_l < epsilon runs on the device.
 *  alpha 0 selects the default. *L receives l, *bound (may be NULL) B_l.
 * Errors: NOT_CONVERGENT (alpha*d_max >= 1), INVALID (epsilon <= 0, or no
 * l <= 4096 qualifies).
 */
GEDWALK_API gedwalk_status gedwalk_truncation(gedwalk_graph_t g, double alpha, double epsilon, int32_t* L, double* bound);

/*
 * Largest singular value of the adjacency matrix A, sigma_max = ||A||_2 (the
 * spectral bound's sigma, Lemma spectral-bound; Appendix E takes alpha =
 * delta / sigma_max). Power iteration on A (undirected or weighted: symmetric,
 * sigma_max = its spectral radius) or on A^T A (directed: sigma_max^2), in FP64
 * sweeps on the device, from the all-ones vector kept positive. Every iterate x
 * certifies rho <= max_v (M x)(v) / x(v) (Collatz-Wielandt bound of a
 * non-negative matrix); *upper is the smallest such value met, inflated by
 * 1e-12 relative against rounding, so upper >= sigma_max always holds. *lower
 * is the last Rayleigh quotient, sqrt(x^T M x / x^T x) <= sigma_max. The graph
 * keeps the smallest upper value as the sigma of its spectral bound.
 *  iters: power iterations, 1..100000. upper/lower: may be NULL.
 */
GEDWALK_API gedwalk_status gedwalk_sigma_max(gedwalk_graph_t g, int32_t iters, double* upper, double* lower);

/*
 * gedwalk_truncation with a choice of bound: GEDWALK_BOUND_COMBINATORIAL as
 * above, or GEDWALK_BOUND_SPECTRAL (Lemma spectral-bound):
 *   B_l = sqrt(n) alpha^{l+1} sigma / (1 - alpha sigma) W_l,  sigma >= sigma_max
 * the graph's certified value (computed on first use with 300 iterations when
 * gedwalk_sigma_max has not run). Errors: NOT_CONVERGENT when alpha * sigma >= 1.
 */
GEDWALK_API gedwalk_status gedwalk_truncation_ex(gedwalk_graph_t g, double alpha, double epsilon, int32_t bound_kind,
                                     int32_t* L, double* bound);

/*
 * GED_{<=L}(S) of one group (problem (i), Algorithm 1), by the two-state
 * hit/miss recurrences of Section 3.1.1 run as a masked two-column SpMV:
 *   h_i = alpha (A h_{i-1} + 1_S . A m_{i-1}),  m_i = alpha 1_{V\S} . A m_{i-1},
 *   score += sum_v h_i(v)  (FP64),
 * starting from h_0 = 1_S, m_0 = 1_{V\S}.
 *  S: host int32[s_len] (s_len >= 0; S may be NULL when s_len is 0).
 *  params: NULL means the defaults; params->precision picks FP64 or FP32 walk
 *  vectors.
 *  score: the partial sum, a lower bound with GED(S) in [score, score + bound].
 *  L_used, tail_bound: may be NULL; receive L and B_L.
 */
GEDWALK_API gedwalk_status gedwalk_score(gedwalk_graph_t g, const int32_t* S, int32_t s_len, const gedwalk_params* params,
                             double* score, int32_t* L_used, double* tail_bound);

/*
 * Scores G groups at once (problem (i) for many groups). Group j is
 * members[offsets[j] .. offsets[j+1]). Groups become the columns of one masked
 * FP32 SpMM over column blocks whose width an on-device autotuner picks; the
 * per-group hit sums are FP64. The hits are counted by first visits:
 *   GED_{<=L}(S) = sum_{s in S} sum_{p=0..L} alpha^p F_p(s) * K_{L-p}(s),
 * F_p(s) the p-walks ending at s whose earlier vertices avoid S, and K_q(s) the
 * alpha-weighted walks of length <= q starting at s (the p = 0 term excludes
 * the empty walk). This equals the two-state sum of gedwalk_score.
 *  offsets: host int32[G+1], offsets[0] = 0, non-decreasing.
 *  members: host int32[offsets[G]].
 *  scores: host double[G]. L_used may be NULL.
 * params->precision is ignored (FP32 vectors, FP64 sums).
 */
GEDWALK_API gedwalk_status gedwalk_score_batch(gedwalk_graph_t g, const int32_t* offsets, const int32_t* members, int32_t G,
                                   const gedwalk_params* params, double* scores, int32_t* L_used);

/*
 * (Measurement of the batched scoring of gedwalk_score_batch; no counterpart in the paper.)
 * The batched-scoring autotuner's record for this graph (empty before the first
 * gedwalk_score_batch): for each column-block width tried, cols[j] and the
 * measured sweep time per column us_per_col[j] (microseconds, one unmasked
 * FP32 sweep of that width divided by its columns); *chosen the width in use
 * (0 before tuning). Up to cap entries are written; *count receives how many
 * exist. count and chosen may be NULL.
 */
GEDWALK_API gedwalk_status gedwalk_batch_tuning(gedwalk_graph_t g, int32_t* cols, double* us_per_col, int32_t cap,
                                    int32_t* count, int32_t* chosen);

/* (Tuning of gedwalk_score_batch; no counterpart in the paper.)
 * Pins the batched-scoring column-block width of this graph to cols (8, 16, 32 or 64; the
 * autotuner does not run), or with 0 lets the next gedwalk_score_batch tune it again. For runs
 * whose timing would mislead the tuner, such as under a profiler. */
GEDWALK_API gedwalk_status gedwalk_batch_set_width(gedwalk_graph_t g, int32_t cols);

/*
 * Exact truncated marginal gain GED_{<=L}(S, x) = GED_{<=L}(S + x) - GED_{<=L}(S)
 * (the lower bound L_l of Section 3.2.1) for every vertex x, counted directly as
 * the alpha-weighted walks of length 1..L that visit x and avoid S (proof of
 * Prop. ged_submod). Members of S get 0.
 *  gains: host double[n] in caller ids. L_used may be NULL.
 */
GEDWALK_API gedwalk_status gedwalk_gains(gedwalk_graph_t g, const int32_t* S, int32_t s_len, const gedwalk_params* params,
                             double* gains, int32_t* L_used);

/*
 * Greedy GED-Walk maximisation (problem (ii), Def. ged-max; the
 * (1-1/e)-approximation of Prop. greedy_approx): k times, add the vertex with
 * the largest truncated marginal gain GED_{<=L}(S, x), lowest id among equal
 * gains, at a fixed L (params: EPS_OVER_K takes L from the bound at
 * epsilon/k, as Algorithm 2 separates at epsilon/k; EPS_PLAIN at epsilon).
 * Each step bounds every gain from above by the smaller of its last exact value
 * (submodularity, Prop. ged_submod) and sum_i alpha^i P_i(S, x) (Lemma
 * initialize), evaluates the best-bounded candidates exactly in batches, and
 * accepts the best once no unevaluated bound can reach it.
 *  k >= 0 and init_len + k <= n.
 *  group: host int32[k], the added vertices in order.
 *  gains: host double[k], the gain of each addition (may be NULL).
 *  score: GED_{<=L} of init + group (may be NULL). Without an init group (and
 *         without GEDWALK_ADAPTIVE_L) it is the sum of the gains: each gain is
 *         GED_{<=L}(S + c) - GED_{<=L}(S), and GED_{<=L} of the empty set is 0.
 *  L_used: may be NULL.
 *  init_group/init_len: resume from this prefix group (may be NULL/0).
 * GEDWALK_GAINS_ALL in params->flags evaluates every vertex at every step.
 * GEDWALK_STOCHASTIC runs stochastic greedy (Appendix D): at step s only a sample
 * competes, vertex v (caller id, not in S) being sampled iff
 *   splitmix64(seed ^ (s << 32) ^ v) < p * 2^64,  p = min(1, m / |V \ S|),
 *   m = ceil((n/k) ln(1/eta)),
 * where splitmix64(x) is the first output of that generator started from state x;
 * an empty sample falls back to all of V \ S. The argmax within the sample is exact.
 * It cannot be combined with GEDWALK_GAINS_ALL or an init group.
 * Without a flag, on an undirected graph, each run of sweeps also computes the
 * next steps' phi^miss vectors and exact gains for guessed winners (lookahead):
 * a step whose winner was guessed needs no sweep. Every pick is still certified
 * against the bounds of the actual group, so the results do not depend on it.
 * params->lookahead (1 = off, 3; 7 in FP32) sets the number of steps per run
 * (0: 7 in FP32, 3 in FP64); params->spec_cols the width of the one-step fused
 * sweep when the lookahead is off. Other values return INVALID.
 * The host drives the steps: one synchronisation per bound pass, to read the
 * selection. With the lookahead on, GEDWALK_DEVICE_LOOP runs the k steps as one
 * device-resident CUDA graph instead (conditional nodes: the certification loop
 * never returns to the host). The picks and gains do not depend on it.
 * GEDWALK_ADAPTIVE_L runs the lazy greedy of Algorithm 2 (Section 3.2.3): the
 * walk length l starts at 1 and only doubles. At each step u, the vertex with the
 * largest L_l(S, u) = GED_{<=l}(S, u), is taken when it is separated from v, the
 * best of the rest: L_l(S, u) > L_l(S, v) + B_l - eps_sep, with B_l the
 * combinatorial bound (Eq. comb-bound) and eps_sep = epsilon/k (EPS_OVER_K) or
 * epsilon (EPS_PLAIN); otherwise l doubles and the step is retried. Then
 * gains[j] is L_l(S, u) at step j's l, *L_used the final l, and score the value
 * computed without the flag (GED_{<=L} of the group, L from the bound at
 * eps_sep). It needs params->L = 0 and cannot be combined with
 * GEDWALK_GAINS_ALL, GEDWALK_STOCHASTIC or an init group (INVALID).
 */
GEDWALK_API gedwalk_status gedwalk_maximize(gedwalk_graph_t g, int32_t k, const gedwalk_params* params, int32_t* group,
                                double* gains, double* score, int32_t* L_used, const int32_t* init_group,
                                int32_t init_len);

/*
 * (Measurement; the paper expects its lazy greedy to evaluate few vertices, Section 3.2.3.)
 * Counters of the last gedwalk_maximize on this graph: exact-gain evaluations
 * (candidate columns), candidate batches, sweep-kernel launches and the
 * batches whose speculation (candidates chosen before the new S was known)
 * failed to certify the winner. Any pointer may be NULL.
 */
GEDWALK_API gedwalk_status gedwalk_maximize_stats(gedwalk_graph_t g, int64_t* evaluations, int64_t* batches, int64_t* sweeps,
                                      int64_t* spec_misses);

/*
 * Walk lengths of the last gedwalk_maximize on this graph: ell[j] (j < min(cap,
 * *count)) is the l at which step j's vertex was taken (the fixed L without
 * GEDWALK_ADAPTIVE_L); *count the number of steps; *separation_failures the
 * number of failed separation tests (doublings of l) of Algorithm 2. ell may be
 * NULL when cap = 0; count and separation_failures may be NULL.
 */
GEDWALK_API gedwalk_status gedwalk_maximize_lengths(gedwalk_graph_t g, int32_t* ell, int32_t cap, int32_t* count,
                                        int64_t* separation_failures);

/* ---------------------------------------------------------------------------
 * Serving: a continuous-batching request loop over device-resident graphs.
 * Its requests are the paper's two problems (Section 2.1): scoring a given
 * group, problem (i), as gedwalk_score_batch computes it, and maximising a
 * group of size k, problem (ii), as gedwalk_maximize does. The loop itself
 * (queues, batching, admission by memory) has no counterpart in the paper.
 * Score requests for the same graph that are pending together are packed as
 * columns of one batched SpMM; maximise requests run on their own streams and
 * overlap with the scoring. Admission is by memory: a request is admitted
 * when its device working set fits in mem_budget beside the requests in
 * flight, otherwise it waits in its queue. Score requests are admitted before
 * maximise requests, and a maximise request only when one of the server's 8
 * maximise workers is free. Results do not depend on which other requests
 * shared a batch.
 * ------------------------------------------------------------------------- */
enum { GEDWALK_REQ_SCORE = 0, GEDWALK_REQ_MAXIMIZE = 1 };

/*
 * graphs: n_graphs uploaded handles, referenced by index in submit; they must
 * outlive the server, and while it runs other calls on them must use the alpha
 * the server serves (the graph's default unless a request set another first).
 * mem_budget: bytes of device working memory the server may hold (0 = 1 GiB;
 * see gedwalk_serve_counters). max_batch: the most score requests packed into
 * one SpMM (0 = 256). The server starts one scoring thread per graph and 8
 * maximise worker threads, each with its own CUDA stream.
 */
GEDWALK_API gedwalk_status gedwalk_serve_create(const gedwalk_graph_t* graphs, int32_t n_graphs, int64_t mem_budget,
                                    int32_t max_batch, gedwalk_server_t* out);

/*
 * Queues a request: problem (i) or (ii) of Section 2.1.
 * kind GEDWALK_REQ_SCORE scores S (s_len members);
 * GEDWALK_REQ_MAXIMIZE runs gedwalk_maximize with k = s_len_or_k (S ignored).
 * params: NULL = defaults (its stream field is ignored). *ticket identifies the
 * request. BUSY when the queue holds 1<<20 requests already. INVALID when the
 * request's alpha differs from the one its graph serves: the graph's walk-total
 * table, which queued score requests read, holds one alpha.
 */
GEDWALK_API gedwalk_status gedwalk_serve_submit(gedwalk_server_t srv, int32_t graph, int32_t kind, const int32_t* S,
                                    int32_t s_len_or_k, const gedwalk_params* params, uint64_t* ticket);

/*
 * (Serving infrastructure; no counterpart in the paper.)
 * Waits up to wait_us microseconds (0 = do not wait, < 0 = wait without limit)
 * for a request. *done = 1 and results written when finished: score, group
 * (int32[k], maximize only), gains (double[k], maximize only; may be NULL),
 * latency_us (submit to completion; may be NULL). The ticket is released once
 * reported done. *done = 0 when still pending. A request that failed reports
 * its own status as the return value with *done = 1.
 */
GEDWALK_API gedwalk_status gedwalk_serve_poll(gedwalk_server_t srv, uint64_t ticket, int32_t wait_us, double* score,
                                  int32_t* group, double* gains, double* latency_us, int32_t* done);

/* (Serving measurement; no counterpart in the paper.)
 * Counters: requests completed, batched SpMM launches, score requests packed into them, and the
 * peak of the charged device bytes (see gedwalk_serve_counters). */
GEDWALK_API gedwalk_status gedwalk_serve_stats(gedwalk_server_t srv, int64_t* completed, int64_t* batches, int64_t* batched_requests,
                                   int64_t* peak_bytes);

/*
 * (Serving measurement; no counterpart in the paper.)
 * Memory admission in detail. Each scoring lane and maximise worker owns a workspace whose device
 * buffers grow to its largest request and stay allocated. The server charges each workspace the
 * bytes it holds or, while it has work, the larger of those and the exact footprint of that work.
 * A request is admitted while the total charge stays within mem_budget; otherwise idle workspaces
 * are released (largest first, counted in releases / released_bytes) and, if that is not enough,
 * the request waits. A request larger than the budget runs when nothing else holds memory. The
 * graphs themselves (their CSR and walk-total tables) are not charged.
 */
typedef struct {
  int64_t completed;             /* requests finished */
  int64_t batches;               /* batched SpMM launches of the scoring lanes */
  int64_t batched_requests;      /* score requests packed into them */
  int64_t peak_bytes;            /* largest total charge seen */
  int64_t budget;                /* mem_budget */
  int64_t charged_bytes;         /* total charge now */
  int64_t idle_held_bytes;       /* device bytes the idle workspaces hold now (measured) */
  int64_t admitted_at_submit;    /* requests admitted by their own submit call */
  int64_t admitted_after_wait;   /* requests that waited in a queue for memory or a worker */
  int64_t peak_maximize_running; /* most maximise requests running at once */
  int64_t releases;              /* idle workspaces released to make room */
  int64_t released_bytes;        /* device bytes they held */
  int64_t pending;               /* requests waiting for admission now */
} gedwalk_serve_counters;

GEDWALK_API gedwalk_status gedwalk_serve_counters_read(gedwalk_server_t srv, gedwalk_serve_counters* out);

/* (Serving infrastructure; no counterpart in the paper.)
 * Stops the server. Requests already admitted finish; requests still waiting
 * for admission end with GEDWALK_ERR_BUSY (a poll reports it). Returns after
 * the server's threads have stopped and every gedwalk_serve_poll call blocked
 * on this server has returned; srv is then freed, and no call on it may start
 * after, or at the same time as, this call. */
GEDWALK_API gedwalk_status gedwalk_serve_destroy(gedwalk_server_t srv);

/*
 * One step of the two-state hit/miss recurrence on caller-owned device memory,
 * allocating nothing. The paper has no counterpart: this exists for callers that
 * cannot allocate device memory, such as code running after its framework has
 * given the whole GPU to its own memory pool, or services that forbid device
 * allocation (its latency and its failure modes) once they are serving. Every
 * other entry point allocates workspaces; this one calls no cudaMalloc, cudaFree
 * or other allocating routine.
 *  d_row_ptr, d_col_idx: device int32[n+1] / int32[nnz], an undirected CSR as in
 *    gedwalk_graph_upload (not validated here; caller ids, no relabelling).
 *  d_mask: device uint32[ceil(n/32)], bit v set iff v is in S.
 *  d_x: device float[n][2], (hit, miss) of the previous length; d_y receives the
 *    next length. Both 8-byte aligned; they must not overlap. A score starts from
 *    x = (1_S, 1_{V\S}) and applies the step L times, swapping x and y.
 *  alpha: the damping factor (> 0).
 *  d_hit_sum: device double[1] (8-byte aligned), receives sum_v hit'(v), the
 *    alpha^i-weighted count of the i-walks that hit S; the score is the sum over
 *    the L steps.
 *  stream: cudaStream_t (0 = default). The call is asynchronous.
 * Scratch: a fixed 512 KiB device array inside the library (per GPU, held until
 * the process exits) limits n to 16,777,216; larger n returns
 * GEDWALK_ERR_INVALID. The first call on each device looks up that array's
 * address, so make the first call on a device before any stream capture. All
 * calls share the array, so calls that overlap on the GPU (different streams,
 * no ordering between them) race and give wrong sums.
 * Errors: INVALID (NULL pointer, n out of range, alpha <= 0, misalignment),
 * DEVICE (launch failure).
 */
GEDWALK_API gedwalk_status gedwalk_score_step_noalloc(const int32_t* d_row_ptr, const int32_t* d_col_idx, int32_t n,
                                                      const uint32_t* d_mask, const float* d_x, float* d_y,
                                                      double alpha, double* d_hit_sum, int64_t stream);

/* ---------------------------------------------------------------------------
 * Profiling: CUDA events around every sweep-kernel launch (the masked SpMV/SpMM
 * step of every algorithm above) and a count of all kernel launches.
 * ------------------------------------------------------------------------- */
typedef struct {
  int64_t launches;        /* every kernel launch of the library since the last reset */
  int64_t sweep_launches;  /* sweep-kernel launches timed */
  double sweep_ms;         /* summed device time of those launches (CUDA events on their stream) */
  double sweep_bytes;      /* summed algorithmic bytes of those launches: per launch the CSR (4 nnz
                              + 4 (n+1)), x read and y written once (2 C s n for C columns of s
                              bytes), the S mask (n/8) where masked, the phi^miss rows written
                              (s n fused, (C-1) s n lookahead) and the vertex scales (s n, weighted) */
  /* the sweep instantiation with the largest summed time: */
  int32_t top_mode;        /* 0 totals, 1 two-state score, 2 fused greedy, 3 candidates, 4 batched,
                              5 greedy lookahead */
  int32_t top_cols;        /* columns per row */
  int32_t top_fp64;        /* 1 for FP64 rows */
  int32_t top_pad;
  int64_t top_launches;
  double top_ms;
  double top_bytes;
} gedwalk_profile_stats;

/* (Measurement; no counterpart in the paper.) enable != 0 starts timing sweep launches; every
 * call resets the counters. */
GEDWALK_API gedwalk_status gedwalk_profile(int32_t enable);

/* (Measurement; no counterpart in the paper.) Waits for the timed launches to finish and reports
 * the counters. */
GEDWALK_API gedwalk_status gedwalk_profile_read(gedwalk_profile_stats* out);

/* Message for the calling thread's last failing call ("" if none). (Error reporting; no
 * counterpart in the paper.) */
GEDWALK_API const char* gedwalk_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* GEDWALK_H */
