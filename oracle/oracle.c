/*
 * GED-Walk CPU oracle (Angriman et al., "Group Centrality Maximization for
 * Large-scale Graphs", ALENEX 2020).
 *
 * TEST INFRASTRUCTURE ONLY: a plain, slow, obviously correct restatement of the
 * paper's definitions and recurrences, used to check the CUDA library. It
 * shares no code, header, table or helper with the library and must never be
 * linked into it; only tests/, the smoke check and the benchmark's CPU-baseline
 * leg load it.
 *
 * The numeric routines live in oracle_impl.inc and are compiled twice: in
 * double (suffix _d) and in long double (suffix _ld).
 *
 * Every routine takes optional CSR entry weights (Section 5.4's weighted walks;
 * NULL for the unweighted graph).
 *
 * Pins (see tests/test_oracle.py): brute-force walk enumeration on graphs of at
 * most 12 vertices (with exact rational weights too), closed forms (complete
 * graph, star, cycle, path; regular graphs for the normalised weights),
 * Prop. katz-relation, monotonicity and submodularity (Prop. ged_submod), the
 * Lemma-initialize upper bound and its equality at L = 1, exhaustive best
 * groups for k <= 3, and double against long double.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Row loops (the SpMV of every recurrence, the two-state step, the per-vertex bound) may run on
 * several threads when the graph has more rows than this; sums over rows stay serial. */
#define ORC_PAR_MIN 4096

/* Threads for the row loops (OpenMP builds; 1 otherwise). Results do not depend on it. */
void orc_set_threads(int t) {
#ifdef _OPENMP
  omp_set_num_threads(t > 0 ? t : 1);
#else
  (void)t;
#endif
}

int orc_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

double orc_delta(int32_t n, const int32_t* rp, const double* w);
double orc_delta2(int32_t n, const int32_t* rp, const double* w, const int32_t* rpt, const double* wt);

#define REAL double
#define ORC(name) orc_##name##_d
#include "oracle_impl.inc"
#undef ORC
#undef REAL

#define REAL long double
#define ORC(name) orc_##name##_ld
#include "oracle_impl.inc"
#undef ORC
#undef REAL

/* maximum degree (the d_max of Eq. comb-bound) */
int32_t orc_dmax(int32_t n, const int32_t* rp) {
  int32_t d = 0;
  for (int32_t v = 0; v < n; ++v)
    if (rp[v + 1] - rp[v] > d) d = rp[v + 1] - rp[v];
  return d;
}

/*
 * The degree bound of Eq. comb-bound for a weighted graph: the largest weighted
 * degree delta = max_v sum_u w(v,u), so that W_{l+1} <= delta W_l still holds (the
 * row sums of the weighted adjacency bound the growth of every walk total). For
 * w = NULL it is d_max.
 */
double orc_delta(int32_t n, const int32_t* rp, const double* w) {
  if (!w) return (double)orc_dmax(n, rp);
  double d = 0;
  for (int32_t v = 0; v < n; ++v) {
    double s = 0;
    for (int32_t j = rp[v]; j < rp[v + 1]; ++j) s += w[j];
    if (s > d) d = s;
  }
  return d;
}

/*
 * For a directed graph (rpt/wt: the transposed CSR) the walk totals grow at most by the largest
 * row sum of either orientation: an l-walk extends at its end along at most d_out arcs and at its
 * start along at most d_in arcs, so W_{l+1} <= min(d_out, d_in) W_l. rpt = NULL: undirected.
 */
double orc_delta2(int32_t n, const int32_t* rp, const double* w, const int32_t* rpt, const double* wt) {
  const double a = orc_delta(n, rp, w);
  if (!rpt) return a;
  const double b = orc_delta(n, rpt, wt);
  return a < b ? a : b;
}

/*
 * Transpose of a CSR (row v of the result lists the u with v in row u), rows sorted, entry
 * weights carried along when w is given. rpt[n+1], cit[nnz], wt[nnz] (wt may be NULL).
 */
void orc_transpose(int32_t n, const int32_t* rp, const int32_t* ci, const double* w, int32_t* rpt, int32_t* cit,
                   double* wt) {
  for (int32_t v = 0; v <= n; ++v) rpt[v] = 0;
  for (int32_t u = 0; u < n; ++u)
    for (int32_t j = rp[u]; j < rp[u + 1]; ++j) rpt[ci[j] + 1]++;
  for (int32_t v = 0; v < n; ++v) rpt[v + 1] += rpt[v];
  int32_t* fill = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  if (!fill) return;
  for (int32_t v = 0; v < n; ++v) fill[v] = rpt[v];
  for (int32_t u = 0; u < n; ++u) /* rows u in increasing order: every transposed row comes out sorted */
    for (int32_t j = rp[u]; j < rp[u + 1]; ++j) {
      const int32_t p = fill[ci[j]]++;
      cit[p] = u;
      if (wt) wt[p] = w[j];
    }
  free(fill);
}

/*
 * Entry weights of the symmetrically normalised adjacency D^{-1/2} A D^{-1/2}
 * (Section 5.4): w(v,u) = 1 / sqrt(deg(v) deg(u)). out receives nnz values.
 */
void orc_normalized_weights(int32_t n, const int32_t* rp, const int32_t* ci, double* out) {
  for (int32_t v = 0; v < n; ++v)
    for (int32_t j = rp[v]; j < rp[v + 1]; ++j) {
      const int32_t u = ci[j];
      out[j] = 1.0 / sqrt((double)(rp[v + 1] - rp[v]) * (double)(rp[u + 1] - rp[u]));
    }
}

/*
 * Brute force (Def. ed-walk): enumerate every walk (x_0, ..., x_i) with
 * (x_{j-1}, x_j) in E by depth-first search and count, in exact integers, the
 * walks that contain at least one vertex of S (phi_i(S)) and all walks (W_i).
 * Exponential; for graphs of at most ~12 vertices and short lengths.
 */
static void brute_rec(const int32_t* rp, const int32_t* ci, const unsigned char* in, int32_t v, int32_t left,
                      int hit, uint64_t* phi, uint64_t* all) {
  if (left == 0) {
    *all += 1;
    if (hit) *phi += 1;
    return;
  }
  for (int32_t j = rp[v]; j < rp[v + 1]; ++j) {
    const int32_t u = ci[j];
    brute_rec(rp, ci, in, u, left - 1, hit || in[u], phi, all);
  }
}

int orc_brute_phi(int32_t n, const int32_t* rp, const int32_t* ci, const int32_t* S, int32_t s_len, int32_t i,
                  uint64_t* phi_out, uint64_t* walks_out) {
  unsigned char* in = (unsigned char*)calloc((size_t)(n > 0 ? n : 1), 1);
  if (!in) return -1;
  for (int32_t j = 0; j < s_len; ++j)
    if (S[j] >= 0 && S[j] < n) in[S[j]] = 1;
  uint64_t phi = 0, all = 0;
  for (int32_t v = 0; v < n; ++v) brute_rec(rp, ci, in, v, i, in[v], &phi, &all);
  free(in);
  *phi_out = phi;
  *walks_out = all;
  return 0;
}

/*
 * Brute force for the marginal gain: the number of i-walks that visit x and
 * avoid S (proof of Prop. ged_submod), by enumeration.
 */
static void brute_gain_rec(const int32_t* rp, const int32_t* ci, const unsigned char* in, int32_t x, int32_t v,
                           int32_t left, int seen, uint64_t* cnt) {
  if (left == 0) {
    if (seen) *cnt += 1;
    return;
  }
  for (int32_t j = rp[v]; j < rp[v + 1]; ++j) {
    const int32_t u = ci[j];
    if (in[u]) continue;
    brute_gain_rec(rp, ci, in, x, u, left - 1, seen || u == x, cnt);
  }
}

int orc_brute_gain(int32_t n, const int32_t* rp, const int32_t* ci, const int32_t* S, int32_t s_len, int32_t x,
                   int32_t i, uint64_t* out) {
  unsigned char* in = (unsigned char*)calloc((size_t)(n > 0 ? n : 1), 1);
  if (!in) return -1;
  for (int32_t j = 0; j < s_len; ++j)
    if (S[j] >= 0 && S[j] < n) in[S[j]] = 1;
  uint64_t cnt = 0;
  if (!in[x])
    for (int32_t v = 0; v < n; ++v)
      if (!in[v]) brute_gain_rec(rp, ci, in, x, v, i, v == x, &cnt);
  free(in);
  *out = cnt;
  return 0;
}

/*
 * Counter-based draw for stochastic greedy (Appendix D): the first output of splitmix64
 * (Steele, Lea & Flood, 2014) started from state seed ^ (step << 32) ^ v. Written here from
 * the published definition; the library implements its own copy.
 */
uint64_t orc_sample_hash(uint64_t seed, uint32_t step, uint32_t v) {
  uint64_t z = (seed ^ ((uint64_t)step << 32) ^ (uint64_t)v) + 0x9e3779b97f4a7c15ULL;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

/* long-double entry points exchange values as double for the ctypes wrapper */
double orc_score_ld_as_d(int32_t n, const int32_t* rp, const int32_t* ci, const double* w, const int32_t* S,
                         int32_t s_len, double alpha, int32_t L) {
  return (double)orc_score_ld(n, rp, ci, w, S, s_len, alpha, L, NULL);
}

double orc_gain_ld_as_d(int32_t n, const int32_t* rp, const int32_t* ci, const double* w, const int32_t* S,
                        int32_t s_len, int32_t x, double alpha, int32_t L) {
  return (double)orc_gain_ld(n, rp, ci, w, S, s_len, x, alpha, L);
}
