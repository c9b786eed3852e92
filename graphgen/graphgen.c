/*
 * Seeded synthetic graph generators (input preparation only).
 *
 * This file produces the undirected, unweighted CSR graphs that the tests and the
 * benchmark feed to both the CPU oracle and the CUDA library. It contains none of
 * the GED-Walk arithmetic: only random-number generation, the three generator
 * families of the paper's synthetic experiments (Erdos-Renyi, Barabasi-Albert,
 * R-MAT with the Graph 500 parameters; Appendix C "Details of the Experimental
 * Setup") and the conversion of an edge list into a symmetric CSR without
 * self-loops or duplicate entries.
 *
 * Random numbers: xoshiro256** (Blackman & Vigna, 2018) seeded through
 * splitmix64 (Steele, Lea & Flood, 2014), both written from their published
 * definitions. Only integer operations decide the output, except the ER skip
 * lengths, which use log() (see gg_er).
 *
 * All routines return a heap-allocated gg_csr that the caller releases with
 * gg_free. NULL means out of memory or invalid arguments.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  int32_t n;
  int64_t nnz;
  int32_t* row_ptr; /* n + 1 entries */
  int32_t* col_idx; /* nnz entries, each row strictly increasing */
} gg_csr;

typedef struct {
  uint64_t s[4];
} gg_rng;

static uint64_t splitmix64_next(uint64_t* x) {
  uint64_t z = (*x += 0x9e3779b97f4a7c15ULL);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

static void rng_seed(gg_rng* r, uint64_t seed) {
  uint64_t x = seed;
  for (int i = 0; i < 4; ++i) r->s[i] = splitmix64_next(&x);
}

static inline uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static inline uint64_t rng_next(gg_rng* r) {
  uint64_t* s = r->s;
  const uint64_t out = rotl64(s[1] * 5u, 7) * 9u;
  const uint64_t t = s[1] << 17;
  s[2] ^= s[0];
  s[3] ^= s[1];
  s[1] ^= s[2];
  s[0] ^= s[3];
  s[2] ^= t;
  s[3] = rotl64(s[3], 45);
  return out;
}

/* uniform double in [0, 1) with 53 random bits */
static inline double rng_unit(gg_rng* r) { return (double)(rng_next(r) >> 11) * (1.0 / 9007199254740992.0); }

/* uniform integer in [0, bound), bound > 0, by rejection (no modulo bias) */
static inline uint64_t rng_below(gg_rng* r, uint64_t bound) {
  const uint64_t limit = UINT64_MAX - (UINT64_MAX % bound);
  uint64_t x;
  do {
    x = rng_next(r);
  } while (x >= limit);
  return x % bound;
}

/* exported so that Python-side helpers can draw from the same stream definition */
void gg_rng_fill(uint64_t seed, uint64_t* out, int64_t count) {
  gg_rng r;
  rng_seed(&r, seed);
  for (int64_t i = 0; i < count; ++i) out[i] = rng_next(&r);
}

void gg_free(gg_csr* g) {
  if (!g) return;
  free(g->row_ptr);
  free(g->col_idx);
  free(g);
}

static int cmp_i32(const void* a, const void* b) {
  const int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

static void sort_small(int32_t* a, int64_t len) {
  if (len < 24) { /* insertion sort */
    for (int64_t i = 1; i < len; ++i) {
      int32_t v = a[i];
      int64_t j = i - 1;
      while (j >= 0 && a[j] > v) {
        a[j + 1] = a[j];
        --j;
      }
      a[j + 1] = v;
    }
  } else {
    qsort(a, (size_t)len, sizeof(int32_t), cmp_i32);
  }
}

/*
 * Undirected edge list (m tuples, vertices in [0, n)) -> symmetric CSR.
 * Each tuple {u, v} with u != v yields the entries (u, v) and (v, u); repeated
 * tuples collapse to one edge; self-loops are dropped.
 */
gg_csr* gg_from_edges(int32_t n, int64_t m, const int32_t* src, const int32_t* dst) {
  if (n < 0 || m < 0) return NULL;
  gg_csr* g = (gg_csr*)calloc(1, sizeof(gg_csr));
  if (!g) return NULL;
  g->n = n;
  int64_t* cnt = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  if (!cnt) {
    free(g);
    return NULL;
  }
  for (int64_t e = 0; e < m; ++e) {
    const int32_t u = src[e], v = dst[e];
    if (u < 0 || v < 0 || u >= n || v >= n) {
      free(cnt);
      free(g);
      return NULL;
    }
    if (u == v) continue;
    cnt[u + 1]++;
    cnt[v + 1]++;
  }
  for (int32_t i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
  const int64_t total = cnt[n];
  int32_t* tmp = (int32_t*)malloc((size_t)(total > 0 ? total : 1) * sizeof(int32_t));
  int64_t* pos = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
  if (!tmp || !pos) {
    free(tmp);
    free(pos);
    free(cnt);
    free(g);
    return NULL;
  }
  memcpy(pos, cnt, (size_t)n * sizeof(int64_t));
  for (int64_t e = 0; e < m; ++e) {
    const int32_t u = src[e], v = dst[e];
    if (u == v) continue;
    tmp[pos[u]++] = v;
    tmp[pos[v]++] = u;
  }
  free(pos);
  /* sort each row, drop duplicates, compact in place */
  g->row_ptr = (int32_t*)malloc(((size_t)n + 1) * sizeof(int32_t));
  if (!g->row_ptr) {
    free(tmp);
    free(cnt);
    free(g);
    return NULL;
  }
  int64_t w = 0;
  g->row_ptr[0] = 0;
  for (int32_t i = 0; i < n; ++i) {
    int32_t* row = tmp + cnt[i];
    const int64_t len = cnt[i + 1] - cnt[i];
    sort_small(row, len);
    for (int64_t j = 0; j < len; ++j) {
      if (j > 0 && row[j] == row[j - 1]) continue;
      tmp[w++] = row[j];
    }
    if (w > INT32_MAX) { /* int32 row_ptr cannot hold it */
      free(tmp);
      free(cnt);
      free(g->row_ptr);
      free(g);
      return NULL;
    }
    g->row_ptr[i + 1] = (int32_t)w;
  }
  free(cnt);
  g->nnz = w;
  g->col_idx = (int32_t*)realloc(tmp, (size_t)(w > 0 ? w : 1) * sizeof(int32_t));
  if (!g->col_idx) g->col_idx = tmp;
  return g;
}

/*
 * Directed arc list (m tuples u -> v) -> CSR of successor lists: row u holds the v with an arc
 * u -> v, sorted; repeated arcs collapse to one; self-loops are dropped.
 */
gg_csr* gg_from_arcs(int32_t n, int64_t m, const int32_t* src, const int32_t* dst) {
  if (n < 0 || m < 0) return NULL;
  gg_csr* g = (gg_csr*)calloc(1, sizeof(gg_csr));
  if (!g) return NULL;
  g->n = n;
  int64_t* cnt = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  if (!cnt) {
    free(g);
    return NULL;
  }
  for (int64_t e = 0; e < m; ++e) {
    const int32_t u = src[e], v = dst[e];
    if (u < 0 || v < 0 || u >= n || v >= n) {
      free(cnt);
      free(g);
      return NULL;
    }
    if (u != v) cnt[u + 1]++;
  }
  for (int32_t i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
  const int64_t total = cnt[n];
  int32_t* tmp = (int32_t*)malloc((size_t)(total > 0 ? total : 1) * sizeof(int32_t));
  int64_t* pos = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
  g->row_ptr = (int32_t*)malloc(((size_t)n + 1) * sizeof(int32_t));
  if (!tmp || !pos || !g->row_ptr) {
    free(tmp);
    free(pos);
    free(cnt);
    free(g->row_ptr);
    free(g);
    return NULL;
  }
  memcpy(pos, cnt, (size_t)n * sizeof(int64_t));
  for (int64_t e = 0; e < m; ++e)
    if (src[e] != dst[e]) tmp[pos[src[e]]++] = dst[e];
  free(pos);
  int64_t w = 0;
  g->row_ptr[0] = 0;
  for (int32_t i = 0; i < n; ++i) {
    int32_t* row = tmp + cnt[i];
    const int64_t len = cnt[i + 1] - cnt[i];
    sort_small(row, len);
    for (int64_t j = 0; j < len; ++j) {
      if (j > 0 && row[j] == row[j - 1]) continue;
      tmp[w++] = row[j];
    }
    g->row_ptr[i + 1] = (int32_t)w;
  }
  free(cnt);
  g->nnz = w;
  g->col_idx = (int32_t*)realloc(tmp, (size_t)(w > 0 ? w : 1) * sizeof(int32_t));
  if (!g->col_idx) g->col_idx = tmp;
  return g;
}

/*
 * Erdos-Renyi G(n, p), undirected. Small graphs (n <= 4096) test every pair
 * against an integer threshold, so the graph is identical on every platform.
 * Larger graphs use geometric skipping over the pair sequence (Batagelj &
 * Brandes, 2005), whose skip lengths go through log().
 */
gg_csr* gg_er(int32_t n, double p, uint64_t seed) {
  if (n < 0 || !(p >= 0.0) || p > 1.0) return NULL;
  gg_rng r;
  rng_seed(&r, seed);
  int64_t cap = 1024, m = 0;
  int32_t* su = (int32_t*)malloc((size_t)cap * sizeof(int32_t));
  int32_t* sv = (int32_t*)malloc((size_t)cap * sizeof(int32_t));
  if (!su || !sv) goto oom;
#define GG_PUSH(a, b)                                                      \
  do {                                                                     \
    if (m == cap) {                                                        \
      cap *= 2;                                                            \
      int32_t* nu = (int32_t*)realloc(su, (size_t)cap * sizeof(int32_t)); \
      if (!nu) goto oom;                                                   \
      su = nu;                                                             \
      int32_t* nv = (int32_t*)realloc(sv, (size_t)cap * sizeof(int32_t)); \
      if (!nv) goto oom;                                                   \
      sv = nv;                                                             \
    }                                                                      \
    su[m] = (a);                                                           \
    sv[m] = (b);                                                           \
    ++m;                                                                   \
  } while (0)
  if (n <= 4096) {
    /* threshold = p * 2^64, saturated */
    const double scaled = p * 18446744073709551616.0;
    const uint64_t thr = scaled >= 18446744073709551615.0 ? UINT64_MAX : (uint64_t)scaled;
    for (int32_t u = 0; u < n; ++u)
      for (int32_t v = u + 1; v < n; ++v)
        if (rng_next(&r) < thr) GG_PUSH(u, v);
  } else if (p > 0.0) {
    const double lq = log(1.0 - p);
    int64_t v = 1, w = -1;
    while (v < n) {
      const double u01 = rng_unit(&r);
      w += 1 + (int64_t)floor(log(1.0 - u01) / lq);
      while (w >= v && v < n) {
        w -= v;
        ++v;
      }
      if (v < n) GG_PUSH((int32_t)v, (int32_t)w);
    }
  }
  {
    gg_csr* g = gg_from_edges(n, m, su, sv);
    free(su);
    free(sv);
    return g;
  }
oom:
  free(su);
  free(sv);
  return NULL;
}

/*
 * Barabasi-Albert preferential attachment: a seed clique on vertices 0..m, then
 * each new vertex v attaches to m distinct earlier vertices, each drawn with
 * probability proportional to its current degree by picking a uniform entry of
 * the endpoint list (Batagelj & Brandes, 2005); a repeated target is redrawn.
 */
gg_csr* gg_ba(int32_t n, int32_t m, uint64_t seed) {
  if (m < 1 || n < m + 1) return NULL;
  gg_rng r;
  rng_seed(&r, seed);
  const int64_t clique = (int64_t)m * (m + 1) / 2;
  const int64_t edges = clique + (int64_t)(n - m - 1) * m;
  int32_t* su = (int32_t*)malloc((size_t)edges * sizeof(int32_t));
  int32_t* sv = (int32_t*)malloc((size_t)edges * sizeof(int32_t));
  int32_t* ends = (int32_t*)malloc((size_t)edges * 2 * sizeof(int32_t));
  int32_t* pick = (int32_t*)malloc((size_t)m * sizeof(int32_t));
  if (!su || !sv || !ends || !pick) {
    free(su);
    free(sv);
    free(ends);
    free(pick);
    return NULL;
  }
  int64_t e = 0, ne = 0;
  for (int32_t u = 0; u <= m; ++u)
    for (int32_t v = u + 1; v <= m; ++v) {
      su[e] = u;
      sv[e] = v;
      ++e;
      ends[ne++] = u;
      ends[ne++] = v;
    }
  for (int32_t v = m + 1; v < n; ++v) {
    const int64_t pool = ne; /* targets come from edges that existed before v */
    for (int32_t j = 0; j < m; ++j) {
      int32_t t;
      int dup;
      do {
        t = ends[rng_below(&r, (uint64_t)pool)];
        dup = 0;
        for (int32_t q = 0; q < j; ++q)
          if (pick[q] == t) dup = 1;
      } while (dup);
      pick[j] = t;
    }
    for (int32_t j = 0; j < m; ++j) {
      su[e] = v;
      sv[e] = pick[j];
      ++e;
      ends[ne++] = v;
      ends[ne++] = pick[j];
    }
  }
  free(ends);
  free(pick);
  gg_csr* g = gg_from_edges(n, edges, su, sv);
  free(su);
  free(sv);
  return g;
}

/*
 * R-MAT (Chakrabarti, Zhan & Faloutsos, 2004) with edge factor ef: ef * 2^scale
 * tuples, each placed by descending `scale` levels of the recursive 2x2
 * partition with probabilities (a, b, c, 1-a-b-c). Vertex labels are then
 * shuffled by a uniform random permutation when `permute` is set (as the
 * Graph 500 generator does), and the result is symmetrised with duplicates and
 * self-loops removed (directed: the tuples are kept as arcs u -> v instead).
 */
gg_csr* gg_rmat_ex(int32_t scale, int32_t ef, double a, double b, double c, uint64_t seed, int32_t permute,
                   int32_t directed) {
  if (scale < 1 || scale > 30 || ef < 1 || a < 0 || b < 0 || c < 0 || a + b + c > 1.0) return NULL;
  const int32_t n = (int32_t)1 << scale;
  const int64_t m = (int64_t)ef * n;
  gg_rng r;
  rng_seed(&r, seed);
  int32_t* su = (int32_t*)malloc((size_t)m * sizeof(int32_t));
  int32_t* sv = (int32_t*)malloc((size_t)m * sizeof(int32_t));
  if (!su || !sv) {
    free(su);
    free(sv);
    return NULL;
  }
  /* integer thresholds on 53-bit draws keep the placement platform-independent */
  const double two53 = 9007199254740992.0;
  const uint64_t ta = (uint64_t)(a * two53), tab = (uint64_t)((a + b) * two53),
                 tabc = (uint64_t)((a + b + c) * two53);
  for (int64_t e = 0; e < m; ++e) {
    uint32_t u = 0, v = 0;
    for (int32_t lev = 0; lev < scale; ++lev) {
      const uint64_t x = rng_next(&r) >> 11;
      uint32_t bu, bv;
      if (x < ta) {
        bu = 0;
        bv = 0;
      } else if (x < tab) {
        bu = 0;
        bv = 1;
      } else if (x < tabc) {
        bu = 1;
        bv = 0;
      } else {
        bu = 1;
        bv = 1;
      }
      u = (u << 1) | bu;
      v = (v << 1) | bv;
    }
    su[e] = (int32_t)u;
    sv[e] = (int32_t)v;
  }
  if (permute) {
    int32_t* perm = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    if (!perm) {
      free(su);
      free(sv);
      return NULL;
    }
    for (int32_t i = 0; i < n; ++i) perm[i] = i;
    for (int32_t i = n - 1; i > 0; --i) {
      const int32_t j = (int32_t)rng_below(&r, (uint64_t)i + 1);
      const int32_t t = perm[i];
      perm[i] = perm[j];
      perm[j] = t;
    }
    for (int64_t e = 0; e < m; ++e) {
      su[e] = perm[su[e]];
      sv[e] = perm[sv[e]];
    }
    free(perm);
  }
  gg_csr* g = directed ? gg_from_arcs(n, m, su, sv) : gg_from_edges(n, m, su, sv);
  free(su);
  free(sv);
  return g;
}

gg_csr* gg_rmat(int32_t scale, int32_t ef, double a, double b, double c, uint64_t seed, int32_t permute) {
  return gg_rmat_ex(scale, ef, a, b, c, seed, permute, 0);
}
