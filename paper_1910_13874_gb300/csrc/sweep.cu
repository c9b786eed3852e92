// The sweep kernel: one masked, alpha-scaled SpMV/SpMM step y = alpha * A x over the
// relabelled CSR, with a fused per-row epilogue selected at compile time.
//
// Every step of GED-Walk's hot path is such a sweep: the walk totals t_r
// (Eq. katz-def terms, used by the combinatorial bound, Eq. comb-bound), the
// two-state hit/miss recurrences of Section 3.1.1, the phi^miss vectors that
// feed the Lemma-initialize bound, and the candidate columns that count the
// walks through a vertex (proof of Prop. ged_submod).
//
// Work distribution. The graph is relabelled by decreasing degree, so rows of
// similar degree are contiguous, and the host cuts the rows into warp-sized
// units (no CTA-wide barrier anywhere after the prologue):
//  - short rows (degree <= 64): W lanes per row with 2W >= degree, so every lane
//    gathers at most two entries; a warp handles two rows per group per
//    iteration and issues all of their loads before reducing (4 gathers in
//    flight per lane);
//  - long rows (64 < degree <= kHeavyDeg): one warp per row, entries strided
//    over the lanes in groups of four loads;
//  - heavy rows (degree > kHeavyDeg): cut into slices of about kSliceEdges
//    entries, one warp per slice; each writes its partial sum and the last warp
//    to arrive (atomic counter) adds the partials in slice order and finishes
//    the row. No warp ever waits for another.
// A row's C-wide sum is reduce-scattered across its lanes (halving the columns
// at every shuffle step), so each lane ends with its own columns and the
// epilogue runs column-parallel. Column sums (sum_v y(v)) are accumulated per lane
// (compensated FP32 for FP32 vectors), reduced per warp in FP64 in a fixed order
// into per-unit slots: every result is bitwise reproducible.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdint>

#include "internal.h"

namespace gw {
namespace {

// [sweep-kernel-source-begin] (the profiles record a hash of the device code up to the end marker)
constexpr unsigned kFull = 0xffffffffu;
constexpr int kWarps = kThreads / 32;

template <int X>
struct Log2 {
  static constexpr int v = 1 + Log2<X / 2>::v;
};
template <>
struct Log2<1> {
  static constexpr int v = 0;
};

// p[0..N) -> out with the widest aligned vector loads (through the read-only path).
template <typename T, int N>
__device__ __forceinline__ void load_vec(const T* __restrict__ p, T (&out)[N]) {
  constexpr int kBytes = int(sizeof(T)) * N;
  if constexpr (kBytes % 16 == 0) {
    constexpr int kPer = 16 / int(sizeof(T));
#pragma unroll
    for (int k = 0; k < kBytes / 16; ++k) {
      const float4 t = __ldg(reinterpret_cast<const float4*>(p) + k);
      memcpy(&out[k * kPer], &t, 16);
    }
  } else if constexpr (kBytes == 8) {
    const float2 t = __ldg(reinterpret_cast<const float2*>(p));
    memcpy(out, &t, 8);
  } else {
#pragma unroll
    for (int e = 0; e < N; ++e) out[e] = __ldg(p + e);
  }
}

template <typename T, int N>
__device__ __forceinline__ void store_vec(T* __restrict__ p, const T (&v)[N]) {
  constexpr int kBytes = int(sizeof(T)) * N;
  if constexpr (kBytes % 16 == 0) {
    constexpr int kPer = 16 / int(sizeof(T));
#pragma unroll
    for (int k = 0; k < kBytes / 16; ++k) {
      float4 t;
      memcpy(&t, &v[k * kPer], 16);
      reinterpret_cast<float4*>(p)[k] = t;
    }
  } else if constexpr (kBytes == 8) {
    float2 t;
    memcpy(&t, v, 8);
    *reinterpret_cast<float2*>(p) = t;
  } else {
#pragma unroll
    for (int e = 0; e < N; ++e) p[e] = v[e];
  }
}

// Gathers of x rows. Vertices are numbered by decreasing degree, so the rows with the
// lowest ids are gathered most often: rows below the hub limit are loaded with high L1
// retention priority, all others without allocating in L1, so the stream of cold rows
// cannot flush the hot ones. 32-byte rows take a single 256-bit load.
#define GW_LD1(Q, TY, R, x, p) asm volatile("ld.global.nc." Q "." TY " %0, [%1];" : "=" R(x[0]) : "l"(p))
#define GW_LD2(Q, TY, R, x, p) \
  asm volatile("ld.global.nc." Q ".v2." TY " {%0,%1}, [%2];" : "=" R(x[0]), "=" R(x[1]) : "l"(p))
#define GW_LD4(Q, TY, R, x, p)                                                                        \
  asm volatile("ld.global.nc." Q ".v4." TY " {%0,%1,%2,%3}, [%4];" : "=" R(x[0]), "=" R(x[1]), "=" R(x[2]), \
               "=" R(x[3]) : "l"(p))
#define GW_LD8(Q, x, p)                                                                                 \
  asm volatile("ld.global.nc." Q ".v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"                              \
               : "=f"(x[0]), "=f"(x[1]), "=f"(x[2]), "=f"(x[3]), "=f"(x[4]), "=f"(x[5]), "=f"(x[6]), \
                 "=f"(x[7])                                                                             \
               : "l"(p))

template <typename T, int N, bool HOT>
__device__ __forceinline__ void gather_vec(const T* __restrict__ p, T* x) {
  if constexpr (sizeof(T) == 4) {
    if constexpr (N == 1) {
      if (HOT) GW_LD1("L1::evict_last", "f32", "f", x, p); else GW_LD1("L1::no_allocate", "f32", "f", x, p);
    } else if constexpr (N == 2) {
      if (HOT) GW_LD2("L1::evict_last", "f32", "f", x, p); else GW_LD2("L1::no_allocate", "f32", "f", x, p);
    } else if constexpr (N == 4) {
      if (HOT) GW_LD4("L1::evict_last", "f32", "f", x, p); else GW_LD4("L1::no_allocate", "f32", "f", x, p);
    } else {
#pragma unroll
      for (int k = 0; k < N / 8; ++k) {
        if (HOT) GW_LD8("L1::evict_last", (x + 8 * k), (p + 8 * k));
        else GW_LD8("L1::no_allocate", (x + 8 * k), (p + 8 * k));
      }
    }
  } else {
    if constexpr (N == 1) {
      if (HOT) GW_LD1("L1::evict_last", "f64", "d", x, p); else GW_LD1("L1::no_allocate", "f64", "d", x, p);
    } else if constexpr (N == 2) {
      if (HOT) GW_LD2("L1::evict_last", "f64", "d", x, p); else GW_LD2("L1::no_allocate", "f64", "d", x, p);
    } else {
#pragma unroll
      for (int k = 0; k < N / 4; ++k) {
        if (HOT) GW_LD4("L1::evict_last", "f64", "d", (x + 4 * k), (p + 4 * k));
        else GW_LD4("L1::no_allocate", "f64", "d", (x + 4 * k), (p + 4 * k));
      }
    }
  }
}

template <typename T, int C>
__device__ __forceinline__ void add_row(T (&acc)[C], const T* __restrict__ X, int v, int hub) {
  T x[C];
  const T* p = X + static_cast<size_t>(v) * C;
  if (v < hub) gather_vec<T, C, true>(p, x);
  else gather_vec<T, C, false>(p, x);
#pragma unroll
  for (int c = 0; c < C; ++c) acc[c] += x[c];
}

// Where gathered rows of x come from.
// GlobalSrc: global memory, rows below `hub` with L1 retention priority.
template <typename T, int C>
struct GlobalSrc {
  const T* __restrict__ X;
  int hub;
  __device__ __forceinline__ void add(T (&acc)[C], int v) const { add_row<T, C>(acc, X, v, hub); }
};

// Column indices are streamed once per sweep: keep them out of L1 (which holds the gathered
// rows of x) and first in line for eviction from L2.
__device__ __forceinline__ uint64_t stream_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

__device__ __forceinline__ int ld_idx(const int32_t* p, uint64_t pol) {
  int v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
  return v;
}

__device__ __forceinline__ bool in_mask(const uint32_t* __restrict__ mask, int r) {
  return (__ldg(mask + (r >> 5)) >> (r & 31)) & 1u;
}

// Reduce-scatter of the C-wide partial sums held by the W = 2^LW lanes of a group.
// On return acc[0..CPL) holds the group totals of columns [blk*CPL, (blk+1)*CPL) with
// blk = lane & (2^HS - 1), HS = min(log2 C, LW), CPL = C >> HS: each halving step keeps
// the upper or lower half of the held columns by one lane bit, highest bit first, so
// the blocks come out in natural order. Every lane of the warp must take part.
template <typename T, int C, int LW>
struct Scatter {
  static constexpr int LC = Log2<C>::v;
  static constexpr int HS = LC < LW ? LC : LW;
  static constexpr int CPL = C >> HS;
  __device__ __forceinline__ static void run(T (&acc)[C], int lane) {
#pragma unroll
    for (int st = HS - 1; st >= 0; --st) {
      const int o = 1 << st;
      const bool up = (lane & o) != 0;
      const int half = (C >> (HS - 1 - st)) / 2;
#pragma unroll
      for (int i = 0; i < C / 2; ++i) {
        if (i < half) {
          const T send = up ? acc[i] : acc[i + half];
          const T keep = up ? acc[i + half] : acc[i];
          acc[i] = keep + __shfl_xor_sync(kFull, send, o);
        }
      }
    }
#pragma unroll
    for (int o = 1 << HS; o < (1 << LW); o <<= 1)
#pragma unroll
      for (int i = 0; i < CPL; ++i) acc[i] += __shfl_xor_sync(kFull, acc[i], o);
  }
};

// Number of FP64 column sums a mode keeps.
template <int MODE, int C>
struct Sums {
  static constexpr int N = MODE == MODE_TOTALS ? 1 : MODE == MODE_SCORE ? 1
                           : (MODE == MODE_FUSED || MODE == MODE_LOOK) ? C - 1 : MODE == MODE_CAND ? C : 0;
  // the sum fed by column c, or -1 (MODE_FUSED and MODE_LOOK: columns 1.., the candidates)
  __device__ __forceinline__ static int slot(int c) {
    constexpr int first = (MODE == MODE_FUSED || MODE == MODE_LOOK) ? 1 : 0;
    return c >= first && c - first < N ? c - first : -1;
  }
};

// Number of candidate ids a mode reads (the only rows whose epilogue differs from y = alpha s).
template <int MODE, int C>
struct Cands {
  static constexpr int N = (MODE == MODE_FUSED || MODE == MODE_LOOK) ? C - 1 : MODE == MODE_CAND ? C : 0;
};

// Per-lane column sums over the rows of one unit. FP64 vectors sum in FP64. FP32 vectors sum with
// compensated FP32 additions (Kahan: the error is at most 2u * sum |y| + O(m u^2), u = 2^-24, over
// m <= 128 rows) and convert once per unit to FP64, in which every later sum (over lanes, units and
// sweeps) is taken. On a GB300 an FP64 addition costs about 64 FP32 ones, and one conversion and
// one FP64 addition per row and column cost more than the rest of the epilogue.
template <typename T, int N>
struct ColAcc {
  double s[N];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int k = 0; k < N; ++k) s[k] = 0.0;
  }
  __device__ __forceinline__ void add(int k, double y) { s[k] += y; }
  __device__ __forceinline__ double get(int k) const { return s[k]; }
};
template <int N>
struct ColAcc<float, N> {
  float s[N], c[N];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int k = 0; k < N; ++k) s[k] = c[k] = 0.0f;
  }
  __device__ __forceinline__ void add(int k, float y) {
    const float t1 = __fsub_rn(y, c[k]);
    const float t = __fadd_rn(s[k], t1);
    c[k] = __fsub_rn(__fsub_rn(t, s[k]), t1);
    s[k] = t;
  }
  __device__ __forceinline__ double get(int k) const { return static_cast<double>(s[k]) - static_cast<double>(c[k]); }
};

// The epilogue of the rows whose warp holds a candidate row (at most kCandSlots rows of the graph;
// every lane of the warp calls it, shuffles inside). y holds alpha * s, zeroed on S.
template <typename T, int C, int MODE, int CPL>
__device__ __forceinline__ void candidate_rows(const SweepArgs& a, const int* __restrict__ s_cand, int r, bool valid,
                                               int c0, int base, T (&y)[CPL]) {
  if constexpr (MODE == MODE_FUSED) {
    // column 0 is phi^miss under S; candidate column j >= 1 takes it at the candidate's row
    // (every S-avoiding walk ending at c_j visits c_j)
    const T m = __shfl_sync(kFull, y[0], base);
#pragma unroll
    for (int k = 0; k < CPL; ++k) {
      const int c = c0 + k;
      if (valid && c >= 1 && s_cand[c - 1] == r) y[k] = m;
    }
  } else if constexpr (MODE == MODE_CAND) {
    const T* min = static_cast<const T*>(a.Min) + (a.level_ptr ? a.level_stride * __ldg(a.level_ptr) : 0);
#pragma unroll
    for (int k = 0; k < CPL; ++k)
      if (valid && s_cand[c0 + k] == r) y[k] = __ldg(min + r);
  }
}

// MODE_LOOK epilogue for row r: D = C - 1 levels of one lookahead run, T_d = S + {c_1..c_d}.
// Column 0 is phi^miss under S; column j >= 1 counts the walks through c_j that avoid T_{j-1}
// (at c_j's own row: all of phi^miss(T_{j-1}), every such walk ending there visits c_j). A walk
// that avoids S either avoids c_1..c_d or has a first c_j among them, so
//   phi^miss(T_d) = column 0 - columns 1..d,
// which gives every level's phi^miss (table d, d = 0..D-1) and c_j's own-row value without
// columns of their own. The differences are clamped at 0 (their exact value is never negative).
// The lane holds columns c0..c0+CPL-1 of the row's group, whose column blocks lie in natural
// order over its first lanes (duplicates beyond them); every lane of the warp calls it.
template <typename T, int C, int CPL>
__device__ __forceinline__ void look_rows(const SweepArgs& a, const int* __restrict__ s_cand, int r, bool valid,
                                          bool store, int c0, int base, T (&y)[CPL], bool maybe_cand) {
  constexpr int NB = C / CPL;  // column blocks of a group
  T y0 = y[0];                 // column 0 sits in block 0, on the group's first lane
  T run = T(0);                // running sum of columns 1.. (starts with the blocks before this lane's)
  if constexpr (NB > 1) {
    const int blk = c0 / CPL;
    y0 = __shfl_sync(kFull, y[0], base);
    T inc = T(0);
#pragma unroll
    for (int k = 0; k < CPL; ++k)
      if (c0 + k >= 1) inc += y[k];
#pragma unroll
    for (int o = 1; o < NB; o <<= 1) {
      const T t = __shfl_up_sync(kFull, inc, o);
      if (blk >= o) inc += t;
    }
    const T t = __shfl_up_sync(kFull, inc, 1);
    run = blk > 0 ? t : T(0);
  }
  bool special = false;  // r is one of the run's candidates (only units that hold one look)
  if (maybe_cand) {
#pragma unroll
    for (int j = 0; j < C - 1; ++j) special |= valid && s_cand[j] == r;
  }
  const bool rare = maybe_cand && __any_sync(kFull, special);
  T* M = static_cast<T*>(a.Mout);
#pragma unroll
  for (int k = 0; k < CPL; ++k) {
    const int d = c0 + k;
    const T before = run;  // columns 1..d-1
    if (d >= 1) run += y[k];
    if (store && d <= C - 2) {  // table d = phi^miss(T_d): column 0 minus columns 1..d, 0 on c_1..c_d
      T m = y0 - run;
      m = m > T(0) ? m : T(0);
      if (rare && special)
        for (int j = 0; j < d; ++j)
          if (s_cand[j] == r) m = T(0);
      M[a.mout_stride * d + r] = m;
    }
    // r = c_m: column m takes phi^miss(T_{m-1}) at r; columns beyond m run under sets that hold r
    if (rare && special && d >= 1) {
      if (s_cand[d - 1] == r) {
        const T e = y0 - before;
        y[k] = e > T(0) ? e : T(0);
      } else {
        for (int j = 0; j < d - 1; ++j)
          if (s_cand[j] == r) y[k] = T(0);
      }
    }
  }
}

// Column-parallel epilogue for row r. The calling lane holds the totals s[0..CPL) of
// columns c0 .. c0+CPL-1; base is the first lane of the row's group. Every lane of the
// warp calls it (shuffles inside); `store` marks the lanes that own distinct columns of a
// valid row. acc accumulates this lane's column sums.
// maybe_cand (warp-uniform): a candidate row may lie among the rows of this unit; otherwise the
// per-row candidate test is skipped.
template <typename T, int C, int MODE, int CPL>
__device__ __forceinline__ void epilogue(const SweepArgs& a, const int* __restrict__ s_cand, int r, bool valid,
                                         bool store, int c0, int base, T (&s)[CPL], ColAcc<T, CPL>& acc,
                                         bool maybe_cand) {
  T* Y = static_cast<T*>(a.Y);
  constexpr bool kMasked = MODE == MODE_SCORE || MODE == MODE_FUSED || MODE == MODE_CAND || MODE == MODE_LOOK;
  const bool inS = kMasked && valid ? in_mask(a.mask, r) : false;
  // weighted graph: the row's scale s_r turns the gathered sum into the true value
  // alpha s_r (A x~)(r), which is summed, and the stored vector is x~ = s_r * value
  const T* rs = sizeof(T) == 8 ? reinterpret_cast<const T*>(a.rs_d) : reinterpret_cast<const T*>(a.rs_f);
  const T sv = rs && valid ? __ldg(rs + r) : T(1);
  const T alpha = static_cast<T>(a.alpha) * sv;
  if constexpr (MODE == MODE_SCORE) {
    // Section 3.1.1: hit_i(v) = sum hit_{i-1}(u) + [v in S] sum miss_{i-1}(u);
    //                miss_i(v) = [v not in S] sum miss_{i-1}(u).  Columns: 0 = hit, 1 = miss.
    T sh, sm;
    if constexpr (CPL == 2) {
      sh = s[0];
      sm = s[1];
    } else {
      sh = s[0];
      sm = __shfl_sync(kFull, s[0], base + 1);
    }
    if (store && c0 == 0) {
      T out[2];
      out[0] = alpha * (inS ? sh + sm : sh);
      out[1] = inS ? T(0) : alpha * sm;
      acc.add(0, out[0]);
      out[0] *= sv;
      out[1] *= sv;
      store_vec<T, 2>(Y + static_cast<size_t>(r) * C, out);
    }
  } else {
    T y[CPL];
#pragma unroll
    for (int k = 0; k < CPL; ++k) y[k] = inS ? T(0) : alpha * s[k];
    if constexpr (MODE == MODE_LOOK) {
      look_rows<T, C, CPL>(a, s_cand, r, valid, store, c0, base, y, maybe_cand);
    } else if (Cands<MODE, C>::N > 0 && maybe_cand) {
      bool special = false;
#pragma unroll
      for (int j = 0; j < Cands<MODE, C>::N; ++j) special |= s_cand[j] == r;
      if (__any_sync(kFull, valid && special)) candidate_rows<T, C, MODE, CPL>(a, s_cand, r, valid, c0, base, y);
    }
    if constexpr (MODE == MODE_FUSED) {
      if (store && c0 == 0) static_cast<T*>(a.Mout)[r] = y[0];
    }
    if (store) {
      if constexpr (Sums<MODE, C>::N > 0) {
#pragma unroll
        for (int k = 0; k < CPL; ++k)
          if (Sums<MODE, C>::slot(c0 + k) >= 0) acc.add(k, y[k]);
      }
#pragma unroll
      for (int k = 0; k < CPL; ++k) y[k] *= sv;
      store_vec<T, CPL>(Y + static_cast<size_t>(r) * C + c0, y);
    }
  }
}

// Whether a candidate row lies in rows [r0, r1) (the unit's rows).
template <int MODE, int C>
__device__ __forceinline__ bool unit_has_cand(const int* __restrict__ s_cand, int r0, int r1) {
  bool any = false;
#pragma unroll
  for (int j = 0; j < Cands<MODE, C>::N; ++j) any |= s_cand[j] >= r0 && s_cand[j] < r1;
  return any;
}

// Writes this lane's column sums (already reduced over the warp) to slot `slot`.
template <int MODE, int C, int CPL>
__device__ __forceinline__ void write_slot(const SweepArgs& a, size_t slot, int c0, const double (&cs)[CPL]) {
  constexpr int NS = Sums<MODE, C>::N;
  if constexpr (NS > 0) {
    double* dst = a.slots + slot * NS;
#pragma unroll
    for (int k = 0; k < CPL; ++k) {
      const int j = Sums<MODE, C>::slot(c0 + k);
      if (j >= 0) dst[j] = a.accumulate ? dst[j] + cs[k] : cs[k];
    }
  }
}

// Short rows (degree <= 2W): W lanes per row, at most two entries per lane, two rows per group.
template <typename T, int C, int MODE, int LW, class Src>
__device__ __forceinline__ void short_rows(const SweepArgs& a, const Src& src, const int4 u, int uidx, int lane,
                                          int* s_rp, const int* s_cand) {
  constexpr int W = 1 << LW;
  constexpr int NG = 32 / W;
  using SC = Scatter<T, C, LW>;
  constexpr int CPL = SC::CPL;
  const int r0 = u.x, nrows = u.y - u.x;
  for (int i = lane; i <= nrows; i += 32) s_rp[i] = __ldcs(a.rp + r0 + i);
  __syncwarp();
  const bool maybe_cand = unit_has_cand<MODE, C>(s_cand, r0, r0 + nrows);
  const int g = lane >> LW, gl = lane & (W - 1);
  const int base = lane & ~(W - 1);
  const int blk = gl & ((1 << SC::HS) - 1);
  const bool owner = (gl >> SC::HS) == 0;
  const int c0 = blk * CPL;
  const int32_t* __restrict__ ci = a.ci;
  const uint64_t pol = stream_policy();
  ColAcc<T, CPL> acc;
  acc.zero();
  for (int it = 0; it < nrows; it += 2 * NG) {
    const int ra = it + g, rb = it + NG + g;
    const bool va = ra < nrows, vb = rb < nrows;
    int ea0 = 0, ea1 = 0, eb0 = 0, eb1 = 0;
    if (va) {
      ea0 = s_rp[ra];
      ea1 = s_rp[ra + 1];
    }
    if (vb) {
      eb0 = s_rp[rb];
      eb1 = s_rp[rb + 1];
    }
    // all index loads first, then all gathers
    const int ja0 = ea0 + gl, ja1 = ea0 + gl + W, jb0 = eb0 + gl, jb1 = eb0 + gl + W;
    const int va0 = ja0 < ea1 ? ld_idx(ci + ja0, pol) : -1;
    const int va1 = ja1 < ea1 ? ld_idx(ci + ja1, pol) : -1;
    const int vb0 = jb0 < eb1 ? ld_idx(ci + jb0, pol) : -1;
    const int vb1 = jb1 < eb1 ? ld_idx(ci + jb1, pol) : -1;
    T acca[C], accb[C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
      acca[c] = T(0);
      accb[c] = T(0);
    }
    if (va0 >= 0) src.add(acca, va0);
    if (va1 >= 0) src.add(acca, va1);
    if (vb0 >= 0) src.add(accb, vb0);
    if (vb1 >= 0) src.add(accb, vb1);
    SC::run(acca, lane);
    SC::run(accb, lane);
    T sa[CPL], sb[CPL];
#pragma unroll
    for (int k = 0; k < CPL; ++k) {
      sa[k] = acca[k];
      sb[k] = accb[k];
    }
    epilogue<T, C, MODE, CPL>(a, s_cand, r0 + ra, va, va && owner, c0, base, sa, acc, maybe_cand);
    epilogue<T, C, MODE, CPL>(a, s_cand, r0 + rb, vb, vb && owner, c0, base, sb, acc, maybe_cand);
  }
  // sum the groups' copies of each column (non-owners hold zeros), in FP64
  double cs[CPL];
#pragma unroll
  for (int k = 0; k < CPL; ++k) cs[k] = acc.get(k);
#pragma unroll
  for (int o = W; o < 32; o <<= 1)
#pragma unroll
    for (int k = 0; k < CPL; ++k) cs[k] += __shfl_xor_sync(kFull, cs[k], o);
  if (lane < W && owner) write_slot<MODE, C, CPL>(a, static_cast<size_t>(uidx), c0, cs);
}

// Long rows: one warp per row, entries strided over the lanes in groups of four loads.
template <typename T, int C, int MODE, class Src>
__device__ __forceinline__ void long_rows(const SweepArgs& a, const Src& src, const int4 u, int uidx, int lane,
                                         int* s_rp, const int* s_cand) {
  using SC = Scatter<T, C, 5>;
  constexpr int CPL = SC::CPL;
  const int r0 = u.x, nrows = u.y - u.x;
  for (int i = lane; i <= nrows; i += 32) s_rp[i] = __ldcs(a.rp + r0 + i);
  __syncwarp();
  const bool maybe_cand = unit_has_cand<MODE, C>(s_cand, r0, r0 + nrows);
  const int blk = lane & ((1 << SC::HS) - 1);
  const bool owner = (lane >> SC::HS) == 0;
  const int c0 = blk * CPL;
  const int32_t* __restrict__ ci = a.ci;
  const uint64_t pol = stream_policy();
  ColAcc<T, CPL> cacc;
  cacc.zero();
  for (int rr = 0; rr < nrows; ++rr) {
    const int e0 = s_rp[rr], e1 = s_rp[rr + 1];
    T acc[C];
#pragma unroll
    for (int c = 0; c < C; ++c) acc[c] = T(0);
    int j = e0 + lane;
    for (; j + 96 < e1; j += 128) {
      const int v0 = ld_idx(ci + j, pol), v1 = ld_idx(ci + j + 32, pol), v2 = ld_idx(ci + j + 64, pol),
                v3 = ld_idx(ci + j + 96, pol);
      src.add(acc, v0);
      src.add(acc, v1);
      src.add(acc, v2);
      src.add(acc, v3);
    }
    for (; j < e1; j += 32) src.add(acc, ld_idx(ci + j, pol));
    SC::run(acc, lane);
    T s[CPL];
#pragma unroll
    for (int k = 0; k < CPL; ++k) s[k] = acc[k];
    epilogue<T, C, MODE, CPL>(a, s_cand, r0 + rr, true, owner, c0, 0, s, cacc, maybe_cand);
  }
  double cs[CPL];
#pragma unroll
  for (int k = 0; k < CPL; ++k) cs[k] = cacc.get(k);
  if (owner) write_slot<MODE, C, CPL>(a, static_cast<size_t>(uidx), c0, cs);
}

// Heavy slice: entries [u.y, u.z) of heavy row u.x, slice u.w.
template <typename T, int C, int MODE, class Src>
__device__ __forceinline__ void heavy_slice(const SweepArgs& a, const Src& src, const int4 u, int uidx, int lane,
                                           const int* s_cand) {
  using SC = Scatter<T, C, 5>;
  constexpr int CPL = SC::CPL;
  constexpr int NS = Sums<MODE, C>::N;
  const int blk = lane & ((1 << SC::HS) - 1);
  const bool owner = (lane >> SC::HS) == 0;
  const int c0 = blk * CPL;
  const int32_t* __restrict__ ci = a.ci;
  const uint64_t pol = stream_policy();
  T acc[C];
#pragma unroll
  for (int c = 0; c < C; ++c) acc[c] = T(0);
  int j = u.y + lane;
  for (; j + 96 < u.z; j += 128) {
    const int v0 = ld_idx(ci + j, pol), v1 = ld_idx(ci + j + 32, pol), v2 = ld_idx(ci + j + 64, pol),
              v3 = ld_idx(ci + j + 96, pol);
    src.add(acc, v0);
    src.add(acc, v1);
    src.add(acc, v2);
    src.add(acc, v3);
  }
  for (; j < u.z; j += 32) src.add(acc, ld_idx(ci + j, pol));
  SC::run(acc, lane);
  // this unit's own slot carries nothing: the row's sums go to the heavy row's slot
  if constexpr (NS > 0) {
    if (lane < NS) a.slots[static_cast<size_t>(uidx) * NS + lane] = 0.0;
  }
  const int4 hr = a.heavy[u.x];  // {row, first slice, slice count, 0}
  T* part = static_cast<T*>(a.partial);
  if (owner) {
    T s[CPL];
#pragma unroll
    for (int k = 0; k < CPL; ++k) s[k] = acc[k];
    store_vec<T, CPL>(part + static_cast<size_t>(u.w) * C + c0, s);
  }
  __threadfence();
  __syncwarp();
  unsigned prev = 0;
  if (lane == 0) prev = atomicAdd(a.counters + u.x, 1u);
  prev = __shfl_sync(kFull, prev, 0);
  if (prev != static_cast<unsigned>(hr.z - 1)) return;  // warp-uniform
  __threadfence();
  T tot[CPL];
#pragma unroll
  for (int k = 0; k < CPL; ++k) tot[k] = T(0);
  for (int s = hr.y; s < hr.y + hr.z; ++s)
#pragma unroll
    for (int k = 0; k < CPL; ++k) tot[k] += __ldcg(part + static_cast<size_t>(s) * C + c0 + k);
  ColAcc<T, CPL> cacc;
  cacc.zero();
  epilogue<T, C, MODE, CPL>(a, s_cand, hr.x, true, owner, c0, 0, tot, cacc, true);
  double cs[CPL];
#pragma unroll
  for (int k = 0; k < CPL; ++k) cs[k] = cacc.get(k);
  if (owner) write_slot<MODE, C, CPL>(a, static_cast<size_t>(a.num_units + u.x), c0, cs);
  if (lane == 0) a.counters[u.x] = 0u;  // ready for the next launch
}

// Runs work unit uidx with the given gather source.
template <typename T, int C, int MODE, class Src>
__device__ __forceinline__ void run_unit(const SweepArgs& a, const Src& src, int uidx, int lane, int* rp,
                                        const int* s_cand) {
  const int4 u = a.units[uidx];
  if (u.w >= 0) {
    heavy_slice<T, C, MODE>(a, src, u, uidx, lane, s_cand);
    return;
  }
  switch (u.z) {
    // the lookahead's 8-column rows of degree <= 2 take two lanes each: one lane holding all eight
    // columns of two rows overflows the register budget of five CTAs per SM
    case 0: short_rows<T, C, MODE, (MODE == MODE_LOOK && C == 8 && sizeof(T) == 4) ? 1 : 0>(a, src, u, uidx, lane, rp, s_cand); break;
    case 1: short_rows<T, C, MODE, 1>(a, src, u, uidx, lane, rp, s_cand); break;
    case 2: short_rows<T, C, MODE, 2>(a, src, u, uidx, lane, rp, s_cand); break;
    case 3: short_rows<T, C, MODE, 3>(a, src, u, uidx, lane, rp, s_cand); break;
    case 4: short_rows<T, C, MODE, 4>(a, src, u, uidx, lane, rp, s_cand); break;
    case 5: short_rows<T, C, MODE, 5>(a, src, u, uidx, lane, rp, s_cand); break;
    default: long_rows<T, C, MODE>(a, src, u, uidx, lane, rp, s_cand); break;
  }
}

constexpr int kCandSlots = 16;

// Resident CTAs per SM each instantiation is compiled for (its register limit). The gathers wait
// on memory, and more resident warps hide more of that latency than a few spilled registers cost:
// the 8-column lookahead sweep is held to 48 registers (five CTAs per SM), the 4-column candidate
// batch to 64 (four), the one-step fused and two-state sweeps of 1-2 columns to 32 (eight) and of 4
// to 40 (six), and the batched-scoring widths to what their C-wide row sums need (measured on R-MAT
// scale 22 and on the Barabasi-Albert graph with n = 10^6).
template <typename T, int C, int MODE>
constexpr int min_ctas() {
  if (sizeof(T) == 8) return 1;
  if (MODE == MODE_LOOK && C == 8) return 5;
  if (MODE == MODE_CAND && C == 4) return 4;
  if ((MODE == MODE_FUSED || MODE == MODE_SCORE) && C <= 2) return 8;
  if (MODE == MODE_FUSED && C == 4) return 6;
  if (MODE == MODE_PLAIN) return C <= 8 ? 5 : C <= 16 ? 3 : C <= 32 ? 2 : 1;
  return 1;
}

// One warp per unit, one CTA per eight units.
template <typename T, int C, int MODE>
__global__ void __launch_bounds__(kThreads, (min_ctas<T, C, MODE>())) sweep_kernel(const SweepArgs a) {
  __shared__ int s_cand[kCandSlots];
  __shared__ int s_rp[kWarps][kUnitRowsMax + 1];
  if (threadIdx.x < kCandSlots)
    s_cand[threadIdx.x] = (MODE == MODE_FUSED || MODE == MODE_CAND || MODE == MODE_LOOK) && a.cand ? a.cand[threadIdx.x] : -1;
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int uidx = blockIdx.x * kWarps + warp;
  if (uidx >= a.num_units) return;
  const GlobalSrc<T, C> src{static_cast<const T*>(a.X), a.hub};
  run_unit<T, C, MODE>(a, src, uidx, lane, s_rp[warp], s_cand);
}

// [sweep-kernel-source-end]

// Deterministic block sum: thread 0 receives the total.
__device__ __forceinline__ double block_sum1(double v, double* sm) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
  if (lane == 0) sm[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = sm[0];
    for (int w = 1; w < kWarps; ++w) s += sm[w];
    v = s;
  }
  __syncthreads();
  return v;
}

// Stage 1: CTA (part, c) sums a fixed stretch of slots for column c; stage 2 adds the
// stretches in order.
__global__ void __launch_bounds__(kThreads) reduce_slots_part(const double* __restrict__ slots, int32_t num_slots,
                                                             int32_t nsum, double* __restrict__ parts) {
  __shared__ double sm[kWarps];
  const int c = blockIdx.y, part = blockIdx.x;
  const int per = (num_slots + kReduceParts - 1) / kReduceParts;
  const int lo = part * per, hi = min(num_slots, lo + per);
  double v = 0.0;
  for (int i = lo + threadIdx.x; i < hi; i += kThreads) v += slots[static_cast<size_t>(i) * nsum + c];
  v = block_sum1(v, sm);
  if (threadIdx.x == 0) parts[c * kReduceParts + part] = v;
}

__global__ void reduce_slots_final(const double* __restrict__ parts, int32_t nsum, double* __restrict__ out) {
  const int c = threadIdx.x;
  if (c >= nsum) return;
  double s = 0.0;
  for (int p = 0; p < kReduceParts; ++p) s += parts[c * kReduceParts + p];
  out[c] = s;
}

// Sets the instantiation's shared-memory carveout on the current device, once per device: a small
// carveout leaves the rest of the unified L1/shared array to cache the gathered rows of x.
template <typename T, int C, int MODE>
void configure() {
  constexpr int kMaxDevices = 64;
  static std::atomic<bool> done[kMaxDevices];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return;
  }
  if (done[dev].load(std::memory_order_acquire)) return;
  cudaFuncSetAttribute(sweep_kernel<T, C, MODE>, cudaFuncAttributePreferredSharedMemoryCarveout, 16);
  cudaGetLastError();
  done[dev].store(true, std::memory_order_release);
}

template <typename T, int C, int MODE>
gedwalk_status run(const SweepArgs& a, cudaStream_t s, bool profile) {
  if (a.num_units == 0) return GEDWALK_OK;
  cudaEvent_t ev = nullptr;
  const bool prof = profile && profiling();
  if (prof) profile_begin(s, &ev);
  configure<T, C, MODE>();
  const int grid = (a.num_units + kWarps - 1) / kWarps;
  SweepArgs b = a;  // rows gathered with L1 priority: about kL1HubBytes of them
  b.hub = static_cast<int32_t>(std::min<int64_t>(a.n, kL1HubBytes / (sizeof(T) * C)));
  sweep_kernel<T, C, MODE><<<grid, kThreads, 0, s>>>(b);
  GW_KCHECK();
  if (prof)
    profile_end(s, ev, sweep_bytes(MODE, sizeof(T) == 8, C, a.n, a.nnz, a.rs_f != nullptr),
                (MODE * 1000 + C) * 2 + (sizeof(T) == 8));
  return GEDWALK_OK;
}

}  // namespace

int sweep_sums(int mode, int cols) {
  switch (mode) {
    case MODE_TOTALS:
    case MODE_SCORE:
      return 1;
    case MODE_FUSED:
    case MODE_LOOK:
      return cols - 1;
    case MODE_CAND:
      return cols;
    default:
      return 0;
  }
}

gedwalk_status configure_sweep(int mode, bool fp64, int cols) {
#define GW_CASE(M, T, C)                                     \
  if (mode == M && fp64 == (sizeof(T) == 8) && cols == C) { \
    configure<T, C, M>();                                    \
    return GEDWALK_OK;                                       \
  }
  GW_CASE(MODE_LOOK, float, 4)
  GW_CASE(MODE_LOOK, float, 8)
  GW_CASE(MODE_LOOK, double, 4)
  GW_CASE(MODE_CAND, float, 4)
  GW_CASE(MODE_CAND, double, 4)
#undef GW_CASE
  return fail(GEDWALK_ERR_INVALID, "no sweep instantiation to configure for mode %d fp64 %d cols %d", mode,
              int(fp64), cols);
}

gedwalk_status launch_sweep(int mode, bool fp64, int cols, const SweepArgs& a, cudaStream_t s, bool profile) {
#define GW_CASE(M, T, C) \
  if (mode == M && fp64 == (sizeof(T) == 8) && cols == C) return run<T, C, M>(a, s, profile);
  GW_CASE(MODE_TOTALS, double, 1)
  GW_CASE(MODE_SCORE, double, 2)
  GW_CASE(MODE_SCORE, float, 2)
  GW_CASE(MODE_FUSED, float, 1)
  GW_CASE(MODE_FUSED, float, 2)
  GW_CASE(MODE_FUSED, float, 4)
  GW_CASE(MODE_FUSED, float, 8)
  GW_CASE(MODE_FUSED, double, 1)
  GW_CASE(MODE_FUSED, double, 2)
  GW_CASE(MODE_FUSED, double, 4)
  GW_CASE(MODE_CAND, float, 4)
  GW_CASE(MODE_CAND, float, 8)
  GW_CASE(MODE_CAND, float, 16)
  GW_CASE(MODE_CAND, double, 4)
  GW_CASE(MODE_CAND, double, 8)
  GW_CASE(MODE_LOOK, float, 4)
  GW_CASE(MODE_LOOK, float, 8)
  GW_CASE(MODE_LOOK, double, 4)
  GW_CASE(MODE_PLAIN, float, 4)
  GW_CASE(MODE_PLAIN, float, 8)
  GW_CASE(MODE_PLAIN, float, 16)
  GW_CASE(MODE_PLAIN, float, 32)
  GW_CASE(MODE_PLAIN, float, 64)
#undef GW_CASE
  return fail(GEDWALK_ERR_INVALID, "no sweep instantiation for mode %d fp64 %d cols %d", mode, int(fp64), cols);
}

gedwalk_status launch_reduce_slots(const double* slots, int32_t num_slots, int32_t nsum, double* out,
                                   double* parts, cudaStream_t s) {
  if (nsum <= 0) return GEDWALK_OK;
  reduce_slots_part<<<dim3(kReduceParts, nsum), kThreads, 0, s>>>(slots, num_slots, nsum, parts);
  GW_KCHECK();
  reduce_slots_final<<<1, 32, 0, s>>>(parts, nsum, out);
  GW_KCHECK();
  return GEDWALK_OK;
}

}  // namespace gw
