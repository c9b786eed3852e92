// The sweep kernel: one masked, alpha-scaled SpMV/SpMM step y = alpha * A x over the
// relabelled CSR, with a fused per-row epilogue selected at compile time.
//
// Every step of GED-Walk's hot path is such a sweep: the walk totals t_r
// (Eq. katz-def terms, used by the combinatorial bound, Eq. comb-bound), the
// two-state hit/miss recurrences of Section 3.1.1, the phi^miss vectors that
// feed the Lemma-initialize bound, and the candidate columns that count the
// walks through a vertex (proof of Prop. ged_submod).
//
// Work distribution (the graph is relabelled by decreasing degree, so rows of
// similar degree are contiguous):
//  - light units: a CTA takes consecutive rows of one degree class and gives
//    each row 2^lw lanes; lanes stride over the row's entries, gather the C-wide
//    rows of x (16-byte vector loads) and reduce with xor shuffles;
//  - heavy slices: rows of degree > kHeavyDeg are cut into slices of about
//    kSliceEdges entries, one CTA per slice; each CTA writes its partial sum,
//    and the last CTA to arrive (atomic counter) adds the partials in slice
//    order and runs the epilogue. No CTA ever waits for another.
// Column sums (sum_v y(v) per column, FP64) are reduced per CTA in a fixed order
// into per-CTA slots, so every result is bitwise reproducible.
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"

namespace gw {
namespace {

constexpr unsigned kFull = 0xffffffffu;

template <typename T>
__device__ __forceinline__ T ldx(const T* p) {
  return __ldg(p);
}

// acc[c] += X[v][c] for c < C with the widest aligned vector loads.
template <typename T, int C>
__device__ __forceinline__ void add_row(T (&acc)[C], const T* __restrict__ X, int v) {
  constexpr int kBytes = int(sizeof(T)) * C;
  const T* p = X + static_cast<size_t>(v) * C;
  if constexpr (kBytes % 16 == 0) {
    constexpr int kPer = 16 / int(sizeof(T));
    const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
    for (int k = 0; k < kBytes / 16; ++k) {
      float4 t = __ldg(q + k);
      T vals[kPer];
      memcpy(vals, &t, 16);
#pragma unroll
      for (int e = 0; e < kPer; ++e) acc[k * kPer + e] += vals[e];
    }
  } else if constexpr (kBytes == 8) {
    float2 t = __ldg(reinterpret_cast<const float2*>(p));
    T vals[8 / sizeof(T)];
    memcpy(vals, &t, 8);
#pragma unroll
    for (int e = 0; e < C; ++e) acc[e] += vals[e];
  } else {
#pragma unroll
    for (int e = 0; e < C; ++e) acc[e] += ldx(p + e);
  }
}

// Y[r][0..C) = vals with vector stores.
template <typename T, int C>
__device__ __forceinline__ void store_row(T* __restrict__ Y, int r, const T (&vals)[C]) {
  constexpr int kBytes = int(sizeof(T)) * C;
  T* p = Y + static_cast<size_t>(r) * C;
  if constexpr (kBytes % 16 == 0) {
    float4* q = reinterpret_cast<float4*>(p);
#pragma unroll
    for (int k = 0; k < kBytes / 16; ++k) {
      float4 t;
      memcpy(&t, &vals[k * (16 / int(sizeof(T)))], 16);
      q[k] = t;
    }
  } else if constexpr (kBytes == 8) {
    float2 t;
    memcpy(&t, vals, 8);
    *reinterpret_cast<float2*>(p) = t;
  } else {
#pragma unroll
    for (int e = 0; e < C; ++e) p[e] = vals[e];
  }
}

__device__ __forceinline__ bool in_mask(const uint32_t* __restrict__ mask, int r) {
  return (__ldg(mask + (r >> 5)) >> (r & 31)) & 1u;
}

// Number of FP64 column sums a mode keeps.
template <int MODE, int C>
struct Sums {
  static constexpr int N = MODE == MODE_TOTALS ? 1 : MODE == MODE_SCORE ? 1 : MODE == MODE_FUSED ? C - 1
                           : MODE == MODE_CAND ? C : 0;
  static constexpr int A = N > 0 ? N : 1;  // storage
};

// The per-row epilogue. acc holds sum_{u ~ r} x(u) for each column.
template <typename T, int C, int MODE>
__device__ __forceinline__ void epilogue(const SweepArgs& a, const int* __restrict__ s_cand, int r,
                                         const T (&acc)[C], double (&cs)[Sums<MODE, C>::A]) {
  const T alpha = static_cast<T>(a.alpha);
  T* Y = static_cast<T*>(a.Y);
  if constexpr (MODE == MODE_TOTALS) {
    T out[C];
    out[0] = alpha * acc[0];
    store_row<T, C>(Y, r, out);
    cs[0] += static_cast<double>(out[0]);
  } else if constexpr (MODE == MODE_SCORE) {
    // Section 3.1.1: hit_i(v) = sum hit_{i-1}(u) + [v in S] sum miss_{i-1}(u);
    //                miss_i(v) = [v not in S] sum miss_{i-1}(u)
    const bool inS = in_mask(a.mask, r);
    T out[C];
    out[0] = alpha * (inS ? acc[0] + acc[1] : acc[0]);
    out[1] = inS ? T(0) : alpha * acc[1];
    store_row<T, C>(Y, r, out);
    cs[0] += static_cast<double>(out[0]);
  } else if constexpr (MODE == MODE_FUSED) {
    // column 0: phi^miss under S; columns j >= 1: walks through candidate c_j that avoid S,
    // whose row c_j takes the phi^miss value (every S-avoiding walk ending at c_j visits it)
    const bool inS = in_mask(a.mask, r);
    T out[C];
    out[0] = inS ? T(0) : alpha * acc[0];
#pragma unroll
    for (int j = 1; j < C; ++j) {
      T y = inS ? T(0) : alpha * acc[j];
      if (s_cand[j - 1] == r) y = out[0];
      out[j] = y;
      cs[j - 1] += static_cast<double>(y);
    }
    store_row<T, C>(Y, r, out);
    static_cast<T*>(a.Mout)[r] = out[0];
  } else if constexpr (MODE == MODE_CAND) {
    const bool inS = in_mask(a.mask, r);
    T out[C];
#pragma unroll
    for (int j = 0; j < C; ++j) {
      T y = inS ? T(0) : alpha * acc[j];
      if (s_cand[j] == r) y = __ldg(static_cast<const T*>(a.Min) + r);
      out[j] = y;
      cs[j] += static_cast<double>(y);
    }
    store_row<T, C>(Y, r, out);
  } else {  // MODE_PLAIN
    T out[C];
#pragma unroll
    for (int j = 0; j < C; ++j) out[j] = alpha * acc[j];
    store_row<T, C>(Y, r, out);
  }
}

// Deterministic block sum: thread 0 receives the totals.
template <typename V, int N>
__device__ __forceinline__ void block_sum(V (&v)[N], V (*sm)[N]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < N; ++c)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[c] += __shfl_down_sync(kFull, v[c], o);
  if (lane == 0)
#pragma unroll
    for (int c = 0; c < N; ++c) sm[warp][c] = v[c];
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int c = 0; c < N; ++c) {
      V s = sm[0][c];
      for (int w = 1; w < kThreads / 32; ++w) s += sm[w][c];
      v[c] = s;
    }
  }
  __syncthreads();
}

template <typename T, int C, int MODE>
__global__ void __launch_bounds__(kThreads) sweep_kernel(const SweepArgs a) {
  constexpr int NS = Sums<MODE, C>::N;
  constexpr int NA = Sums<MODE, C>::A;
  __shared__ int s_cand[C];
  __shared__ double s_cs[kThreads / 32][NA];
  __shared__ T s_acc[kThreads / 32][C];
  __shared__ int s_last;
  if (threadIdx.x < C)
    s_cand[threadIdx.x] = (MODE == MODE_FUSED || MODE == MODE_CAND) && a.cand ? a.cand[threadIdx.x] : -1;
  __syncthreads();

  const int4 u = a.units[blockIdx.x];
  const int32_t* __restrict__ ci = a.ci;
  const T* __restrict__ X = static_cast<const T*>(a.X);
  double cs[NA];
#pragma unroll
  for (int c = 0; c < NA; ++c) cs[c] = 0.0;

  if (u.w >= 0) {
    // ---- heavy slice: entries [u.y, u.z) of heavy row u.x
    T acc[C];
#pragma unroll
    for (int c = 0; c < C; ++c) acc[c] = T(0);
    int j = u.y + threadIdx.x;
    for (; j + 3 * kThreads < u.z; j += 4 * kThreads) {
      const int v0 = __ldcs(ci + j), v1 = __ldcs(ci + j + kThreads), v2 = __ldcs(ci + j + 2 * kThreads),
                v3 = __ldcs(ci + j + 3 * kThreads);
      add_row<T, C>(acc, X, v0);
      add_row<T, C>(acc, X, v1);
      add_row<T, C>(acc, X, v2);
      add_row<T, C>(acc, X, v3);
    }
    for (; j < u.z; j += kThreads) add_row<T, C>(acc, X, __ldcs(ci + j));
    block_sum<T, C>(acc, s_acc);
    const int4 hr = a.heavy[u.x];  // {row, first slice, slice count, 0}
    if constexpr (NS > 0) {
      // this CTA's own slot carries nothing: the row's sums go to the heavy row's slot
      if (threadIdx.x < NS) a.slots[static_cast<size_t>(blockIdx.x) * NS + threadIdx.x] = 0.0;
    }
    if (threadIdx.x == 0) {
      T* part = static_cast<T*>(a.partial) + static_cast<size_t>(u.w) * C;
#pragma unroll
      for (int c = 0; c < C; ++c) part[c] = acc[c];
      __threadfence();
      const unsigned prev = atomicAdd(a.counters + u.x, 1u);
      s_last = (prev == static_cast<unsigned>(hr.z - 1));
    }
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
      __threadfence();
      T tot[C];
#pragma unroll
      for (int c = 0; c < C; ++c) tot[c] = T(0);
      const T* part = static_cast<const T*>(a.partial);
      for (int s = hr.y; s < hr.y + hr.z; ++s)
#pragma unroll
        for (int c = 0; c < C; ++c) tot[c] += __ldcg(part + static_cast<size_t>(s) * C + c);
      epilogue<T, C, MODE>(a, s_cand, hr.x, tot, cs);
      if constexpr (NS > 0) {
        double* slot = a.slots + static_cast<size_t>(a.num_units + u.x) * NS;
#pragma unroll
        for (int c = 0; c < NS; ++c) slot[c] = a.accumulate ? slot[c] + cs[c] : cs[c];
      }
      a.counters[u.x] = 0u;  // ready for the next launch
    }
    return;
  }

  // ---- light unit: rows [u.x, u.y), 2^u.z lanes per row
  const int lw = u.z;
  const int w = 1 << lw;
  const int lane = threadIdx.x & (w - 1);
  const int grp = threadIdx.x >> lw;
  const int ngrp = kThreads >> lw;
  const int rows = u.y - u.x;
  const int iters = (rows + ngrp - 1) / ngrp;
  for (int it = 0; it < iters; ++it) {
    const int r = u.x + it * ngrp + grp;
    const bool valid = r < u.y;
    T acc[C];
#pragma unroll
    for (int c = 0; c < C; ++c) acc[c] = T(0);
    if (valid) {
      const int e0 = __ldcs(a.rp + r), e1 = __ldcs(a.rp + r + 1);
      int j = e0 + lane;
      for (; j + 3 * w < e1; j += 4 * w) {
        const int v0 = __ldcs(ci + j), v1 = __ldcs(ci + j + w), v2 = __ldcs(ci + j + 2 * w),
                  v3 = __ldcs(ci + j + 3 * w);
        add_row<T, C>(acc, X, v0);
        add_row<T, C>(acc, X, v1);
        add_row<T, C>(acc, X, v2);
        add_row<T, C>(acc, X, v3);
      }
      for (; j < e1; j += w) add_row<T, C>(acc, X, __ldcs(ci + j));
    }
    // butterfly over the row's lanes; every lane of the warp takes part
    for (int o = w >> 1; o > 0; o >>= 1)
#pragma unroll
      for (int c = 0; c < C; ++c) acc[c] += __shfl_xor_sync(kFull, acc[c], o);
    if (valid && lane == 0) epilogue<T, C, MODE>(a, s_cand, r, acc, cs);
  }
  if constexpr (NS > 0) {
    block_sum<double, NA>(cs, s_cs);
    if (threadIdx.x == 0) {
      double* slot = a.slots + static_cast<size_t>(blockIdx.x) * NS;
#pragma unroll
      for (int c = 0; c < NS; ++c) slot[c] = a.accumulate ? slot[c] + cs[c] : cs[c];
    }
  }
}

// Sum of slots[i][c] over i, one CTA per column, fixed order.
__global__ void __launch_bounds__(kThreads) reduce_slots_kernel(const double* __restrict__ slots, int32_t num_slots,
                                                               int32_t nsum, double* __restrict__ out) {
  __shared__ double sm[kThreads / 32][1];
  const int c = blockIdx.x;
  double v[1] = {0.0};
  for (int i = threadIdx.x; i < num_slots; i += kThreads) v[0] += slots[static_cast<size_t>(i) * nsum + c];
  block_sum<double, 1>(v, sm);
  if (threadIdx.x == 0) out[c] = v[0];
}

template <typename T, int C, int MODE>
gedwalk_status run(const SweepArgs& a, cudaStream_t s) {
  if (a.num_units == 0) return GEDWALK_OK;
  cudaEvent_t ev = nullptr;
  const bool prof = profiling();
  if (prof) profile_begin(s, &ev);
  sweep_kernel<T, C, MODE><<<a.num_units, kThreads, 0, s>>>(a);
  GW_KCHECK();
  if (prof) profile_end(s, ev, sweep_bytes(MODE, sizeof(T) == 8, C, a.n, a.nnz));
  return GEDWALK_OK;
}

}  // namespace

int sweep_sums(int mode, int cols) {
  switch (mode) {
    case MODE_TOTALS:
    case MODE_SCORE:
      return 1;
    case MODE_FUSED:
      return cols - 1;
    case MODE_CAND:
      return cols;
    default:
      return 0;
  }
}

gedwalk_status launch_sweep(int mode, bool fp64, int cols, const SweepArgs& a, cudaStream_t s) {
#define GW_CASE(M, T, C) \
  if (mode == M && fp64 == (sizeof(T) == 8) && cols == C) return run<T, C, M>(a, s);
  GW_CASE(MODE_TOTALS, double, 1)
  GW_CASE(MODE_SCORE, double, 2)
  GW_CASE(MODE_SCORE, float, 2)
  GW_CASE(MODE_FUSED, float, 1)
  GW_CASE(MODE_FUSED, float, 8)
  GW_CASE(MODE_FUSED, double, 1)
  GW_CASE(MODE_FUSED, double, 4)
  GW_CASE(MODE_CAND, float, 8)
  GW_CASE(MODE_CAND, float, 16)
  GW_CASE(MODE_CAND, double, 4)
  GW_CASE(MODE_CAND, double, 8)
  GW_CASE(MODE_PLAIN, float, 4)
  GW_CASE(MODE_PLAIN, float, 8)
  GW_CASE(MODE_PLAIN, float, 16)
  GW_CASE(MODE_PLAIN, float, 32)
#undef GW_CASE
  return fail(GEDWALK_ERR_INVALID, "no sweep instantiation for mode %d fp64 %d cols %d", mode, int(fp64), cols);
}

gedwalk_status launch_reduce_slots(const double* slots, int32_t num_slots, int32_t nsum, double* out,
                                   cudaStream_t s) {
  if (nsum <= 0) return GEDWALK_OK;
  reduce_slots_kernel<<<nsum, kThreads, 0, s>>>(slots, num_slots, nsum, out);
  GW_KCHECK();
  return GEDWALK_OK;
}

}  // namespace gw
