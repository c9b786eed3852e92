// Greedy GED-Walk maximisation (problem (ii), Def. ged-max; Prop. greedy_approx) and
// all-vertex exact marginal gains.
//
// A step with current group S:
//  1. L fused sweeps compute phi^miss_1..L under S (column 0, stored in a table) and,
//     in the same pass, the exact gains of up to kSpec "speculative" candidates
//     (columns 1..), chosen before S was known from bounds that stay valid when S
//     grows: the last exact gain (submodularity, Prop. ged_submod) and the previous
//     step's Lemma-initialize bound (P_i is non-increasing in S).
//  2. One pass over all vertices forms the Lemma-initialize bound
//       ub(x) = sum_{i=1..L} alpha^i P_i(S, x) = sum_{1 <= a+b <= L} y_a(x) y_b(x),
//     y_a = alpha^a phi^miss_a (psi^miss = phi^miss on an undirected graph), takes
//     min(ub, last exact gain), and selects the best-bounded unevaluated vertices.
//  3. The best evaluated candidate wins once no unevaluated bound (inflated by the
//     rounding tolerance) reaches its gain; otherwise the next batch of candidates
//     is evaluated exactly and step 2 repeats. A vertex whose bound is exactly 0
//     has gain exactly 0. Among equal gains the lowest caller id wins.
// The gain of candidate c counts walks of length 1..L in G[V\S] through c
// (proof of Prop. ged_submod): h_0 = e_c, h_t = alpha 1_{V\S} . A h_{t-1} except
// h_t(c) = phi^miss_t(c); gain = sum_t sum_v h_t(v) in FP64.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdlib>

#include "internal.h"

namespace gw {
namespace {

constexpr int kTopK = 16;
constexpr int kSelPerSM = 4;               // resident blocks of the bound pass per SM
constexpr int kSelU = 2;                   // vertices per lane and iteration of the bound pass
constexpr int kSelBlocks = 152 * kSelPerSM;

struct Stale {
  float ub;      // last exact gain rounded up (an upper bound for every later step)
  int32_t step;  // step in which it was evaluated, -1 if never
};

struct SelOut {  // device -> host after each selection pass
  float val[kTopK];
  int32_t id[kTopK];
  // the unevaluated vertex with bound exactly 0 and the smallest caller id, packed as
  // (caller id << 32) | internal id (all ones: none)
  unsigned long long zero_min;
  int32_t sampled;  // stochastic greedy: sampled vertices outside S seen by the pass
  int32_t done;     // blocks of the pass that have finished
  double gains[16];  // exact gains of the last candidate batch
};

constexpr unsigned long long kNoZero = ~0ull;
__host__ __device__ inline int32_t zero_caller(unsigned long long z) {
  return z == kNoZero ? INT_MAX : static_cast<int32_t>(z >> 32);
}
__host__ __device__ inline int32_t zero_internal(unsigned long long z) {
  return static_cast<int32_t>(z & 0xffffffffull);
}

__device__ __forceinline__ bool better(float a, int ia, float b, int ib) { return a > b || (a == b && ia < ib); }

// Stochastic greedy's counter-based draw: the first output of splitmix64 (Steele, Lea & Flood,
// 2014) started from state seed ^ (step << 32) ^ v, v a caller id.
__device__ __forceinline__ uint64_t sample_hash(uint64_t seed, uint32_t step, uint32_t v) {
  uint64_t z = (seed ^ (static_cast<uint64_t>(step) << 32) ^ static_cast<uint64_t>(v)) + 0x9e3779b97f4a7c15ULL;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

// Sampling of one selection pass; thr == UINT64_MAX means every vertex takes part.
struct Sampling {
  uint64_t thr;
  uint64_t seed;
  uint32_t step;
};

constexpr unsigned kFullMask = 0xffffffffu;

// A warp's sorted list of its kTopK best (value, id) pairs in the order of `better`: lane i <
// kTopK holds the i-th entry (value -1, id INT_MAX: empty); `tag` travels with its entry.
struct WarpList {
  float v = -1.0f;
  int id = INT_MAX;
  int tag = 0;
};

// Offers every lane's (x, ix, tag) where `want` holds. Only the lanes that beat the list's last
// entry are inserted, one at a time (lowest lane first); after each insertion the others are
// checked again against the new last entry. Ids must be distinct. All 32 lanes take part.
__device__ __forceinline__ void warp_list_offer(WarpList& w, bool want, float x, int ix, int tag) {
  const int lane = threadIdx.x & 31;
  float tv = __shfl_sync(kFullMask, w.v, kTopK - 1);
  int ti = __shfl_sync(kFullMask, w.id, kTopK - 1);
  unsigned m = __ballot_sync(kFullMask, want && better(x, ix, tv, ti));
  while (m) {
    const int src = __ffs(m) - 1;
    const float cv = __shfl_sync(kFullMask, x, src);
    const int ci = __shfl_sync(kFullMask, ix, src);
    const int ct = __shfl_sync(kFullMask, tag, src);
    // the entries ahead of the new one form a prefix of the sorted list
    const int pos = __popc(__ballot_sync(kFullMask, lane < kTopK && better(w.v, w.id, cv, ci)));
    const float uv = __shfl_up_sync(kFullMask, w.v, 1);
    const int ui = __shfl_up_sync(kFullMask, w.id, 1);
    const int ut = __shfl_up_sync(kFullMask, w.tag, 1);
    if (lane == pos) {
      w.v = cv;
      w.id = ci;
      w.tag = ct;
    } else if (lane > pos && lane < kTopK) {
      w.v = uv;
      w.id = ui;
      w.tag = ut;
    }
    tv = __shfl_sync(kFullMask, w.v, kTopK - 1);
    ti = __shfl_sync(kFullMask, w.id, kTopK - 1);
    m &= m - 1;
    m &= __ballot_sync(kFullMask, want && better(x, ix, tv, ti));
  }
}

// Merges the NW warp lists of a block into warp 0's list (staged through shared memory sv/si/st,
// NW * kTopK entries each). Every thread of the block calls it.
template <int NW>
__device__ void block_list_merge(WarpList& w, float* sv, int* si, int* st) {
  static_assert(kTopK == 16, "two warp lists per 32-lane offer");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane < kTopK) {
    sv[warp * kTopK + lane] = w.v;
    si[warp * kTopK + lane] = w.id;
    st[warp * kTopK + lane] = w.tag;
  }
  __syncthreads();
  if (warp == 0) {
    for (int j = 1; j < NW; j += 2) {  // lists j and j + 1 on lanes 0-15 and 16-31
      const int src = j + (lane >> 4);
      const bool ok = src < NW;
      const int e = src * kTopK + (lane & 15);
      const float x = ok ? sv[e] : -1.0f;
      const int ix = ok ? si[e] : INT_MAX;
      const int t = ok ? st[e] : 0;
      warp_list_offer(w, ix != INT_MAX, x, ix, t);
    }
  }
  __syncthreads();
}

// mtab row 0 = phi^miss_0 = 1_{V\S}; X column 0 (fused) = the same; candidate columns = e_c.
// On a weighted graph X holds the scaled vectors (times s_v, rs); the table the true values.
template <typename T>
__global__ void greedy_init(T* __restrict__ m0, T* __restrict__ X, int cols, int first_cand_col,
                            const int32_t* __restrict__ cand, const uint32_t* __restrict__ mask, int32_t n,
                            const T* __restrict__ rs) {
  __shared__ int sc[16];
  if (threadIdx.x < 16) sc[threadIdx.x] = threadIdx.x < cols - first_cand_col ? cand[threadIdx.x] : -1;
  __syncthreads();
  for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const bool inS = (mask[v >> 5] >> (v & 31)) & 1u;
    const T m = inS ? T(0) : T(1);
    const T sv = rs ? rs[v] : T(1);
    if (m0) m0[v] = m;
    T* row = X + static_cast<size_t>(v) * cols;
    if (first_cand_col == 1) row[0] = m * sv;
    for (int j = first_cand_col; j < cols; ++j) row[j] = (sc[j - first_cand_col] == v) ? sv : T(0);
  }
}

// MODE_LOOK initialisation for a run of C - 1 levels with guesses c_1..c_{C-1}: column 0 is
// phi^miss_0 under S, column j >= 1 the unit vector of c_j (0 without one); table d, row 0, is
// phi^miss_0 under S + {c_1..c_d}. The walk vectors are written 16 bytes per thread (consecutive
// threads, consecutive chunks).
template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
  using type = float4;
  __device__ static float4 make(const float* e) { return make_float4(e[0], e[1], e[2], e[3]); }
};
template <>
struct Vec16<double> {
  using type = double2;
  __device__ static double2 make(const double* e) { return make_double2(e[0], e[1]); }
};

template <typename T, int C>
__global__ void look_init(T* __restrict__ tab, int64_t tab_stride, T* __restrict__ X,
                          const int32_t* __restrict__ cand, const uint32_t* __restrict__ mask, int32_t n,
                          const T* __restrict__ rs) {
  constexpr int LV = C - 1;                               // levels
  constexpr int per = 16 / static_cast<int>(sizeof(T));  // elements per 16-byte chunk
  static_assert(C % per == 0, "a row is whole 16-byte chunks");
  constexpr int cpr = C / per;                            // chunks per row
  __shared__ int sc[LV];
  if (threadIdx.x < LV) sc[threadIdx.x] = cand[threadIdx.x];
  __syncthreads();
  const int64_t chunks = static_cast<int64_t>(n) * cpr;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  using V = typename Vec16<T>::type;
  for (int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; q < chunks; q += stride) {
    const int32_t v = static_cast<int32_t>(q / cpr);
    const int part = static_cast<int>(q % cpr);
    const bool inS = (__ldg(mask + (v >> 5)) >> (v & 31)) & 1u;
    const T sv = rs ? rs[v] : T(1);
    T e[per];
#pragma unroll
    for (int j = 0; j < per; ++j) {
      const int col = part * per + j;
      if (col == 0) e[j] = inS ? T(0) : sv;
      else e[j] = sc[col - 1] == v ? sv : T(0);
    }
    reinterpret_cast<V*>(X)[q] = Vec16<T>::make(e);
  }
  for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    bool out = (__ldg(mask + (v >> 5)) >> (v & 31)) & 1u;
#pragma unroll
    for (int d = 0; d < LV; ++d) {
      if (d > 0 && sc[d - 1] == v) out = true;
      tab[tab_stride * d + v] = out ? T(0) : T(1);
    }
  }
}

// cols = levels + 1: 4 or (FP32) 8, the only shapes greedy_shape admits
template <typename T>
void launch_look_init(int cols, int blocks, cudaStream_t s, T* tab, int64_t tab_stride, T* X, const int32_t* cand,
                      const uint32_t* mask, int32_t n, const T* rs) {
  if (cols == 4 || sizeof(T) == 8) look_init<T, 4><<<blocks, 256, 0, s>>>(tab, tab_stride, X, cand, mask, n, rs);
  else look_init<T, 8><<<blocks, 256, 0, s>>>(tab, tab_stride, X, cand, mask, n, rs);
}

// Records one exact gain known on the host (a lookahead level's candidate) for this step.
__global__ void set_stale(Stale* __restrict__ stale, int32_t v, double gain, int32_t step, double* __restrict__ out) {
  Stale st;
  st.ub = __double2float_ru(gain);
  st.step = step;
  stale[v] = st;
  out[0] = gain;
}

__global__ void update_stale(Stale* __restrict__ stale, const int32_t* __restrict__ cand,
                             const double* __restrict__ gains, int count, int32_t step, double* __restrict__ out) {
  const int j = threadIdx.x;
  if (j >= count) return;
  const int c = cand[j];
  if (out) out[j] = gains[j];
  if (c < 0) return;
  Stale st;
  st.ub = __double2float_ru(gains[j]);
  st.step = step;
  stale[c] = st;
}

__device__ __forceinline__ float to_f32_up(float v) { return v; }
__device__ __forceinline__ float to_f32_up(double v) { return __double2float_ru(v); }

// Lemma-initialize bound of vertex x:
//   ub(x) = sum_{i=1..L} alpha^i P_i(S, x) = sum over ordered pairs 1 <= a+b <= L of y_a(x) z_b(x)
//         = y_0 (Q_L - z_0) + sum_{a=1..L} y_a Q_{L-a},   Q_q = sum_{b <= q} z_b,
// y_a = alpha^a phi^miss_a(x) and z_b = alpha^b psi^miss_b(x), the S-avoiding walks in the other
// orientation (a directed graph's reverse; on an undirected graph z = y, zcol == col). Evaluated
// in FP32 with every operation rounded toward +infinity on non-negative inputs (FP64 inputs are
// first rounded up), so the result never falls below the bound of the stored vectors.
template <typename T, int L>
__device__ __forceinline__ float ub_fixed(const T* __restrict__ col, const T* __restrict__ zcol, int32_t n, float m0) {
  // row 0 is phi^miss_0 = psi^miss_0 = 1_{V\S}: m0, not read from the tables
  float y[L + 1], z[L + 1];
  y[0] = m0;
#pragma unroll
  for (int a = 1; a <= L; ++a) y[a] = to_f32_up(__ldcs(col + static_cast<size_t>(a) * n));
  if (zcol == col) {
#pragma unroll
    for (int a = 0; a <= L; ++a) z[a] = y[a];
  } else {
    z[0] = m0;
#pragma unroll
    for (int a = 1; a <= L; ++a) z[a] = to_f32_up(__ldcs(zcol + static_cast<size_t>(a) * n));
  }
  float Q[L + 1];
  Q[0] = z[0];
  float R = 0.0f;
#pragma unroll
  for (int q = 1; q <= L; ++q) {
    Q[q] = __fadd_ru(Q[q - 1], z[q]);
    R = __fadd_ru(R, z[q]);
  }
  float ub = __fmul_ru(y[0], R);
#pragma unroll
  for (int a = 1; a <= L; ++a) ub = __fmaf_ru(y[a], Q[L - a], ub);
  return ub;
}

// The same sum for any L in one pass: a runs down from L while Q_{L-a} = z_0 + ... + z_{L-a}
// grows, so every pair (a, b) with 1 <= a + b <= L is met once: y_a Q_{L-a} for a >= 1, and
// y_0 (Q_L - z_0) at the end. Two table reads per step, every operation rounded up.
template <typename T>
__device__ float ub_any(const T* __restrict__ col, const T* __restrict__ zcol, int32_t n, int32_t L, float m0) {
  float Q = m0;     // Q_0 = z_0
  float R = 0.0f;   // z_1 + ... + z_{L-a}
  float ub = 0.0f;
  for (int a = L; a >= 1; --a) {
    if (a < L) {
      const float zb = to_f32_up(__ldcs(zcol + static_cast<size_t>(L - a) * n));
      Q = __fadd_ru(Q, zb);
      R = __fadd_ru(R, zb);
    }
    ub = __fmaf_ru(to_f32_up(__ldcs(col + static_cast<size_t>(a) * n)), Q, ub);
  }
  R = __fadd_ru(R, to_f32_up(__ldcs(zcol + static_cast<size_t>(L) * n)));
  return __fmaf_ru(m0, R, ub);
}

// Lemma-initialize bound + selection over vertices [0, n_scan) (the tables have n rows apart):
// the kTopK unevaluated vertices outside S with the largest bounds go to out->val / out->id.
// Each warp keeps its own list (bounds offered 32 at a time, two per lane per iteration), a block
// merges its warps' lists into sel_v / sel_id[block], and the last block to finish merges the
// blocks' lists: only the kTopK blocks whose heads rank among the best kTopK heads can hold an
// entry of the result (any other head has kTopK better entries ahead of it). out->done counts the
// finished blocks (0 before the pass). LF = L when L <= 16, else 0 (any L).
template <typename T, int LF>
__global__ void __launch_bounds__(kThreads, kSelPerSM) ub_select(const T* __restrict__ mtab, const T* __restrict__ ztab,
                                                     int32_t L, int32_t n, int32_t n_scan,
                                                     const uint32_t* __restrict__ mask,
                                                     const Stale* __restrict__ stale, int32_t step,
                                                     const int32_t* __restrict__ perm, float* __restrict__ sel_v,
                                                     int* __restrict__ sel_id, SelOut* __restrict__ out,
                                                     const Sampling smp, const int32_t* level_ptr,
                                                     int64_t level_stride, const int32_t* step_ptr) {
  constexpr int NW = kThreads / 32;
  static_assert(2 * NW >= kTopK, "the final merge gives each warp two block lists");
  constexpr int U = kSelU;
  if (level_ptr) {  // the table (lookahead level) the device-resident loop chose for this step
    const int64_t off = level_stride * __ldg(level_ptr);
    mtab += off;
    ztab += off;
  }
  if (step_ptr) step = __ldg(step_ptr);  // the device-resident loop's step
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int nsampled = 0;
  WarpList w;
  // U * 32 consecutive vertices per warp and iteration, all loads issued before any decision
  const int32_t wid = blockIdx.x * NW + warp;
  const int32_t wstride = gridDim.x * NW * (U * 32);
  for (int32_t base = wid * (U * 32); base < n_scan; base += wstride) {
    float b[U];
    bool live[U];
#pragma unroll
    for (int k = 0; k < U; ++k) {
      const int32_t xr = base + k * 32 + lane;
      const int32_t x = xr < n_scan ? xr : n_scan - 1;
      const bool inS = (__ldg(mask + (x >> 5)) >> (x & 31)) & 1u;
      const Stale st = stale[x];
      const float m0 = inS ? 0.0f : 1.0f;
      float ub = LF > 0 ? ub_fixed<T, (LF > 0 ? LF : 1)>(mtab + x, ztab + x, n, m0)
                        : ub_any<T>(mtab + x, ztab + x, n, L, m0);
      if (st.step >= 0 && st.ub < ub) ub = st.ub;
      b[k] = ub;
      bool in_sample = true;
      if (smp.thr != ~0ull && xr < n_scan && !inS)
        in_sample = sample_hash(smp.seed, smp.step, static_cast<uint32_t>(__ldg(perm + x))) < smp.thr;
      if (xr < n_scan && !inS && in_sample) ++nsampled;
      // evaluated with the current S: its exact gain is known
      live[k] = xr < n_scan && !inS && in_sample && st.step != step;
    }
#pragma unroll
    for (int k = 0; k < U; ++k) {
      const int32_t x = base + k * 32 + lane;
      if (live[k] && b[k] == 0.0f)
        atomicMin(&out->zero_min, (static_cast<unsigned long long>(__ldg(perm + x)) << 32) | static_cast<uint32_t>(x));
      warp_list_offer(w, live[k] && b[k] != 0.0f, b[k], x, 0);
    }
  }
  if (smp.thr != ~0ull) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nsampled += __shfl_xor_sync(kFullMask, nsampled, o);
    if (lane == 0 && nsampled) atomicAdd(&out->sampled, nsampled);
  }
  __shared__ float sv[NW * kTopK];
  __shared__ int si[NW * kTopK], st[NW * kTopK];
  __shared__ int is_last;
  block_list_merge<NW>(w, sv, si, st);
  if (warp == 0) {
    if (lane < kTopK) {
      sel_v[blockIdx.x * kTopK + lane] = w.v;
      sel_id[blockIdx.x * kTopK + lane] = w.id;
    }
    __threadfence();
    __syncwarp();
    int done = 0;
    if (lane == 0) done = atomicAdd(&out->done, 1);
    if (lane == 0) is_last = done == static_cast<int>(gridDim.x) - 1;
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  // the best kTopK block heads (tag: the block)
  WarpList h;
  for (int32_t b0 = warp * 32; b0 < static_cast<int32_t>(gridDim.x); b0 += NW * 32) {
    const int32_t blk = b0 + lane;
    const bool ok = blk < static_cast<int32_t>(gridDim.x);
    const float x = ok ? __ldcg(sel_v + static_cast<size_t>(blk) * kTopK) : -1.0f;
    const int ix = ok ? __ldcg(sel_id + static_cast<size_t>(blk) * kTopK) : INT_MAX;
    warp_list_offer(h, ix != INT_MAX, x, ix, blk);
  }
  block_list_merge<NW>(h, sv, si, st);
  __shared__ int heads[kTopK];
  if (warp == 0 && lane < kTopK) heads[lane] = h.id != INT_MAX ? h.tag : -1;
  __syncthreads();
  // the entries of those blocks, two block lists per warp
  WarpList f;
  {
    const int j = 2 * warp + (lane >> 4);
    const int blk = j < kTopK ? heads[j] : -1;
    const bool ok = blk >= 0;
    const size_t e = static_cast<size_t>(ok ? blk : 0) * kTopK + (lane & 15);
    const float x = ok ? __ldcg(sel_v + e) : -1.0f;
    const int ix = ok ? __ldcg(sel_id + e) : INT_MAX;
    warp_list_offer(f, ix != INT_MAX, x, ix, 0);
  }
  block_list_merge<NW>(f, sv, si, st);
  if (warp == 0 && lane < kTopK) {
    out->val[lane] = f.v;
    out->id[lane] = f.id;
  }
}

template <typename T>
cudaError_t launch_ub_select(int nb, cudaStream_t s, const T* mtab, const T* ztab, int32_t L, int32_t n,
                             int32_t n_scan, const uint32_t* mask,
                             const Stale* stale, int32_t step, const int32_t* perm, float* sel_v, int* sel_id,
                             SelOut* out, const Sampling& smp,
                             const int32_t* level_ptr = nullptr, int64_t level_stride = 0,
                             const int32_t* step_ptr = nullptr) {
#define GW_UB(LL)                                                                                          \
  case LL:                                                                                                 \
    ub_select<T, LL><<<nb, kThreads, 0, s>>>(mtab, ztab, L, n, n_scan, mask, stale, step, perm, sel_v, sel_id, \
                                             out, smp, level_ptr, level_stride, step_ptr);                 \
    break;
  switch (L) {
    GW_UB(1) GW_UB(2) GW_UB(3) GW_UB(4) GW_UB(5) GW_UB(6) GW_UB(7) GW_UB(8)
    GW_UB(9) GW_UB(10) GW_UB(11) GW_UB(12) GW_UB(13) GW_UB(14) GW_UB(15) GW_UB(16)
    default:
      ub_select<T, 0><<<nb, kThreads, 0, s>>>(mtab, ztab, L, n, n_scan, mask, stale, step, perm, sel_v, sel_id,
                                              out, smp, level_ptr, level_stride, step_ptr);
  }
#undef GW_UB
  return cudaGetLastError();
}

// Blocks of a selection pass: one wave at kSelPerSM blocks per SM, one iteration per lane at least.
int sel_blocks(int32_t n_scan) {
  constexpr int64_t per_block = int64_t(kThreads) * kSelU;
  return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(kSelBlocks, (int64_t(n_scan) + per_block - 1) / per_block)));
}

// Resets the per-pass counters of a selection pass.
__global__ void reset_selection(SelOut* out) {
  out->zero_min = kNoZero;
  out->sampled = 0;
  out->done = 0;
}

int blocks_for(int64_t n) { return static_cast<int>(std::min<int64_t>((n + 255) / 256, 152 * 16)); }

// Rows 1..L of the phi^miss table at isolated vertices: the sweeps never write them (no walk
// of length >= 1 ends there), so they are set to 0 once.
gedwalk_status zero_isolated_tail(Graph& g, void* tab, size_t es, int32_t L, cudaStream_t s) {
  if (g.n_active >= g.n || L < 1) return GEDWALK_OK;
  char* base = static_cast<char*>(tab) + static_cast<size_t>(g.n) * es + static_cast<size_t>(g.n_active) * es;
  GW_CUDA(cudaMemset2DAsync(base, static_cast<size_t>(g.n) * es, 0, static_cast<size_t>(g.n - g.n_active) * es, L, s));
  return GEDWALK_OK;
}

struct Cand {
  double g;
  int32_t v;       // internal id
  int32_t caller;  // caller id
};
// exact-gain order: larger gain first, then the lower caller id
bool cand_before(const Cand& a, const Cand& b) { return a.g > b.g || (a.g == b.g && a.caller < b.caller); }

struct GreedyCtx {
  Graph& g;
  Workspace& ws;
  const Resolved& r;
  cudaStream_t s;
  int32_t L;
  size_t es;
  SelOut* d_out;
  int32_t* d_cand;
  double* d_gains;
  SelOut* h_out;
  int64_t sweeps = 0;
  size_t tab_off = 0;  // elements: the phi^miss table in use (lookahead level) within ws.mtab
  // device-resident loop: candidate rows read the table level the device chose (nullptr: none)
  const int32_t* level_ptr = nullptr;
  int64_t level_stride = 0;
  // device-resident loop: a kernel stamps the device clock around the sweeps (stamp >= 0)
  void* stamp_ctl = nullptr;
  int stamp_end = 0;
};

// Stamps the device clock (%globaltimer, nanoseconds) into the controller: kind 0 opens an
// interval, kind 1 adds it to the lookahead runs' time, kind 2 to the candidate batches'.
__global__ void ctl_stamp(unsigned long long* __restrict__ t, int kind) {
  if (threadIdx.x != 0) return;
  unsigned long long now;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
  if (kind == 0) t[0] = now;
  else t[kind] += now - t[0];
}

// Issues init + L sweeps + column-sum reduction on c.s. ev (optional): two external events
// around each sweep (graph capture).
// rev (directed graphs, MODE_FUSED with one column): the sweeps run on the reverse CSR and fill
// the psi^miss table instead.
gedwalk_status issue_sweeps(GreedyCtx& c, int mode, int cols, bool profile, const std::vector<cudaEvent_t>* ev,
                            bool rev) {
  Graph& g = c.g;
  Workspace& ws = c.ws;
  const bool fp64 = c.r.fp64;
  const int first = mode == MODE_FUSED ? 1 : 0;
  DevBuf& tab = rev ? ws.ztab : ws.mtab;
  const size_t off = rev ? 0 : c.tab_off;  // elements
  const int64_t look_stride = static_cast<int64_t>(c.L + 1) * g.n;  // elements between level tables
  void* m0 = mode == MODE_FUSED ? tab.as<char>() + off * c.es : nullptr;
  if (mode == MODE_LOOK) {
    // cols - 1 lookahead levels: 3 or (FP32) 7 (the shape admits no other)
    const int64_t chunks = static_cast<int64_t>(g.n) * cols * static_cast<int64_t>(c.es) / 16;
    if (fp64)
      launch_look_init<double>(cols, blocks_for(chunks), c.s, ws.mtab.as<double>(), look_stride, ws.x0.as<double>(),
                               c.d_cand, ws.mask.as<uint32_t>(), g.n, g.weighted ? g.rs_d.as<double>() : nullptr);
    else
      launch_look_init<float>(cols, blocks_for(chunks), c.s, ws.mtab.as<float>(), look_stride, ws.x0.as<float>(),
                              c.d_cand, ws.mask.as<uint32_t>(), g.n, g.weighted ? g.rs_f.as<float>() : nullptr);
  } else if (fp64)
    greedy_init<double><<<blocks_for(g.n), 256, 0, c.s>>>(static_cast<double*>(m0), ws.x0.as<double>(), cols, first,
                                                           c.d_cand, ws.mask.as<uint32_t>(), g.n,
                                                           g.weighted ? g.rs_d.as<double>() : nullptr);
  else
    greedy_init<float><<<blocks_for(g.n), 256, 0, c.s>>>(static_cast<float*>(m0), ws.x0.as<float>(), cols, first,
                                                          c.d_cand, ws.mask.as<uint32_t>(), g.n,
                                                          g.weighted ? g.rs_f.as<float>() : nullptr);
  GW_KCHECK();
  SweepArgs a = rev ? base_args_rev(g, ws) : base_args(g, ws);
  a.alpha = c.r.alpha;
  a.cand = c.d_cand;
  void* cur = ws.x0.p;
  void* nxt = ws.x1.p;
  for (int32_t t = 1; t <= c.L; ++t) {
    a.X = cur;
    a.Y = nxt;
    a.accumulate = t > 1;
    char* row = tab.as<char>() + (off + static_cast<size_t>(t) * g.n) * c.es;
    if (mode == MODE_FUSED) a.Mout = row;
    else if (mode == MODE_LOOK) a.Mout = tab.as<char>() + static_cast<size_t>(t) * g.n * c.es;
    else a.Min = row;
    a.mout_stride = look_stride;
    a.level_ptr = c.level_ptr;
    a.level_stride = c.level_stride;
    // external events bracket the whole run of sweeps (event nodes between kernel nodes cost
    // a few microseconds each)
    if (ev && t == 1) GW_CUDA(cudaEventRecordWithFlags((*ev)[0], c.s, cudaEventRecordExternal));
    if (c.stamp_ctl && t == 1) {
      ctl_stamp<<<1, 32, 0, c.s>>>(static_cast<unsigned long long*>(c.stamp_ctl), 0);
      GW_KCHECK();
    }
    GW_TRY(launch_sweep(mode, fp64, cols, a, c.s, profile));
    if (ev && t == c.L) GW_CUDA(cudaEventRecordWithFlags((*ev)[1], c.s, cudaEventRecordExternal));
    if (c.stamp_ctl && t == c.L) {
      ctl_stamp<<<1, 32, 0, c.s>>>(static_cast<unsigned long long*>(c.stamp_ctl), c.stamp_end);
      GW_KCHECK();
    }
    std::swap(cur, nxt);
  }
  const int nsum = sweep_sums(mode, cols);
  if (nsum > 0) GW_TRY(reduce_slots(g, ws, nsum, c.d_gains, c.s, rev));
  return GEDWALK_OK;
}

uint64_t mix_key(uint64_t h, uint64_t v) {
  h ^= v + 0x9e3779b97f4a7c15ULL + (h << 6) + (h >> 2);
  return h;
}

// Runs L sweeps. mode MODE_FUSED (column 0 = phi^miss, table rows written) or MODE_CAND. On a
// capturable stream the sequence is captured once per configuration (on its second use) and
// replayed as a CUDA graph.
gedwalk_status run_sweeps(GreedyCtx& c, int mode, int cols, const std::vector<int32_t>& cand, bool rev = false) {
  Graph& g = c.g;
  Workspace& ws = c.ws;
  const bool fp64 = c.r.fp64;
  int32_t hc[16];
  for (int j = 0; j < 16; ++j) hc[j] = j < static_cast<int>(cand.size()) ? cand[j] : -1;
  GW_CUDA(cudaMemcpyAsync(c.d_cand, hc, sizeof hc, cudaMemcpyHostToDevice, c.s));
  const size_t vbytes = static_cast<size_t>(g.n) * cols * c.es;
  GW_TRY(ws.x0.ensure(vbytes, c.s));
  GW_TRY(ws.x1.ensure(vbytes, c.s));
  GW_TRY(ensure_sweep_scratch(g, ws, cols, fp64, c.s));
  c.sweeps += c.L;
  if (c.s == nullptr || g.plan.num_units == 0) return issue_sweeps(c, mode, cols, true, nullptr, rev);
  uint64_t key = 0;
  for (uint64_t v : {uint64_t(mode), uint64_t(cols), uint64_t(fp64), uint64_t(c.L), uint64_t(g.n), uint64_t(rev),
                     uint64_t(c.tab_off),
                     reinterpret_cast<uint64_t>(ws.ztab.p),
                     reinterpret_cast<uint64_t>(&g), reinterpret_cast<uint64_t>(c.s),
                     reinterpret_cast<uint64_t>(ws.x0.p), reinterpret_cast<uint64_t>(ws.x1.p),
                     reinterpret_cast<uint64_t>(ws.mtab.p), reinterpret_cast<uint64_t>(ws.slots.p),
                     reinterpret_cast<uint64_t>(ws.parts.p), reinterpret_cast<uint64_t>(ws.partial.p),
                     reinterpret_cast<uint64_t>(ws.counters.p), reinterpret_cast<uint64_t>(ws.mask.p),
                     reinterpret_cast<uint64_t>(c.d_cand), reinterpret_cast<uint64_t>(c.d_gains)}) {
    key = mix_key(key, v);
  }
  uint64_t abits;
  memcpy(&abits, &c.r.alpha, 8);
  key = mix_key(key, abits);
  if (key == 0) key = 1;  // 0 marks a free cache entry
  // the workspace's entry for this configuration, else the least recently used one
  SweepGraph* hit = nullptr;
  SweepGraph* lru = &ws.graphs[0];
  for (SweepGraph& e : ws.graphs) {
    if (e.key == key) hit = &e;
    if (e.last_use < lru->last_use) lru = &e;
  }
  if (!hit) {
    lru->reset();
    lru->key = key;
    hit = lru;
  }
  SweepGraph& sg = *hit;
  sg.last_use = ++ws.graph_clock;
  if (!sg.exec) {
    if (sg.uses++ < 1) return issue_sweeps(c, mode, cols, true, nullptr, rev);  // set-up happens outside capture
    sg.ev.assign(2, nullptr);
    for (cudaEvent_t& e : sg.ev) GW_CUDA(cudaEventCreate(&e));
    GW_CUDA(cudaStreamBeginCapture(c.s, cudaStreamCaptureModeThreadLocal));
    set_capturing(true);
    const gedwalk_status st = issue_sweeps(c, mode, cols, false, &sg.ev, rev);
    set_capturing(false);
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(c.s, &graph);
    if (st != GEDWALK_OK || ce != cudaSuccess || !graph) {
      // Nothing captured has run. Another thread can invalidate a capture (a call that waits for
      // the whole device, such as cudaFree); the sequence then runs directly, and a genuine error
      // shows up again there.
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      sg.reset();
      return issue_sweeps(c, mode, cols, true, nullptr, rev);
    }
    const cudaError_t ie = cudaGraphInstantiate(&sg.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
      sg.exec = nullptr;
      sg.reset();
      return fail(GEDWALK_ERR_DEVICE, "graph instantiation failed: %s", cudaGetErrorString(ie));
    }
    sg.kernels = 1 + c.L + (sweep_sums(mode, cols) > 0 ? 2 : 0);
    sg.sweeps = c.L;
    sg.bytes = sweep_bytes(mode, fp64, cols, g.n, g.nnz, g.weighted);
    sg.prof_key = (mode * 1000 + cols) * 2 + (fp64 ? 1 : 0);
  }
  GW_CUDA(cudaGraphLaunch(sg.exec, c.s));
  count_launches(sg.kernels);
  sg.timing_pending = profiling();
  return GEDWALK_OK;
}

// After a synchronisation: hands the sweep timings of graph replays to the profiler.
void read_graph_timing(Workspace& ws) {
  for (SweepGraph& sg : ws.graphs) {
    if (!sg.timing_pending) continue;
    sg.timing_pending = false;
    float ms = 0.0f;  // the run of sweeps, shared evenly among them
    if (sg.ev.size() == 2 && cudaEventElapsedTime(&ms, sg.ev[0], sg.ev[1]) == cudaSuccess) {
      for (int t = 0; t < sg.sweeps; ++t) profile_add(ms / sg.sweeps, sg.bytes, sg.prof_key);
    } else {
      cudaGetLastError();
    }
  }
}

// The stream a greedy run uses: the caller's, or (for the legacy default stream, which cannot
// be captured) the workspace's own stream, ordered after the caller's.
gedwalk_status greedy_stream(Workspace& ws, cudaStream_t caller, cudaStream_t* out) {
  if (caller != nullptr) {
    *out = caller;
    return GEDWALK_OK;
  }
  if (!ws.own_stream) GW_CUDA(cudaStreamCreateWithFlags(&ws.own_stream, cudaStreamNonBlocking));
  if (!ws.order_ev) GW_CUDA(cudaEventCreateWithFlags(&ws.order_ev, cudaEventDisableTiming));
  GW_CUDA(cudaEventRecord(ws.order_ev, caller));
  GW_CUDA(cudaStreamWaitEvent(ws.own_stream, ws.order_ev, 0));
  *out = ws.own_stream;
  return GEDWALK_OK;
}

// ---------------------------------------------------------------- device-resident greedy loop
// The plain greedy with lookahead runs as one CUDA graph: an outer WHILE node over the k steps; in
// each, a controller kernel either takes the next lookahead level (its table and its candidate's
// exact gain are already there) or starts a new run (IF node: the L lookahead sweeps), then an
// inner WHILE node repeats bound pass -> merge -> certification, with a candidate batch (IF node)
// whenever the best exact value does not beat every unevaluated bound. The decisions the host loop
// takes (certification, the next candidates, the speculative guesses, the lookahead level) are
// taken by single-thread kernels on the same data, in the same order and with the same ties, so
// the picks and gains are those of the host loop. A step that needs more than `max_batches`
// candidate batches stops the loop with an error flag instead of running on.
constexpr int kMaxEval = 64;  // exact values one step keeps (the largest, if more)

struct DevCtl {
  int32_t step, k, levels, L;
  int32_t look_lvl, tab_level;  // the level the next step may take; the table this step reads
  int32_t run_look, looping, run_cand, n_last;
  int32_t first_batch, guessed, e_n, spec_n;
  int32_t iso_next, batches_step, err, cols_cand;
  int32_t look_c[8];
  int32_t spec_v[8];
  int32_t e_v[kMaxEval];
  double look_g[8];
  double spec_g[8];
  double e_g[kMaxEval];
  long long evals, batches, spec_miss, runs, cand_batches, iters;
  unsigned long long t[3];  // device clock: interval start, lookahead-run sweeps, candidate-batch sweeps
};

__device__ __forceinline__ bool dev_in(const uint32_t* mask, int32_t v) { return (mask[v >> 5] >> (v & 31)) & 1u; }

// Opens a step: the next lookahead level, or a new run whose guesses are the best remaining values
// (at the first step without any, the highest-degree vertices outside S).
__global__ void ctl_begin(DevCtl* __restrict__ c, Stale* __restrict__ stale, const uint32_t* __restrict__ mask,
                          int32_t n, int32_t* __restrict__ cand, cudaGraphConditionalHandle h_run,
                          cudaGraphConditionalHandle h_loop) {
  if (threadIdx.x != 0) return;
  c->e_n = 0;
  c->first_batch = 1;
  c->guessed = 0;
  c->batches_step = 0;
  c->n_last = 0;
  c->looping = 1;
  const int lvl = c->look_lvl;
  if (lvl > 0 && lvl < c->levels && c->look_c[lvl] >= 0) {
    const int32_t v = c->look_c[lvl];
    c->tab_level = lvl;
    Stale st;
    st.ub = __double2float_ru(c->look_g[lvl]);
    st.step = c->step;
    stale[v] = st;
    c->e_v[0] = v;
    c->e_g[0] = c->look_g[lvl];
    c->e_n = 1;
    c->guessed = 1;
    c->run_look = 0;
  } else {
    int m = 0;
    for (int j = 0; j < c->spec_n && m < c->levels; ++j) cand[m++] = c->spec_v[j];
    if (m == 0 && c->step == 0)
      for (int32_t v = 0; v < n && m < c->levels; ++v)
        if (!dev_in(mask, v)) cand[m++] = v;
    for (int j = m; j < 16; ++j) cand[j] = -1;
    for (int j = 0; j < c->levels; ++j) c->look_c[j] = cand[j];
    c->look_lvl = 0;
    c->tab_level = 0;
    c->guessed = m > 0;
    c->n_last = m > 0 ? 1 : 0;  // level 0's guess has its exact gain once the run is done
    c->evals += m;
    c->batches += m > 0;
    c->runs += 1;
    c->run_look = 1;
  }
  cudaGraphSetConditional(h_run, c->run_look ? 1u : 0u);
  cudaGraphSetConditional(h_loop, 1u);
}

// After a run: the exact gains of every level's guess (each under S + the earlier guesses).
__global__ void ctl_after_run(DevCtl* __restrict__ c, const double* __restrict__ gains) {
  if (threadIdx.x < c->levels) c->look_g[threadIdx.x] = gains[threadIdx.x];
}

// Records the exact gains of the last evaluated candidates (as the stale bounds of this step and
// in the step's list of exact values, which keeps the kMaxEval largest).
__global__ void ctl_record(DevCtl* __restrict__ c, Stale* __restrict__ stale, const int32_t* __restrict__ cand,
                           const double* __restrict__ gains, const int32_t* __restrict__ perm) {
  if (threadIdx.x != 0) return;
  for (int j = 0; j < c->n_last; ++j) {
    const int32_t v = cand[j];
    if (v < 0) continue;
    Stale st;
    st.ub = __double2float_ru(gains[j]);
    st.step = c->step;
    stale[v] = st;
    if (c->e_n < kMaxEval) {
      c->e_v[c->e_n] = v;
      c->e_g[c->e_n] = gains[j];
      ++c->e_n;
    } else {  // replace the smallest exact value (never the best: certification needs only that)
      int w = 0;
      for (int i = 1; i < kMaxEval; ++i)
        if (c->e_g[i] < c->e_g[w] || (c->e_g[i] == c->e_g[w] && perm[c->e_v[i]] > perm[c->e_v[w]])) w = i;
      if (gains[j] > c->e_g[w]) {
        c->e_v[w] = v;
        c->e_g[w] = gains[j];
      }
    }
  }
  c->n_last = 0;
}

__device__ __forceinline__ bool cand_first(double ga, int32_t ca, double gb, int32_t cb) {
  return ga > gb || (ga == gb && ca < cb);
}

// Certification after a bound pass: the best exact value wins once it beats every unevaluated
// bound (inflated by tol); then the step's outputs, the vertex joins S, the next step's guesses and
// lookahead level are set. Otherwise the best-bounded unevaluated vertices become a candidate batch.
__global__ void ctl_certify(DevCtl* __restrict__ c, const SelOut* __restrict__ sel, uint32_t* __restrict__ mask,
                            const int32_t* __restrict__ perm, int32_t n, int32_t* __restrict__ cand,
                            int32_t* __restrict__ out_group, double* __restrict__ out_gains, double tol,
                            int32_t max_batches, cudaGraphConditionalHandle h_loop,
                            cudaGraphConditionalHandle h_cand) {
  if (threadIdx.x != 0) return;
  ++c->iters;
  // the zero-gain candidate: the bound pass's, or the smallest isolated row outside S
  unsigned long long z = sel->zero_min;
  while (c->iso_next < n && dev_in(mask, c->iso_next)) ++c->iso_next;
  if (c->iso_next < n) {
    const unsigned long long iso =
        (static_cast<unsigned long long>(perm[c->iso_next]) << 32) | static_cast<uint32_t>(c->iso_next);
    if (iso < z) z = iso;
  }
  // the best exact value (larger gain first, then the lower caller id)
  int32_t bv = -1, bc = INT_MAX;
  double bg = -1.0;
  for (int j = 0; j < c->e_n; ++j) {
    const int32_t cc = perm[c->e_v[j]];
    if (bv < 0 || cand_first(c->e_g[j], cc, bg, bc)) {
      bv = c->e_v[j];
      bc = cc;
      bg = c->e_g[j];
    }
  }
  if (z != kNoZero && (bv < 0 || cand_first(0.0, zero_caller(z), bg, bc))) {
    bv = zero_internal(z);
    bc = zero_caller(z);
    bg = 0.0;
  }
  const bool top_empty = sel->id[0] == INT_MAX;
  const double ub0 = top_empty ? -1.0 : static_cast<double>(sel->val[0]) * (1.0 + tol);
  const bool certified = top_empty || (bv >= 0 && ub0 < bg);
  if (certified) {
    if (bv < 0) {  // no vertex left to add
      c->err = 2;
      c->looping = 0;
      c->run_cand = 0;
    } else {
      out_group[c->step] = bc;
      out_gains[c->step] = bg;
      mask[bv >> 5] |= 1u << (bv & 31);
      // the next run's guesses: the best remaining values, exact or bounds, positive only
      int32_t pv[kMaxEval + kTopK];
      double pg[kMaxEval + kTopK];
      int np = 0;
      for (int j = 0; j < c->e_n; ++j)
        if (c->e_v[j] != bv) {
          pv[np] = c->e_v[j];
          pg[np++] = c->e_g[j];
        }
      for (int j = 0; j < kTopK; ++j)
        if (sel->id[j] != INT_MAX && sel->id[j] != bv) {
          pv[np] = sel->id[j];
          pg[np++] = static_cast<double>(sel->val[j]);
        }
      int ns = 0;
      while (ns < c->levels) {
        int w = -1;
        for (int j = 0; j < np; ++j) {
          if (pv[j] < 0 || !(pg[j] > 0.0)) continue;
          if (w < 0 || cand_first(pg[j], perm[pv[j]], pg[w], perm[pv[w]])) w = j;
        }
        if (w < 0) break;
        c->spec_v[ns] = pv[w];
        c->spec_g[ns++] = pg[w];
        pv[w] = -1;
      }
      c->spec_n = ns;
      const int lvl = c->look_lvl;
      if (lvl >= 0 && bv == c->look_c[lvl] && lvl + 1 < c->levels && c->look_c[lvl + 1] >= 0) c->look_lvl = lvl + 1;
      else c->look_lvl = -1;
      ++c->step;
      c->looping = 0;
      c->run_cand = 0;
    }
  } else {
    if (c->first_batch && c->guessed) ++c->spec_miss;
    c->first_batch = 0;
    int m = 0;
    for (int j = 0; j < kTopK && m < c->cols_cand; ++j)
      if (sel->id[j] != INT_MAX) cand[m++] = sel->id[j];
    for (int j = m; j < 16; ++j) cand[j] = -1;
    c->n_last = m;
    c->evals += m;
    c->batches += 1;
    c->cand_batches += 1;
    if (++c->batches_step > max_batches) {
      c->err = 1;
      c->looping = 0;
      c->run_cand = 0;
    } else {
      c->looping = 1;
      c->run_cand = 1;
    }
  }
  cudaGraphSetConditional(h_loop, c->looping ? 1u : 0u);
  cudaGraphSetConditional(h_cand, c->run_cand ? 1u : 0u);
}

__global__ void ctl_end(const DevCtl* __restrict__ c, cudaGraphConditionalHandle h_step) {
  if (threadIdx.x == 0) cudaGraphSetConditional(h_step, (c->step < c->k && c->err == 0) ? 1u : 0u);
}

// Adds a conditional node (IF or WHILE, one body) at the current point of a capture on s.
gedwalk_status add_conditional(cudaStream_t s, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type,
                               cudaGraph_t* body) {
  cudaStreamCaptureStatus st;
  cudaGraph_t graph = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  GW_CUDA(cudaStreamGetCaptureInfo(s, &st, nullptr, &graph, &deps, nullptr, &nd));
  if (st != cudaStreamCaptureStatusActive) return fail(GEDWALK_ERR_DEVICE, "stream is not capturing");
  cudaGraphNodeParams p{};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = h;
  p.conditional.type = type;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  GW_CUDA(cudaGraphAddNode(&node, graph, deps, nullptr, nd, &p));
  GW_CUDA(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  *body = p.conditional.phGraph_out[0];
  return GEDWALK_OK;
}

// Captures `fill` into `graph` on s (BeginCaptureToGraph); the capture ends whatever fill returns.
template <class F>
gedwalk_status capture_into(cudaStream_t s, cudaGraph_t graph, F&& fill) {
  GW_CUDA(cudaStreamBeginCaptureToGraph(s, graph, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  set_capturing(true);
  const gedwalk_status st = fill();
  set_capturing(false);
  cudaGraph_t out = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(s, &out);
  if (st != GEDWALK_OK) {
    cudaGetLastError();
    return st;
  }
  if (ce != cudaSuccess) return fail(GEDWALK_ERR_DEVICE, "capture of the greedy loop failed: %s", cudaGetErrorString(ce));
  return GEDWALK_OK;
}

}  // namespace

gedwalk_status greedy_shape(const Graph& g, const Resolved& r, int32_t flags, GreedyShape* out) {
  GreedyShape sh{};
  const bool adaptive = (flags & GEDWALK_ADAPTIVE_L) != 0;
  // phi^miss + speculative candidates. Every gather costs one L2 sector whatever the row width,
  // so narrow rows are cheapest; one speculative candidate certifies most steps (a miss costs one
  // extra candidate batch). The adaptive variant certifies the best two exact gains (u and v of
  // its separation test), so it speculates on three candidates.
  sh.cols_fused = adaptive ? 4 : 2;
  if (r.spec_cols != 0) {
    if (!(r.spec_cols == 2 || r.spec_cols == 4 || (r.spec_cols == 8 && !r.fp64)))
      return fail(GEDWALK_ERR_INVALID, "spec_cols must be 0, 2, 4 or (FP32) 8");
    sh.cols_fused = r.spec_cols;
  }
  // Lookahead (plain greedy on an undirected graph): one run of sweeps carries `levels` steps,
  // level d under S + {c_1..c_d} with the guessed winners c_d; a step whose winner was guessed
  // needs no sweep of its own. The run's rows hold levels + 1 columns (phi^miss under S and one
  // column per guess; every level's phi^miss is a difference of them). A gather costs one L2
  // sector request whatever the row width up to 32 bytes, so 7 FP32 levels (3 FP64) cost little
  // more per sweep than one.
  sh.levels = 1;
  if (!(flags & (GEDWALK_ADAPTIVE_L | GEDWALK_STOCHASTIC | GEDWALK_GAINS_ALL)) && !g.directed) {
    sh.levels = r.fp64 ? 3 : 7;
    if (r.lookahead != 0) {
      if (!(r.lookahead == 1 || r.lookahead == 3 || (!r.fp64 && r.lookahead == 7)))
        return fail(GEDWALK_ERR_INVALID, "lookahead must be 0, 1, 3 or (FP32) 7");
      sh.levels = r.lookahead;
    }
  }
  // Candidate batches run when the evaluated guess is not certified; the winner is nearly always
  // among the best few bounds, and a narrower batch is a cheaper sweep.
  sh.cols_cand = 4;
  sh.cols_all = r.fp64 ? 8 : 16;
  sh.ell_max = 1;
  while (adaptive && sh.ell_max < r.L) sh.ell_max *= 2;
  sh.tab_L = adaptive ? sh.ell_max : r.L;
  sh.cols_max = std::max({sh.levels > 1 ? sh.levels + 1 : sh.cols_fused, sh.cols_cand,
                          (flags & GEDWALK_GAINS_ALL) ? sh.cols_all : 0, 2});
  *out = sh;
  return GEDWALK_OK;
}

namespace {
// GEDWALK_DEVICE_LOOP: the plain greedy with lookahead runs its k steps as one CUDA graph.
bool uses_device_loop(const Graph& g, const GreedyShape& sh, int32_t flags, int32_t k) {
  return (flags & GEDWALK_DEVICE_LOOP) && sh.levels > 1 &&
         (flags & (GEDWALK_GAINS_ALL | GEDWALK_STOCHASTIC | GEDWALK_ADAPTIVE_L)) == 0 && !g.directed && k > 0 &&
         g.plan.num_units > 0;
}
// Its controller block: the state, then the group and the gains of up to kcap steps.
int32_t loop_kcap(int32_t k) {
  int32_t kcap = 64;
  while (kcap < k) kcap *= 2;
  return kcap;
}
size_t loop_ctl_bytes(int32_t k) {
  return (sizeof(DevCtl) + 255) / 256 * 256 + static_cast<size_t>(loop_kcap(k)) * (sizeof(double) + sizeof(int32_t)) +
         256;
}
}  // namespace

int64_t maximize_footprint(const Graph& g, const Resolved& r, int32_t flags, int32_t k) {
  GreedyShape sh{};
  if (greedy_shape(g, r, flags, &sh) != GEDWALK_OK) return 0;
  const int64_t n = g.n, es = r.fp64 ? 8 : 4;
  const int64_t slices = std::max(std::max(g.plan.num_slices, g.directed ? g.plan_r.num_slices : 0), 1);
  const int64_t heavy = std::max(std::max(g.plan.num_heavy, g.directed ? g.plan_r.num_heavy : 0), 1);
  const int64_t slots = std::max(std::max(g.plan.num_slots, g.directed ? g.plan_r.num_slots : 0), 1);
  int64_t b = 0;
  b += static_cast<int64_t>(sh.tab_L + 1) * n * es * sh.levels;  // phi^miss tables
  if (g.directed) b += static_cast<int64_t>(sh.tab_L + 1) * n * es;  // psi^miss table
  b += 2 * n * sh.cols_max * es;                                    // walk vectors x0, x1
  b += slices * sh.cols_max * es + heavy * 4 + slots * sh.cols_max * 8 + sh.cols_max * kReduceParts * 8;
  b += (n + 31) / 32 * 4;                                           // S bitmask
  b += n * static_cast<int64_t>(sizeof(Stale)) + static_cast<int64_t>(kSelBlocks) * kTopK * 8;
  b += static_cast<int64_t>(sizeof(SelOut)) + 16 * 4 + 16 * 8 + 256;
  if (uses_device_loop(g, sh, flags, k)) b += static_cast<int64_t>(loop_ctl_bytes(k));
  return b;
}

namespace {

uint64_t mix_all(std::initializer_list<uint64_t> vs) {
  uint64_t key = 0;
  for (uint64_t v : vs) key ^= v + 0x9e3779b97f4a7c15ULL + (key << 6) + (key >> 2);
  return key;
}

// Runs the k steps of the plain greedy with lookahead as one CUDA graph launch (the loop's graph is
// built once per configuration of the workspace) and reads back the group and the gains.
gedwalk_status run_device_loop(GreedyCtx& c, int32_t k, int levels, int cols_cand, int cols_max, size_t tab_elems,
                               int nb_sel, int32_t n_scan, double tol, Stale* stale, float* sel_v, int* sel_id,
                               int32_t* group, double* gains, bool* launched) {
  *launched = false;
  Graph& g = c.g;
  Workspace& ws = c.ws;
  const cudaStream_t s = c.s;
  const bool fp64 = c.r.fp64;
  const int32_t L = c.L;
  // controller state, then the outputs for up to kcap steps
  const int32_t kcap = loop_kcap(k);
  const size_t ctl_bytes = (sizeof(DevCtl) + 255) / 256 * 256;
  GW_TRY(ws.ctl.ensure(loop_ctl_bytes(k), s));
  char* base = ws.ctl.as<char>();
  DevCtl* dctl = reinterpret_cast<DevCtl*>(base);
  double* d_ogains = reinterpret_cast<double*>(base + ctl_bytes);
  int32_t* d_ogroup = reinterpret_cast<int32_t*>(d_ogains + kcap);
  const int32_t* d_level = reinterpret_cast<const int32_t*>(base + offsetof(DevCtl, tab_level));
  const int32_t* d_step = reinterpret_cast<const int32_t*>(base + offsetof(DevCtl, step));
  void* d_stamp = base + offsetof(DevCtl, t);
  // buffers the captured sweeps use, sized before the capture
  const size_t es = fp64 ? 8 : 4;
  GW_TRY(ws.x0.ensure(static_cast<size_t>(g.n) * cols_max * es, s));
  GW_TRY(ws.x1.ensure(static_cast<size_t>(g.n) * cols_max * es, s));
  GW_TRY(ensure_sweep_scratch(g, ws, cols_max, fp64, s));
  GW_TRY(configure_sweep(MODE_LOOK, fp64, levels + 1));
  GW_TRY(configure_sweep(MODE_CAND, fp64, cols_cand));
  DevCtl h{};
  h.k = k;
  h.levels = levels;
  h.L = L;
  h.look_lvl = -1;
  h.iso_next = n_scan;
  h.cols_cand = cols_cand;
  for (int j = 0; j < 8; ++j) h.look_c[j] = -1;
  GW_CUDA(cudaMemcpyAsync(dctl, &h, sizeof h, cudaMemcpyHostToDevice, s));
  const int32_t max_batches = n_scan / std::max(cols_cand, 1) + 64;
  uint64_t abits;
  memcpy(&abits, &c.r.alpha, 8);
  uint64_t tbits;
  memcpy(&tbits, &tol, 8);
  const uint64_t key = mix_all(
      {uint64_t(levels), uint64_t(cols_cand), uint64_t(fp64), uint64_t(L), uint64_t(g.n), uint64_t(kcap),
       uint64_t(nb_sel), uint64_t(n_scan), abits, tbits, reinterpret_cast<uint64_t>(&g), reinterpret_cast<uint64_t>(s),
       reinterpret_cast<uint64_t>(ws.x0.p), reinterpret_cast<uint64_t>(ws.x1.p), reinterpret_cast<uint64_t>(ws.mtab.p),
       reinterpret_cast<uint64_t>(ws.slots.p), reinterpret_cast<uint64_t>(ws.parts.p),
       reinterpret_cast<uint64_t>(ws.partial.p), reinterpret_cast<uint64_t>(ws.counters.p),
       reinterpret_cast<uint64_t>(ws.mask.p), reinterpret_cast<uint64_t>(ws.stale.p),
       reinterpret_cast<uint64_t>(ws.sel.p), reinterpret_cast<uint64_t>(ws.small.p),
       reinterpret_cast<uint64_t>(ws.ctl.p)});
  SweepGraph& sg = ws.greedy_loop;
  if (sg.key != key || !sg.exec) {
    sg.reset();
    cudaGraph_t root = nullptr;
    GW_CUDA(cudaGraphCreate(&root, 0));
    struct Owner {
      cudaGraph_t g;
      ~Owner() {
        if (g) cudaGraphDestroy(g);
      }
    } owner{root};
    cudaGraphConditionalHandle h_step, h_run, h_loop, h_cand;
    GW_CUDA(cudaGraphConditionalHandleCreate(&h_step, root, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams p{};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h_step;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t n_step;
    GW_CUDA(cudaGraphAddNode(&n_step, root, nullptr, nullptr, 0, &p));
    cudaGraph_t body_step = p.conditional.phGraph_out[0];
    GW_CUDA(cudaGraphConditionalHandleCreate(&h_run, body_step, 0, 0));
    GW_CUDA(cudaGraphConditionalHandleCreate(&h_loop, body_step, 0, 0));
    cudaGraph_t body_run = nullptr, body_loop = nullptr, body_cand = nullptr;
    uint32_t* mask = ws.mask.as<uint32_t>();
    const int32_t* perm = g.perm_d.as<int32_t>();
    // step: open (level or run), the run, the certification loop, close
    GW_TRY(capture_into(s, body_step, [&]() -> gedwalk_status {
      ctl_begin<<<1, 32, 0, s>>>(dctl, stale, mask, g.n, c.d_cand, h_run, h_loop);
      GW_CUDA(cudaGetLastError());
      GW_TRY(add_conditional(s, h_run, cudaGraphCondTypeIf, &body_run));
      GW_TRY(add_conditional(s, h_loop, cudaGraphCondTypeWhile, &body_loop));
      ctl_end<<<1, 32, 0, s>>>(dctl, h_step);
      GW_CUDA(cudaGetLastError());
      return GEDWALK_OK;
    }));
    // the lookahead run: init, L sweeps (device-clock stamps around them), column sums, the gains
    GW_TRY(capture_into(s, body_run, [&]() -> gedwalk_status {
      c.tab_off = 0;
      c.stamp_ctl = d_stamp;
      c.stamp_end = 1;
      const gedwalk_status st = issue_sweeps(c, MODE_LOOK, levels + 1, false, nullptr, false);
      c.stamp_ctl = nullptr;
      GW_TRY(st);
      ctl_after_run<<<1, 32, 0, s>>>(dctl, c.d_gains);
      GW_CUDA(cudaGetLastError());
      return GEDWALK_OK;
    }));
    // one certification round: record the last gains, bound pass, merge, certify, maybe a batch
    GW_CUDA(cudaGraphConditionalHandleCreate(&h_cand, body_loop, 0, 0));
    GW_TRY(capture_into(s, body_loop, [&]() -> gedwalk_status {
      ctl_record<<<1, 32, 0, s>>>(dctl, stale, c.d_cand, c.d_gains, perm);
      GW_CUDA(cudaGetLastError());
      reset_selection<<<1, 1, 0, s>>>(c.d_out);
      GW_CUDA(cudaGetLastError());
      const Sampling all{~0ull, 0, 0};
      if (fp64)
        GW_CUDA(launch_ub_select<double>(nb_sel, s, ws.mtab.as<double>(), ws.mtab.as<double>(), L, g.n, n_scan, mask,
                                         stale, 0, perm, sel_v, sel_id, c.d_out, all, d_level,
                                         static_cast<int64_t>(tab_elems), d_step));
      else
        GW_CUDA(launch_ub_select<float>(nb_sel, s, ws.mtab.as<float>(), ws.mtab.as<float>(), L, g.n, n_scan, mask,
                                        stale, 0, perm, sel_v, sel_id, c.d_out, all, d_level,
                                        static_cast<int64_t>(tab_elems), d_step));
      ctl_certify<<<1, 32, 0, s>>>(dctl, c.d_out, mask, perm, g.n, c.d_cand, d_ogroup, d_ogains, tol, max_batches,
                                   h_loop, h_cand);
      GW_CUDA(cudaGetLastError());
      return add_conditional(s, h_cand, cudaGraphCondTypeIf, &body_cand);
    }));
    // the candidate batch: candidate rows read the table of the step's level
    GW_TRY(capture_into(s, body_cand, [&]() -> gedwalk_status {
      c.tab_off = 0;
      c.level_ptr = d_level;
      c.level_stride = static_cast<int64_t>(tab_elems);
      c.stamp_ctl = d_stamp;
      c.stamp_end = 2;
      const gedwalk_status st = issue_sweeps(c, MODE_CAND, cols_cand, false, nullptr, false);
      c.stamp_ctl = nullptr;
      c.level_ptr = nullptr;
      c.level_stride = 0;
      return st;
    }));
    GW_CUDA(cudaGraphInstantiate(&sg.exec, root, 0));
    sg.key = key;
  }
  *launched = true;
  GW_CUDA(cudaGraphLaunch(sg.exec, s));
  DevCtl out{};
  std::vector<double> og(k);
  std::vector<int32_t> ogr(k);
  GW_CUDA(cudaMemcpyAsync(&out, dctl, sizeof out, cudaMemcpyDeviceToHost, s));
  GW_CUDA(cudaMemcpyAsync(og.data(), d_ogains, sizeof(double) * k, cudaMemcpyDeviceToHost, s));
  GW_CUDA(cudaMemcpyAsync(ogr.data(), d_ogroup, sizeof(int32_t) * k, cudaMemcpyDeviceToHost, s));
  GW_CUDA(cudaStreamSynchronize(s));
  if (out.err == 2) return fail(GEDWALK_ERR_INVALID, "no vertex left to add");
  if (out.err != 0 || out.step != k)
    return fail(GEDWALK_ERR_DEVICE, "the greedy loop stopped at step %d of %d (certification exceeded %d batches)",
                out.step, k, max_batches);
  for (int32_t j = 0; j < k; ++j) {
    group[j] = ogr[j];
    if (gains) gains[j] = og[j];
  }
  ws.st_evals = out.evals;
  ws.st_batches = out.batches;
  ws.st_spec_miss = out.spec_miss;
  ws.st_sweeps = (out.runs + out.cand_batches) * L;
  ws.st_ell.assign(k, L);
  // launches the graph ran: per step open/close, per run init + L sweeps + 2 stamps + 2 reduce +
  // after_run, per certification round 4 kernels, per batch init + L sweeps + 2 stamps + 2 reduce
  count_launches(static_cast<int>(2 * k + out.runs * (L + 6) + out.iters * 4 + out.cand_batches * (L + 5)));
  if (profiling()) {  // the sweeps' device time, from the device-clock stamps around each run / batch
    const double b_look = sweep_bytes(MODE_LOOK, fp64, levels + 1, g.n, g.nnz, g.weighted);
    const double b_cand = sweep_bytes(MODE_CAND, fp64, cols_cand, g.n, g.nnz, g.weighted);
    const int64_t n_look = out.runs * L, n_cand = out.cand_batches * L;
    for (int64_t i = 0; i < n_look; ++i)
      profile_add(static_cast<double>(out.t[1]) / 1e6 / n_look, b_look, (MODE_LOOK * 1000 + levels + 1) * 2 + fp64);
    for (int64_t i = 0; i < n_cand; ++i)
      profile_add(static_cast<double>(out.t[2]) / 1e6 / n_cand, b_cand, (MODE_CAND * 1000 + cols_cand) * 2 + fp64);
  }
  return GEDWALK_OK;
}

}  // namespace

namespace {
// Waits for a stream when a call leaves early with an error, so that nothing it launched still
// runs when its buffers are reused or freed.
struct SyncOnError {
  cudaStream_t s = nullptr;
  bool ok = false;
  ~SyncOnError() {
    if (!ok && s) {
      cudaStreamSynchronize(s);
      cudaGetLastError();
    }
  }
};
}  // namespace

gedwalk_status maximize_impl(Graph& g, Workspace& ws, int32_t k, const Resolved& r_in, int32_t flags,
                             const std::vector<int32_t>& init_int, int32_t* group, double* gains, double* score) {
  Resolved r = r_in;
  GW_TRY(greedy_stream(ws, r_in.stream, &r.stream));
  SyncOnError guard{r.stream};
  cudaStream_t s = r.stream;
  const size_t es = r.fp64 ? 8 : 4;
  const bool adaptive = (flags & GEDWALK_ADAPTIVE_L) != 0;
  GreedyShape shape{};
  GW_TRY(greedy_shape(g, r, flags, &shape));
  const int cols_fused = shape.cols_fused;
  const int levels = shape.levels;
  const bool look = levels > 1;
  const int n_spec = look ? levels : cols_fused - 1;
  const int cols_cand = shape.cols_cand;
  const int cols_all = shape.cols_all;
  const double tol = r.fp64 ? 1e-11 : 1e-5;  // relative inflation of bounds against rounding
  const bool gains_all = (flags & GEDWALK_GAINS_ALL) != 0;
  const bool stochastic = (flags & GEDWALK_STOCHASTIC) != 0;
  if (stochastic && (gains_all || !init_int.empty()))
    return fail(GEDWALK_ERR_INVALID, "stochastic greedy cannot be combined with GEDWALK_GAINS_ALL or an init group");
  if (stochastic && !(r.eta > 0.0 && r.eta < 1.0)) return fail(GEDWALK_ERR_INVALID, "eta must lie in (0, 1)");
  if (adaptive && (gains_all || stochastic || !init_int.empty()))
    return fail(GEDWALK_ERR_INVALID,
                "GEDWALK_ADAPTIVE_L cannot be combined with GEDWALK_GAINS_ALL, GEDWALK_STOCHASTIC or an init group");
  if (adaptive && !(r.eps > 0.0)) return fail(GEDWALK_ERR_INVALID, "GEDWALK_ADAPTIVE_L needs epsilon (L must be 0)");
  // stochastic greedy: about m vertices outside S are sampled per step (Appendix D)
  const double sample_m = std::ceil(static_cast<double>(g.n) / std::max(k, 1) * std::log(1.0 / (stochastic ? r.eta : 0.5)));
  // adaptive: l runs through the powers of two from 1; B_l < eps_sep separates any pair, and r.L
  // (the first l with B_l < eps_sep) bounds the largest power reached.
  const double eps_sep = r.eps;
  const int32_t ell_max = shape.ell_max;
  const int32_t L = shape.tab_L;  // rows of the miss table
  double coef = 0.0;  // B_l = coef * Wa_l (Eq. comb-bound, or Lemma spectral-bound)
  std::vector<double> Wa;  // the walk totals this run needs, copied under the table's lock
  if (adaptive) {
    GW_TRY(bound_coef(g, r.alpha, r.bound_kind, s, &coef));
    GW_TRY(ensure_totals(g, r.alpha, ell_max + 1, s));
    std::shared_lock<std::shared_mutex> rl(g.tt_lock);
    if (g.tt_alpha != r.alpha || g.tt_rows < ell_max + 1)
      return fail(GEDWALK_ERR_INVALID, "the walk-total table was replaced for another alpha during the call");
    Wa.assign(g.Wa.begin(), g.Wa.begin() + ell_max + 1);
  }
  auto bound_at = [&](int32_t l) { return coef * Wa[l]; };
  ws.st_evals = ws.st_batches = ws.st_sweeps = ws.st_spec_miss = ws.st_sep_fail = 0;
  ws.st_ell.clear();

  const size_t tab_elems = static_cast<size_t>(L + 1) * g.n;  // one phi^miss table
  GW_TRY(ws.mtab.ensure(tab_elems * levels * es, s));
  for (int d = 0; d < levels; ++d) GW_TRY(zero_isolated_tail(g, ws.mtab.as<char>() + d * tab_elems * es, es, L, s));
  if (g.directed) {
    GW_TRY(ws.ztab.ensure(static_cast<size_t>(L + 1) * g.n * es, s));
    GW_TRY(zero_isolated_tail(g, ws.ztab.p, es, L, s));
  }
  GW_TRY(ws.stale.ensure(static_cast<size_t>(g.n) * sizeof(Stale), s));
  GW_TRY(ws.sel.ensure(static_cast<size_t>(kSelBlocks) * kTopK * 8, s));
  GW_TRY(ws.small.ensure(sizeof(SelOut) + 16 * sizeof(int32_t) + 16 * sizeof(double) + 256, s));
  GW_TRY(ws.ensure_pinned(sizeof(SelOut) + 64 + 8 * sizeof(double)));
  double* h_look = reinterpret_cast<double*>(static_cast<char*>(ws.pinned) + sizeof(SelOut) + 64);
  GW_TRY(upload_mask(g, ws, init_int, s));
  GW_CUDA(cudaMemsetAsync(ws.stale.p, 0xff, static_cast<size_t>(g.n) * sizeof(Stale), s));  // step -1, ub NaN

  GreedyCtx c{g, ws, r, s, adaptive ? 1 : r.L, es};
  const int need = adaptive ? 2 : 1;
  c.d_out = ws.small.as<SelOut>();
  c.d_cand = reinterpret_cast<int32_t*>(c.d_out + 1);
  c.d_gains = reinterpret_cast<double*>(c.d_cand + 16);
  c.h_out = static_cast<SelOut*>(ws.pinned);
  float* sel_v = ws.sel.as<float>();
  int* sel_id = reinterpret_cast<int*>(sel_v + kSelBlocks * kTopK);
  Stale* stale = ws.stale.as<Stale>();

  std::vector<uint32_t> hmask((static_cast<size_t>(g.n) + 31) / 32, 0u);
  std::vector<char> inS(g.n, 0);
  for (int32_t v : init_int) {
    hmask[v >> 5] |= 1u << (v & 31);
    inS[v] = 1;
  }
  std::vector<int32_t> S_all = init_int;
  std::vector<Cand> spec;  // next step's speculative candidates (internal ids)
  int look_lvl = -1;                  // lookahead level of the next step (-1: none valid)
  std::vector<int32_t> look_c;        // guessed winners c_1..c_levels of the last lookahead run
  double look_g[8] = {0};             // their exact gains, each under S + {c_1..c_d}
  // The step's sample: vertex v (caller id) is drawn when hash(seed, step, v) < thr, i.e. with
  // probability p = m / |V \ S| (all of V \ S when p >= 1).
  auto sampling_for = [&](int32_t st) {
    Sampling smp{~0ull, r.seed, static_cast<uint32_t>(st)};
    if (stochastic) {
      const double p = sample_m / static_cast<double>(g.n - st);
      const double scaled = p * 18446744073709551616.0;
      if (p < 1.0 && scaled < 18446744073709551615.0) smp.thr = static_cast<uint64_t>(scaled);
    }
    return smp;
  };
  // Isolated vertices (rows [n_active, n)) start and end no walk: their bound and gain are exactly
  // 0. The bound pass skips them, and the smallest caller id among those outside S stands for
  // them among the zero gains. Stochastic greedy scans them all: they belong to its samples.
  // The relabelling is a stable sort by degree, so the isolated rows hold increasing caller ids.
  const int32_t n_scan = stochastic ? g.n : g.n_active;
  int32_t iso_next = stochastic ? g.n : g.n_active;  // first isolated row not in S
  const int nb_sel = sel_blocks(n_scan);
  // One bound + selection pass into c.d_out / c.h_out; `step` decides which stale gains are exact.
  auto select_pass = [&](int32_t st, const Sampling& smp) -> gedwalk_status {
    reset_selection<<<1, 1, 0, s>>>(c.d_out);
    GW_KCHECK();
    if (r.fp64)
      GW_CUDA(launch_ub_select<double>(nb_sel, s, ws.mtab.as<double>() + c.tab_off,
                                       g.directed ? ws.ztab.as<double>() : ws.mtab.as<double>() + c.tab_off, c.L, g.n,
                                       n_scan, ws.mask.as<uint32_t>(), stale, st, g.perm_d.as<int32_t>(), sel_v,
                                       sel_id, c.d_out, smp));
    else
      GW_CUDA(launch_ub_select<float>(nb_sel, s, ws.mtab.as<float>() + c.tab_off,
                                      g.directed ? ws.ztab.as<float>() : ws.mtab.as<float>() + c.tab_off, c.L, g.n,
                                      n_scan, ws.mask.as<uint32_t>(), stale, st, g.perm_d.as<int32_t>(), sel_v,
                                      sel_id, c.d_out, smp));
    count_launch();
    GW_CUDA(cudaMemcpyAsync(c.h_out, c.d_out, sizeof(SelOut), cudaMemcpyDeviceToHost, s));
    GW_CUDA(cudaStreamSynchronize(s));
    read_graph_timing(ws);
    while (iso_next < g.n && inS[iso_next]) ++iso_next;
    if (iso_next < g.n) {
      const unsigned long long iso =
          (static_cast<unsigned long long>(g.perm[iso_next]) << 32) | static_cast<uint32_t>(iso_next);
      c.h_out->zero_min = std::min(c.h_out->zero_min, iso);
    }
    return GEDWALK_OK;
  };

  // The plain greedy with lookahead runs as one CUDA graph (device-resident loop); the others keep
  // the host loop below.
  // GED_{<=L} of the final group. From an empty start it is the sum of the picks' exact gains
  // g_L(S_j, c_j) = GED_{<=L}(S_j + c_j) - GED_{<=L}(S_j), telescoping from GED_{<=L}(empty) = 0;
  // otherwise (an init group, or gains at shorter walk lengths) two-state sweeps over the group.
  auto group_score = [&](const std::vector<int32_t>& S_fin) -> gedwalk_status {
    if (init_int.empty() && !adaptive && gains) {
      double v = 0.0;
      for (int32_t j = 0; j < k; ++j) v += gains[j];
      *score = v;
      return GEDWALK_OK;
    }
    double v = 0;
    GW_TRY(score_one(g, ws, S_fin, r, &v));
    *score = v;
    return GEDWALK_OK;
  };
  bool device_loop = uses_device_loop(g, shape, flags, k);
  if (device_loop) {
    bool launched = false;
    const gedwalk_status st = run_device_loop(c, k, levels, cols_cand, shape.cols_max, tab_elems, nb_sel, n_scan, tol,
                                              stale, sel_v, sel_id, group, gains, &launched);
    if (st != GEDWALK_OK && launched) return st;
    if (st != GEDWALK_OK) {  // the loop's graph could not be built: the host loop below runs instead
      cudaGetLastError();
      ws.greedy_loop.reset();
      device_loop = false;
    }
  }
  if (device_loop) {
    std::vector<int32_t> S_dev = init_int;
    for (int32_t j = 0; j < k; ++j) S_dev.push_back(g.inv[group[j]]);
    if (score) GW_TRY(group_score(S_dev));
    GW_CUDA(cudaStreamSynchronize(s));
    guard.ok = true;
    return GEDWALK_OK;
  }

  for (int32_t step = 0; step < k; ++step) {
    std::vector<Cand> E;  // evaluated with the current S
    Cand best{-1.0, -1, INT_MAX};
    if (gains_all) {
      GW_TRY(run_sweeps(c, MODE_FUSED, 1, {}));
      std::vector<int32_t> batch;
      for (int32_t v = 0; v <= g.n; ++v) {
        if (v < g.n && !inS[v]) batch.push_back(v);
        if (static_cast<int>(batch.size()) == cols_all || (v == g.n && !batch.empty())) {
          GW_TRY(run_sweeps(c, MODE_CAND, cols_all, batch));
          double hg[16];
          GW_CUDA(cudaMemcpyAsync(hg, c.d_gains, sizeof(double) * cols_all, cudaMemcpyDeviceToHost, s));
          GW_CUDA(cudaStreamSynchronize(s));
          read_graph_timing(ws);
          for (size_t j = 0; j < batch.size(); ++j) {
            Cand e{hg[j], batch[j], g.perm[batch[j]]};
            if (best.v < 0 || cand_before(e, best)) best = e;
          }
          ws.st_evals += static_cast<int64_t>(batch.size());
          ++ws.st_batches;
          batch.clear();
        }
      }
    } else {
      Sampling smp = sampling_for(step);
      for (;;) {  // one attempt per walk length (a single attempt unless adaptive)
        // 1. fused sweeps: phi^miss under S plus the speculative candidates (on a directed graph
        // first psi^miss, the walks of the other orientation, on the reverse CSR)
        std::vector<int32_t> sc, last;
        E.clear();
        bool look_run = false;
        if (look && look_lvl > 0 && look_lvl < levels && look_c[look_lvl] >= 0) {
          // the last winner was this level's predecessor: its table and its candidate's exact gain
          // were computed with the current S
          const int32_t cl = look_c[look_lvl];
          c.tab_off = static_cast<size_t>(look_lvl) * tab_elems;
          set_stale<<<1, 1, 0, s>>>(stale, cl, look_g[look_lvl], step, c.d_out->gains);
          GW_KCHECK();
          E.push_back(Cand{look_g[look_lvl], cl, g.perm[cl]});
          sc.push_back(cl);
        } else if (look && (!spec.empty() || step == 0)) {
          if (spec.empty()) {
            // the first step has no bounds yet: guess the highest-degree vertices outside S (new
            // ids run by decreasing degree), GED-Walk's leading order for small alpha
            for (int32_t v = 0; v < g.n && static_cast<int>(spec.size()) < levels; ++v)
              if (!inS[v]) spec.push_back(Cand{0.0, v, g.perm[v]});
          }
          sc.assign(levels, -1);
          for (size_t j = 0; j < spec.size() && j < static_cast<size_t>(levels); ++j) sc[j] = spec[j].v;
          c.tab_off = 0;
          GW_TRY(run_sweeps(c, MODE_LOOK, levels + 1, sc));
          GW_CUDA(cudaMemcpyAsync(h_look, c.d_gains, sizeof(double) * levels, cudaMemcpyDeviceToHost, s));
          look_lvl = 0;
          look_c = sc;
          look_run = true;
          last.push_back(sc[0]);  // level 0's candidate is exact now; deeper levels wait for theirs
          for (int32_t v : sc) ws.st_evals += v >= 0;
          ++ws.st_batches;
          sc.resize(1);
        } else {
          if (g.directed) GW_TRY(run_sweeps(c, MODE_FUSED, 1, {}, true));
          for (const Cand& e : spec) sc.push_back(e.v);
          const int cf = sc.empty() ? 1 : cols_fused;
          c.tab_off = 0;
          look_lvl = -1;
          GW_TRY(run_sweeps(c, MODE_FUSED, cf, sc));
          last = sc;
        }
        bool first_batch = true;
        std::vector<Cand> X;  // exact values for the current S, best first
        std::vector<int32_t> top;
        for (;;) {
          if (!last.empty()) {
            update_stale<<<1, 32, 0, s>>>(stale, c.d_cand, c.d_gains, static_cast<int>(last.size()), step,
                                          c.d_out->gains);
            GW_KCHECK();
          }
          // 2. bound + selection pass
          GW_TRY(select_pass(step, smp));
          if (smp.thr != ~0ull && c.h_out->sampled == 0) {  // empty sample: all of V \ S competes
            smp.thr = ~0ull;
            continue;
          }
          if (look_run) {  // the gains of every level arrived with the first synchronisation
            for (int d = 0; d < levels; ++d) look_g[d] = h_look[d];
            look_run = false;
            for (size_t j = 0; j < last.size(); ++j) E.push_back(Cand{c.h_out->gains[j], last[j], g.perm[last[j]]});
          } else {
            for (size_t j = 0; j < last.size(); ++j) E.push_back(Cand{c.h_out->gains[j], last[j], g.perm[last[j]]});
            ws.st_evals += static_cast<int64_t>(last.size());
            if (!last.empty()) ++ws.st_batches;
          }
          // 3. certify: the first `need` exact values beat every bound not yet evaluated (a zero
          // bound is an exact zero gain; the lowest such caller id stands for all of them)
          top.clear();
          for (int j = 0; j < kTopK; ++j)
            if (c.h_out->id[j] != INT_MAX) top.push_back(c.h_out->id[j]);
          X = E;
          const unsigned long long zmin = c.h_out->zero_min;
          if (zmin != kNoZero) X.push_back(Cand{0.0, zero_internal(zmin), zero_caller(zmin)});
          std::sort(X.begin(), X.end(), cand_before);
          const double ub0 = top.empty() ? -1.0 : static_cast<double>(c.h_out->val[0]) * (1.0 + tol);
          const bool certified =
              top.empty() || (static_cast<int>(X.size()) >= need && ub0 < X[need - 1].g);
          if (certified) break;
          if (first_batch && !sc.empty()) ++ws.st_spec_miss;
          first_batch = false;
          last.assign(top.begin(), top.begin() + std::min<size_t>(top.size(), cols_cand));
          GW_TRY(run_sweeps(c, MODE_CAND, cols_cand, last));
        }
        best = X.empty() ? Cand{-1.0, -1, INT_MAX} : X[0];
        // speculative candidates for the next step (or attempt): best remaining values, exact or not
        std::vector<Cand> pool(X.begin() + (X.empty() ? 0 : 1), X.end());
        for (size_t j = 0; j < top.size(); ++j)
          pool.push_back(Cand{static_cast<double>(c.h_out->val[j]), top[j], g.perm[top[j]]});
        std::sort(pool.begin(), pool.end(), cand_before);
        spec.clear();
        for (const Cand& e : pool) {
          if (static_cast<int>(spec.size()) == n_spec) break;
          if (e.g > 0.0) spec.push_back(e);
        }
        if (!adaptive) break;
        // separation test (Algorithm 2): u = best is taken when L(u) > U(v) - eps_sep, where v is
        // the best of the rest and U = L + B_l. With every other vertex unevaluated the rest has
        // zero gains; with u the last vertex outside S there is no v.
        const int32_t left = g.n - static_cast<int32_t>(S_all.size());
        const double gv = X.size() >= 2 ? X[1].g : 0.0;
        if (left <= 1 || best.g > (gv + bound_at(c.L)) - eps_sep) break;
        ++ws.st_sep_fail;
        if (2 * c.L > ell_max) return fail(GEDWALK_ERR_DEVICE, "walk length passed %d without separation", ell_max);
        c.L *= 2;
        // the bounds of the shorter length are no upper bounds for the longer one: reset them
        GW_CUDA(cudaMemsetAsync(ws.stale.p, 0xff, static_cast<size_t>(g.n) * sizeof(Stale), s));
        spec.clear();  // u and the runners-up are the best guesses at the longer length
        for (const Cand& e : X) {
          if (static_cast<int>(spec.size()) == n_spec) break;
          if (e.g > 0.0) spec.push_back(e);
        }
      }
    }
    ws.st_ell.push_back(c.L);
    if (look) {  // the next level is valid only when this step took the vertex it assumed
      if (look_lvl >= 0 && best.v == look_c[look_lvl] && look_lvl + 1 < levels && look_c[look_lvl + 1] >= 0)
        ++look_lvl;
      else
        look_lvl = -1;
    }
    if (best.v < 0) return fail(GEDWALK_ERR_INVALID, "no vertex left to add");
    group[step] = best.caller;
    if (gains) gains[step] = best.g;
    const int32_t w = best.v;
    inS[w] = 1;
    S_all.push_back(w);
    hmask[w >> 5] |= 1u << (w & 31);
    GW_CUDA(cudaMemcpyAsync(ws.mask.as<uint32_t>() + (w >> 5), &hmask[w >> 5], 4, cudaMemcpyHostToDevice, s));
    spec.erase(std::remove_if(spec.begin(), spec.end(), [&](const Cand& e) { return e.v == w; }), spec.end());
    if (stochastic && step + 1 < k) {
      // The next step draws a new sample, so its speculative candidates are the best bounds
      // inside that sample: bounds and exact gains under the current S stay upper bounds once
      // w joins S (submodularity), which is all a speculative choice needs.
      spec.clear();
      const Sampling nxt = sampling_for(step + 1);
      GW_TRY(select_pass(step + 1, nxt));
      for (int j = 0; j < kTopK && static_cast<int>(spec.size()) < n_spec; ++j) {
        const int32_t id = c.h_out->id[j];
        if (id == INT_MAX || !(c.h_out->val[j] > 0.0f)) break;
        spec.push_back(Cand{static_cast<double>(c.h_out->val[j]), id, g.perm[id]});
      }
    }
  }
  ws.st_sweeps = c.sweeps;
  if (score) GW_TRY(group_score(S_all));
  GW_CUDA(cudaStreamSynchronize(s));
  guard.ok = true;
  return GEDWALK_OK;
}

gedwalk_status gains_impl(Graph& g, Workspace& ws, const std::vector<int32_t>& S_int, const Resolved& r_in,
                          double* gains_caller) {
  Resolved r = r_in;
  GW_TRY(greedy_stream(ws, r_in.stream, &r.stream));
  SyncOnError guard{r.stream};
  cudaStream_t s = r.stream;
  const size_t es = r.fp64 ? 8 : 4;
  const int cols_all = r.fp64 ? 8 : 16;
  GW_TRY(ws.mtab.ensure(static_cast<size_t>(r.L + 1) * g.n * es, s));
  GW_TRY(zero_isolated_tail(g, ws.mtab.p, es, r.L, s));
  GW_TRY(ws.small.ensure(sizeof(SelOut) + 16 * sizeof(int32_t) + 16 * sizeof(double) + 256, s));
  GW_TRY(upload_mask(g, ws, S_int, s));
  GreedyCtx c{g, ws, r, s, r.L, es};
  c.d_out = ws.small.as<SelOut>();
  c.d_cand = reinterpret_cast<int32_t*>(c.d_out + 1);
  c.d_gains = reinterpret_cast<double*>(c.d_cand + 16);
  std::vector<char> inS(g.n, 0);
  for (int32_t v : S_int) inS[v] = 1;
  for (int32_t v = 0; v < g.n; ++v) gains_caller[v] = 0.0;
  GW_TRY(run_sweeps(c, MODE_FUSED, 1, {}));
  std::vector<int32_t> batch;
  for (int32_t v = 0; v <= g.n; ++v) {
    if (v < g.n && !inS[v]) batch.push_back(v);
    if (static_cast<int>(batch.size()) == cols_all || (v == g.n && !batch.empty())) {
      GW_TRY(run_sweeps(c, MODE_CAND, cols_all, batch));
      double hg[16];
      GW_CUDA(cudaMemcpyAsync(hg, c.d_gains, sizeof(double) * cols_all, cudaMemcpyDeviceToHost, s));
      GW_CUDA(cudaStreamSynchronize(s));
      read_graph_timing(ws);
      for (size_t j = 0; j < batch.size(); ++j) gains_caller[g.perm[batch[j]]] = hg[j];
      batch.clear();
    }
  }
  guard.ok = true;
  return GEDWALK_OK;
}

}  // namespace gw

using namespace gw;

extern "C" {

gedwalk_status gedwalk_maximize(gedwalk_graph_t h, int32_t k, const gedwalk_params* params, int32_t* group,
                                double* gains, double* score, int32_t* L_used, const int32_t* init_group,
                                int32_t init_len) {
  if (!h) return fail(GEDWALK_ERR_INVALID, "graph is NULL");
  if (k < 0) return fail(GEDWALK_ERR_INVALID, "k must be >= 0");
  if (k > 0 && !group) return fail(GEDWALK_ERR_INVALID, "group is NULL");
  Graph* g = G(h);
  std::lock_guard<std::mutex> lk(g->mu);
  GW_CUDA(cudaSetDevice(g->device));
  std::vector<int32_t> init;
  GW_TRY(map_group(*g, init_group, init_len, &init));
  if (static_cast<int64_t>(init.size()) + k > g->n)
    return fail(GEDWALK_ERR_INVALID, "init group (%zu) + k (%d) exceeds n (%d)", init.size(), k, g->n);
  gedwalk_params d;
  gedwalk_params_default(&d);
  const gedwalk_params* p = params ? params : &d;
  const double eps = (p->greedy_eps_rule == GEDWALK_EPS_OVER_K && k > 0) ? p->epsilon / k : p->epsilon;
  Resolved r;
  GW_TRY(resolve(*g, p, eps, &r));
  std::vector<int32_t> grp(std::max(k, 1));
  std::vector<double> gn(std::max(k, 1));
  double sc = 0;
  GW_TRY(maximize_impl(*g, g->ws, k, r, p->flags, init, grp.data(), gn.data(), score ? &sc : nullptr));
  g->st_evals = g->ws.st_evals;
  g->st_batches = g->ws.st_batches;
  g->st_sweeps = g->ws.st_sweeps;
  g->st_spec_miss = g->ws.st_spec_miss;
  g->st_ell = g->ws.st_ell;
  g->st_sep_fail = g->ws.st_sep_fail;
  for (int32_t j = 0; j < k; ++j) {
    group[j] = grp[j];
    if (gains) gains[j] = gn[j];
  }
  if (score) *score = sc;
  if (L_used) *L_used = (p->flags & GEDWALK_ADAPTIVE_L) ? (g->st_ell.empty() ? 1 : g->st_ell.back()) : r.L;
  return GEDWALK_OK;
}

gedwalk_status gedwalk_maximize_lengths(gedwalk_graph_t h, int32_t* ell, int32_t cap, int32_t* count,
                                        int64_t* separation_failures) {
  if (!h) return fail(GEDWALK_ERR_INVALID, "graph is NULL");
  if (cap < 0 || (cap > 0 && !ell)) return fail(GEDWALK_ERR_INVALID, "ell is NULL or cap < 0");
  Graph* g = G(h);
  std::lock_guard<std::mutex> lk(g->mu);
  const int32_t m = static_cast<int32_t>(g->st_ell.size());
  for (int32_t j = 0; j < std::min(m, cap); ++j) ell[j] = g->st_ell[j];
  if (count) *count = m;
  if (separation_failures) *separation_failures = g->st_sep_fail;
  return GEDWALK_OK;
}

gedwalk_status gedwalk_maximize_stats(gedwalk_graph_t h, int64_t* evaluations, int64_t* batches, int64_t* sweeps,
                                      int64_t* spec_misses) {
  if (!h) return fail(GEDWALK_ERR_INVALID, "graph is NULL");
  Graph* g = G(h);
  std::lock_guard<std::mutex> lk(g->mu);
  if (evaluations) *evaluations = g->st_evals;
  if (batches) *batches = g->st_batches;
  if (sweeps) *sweeps = g->st_sweeps;
  if (spec_misses) *spec_misses = g->st_spec_miss;
  return GEDWALK_OK;
}

gedwalk_status gedwalk_gains(gedwalk_graph_t h, const int32_t* S, int32_t s_len, const gedwalk_params* params,
                             double* gains, int32_t* L_used) {
  if (!h || !gains) return fail(GEDWALK_ERR_INVALID, "graph or gains is NULL");
  Graph* g = G(h);
  std::lock_guard<std::mutex> lk(g->mu);
  GW_CUDA(cudaSetDevice(g->device));
  std::vector<int32_t> S_int;
  GW_TRY(map_group(*g, S, s_len, &S_int));
  Resolved r;
  GW_TRY(resolve(*g, params, 0.0, &r));
  GW_TRY(gains_impl(*g, g->ws, S_int, r, gains));
  if (L_used) *L_used = r.L;
  return GEDWALK_OK;
}

}  // extern "C"
