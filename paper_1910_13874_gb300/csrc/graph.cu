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

// While a thread captures a CUDA graph its launches are not executions: they are counted when the
// graph runs.
static thread_local bool t_capturing = false;
void set_capturing(bool on) { t_capturing = on; }
void count_launch() {
  if (!t_capturing) prof().launches.fetch_add(1, std::memory_order_relaxed);
}
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

double sweep_bytes(int mode, bool fp64, int cols, int32_t n, int64_t nnz, bool weighted) {
  const double es = mode == MODE_TOTALS ? 8.0 : (fp64 ? 8.0 : 4.0);
  double b = 4.0 * double(nnz) + 4.0 * (double(n) + 1.0) + 2.0 * cols * es * double(n);
  if (mode == MODE_SCORE || mode == MODE_FUSED || mode == MODE_CAND || mode == MODE_LOOK) b += double(n) / 8.0;
  if (mode == MODE_FUSED) b += es * double(n);
  if (mode == MODE_LOOK) b += es * double(n) * (cols - 1);  // one phi^miss row per level
  if (weighted) b += es * double(n);  // the vertex scales
  return b;
}

// ---------------------------------------------------------------- device memory
static gedwalk_alloc_fn g_alloc = nullptr;
static gedwalk_free_fn g_free = nullptr;
static void* g_alloc_ctx = nullptr;

void* dalloc(size_t bytes, cudaStream_t s, Allocator* from) {
  if (bytes == 0) bytes = 16;
  if (g_alloc) {
    from->release = g_free;
    from->ctx = g_alloc_ctx;
    return g_alloc(bytes, reinterpret_cast<int64_t>(s), g_alloc_ctx);
  }
  from->release = nullptr;
  from->ctx = nullptr;
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();  // clear the sticky-free error state of a failed allocation
    return nullptr;
  }
  return p;
}

void dfree(void* p, size_t bytes, cudaStream_t s, const Allocator& from) {
  if (!p) return;
  if (from.release) {
    // A caching allocator (PyTorch's) may hand the block to its next user at once, while cudaFree
    // would first wait for the device. The library frees only blocks no kernel uses any more:
    // every call synchronises the stream it ran on before it returns (on success and on error),
    // the walk-total table grows only after its readers have finished, and a graph is freed after
    // the whole device has. (No device-wide wait here: it would break a CUDA graph capture that
    // another thread has in progress.)
    from.release(p, bytes, reinterpret_cast<int64_t>(s), from.ctx);
    return;
  }
  if (cudaFree(p) != cudaSuccess) cudaGetLastError();  // leave no error behind for the next check
}

gedwalk_status DevBuf::ensure(size_t need, cudaStream_t s, bool zero) {
  if (need == 0) need = 16;
  if (p && bytes >= need) return GEDWALK_OK;
  release();
  p = dalloc(need, s, &from);
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

int64_t Workspace::device_bytes() const {
  int64_t b = 0;
  for (const DevBuf* d : {&x0, &x1, &mtab, &ztab, &pvec, &partial, &counters, &slots, &parts, &mask, &stale, &sel,
                          &small, &members, &ctl})
    b += static_cast<int64_t>(d->bytes);
  return b;
}

void Workspace::release_device() {
  for (SweepGraph& sg : graphs) sg.reset();
  greedy_loop.reset();
  for (DevBuf* d : {&x0, &x1, &mtab, &ztab, &pvec, &partial, &counters, &slots, &parts, &mask, &stale, &sel, &small,
                    &members, &ctl})
    d->release();
}

Workspace::~Workspace() {
  for (SweepGraph& sg : graphs) sg.reset();
  greedy_loop.reset();
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


// First malformed row (or -1) and a reason.
// Entry checks of an uploaded CSR: column in range, and (full) no self-loop, strictly increasing
// rows and (symmetric) every entry mirrored. The smallest offending (row << 3 | kind) wins.
// Entries [b, e) of row v, whose row starts at r0.
// Symmetry: order the vertices by (degree, id). An entry (v, u) is "down" when u comes before v;
// only down entries look for their mirror (v in row u, the shorter row, by binary search), and
// counts[0] / counts[1] receive the numbers of down / up entries. The mirror of a down entry is an
// up entry and distinct entries have distinct mirrors (rows have no repeats), so if every down
// entry is mirrored and the two counts agree, the mirrors are all the up entries: the CSR is
// symmetric. all_up = 1 checks every entry (locates the row after the counts disagreed).
__device__ __forceinline__ void check_entries(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                              int32_t n, int full, int symmetric, int all_up, int64_t v, int32_t r0,
                                              int32_t b, int32_t e, int32_t dv, int lane,
                                              unsigned long long* __restrict__ bad, unsigned long long& down,
                                              unsigned long long& up) {
  for (int32_t j = b + lane; j < e; j += 32) {
    const int32_t u = ci[j];
    int k = 0;
    if (u < 0 || u >= n) {
      k = 1;
    } else if (full) {
      if (u == v) {
        k = 2;
      } else if (j > r0 && ci[j - 1] >= u) {
        k = 3;
      } else if (symmetric) {
        int32_t lo = rp[u], hi = rp[u + 1];
        const int32_t du = hi - lo;
        const bool is_down = du < dv || (du == dv && u < v);
        if (is_down) ++down;
        else ++up;
        if (is_down || all_up) {
          const int32_t end = hi;
          while (lo < hi) {  // first entry of row u that is >= v
            const int32_t mid = lo + ((hi - lo) >> 1);
            if (ci[mid] < v) lo = mid + 1;
            else hi = mid;
          }
          if (lo == end || ci[lo] != v) k = 4;
        }
      }
    }
    if (k) atomicMin(bad, (static_cast<unsigned long long>(v) << 3) | static_cast<unsigned long long>(k));
  }
}

// One warp per row of at most kCheckPiece entries; longer rows come as pieces in `pieces`
// ({row, first entry, end}), so that no warp walks a hub row alone.
constexpr int32_t kCheckPiece = 1024;
__global__ void validate_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, int32_t n,
                                int full, int symmetric, int all_up, const int4* __restrict__ pieces, int64_t npieces,
                                unsigned long long* __restrict__ bad, unsigned long long* __restrict__ counts) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t(gridDim.x) * blockDim.x) >> 5;
  unsigned long long down = 0, up = 0;
  for (int64_t w = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; w < n + npieces; w += warps) {
    if (w < n) {
      const int32_t b = rp[w], e = rp[w + 1];
      if (e - b <= kCheckPiece)
        check_entries(rp, ci, n, full, symmetric, all_up, w, b, b, e, e - b, lane, bad, down, up);
    } else {
      const int4 pc = pieces[w - n];
      const int32_t r0 = rp[pc.x];
      check_entries(rp, ci, n, full, symmetric, all_up, pc.x, r0, pc.y, pc.z, rp[pc.x + 1] - r0, lane, bad, down,
                    up);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    down += __shfl_xor_sync(0xffffffffu, down, o);
    up += __shfl_xor_sync(0xffffffffu, up, o);
  }
  if (lane == 0 && (down | up)) {
    atomicAdd(counts, down);
    atomicAdd(counts + 1, up);
  }
}

// Row-pointer check of an uploaded CSR (rp[0] = 0 and rp[n] = nnz already hold): out[0] = the
// first row whose pointer decreases (min over rows; all ones if none), out[1] = the largest row
// length, out[2] = the number of kCheckPiece pieces of the longer rows.
__global__ void rowptr_check_kernel(const int32_t* __restrict__ rp, int32_t n, unsigned long long* __restrict__ out) {
  unsigned long long dmax = 0, pcs = 0;
  for (int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; v < n; v += int64_t(gridDim.x) * blockDim.x) {
    const int64_t d = static_cast<int64_t>(rp[v + 1]) - rp[v];
    if (d < 0) {
      atomicMin(out, static_cast<unsigned long long>(v));
    } else {
      dmax = static_cast<unsigned long long>(d) > dmax ? static_cast<unsigned long long>(d) : dmax;
      if (d > kCheckPiece) pcs += static_cast<unsigned long long>((d + kCheckPiece - 1) / kCheckPiece);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long m = __shfl_xor_sync(0xffffffffu, dmax, o);
    dmax = m > dmax ? m : dmax;
    pcs += __shfl_xor_sync(0xffffffffu, pcs, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (dmax) atomicMax(out + 1, dmax);
    if (pcs) atomicAdd(out + 2, pcs);
  }
}

// The pieces {row, first entry, end, 0} of the rows above kCheckPiece entries, in any order.
__global__ void check_pieces_kernel(const int32_t* __restrict__ rp, int32_t n, unsigned long long* __restrict__ count,
                                    int4* __restrict__ pieces) {
  for (int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; v < n; v += int64_t(gridDim.x) * blockDim.x) {
    const int32_t b0 = rp[v], e = rp[v + 1];
    if (e - b0 <= kCheckPiece) continue;
    const int32_t np = (e - b0 + kCheckPiece - 1) / kCheckPiece;
    const unsigned long long at = atomicAdd(count, static_cast<unsigned long long>(np));
    for (int32_t k = 0; k < np; ++k) {
      const int32_t b = b0 + k * kCheckPiece;
      pieces[at + k] = make_int4(static_cast<int32_t>(v), b, min(e, b + kCheckPiece), 0);
    }
  }
}

// Relabelled CSR, one warp per new row i: the entries of old row perm[i], each mapped to its new
// id, in their old order.
__global__ void relabel_kernel(const int32_t* __restrict__ raw_rp, const int32_t* __restrict__ raw_ci,
                               const int32_t* __restrict__ rp, const int32_t* __restrict__ perm,
                               const int32_t* __restrict__ inv, int32_t n, int32_t* __restrict__ ci) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t i = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
    const int32_t src = raw_rp[perm[i]], dst = rp[i], len = rp[i + 1] - rp[i];
    for (int32_t j = lane; j < len; j += 32) ci[dst + j] = inv[raw_ci[src + j]];
  }
}

static int grid_for(int64_t n) { return static_cast<int>(std::min<int64_t>((n + 255) / 256, 152 * 16)); }

// ---------------------------------------------------------------- device relabelling
// Exclusive scan of m unsigned counts (m >= 1), in tiles of kScanTile: each tile is scanned by one
// block, the tiles' totals are scanned the same way (recursively), then added back.
constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int64_t kScanTile = int64_t(kScanThreads) * kScanItems;

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t x, uint32_t* warp_tot, uint32_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) warp_tot[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    constexpr int NW = kScanThreads / 32;
    uint32_t t = lane < NW ? warp_tot[lane] : 0u;
    uint32_t ti = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, ti, o);
      if (lane >= o) ti += y;
    }
    if (lane < NW) warp_tot[lane] = ti - t;  // exclusive offsets of the warps
    if (lane == NW - 1) *total = ti;
  }
  __syncthreads();
  return warp_tot[warp] + inc - x;
}

// out[i] = sum of in[tile start .. i) within each tile; sums[tile] = the tile's total.
__global__ void __launch_bounds__(kScanThreads) scan_tiles_kernel(const uint32_t* __restrict__ in, int64_t m,
                                                                  uint32_t* __restrict__ out,
                                                                  uint32_t* __restrict__ sums) {
  __shared__ uint32_t warp_tot[kScanThreads / 32];
  __shared__ uint32_t total;
  const int64_t base = int64_t(blockIdx.x) * kScanTile + int64_t(threadIdx.x) * kScanItems;
  uint32_t v[kScanItems];
  uint32_t acc = 0;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    v[j] = base + j < m ? in[base + j] : 0u;
    acc += v[j];
  }
  uint32_t run = block_exclusive_scan(acc, warp_tot, &total);
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    if (base + j < m) out[base + j] = run;
    run += v[j];
  }
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void scan_add_kernel(uint32_t* __restrict__ out, int64_t m, const uint32_t* __restrict__ offs) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < m; i += int64_t(gridDim.x) * blockDim.x)
    out[i] += offs[i / kScanTile];
}

// out[0..m) = exclusive scan of in[0..m); *total_out (device, may be null) = the sum. Scratch is
// allocated per level.
static gedwalk_status exclusive_scan(const uint32_t* in, int64_t m, uint32_t* out, uint32_t* total_out) {
  const int64_t tiles = (m + kScanTile - 1) / kScanTile;
  DevBuf sums, sums_scan;
  GW_TRY(sums.ensure(static_cast<size_t>(tiles) * sizeof(uint32_t), 0));
  scan_tiles_kernel<<<static_cast<int>(tiles), kScanThreads>>>(in, m, out, sums.as<uint32_t>());
  GW_KCHECK();
  if (tiles == 1) {
    if (total_out) GW_CUDA(cudaMemcpy(total_out, sums.p, sizeof(uint32_t), cudaMemcpyDeviceToDevice));
    return GEDWALK_OK;
  }
  GW_TRY(sums_scan.ensure(static_cast<size_t>(tiles) * sizeof(uint32_t), 0));
  GW_TRY(exclusive_scan(sums.as<uint32_t>(), tiles, sums_scan.as<uint32_t>(), total_out));
  scan_add_kernel<<<grid_for(m), 256>>>(out, m, sums_scan.as<uint32_t>());
  GW_KCHECK();
  return GEDWALK_OK;
}

// Stable LSD radix sort of (key, value) pairs by 8-bit digits. A block takes kRadixTile
// consecutive pairs, each of its warps kRadixTile / 8 consecutive ones in chunks of 32 lanes in
// index order; equal digits are ranked by __match_any_sync, so the order of equal keys is kept.
constexpr int kRadixThreads = 256;
constexpr int kRadixWarps = kRadixThreads / 32;
constexpr int64_t kRadixTile = 4096;
constexpr int kRadixChunks = static_cast<int>(kRadixTile / kRadixWarps / 32);

// counts[digit * blocks + block] = pairs of the block with that digit
__global__ void __launch_bounds__(kRadixThreads) radix_count_kernel(const uint32_t* __restrict__ keys, int64_t n,
                                                                    int shift, uint32_t* __restrict__ counts) {
  __shared__ uint32_t h[256];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < 256; i += kRadixThreads) h[i] = 0;
  __syncthreads();
  const int64_t base = int64_t(blockIdx.x) * kRadixTile + int64_t(warp) * (kRadixTile / kRadixWarps);
  for (int c = 0; c < kRadixChunks; ++c) {
    const int64_t j = base + c * 32 + lane;
    const bool ok = j < n;
    const uint32_t d = ok ? (keys[j] >> shift) & 255u : 256u;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    if (ok && lane == __ffs(peers) - 1) atomicAdd(&h[d], static_cast<uint32_t>(__popc(peers)));
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 256; i += kRadixThreads) counts[int64_t(i) * gridDim.x + blockIdx.x] = h[i];
}

// Scatters the block's pairs to offs[digit * blocks + block] + their stable rank. vals_in null:
// the values are the indices.
__global__ void __launch_bounds__(kRadixThreads) radix_scatter_kernel(const uint32_t* __restrict__ keys_in,
                                                                      const int32_t* __restrict__ vals_in, int64_t n,
                                                                      int shift, const uint32_t* __restrict__ offs,
                                                                      uint32_t* __restrict__ keys_out,
                                                                      int32_t* __restrict__ vals_out) {
  __shared__ uint32_t wc[kRadixWarps][256];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < kRadixWarps * 256; i += kRadixThreads) wc[i / 256][i % 256] = 0;
  __syncthreads();
  const int64_t base = int64_t(blockIdx.x) * kRadixTile + int64_t(warp) * (kRadixTile / kRadixWarps);
  const unsigned lt = (1u << lane) - 1u;
  for (int c = 0; c < kRadixChunks; ++c) {  // per-warp digit counts
    const int64_t j = base + c * 32 + lane;
    const bool ok = j < n;
    const uint32_t d = ok ? (keys_in[j] >> shift) & 255u : 256u;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    if (ok && lane == __ffs(peers) - 1) wc[warp][d] += __popc(peers);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < 256; d += kRadixThreads) {  // warp offsets within the digit's range
    uint32_t run = offs[int64_t(d) * gridDim.x + blockIdx.x];
    for (int w = 0; w < kRadixWarps; ++w) {
      const uint32_t t = wc[w][d];
      wc[w][d] = run;
      run += t;
    }
  }
  __syncthreads();
  for (int c = 0; c < kRadixChunks; ++c) {
    const int64_t j = base + c * 32 + lane;
    const bool ok = j < n;
    const uint32_t key = ok ? keys_in[j] : 0u;
    const uint32_t d = ok ? (key >> shift) & 255u : 256u;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    if (ok) {
      const uint32_t pos = wc[warp][d] + __popc(peers & lt);
      keys_out[pos] = key;
      vals_out[pos] = vals_in ? vals_in[j] : static_cast<int32_t>(j);
    }
    __syncwarp();
    if (ok && lane == __ffs(peers) - 1) wc[warp][d] += __popc(peers);
    __syncwarp();
  }
}

// key[v] = dmax - degree(v): ascending keys order the rows by decreasing degree
__global__ void degree_key_kernel(const int32_t* __restrict__ rp, int32_t n, int32_t dmax, uint32_t* __restrict__ key) {
  for (int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; v < n; v += int64_t(gridDim.x) * blockDim.x)
    key[v] = static_cast<uint32_t>(dmax - (rp[v + 1] - rp[v]));
}

// inv[perm[i]] = i and deg[i] = dmax - key[i] (the sorted keys)
__global__ void perm_finish_kernel(const int32_t* __restrict__ perm, const uint32_t* __restrict__ key, int32_t n,
                                   int32_t dmax, int32_t* __restrict__ inv, uint32_t* __restrict__ deg) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    inv[perm[i]] = static_cast<int32_t>(i);
    deg[i] = static_cast<uint32_t>(dmax) - key[i];
  }
}

// perm: new -> caller id (decreasing degree, equal degrees by caller id), inv its inverse, deg
// and rp the relabelled degrees and row pointers (rp[n] = nnz), all on the device.
static gedwalk_status degree_order(const int32_t* raw_rp, int32_t n, int32_t dmax, int32_t* perm, int32_t* inv,
                                   int32_t* deg, int32_t* rp) {
  const int64_t blocks = (int64_t(n) + kRadixTile - 1) / kRadixTile;
  DevBuf k0, k1, v1, counts, offs;
  GW_TRY(k0.ensure(static_cast<size_t>(n) * sizeof(uint32_t), 0));
  GW_TRY(k1.ensure(static_cast<size_t>(n) * sizeof(uint32_t), 0));
  GW_TRY(v1.ensure(static_cast<size_t>(n) * sizeof(int32_t), 0));
  GW_TRY(counts.ensure(static_cast<size_t>(blocks) * 256 * sizeof(uint32_t), 0));
  GW_TRY(offs.ensure(static_cast<size_t>(blocks) * 256 * sizeof(uint32_t), 0));
  degree_key_kernel<<<grid_for(n), 256>>>(raw_rp, n, dmax, k0.as<uint32_t>());
  GW_KCHECK();
  int bits = 0;
  while (bits < 32 && (static_cast<uint32_t>(dmax) >> bits) != 0) ++bits;
  const int passes = std::max(1, (bits + 7) / 8);
  // ping-pong so that the last pass writes perm: passes odd -> k0/perm first
  uint32_t* kin = k0.as<uint32_t>();
  const int32_t* vin = nullptr;
  for (int ps = 0; ps < passes; ++ps) {
    const bool last_to_perm = ((passes - 1 - ps) % 2) == 0;
    uint32_t* kout = (kin == k0.as<uint32_t>()) ? k1.as<uint32_t>() : k0.as<uint32_t>();
    int32_t* vout = last_to_perm ? perm : v1.as<int32_t>();
    radix_count_kernel<<<static_cast<int>(blocks), kRadixThreads>>>(kin, n, 8 * ps, counts.as<uint32_t>());
    GW_KCHECK();
    GW_TRY(exclusive_scan(counts.as<uint32_t>(), blocks * 256, offs.as<uint32_t>(), nullptr));
    radix_scatter_kernel<<<static_cast<int>(blocks), kRadixThreads>>>(kin, vin, n, 8 * ps, offs.as<uint32_t>(), kout,
                                                                      vout);
    GW_KCHECK();
    kin = kout;
    vin = vout;
  }
  perm_finish_kernel<<<grid_for(n), 256>>>(perm, kin, n, dmax, inv, reinterpret_cast<uint32_t*>(deg));
  GW_KCHECK();
  GW_TRY(exclusive_scan(reinterpret_cast<const uint32_t*>(deg), n, reinterpret_cast<uint32_t*>(rp),
                        reinterpret_cast<uint32_t*>(rp + n)));
  return GEDWALK_OK;
}

// Sorts segments of the relabelled CSR (one warp per segment of at most 1024 entries): the
// 1024-entry pieces of rows longer than that (listed in seg; those rows are summed slice by slice
// anyway), then the whole rows [r0, r1). Ascending neighbour ids put the high-degree neighbours,
// the most gathered rows, first in every row. A bitonic network: in registers up to 32 entries,
// in the warp's shared memory above.
constexpr int kSortSeg = 1024;
__global__ void __launch_bounds__(256) sort_segments_kernel(const int2* __restrict__ seg, int64_t nseg,
                                                            const int32_t* __restrict__ rp, int32_t r0, int32_t r1,
                                                            int32_t* __restrict__ ci) {
  __shared__ int32_t buf[8][kSortSeg];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t warps = (int64_t(gridDim.x) * blockDim.x) >> 5;
  const int64_t total = nseg + (r1 - r0);
  for (int64_t sidx = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; sidx < total; sidx += warps) {
    int2 sg;
    if (sidx < nseg) {
      sg = seg[sidx];
    } else {
      const int32_t r = r0 + static_cast<int32_t>(sidx - nseg);
      sg = make_int2(rp[r], rp[r + 1] - rp[r]);
    }
    if (sg.y <= 1) continue;
    int32_t* p = ci + sg.x;
    const int len = sg.y;
    if (len <= 32) {
      int32_t x = lane < len ? p[lane] : INT_MAX;
      for (int k = 2; k <= 32; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
          const int32_t y = __shfl_xor_sync(0xffffffffu, x, j);
          const bool up = (lane & k) == 0, low = (lane & j) == 0;
          x = (low == up) ? min(x, y) : max(x, y);
        }
      if (lane < len) p[lane] = x;
      continue;
    }
    int P = 64;
    while (P < len) P <<= 1;
    int32_t* b = buf[w];
    for (int i = lane; i < P; i += 32) b[i] = i < len ? p[i] : INT_MAX;
    __syncwarp();
    for (int k = 2; k <= P; k <<= 1)
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int t = lane; t < P / 2; t += 32) {
          const int i = 2 * j * (t / j) + (t % j), q = i + j;
          const int32_t a = b[i], c = b[q];
          if (((i & k) == 0) == (a > c)) {
            b[i] = c;
            b[q] = a;
          }
        }
        __syncwarp();
      }
    for (int i = lane; i < len; i += 32) p[i] = b[i];
    __syncwarp();
  }
}

// Validates a CSR: row_ptr on the host (the kernels index with it), the entries on the device
// (drp/dci: copies of the same arrays). Returns the first offending row or -1.
static int64_t validate_csr(const int32_t* rp, const int32_t* drp, const int32_t* dci, int32_t n, int64_t nnz,
                            bool full, std::string* why, bool symmetric, gedwalk_status* st, int32_t* dmax_out) {
  *st = GEDWALK_OK;
  if (rp[0] != 0) {
    *why = "row_ptr[0] != 0";
    return 0;
  }
  if (static_cast<int64_t>(rp[n]) != nnz) {
    *why = "row_ptr[n] != nnz";
    return n;
  }
  // on the device: monotone row pointers, the largest degree, the pieces of rows above kCheckPiece
  DevBuf dbad, dpieces;
  // first {first decreasing row, d_max, pieces}, then {worst entry, down and up entry counts}
  unsigned long long hbad[3] = {~0ull, 0ull, 0ull};
  if ((*st = dbad.ensure(sizeof(hbad), 0)) != GEDWALK_OK) return -1;
  cudaError_t e = cudaMemcpy(dbad.p, hbad, sizeof(hbad), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    rowptr_check_kernel<<<grid_for(n), 256>>>(drp, n, dbad.as<unsigned long long>());
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(hbad, dbad.p, sizeof(hbad), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    *st = fail(GEDWALK_ERR_DEVICE, "CSR validation: %s", cudaGetErrorString(e));
    return -1;
  }
  if (hbad[0] != ~0ull) {
    *why = "row_ptr decreases";
    return static_cast<int64_t>(hbad[0]);
  }
  *dmax_out = static_cast<int32_t>(hbad[1]);
  if (nnz == 0) return -1;
  const int64_t npieces = static_cast<int64_t>(hbad[2]);
  if ((*st = dpieces.ensure(std::max<size_t>(static_cast<size_t>(npieces), 1) * sizeof(int4), 0)) != GEDWALK_OK)
    return -1;
  if (npieces > 0) {
    hbad[2] = 0;
    e = cudaMemcpy(dbad.as<unsigned long long>() + 2, &hbad[2], sizeof(hbad[2]), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
      check_pieces_kernel<<<grid_for(n), 256>>>(drp, n, dbad.as<unsigned long long>() + 2, dpieces.as<int4>());
      e = cudaGetLastError();
    }
  }
  const int64_t work = static_cast<int64_t>(n) + npieces;
  const int64_t blocks = std::min<int64_t>((work * 32 + 255) / 256, 152 * 32);
  // first the down entries only; if every one is mirrored but the counts disagree, every entry
  for (int all_up = 0; all_up < 2 && e == cudaSuccess; ++all_up) {
    hbad[0] = ~0ull;
    hbad[1] = hbad[2] = 0;
    e = cudaMemcpy(dbad.p, hbad, sizeof(hbad), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) break;
    validate_kernel<<<static_cast<int>(blocks), 256>>>(drp, dci, n, full ? 1 : 0, symmetric ? 1 : 0, all_up,
                                                       dpieces.as<int4>(), npieces,
                                                       dbad.as<unsigned long long>(),
                                                       dbad.as<unsigned long long>() + 1);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(hbad, dbad.p, sizeof(hbad), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess || hbad[0] != ~0ull || !full || !symmetric || hbad[1] == hbad[2]) break;
  }
  if (e != cudaSuccess) {
    *st = fail(GEDWALK_ERR_DEVICE, "CSR validation: %s", cudaGetErrorString(e));
    return -1;
  }
  static const char* reasons[] = {"", "column index out of range", "self-loop", "row not strictly increasing",
                                  "graph is not symmetric (undirected graphs only)"};
  if (hbad[0] != ~0ull) {
    *why = reasons[hbad[0] & 7];
    return static_cast<int64_t>(hbad[0] >> 3);
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

// The first row in [lo, hi) where pred holds, for a pred that holds on a suffix of the range
// (hi if none): a binary search.
template <class P>
static int32_t first_row(int32_t lo, int32_t hi, P pred) {
  while (lo < hi) {
    const int32_t mid = lo + (hi - lo) / 2;
    if (pred(mid)) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

static gedwalk_status finish_plan(Plan& plan, const std::vector<int4>& units, const std::vector<int4>& heavy) {
  plan.num_units = static_cast<int32_t>(units.size());
  plan.num_slots = plan.num_units + plan.num_heavy;
  GW_TRY(plan.units.ensure(units.size() * sizeof(int4) + 16, 0));
  GW_TRY(plan.heavy.ensure(heavy.size() * sizeof(int4) + 16, 0));
  if (!units.empty()) GW_CUDA(cudaMemcpy(plan.units.p, units.data(), units.size() * sizeof(int4), cudaMemcpyHostToDevice));
  if (!heavy.empty()) GW_CUDA(cudaMemcpy(plan.heavy.p, heavy.data(), heavy.size() * sizeof(int4), cudaMemcpyHostToDevice));
  return GEDWALK_OK;
}

// Work units of one CSR. Heavy rows (degree > kHeavyDeg) are cut into slices wherever they sit;
// the other rows [0, n_active) form contiguous runs of one degree class. Rows from n_active on have
// no units (isolated vertices: nothing gathers them). With rows sorted by decreasing degree (the
// relabelled forward CSR) the heavy rows are the prefix and every class is one contiguous run; the
// reverse CSR of a directed graph keeps the forward order, so its runs are shorter.
// With `sorted` (the forward CSR) the runs are found by binary search over degrees and row
// pointers; otherwise the rows are walked one by one.
static gedwalk_status build_plan(Plan& plan, const std::vector<int32_t>& deg, const std::vector<int32_t>& rp,
                                 int32_t n_active, int32_t n, bool sorted) {
  if (!sorted) {
    std::vector<int4> units, heavy;
    int32_t slice = 0;
    for (int32_t r = 0; r < n_active; ++r) {
      const int32_t d = deg[r];
      if (d <= kHeavyDeg) continue;
      const int32_t ns = (d + kSliceEdges - 1) / kSliceEdges;
      const int32_t hi = static_cast<int32_t>(heavy.size());
      heavy.push_back(make_int4(r, slice, ns, 0));
      for (int32_t k = 0; k < ns; ++k) {
        const int32_t e0 = rp[r] + static_cast<int32_t>(static_cast<int64_t>(d) * k / ns);
        const int32_t e1 = rp[r] + static_cast<int32_t>(static_cast<int64_t>(d) * (k + 1) / ns);
        units.push_back(make_int4(hi, e0, e1, slice + k));
      }
      slice += ns;
    }
    plan.num_slices = slice;
    plan.num_heavy = static_cast<int32_t>(heavy.size());
    int32_t r = 0;
    while (r < n_active) {
      if (deg[r] > kHeavyDeg) {
        ++r;
        continue;
      }
      const int cls = row_class(deg[r]);
      // a short-row unit takes up to kUnitRowsMax rows; on small graphs fewer, down to one
      // iteration of its warp (2 rows per lane group), so that every SM gets work
      const int32_t iter_rows = cls == 6 ? 1 : 2 * (32 >> cls);
      const int32_t small_cap = std::max<int32_t>(iter_rows, n_active / kTargetUnits);
      const int32_t max_rows = std::min<int32_t>(cls == 6 ? 32 : kUnitRowsMax, small_cap);
      const int64_t max_edges = cls == 6 ? kLongUnitEdges : kUnitEdges;
      int32_t r1 = r;
      int64_t edges = 0;
      while (r1 < n_active && deg[r1] <= kHeavyDeg && row_class(deg[r1]) == cls && r1 - r < max_rows &&
             (r1 == r || edges + deg[r1] <= max_edges)) {
        edges += deg[r1];
        ++r1;
      }
      units.push_back(make_int4(r, r1, cls, -1));
      r = r1;
    }
    return finish_plan(plan, units, heavy);
  }
  // rows are ordered by decreasing degree: the heavy rows form a prefix, then runs of one class
  // (row lengths from the row pointers)
  auto deg_at = [&](int32_t i) { return rp[i + 1] - rp[i]; };
  std::vector<int4> units, heavy;
  int32_t slice = 0;
  int32_t r = 0;
  for (; r < n_active && deg_at(r) > kHeavyDeg; ++r) {
    const int32_t d = deg_at(r);
    const int32_t ns = (d + kSliceEdges - 1) / kSliceEdges;
    const int32_t hi = static_cast<int32_t>(heavy.size());
    heavy.push_back(make_int4(r, slice, ns, 0));
    for (int32_t k = 0; k < ns; ++k) {
      const int32_t e0 = rp[r] + static_cast<int32_t>(static_cast<int64_t>(d) * k / ns);
      const int32_t e1 = rp[r] + static_cast<int32_t>(static_cast<int64_t>(d) * (k + 1) / ns);
      units.push_back(make_int4(hi, e0, e1, slice + k));
    }
    slice += ns;
  }
  plan.num_slices = slice;
  plan.num_heavy = static_cast<int32_t>(heavy.size());
  while (r < n_active) {
    const int cls = row_class(deg_at(r));
    // the run of this class: classes do not increase along the rows
    const int32_t cls_end = first_row(r, n_active, [&](int32_t i) { return row_class(deg_at(i)) != cls; });
    // a short-row unit takes up to kUnitRowsMax rows; on small graphs fewer, down to one
    // iteration of its warp (2 rows per lane group), so that every SM gets work
    const int32_t iter_rows = cls == 6 ? 1 : 2 * (32 >> cls);
    const int32_t small_cap = std::max<int32_t>(iter_rows, n_active / kTargetUnits);
    const int32_t max_rows = std::min<int32_t>(cls == 6 ? 32 : kUnitRowsMax, small_cap);
    const int64_t max_edges = cls == 6 ? kLongUnitEdges : kUnitEdges;
    while (r < cls_end) {
      // the most rows from r whose entries stay within max_edges (at least one row)
      const int64_t cap = static_cast<int64_t>(rp[r]) + max_edges;
      const auto it = std::upper_bound(rp.begin() + r + 1, rp.begin() + cls_end + 1, cap,
                                       [](int64_t c, int32_t x) { return c < x; });
      int32_t r1 = static_cast<int32_t>(it - rp.begin()) - 1;
      r1 = std::max(r + 1, std::min({r1, r + max_rows, cls_end}));
      units.push_back(make_int4(r, r1, cls, -1));
      r = r1;
    }
  }
  (void)n;
  return finish_plan(plan, units, heavy);
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
  a.rs_f = g.weighted ? g.rs_f.as<float>() : nullptr;
  a.rs_d = g.weighted ? g.rs_d.as<double>() : nullptr;
  return a;
}

SweepArgs base_args_rev(Graph& g, Workspace& ws) {
  SweepArgs a = base_args(g, ws);
  a.rp = g.rp_r.as<int32_t>();
  a.ci = g.ci_r.as<int32_t>();
  a.units = g.plan_r.units.as<int4>();
  a.heavy = g.plan_r.heavy.as<int4>();
  a.num_units = g.plan_r.num_units;
  return a;
}

gedwalk_status ensure_sweep_scratch(Graph& g, Workspace& ws, int cols, bool fp64, cudaStream_t s) {
  const size_t es = fp64 ? 8 : 4;
  // sized for the larger of the two plans of a directed graph
  const int32_t slices = std::max(g.plan.num_slices, g.directed ? g.plan_r.num_slices : 0);
  const int32_t heavy = std::max(g.plan.num_heavy, g.directed ? g.plan_r.num_heavy : 0);
  const int32_t slots = std::max(g.plan.num_slots, g.directed ? g.plan_r.num_slots : 0);
  GW_TRY(ws.partial.ensure(static_cast<size_t>(std::max(slices, 1)) * cols * es, s));
  const size_t cbytes = static_cast<size_t>(std::max(heavy, 1)) * sizeof(unsigned);
  if (ws.counters.bytes < cbytes || !ws.counters.p) GW_TRY(ws.counters.ensure(cbytes, s, /*zero=*/true));
  GW_TRY(ws.slots.ensure(static_cast<size_t>(std::max(slots, 1)) * cols * sizeof(double), s));
  GW_TRY(ws.parts.ensure(static_cast<size_t>(cols) * kReduceParts * sizeof(double), s));
  return GEDWALK_OK;
}

gedwalk_status reduce_slots(Graph& g, Workspace& ws, int nsum, double* out, cudaStream_t s, bool rev) {
  return launch_reduce_slots(ws.slots.as<double>(), rev ? g.plan_r.num_slots : g.plan.num_slots, nsum, out,
                             ws.parts.as<double>(), s);
}

// ---------------------------------------------------------------- walk totals
gedwalk_status ensure_totals(Graph& g, double alpha, int32_t rows, cudaStream_t s) {
  {
    std::shared_lock<std::shared_mutex> rl(g.tt_lock);
    if (g.tt_alpha == alpha && rows <= g.tt_rows) return GEDWALK_OK;
  }
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
    g.ttab.swap(fresh);
    GW_CUDA(cudaStreamSynchronize(s));
  }
  if (g.Wa_d.bytes < static_cast<size_t>(rows) * sizeof(double)) {
    // grow the device sums, keeping the rows already computed
    DevBuf fresh;
    GW_TRY(fresh.ensure(static_cast<size_t>(std::max(rows, 64)) * sizeof(double), s));
    if (g.tt_rows > 0)
      GW_CUDA(cudaMemcpyAsync(fresh.p, g.Wa_d.p, static_cast<size_t>(g.tt_rows) * sizeof(double),
                              cudaMemcpyDeviceToDevice, s));
    g.Wa_d.swap(fresh);
    GW_CUDA(cudaStreamSynchronize(s));
  }
  Workspace& ws = g.ws;
  GW_TRY(ensure_sweep_scratch(g, ws, 1, true, s));
  double* T = g.ttab.as<double>();
  double* dWa = g.Wa_d.as<double>();
  int32_t r0 = g.tt_rows;
  if (r0 == 0) {
    // t_0 = 1, stored scaled (t~_0 = s) on a weighted graph: the rows of the table are sweep inputs
    if (g.weighted) {
      GW_CUDA(cudaMemcpyAsync(T, g.rs_d.p, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    } else {
      fill_f64_kernel<<<grid_for(g.n), 256, 0, s>>>(T, g.n, 1.0);
      GW_KCHECK();
    }
    g.Wa.assign(1, static_cast<double>(g.n));
    fill_f64_kernel<<<1, 32, 0, s>>>(dWa, 1, static_cast<double>(g.n));
    GW_KCHECK();
    r0 = 1;
  }
  // t_r counts the walks that start at a vertex; on a directed graph batched scoring needs the
  // walks that end there (the sweeps' other orientation), so the table runs on the reverse CSR.
  // The totals W_r are the same either way.
  SweepArgs a = g.directed ? base_args_rev(g, ws) : base_args(g, ws);
  a.alpha = alpha;
  a.accumulate = 0;
  for (int32_t r = r0; r < rows; ++r) {
    a.X = T + static_cast<size_t>(r - 1) * n;
    a.Y = T + static_cast<size_t>(r) * n;
    if (g.n_active < g.n)  // isolated vertices start no walk of length >= 1
      GW_CUDA(cudaMemsetAsync(T + static_cast<size_t>(r) * n + g.n_active, 0,
                              sizeof(double) * (n - static_cast<size_t>(g.n_active)), s));
    GW_TRY(launch_sweep(MODE_TOTALS, true, 1, a, s));
    GW_TRY(reduce_slots(g, ws, 1, dWa + r, s, g.directed));
  }
  std::vector<double> tmp(rows);
  GW_CUDA(cudaMemcpyAsync(tmp.data() + r0, dWa + r0, sizeof(double) * (rows - r0), cudaMemcpyDeviceToHost, s));
  GW_CUDA(cudaStreamSynchronize(s));
  g.Wa.resize(rows);
  for (int32_t r = r0; r < rows; ++r) g.Wa[r] = tmp[r];
  g.tt_rows = rows;
  return GEDWALK_OK;
}

// ---------------------------------------------------------------- sigma_max by power iteration
// Statistics of one power step y = M x on the true vectors (a weighted graph stores s * x; the
// scale cancels in the ratio): per block the largest y(v)/x(v) over x(v) > 0 (Collatz-Wielandt),
// sum x(v) y(v), sum x(v)^2 and the largest y(v). rs: vertex scales or nullptr.
constexpr int kPiBlocks = 304;
__global__ void pi_stats_kernel(const double* __restrict__ X, const double* __restrict__ Y,
                                const double* __restrict__ rs, int32_t n, double* __restrict__ part) {
  double rmax = 0.0, num = 0.0, den = 0.0, ymax = 0.0;
  for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const double xs = X[v], ys = Y[v];
    if (!(xs > 0.0)) continue;  // a weighted vertex without edges (scale 0)
    rmax = fmax(rmax, ys / xs);
    const double sv = rs ? rs[v] : 1.0;
    const double x = xs / sv, y = ys / sv;
    num += x * y;
    den += x * x;
    ymax = fmax(ymax, y);
  }
  __shared__ double sm[4][256];
  sm[0][threadIdx.x] = rmax;
  sm[1][threadIdx.x] = num;
  sm[2][threadIdx.x] = den;
  sm[3][threadIdx.x] = ymax;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sm[0][threadIdx.x] = fmax(sm[0][threadIdx.x], sm[0][threadIdx.x + o]);
      sm[1][threadIdx.x] += sm[1][threadIdx.x + o];
      sm[2][threadIdx.x] += sm[2][threadIdx.x + o];
      sm[3][threadIdx.x] = fmax(sm[3][threadIdx.x], sm[3][threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x < 4) part[threadIdx.x * kPiBlocks + blockIdx.x] = sm[threadIdx.x][0];
}

// st = {smallest Collatz-Wielandt value so far, last Rayleigh quotient, normaliser for the next x}
__global__ void pi_finish_kernel(const double* __restrict__ part, double* __restrict__ st) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double rmax = 0.0, num = 0.0, den = 0.0, ymax = 0.0;
  for (int b = 0; b < kPiBlocks; ++b) {
    rmax = fmax(rmax, part[b]);
    num += part[kPiBlocks + b];
    den += part[2 * kPiBlocks + b];
    ymax = fmax(ymax, part[3 * kPiBlocks + b]);
  }
  st[0] = fmin(st[0], rmax);
  st[1] = den > 0.0 ? num / den : 0.0;
  st[2] = ymax > 0.0 ? ymax : 1.0;
}

// x <- y / ymax + tau (true values): positive everywhere, as the Collatz-Wielandt bound needs.
__global__ void pi_next_kernel(double* __restrict__ X, const double* __restrict__ Y, const double* __restrict__ rs,
                               int32_t n, const double* __restrict__ st, double tau) {
  const double inv = 1.0 / st[2];
  for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    X[v] = Y[v] * inv + tau * (rs ? rs[v] : 1.0);
}

__global__ void pi_init_kernel(double* __restrict__ X, double* __restrict__ Y, double* __restrict__ Z,
                               const double* __restrict__ rs, int32_t n, double* __restrict__ st) {
  for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    X[v] = rs ? rs[v] : 1.0;  // x = 1, stored scaled
    Y[v] = 0.0;               // rows without units are never written: they stay 0
    Z[v] = 0.0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st[0] = INFINITY;
    st[1] = 0.0;
    st[2] = 1.0;
  }
}

static gedwalk_status power_iteration(Graph& g, int32_t iters, cudaStream_t s) {
  Workspace& ws = g.ws;
  const size_t n = static_cast<size_t>(g.n);
  GW_TRY(ws.pvec.ensure((3 * n + 4 * kPiBlocks + 8) * sizeof(double), s));
  GW_TRY(ensure_sweep_scratch(g, ws, 1, true, s));
  double* X = ws.pvec.as<double>();
  double* Y = X + n;
  double* Z = Y + n;  // directed: A x before A^T
  double* part = Z + n;
  double* st = part + 4 * kPiBlocks;
  const double* rs = g.weighted ? g.rs_d.as<double>() : nullptr;
  pi_init_kernel<<<grid_for(g.n), 256, 0, s>>>(X, Y, Z, rs, g.n, st);
  GW_KCHECK();
  SweepArgs a = base_args(g, ws);
  a.alpha = 1.0;
  a.accumulate = 0;
  SweepArgs ar = g.directed ? base_args_rev(g, ws) : a;
  ar.alpha = 1.0;
  ar.accumulate = 0;
  for (int32_t it = 0; it < iters; ++it) {
    if (g.directed) {  // M = A^T A: sigma_max^2 = rho(M)
      a.X = X;
      a.Y = Z;
      GW_TRY(launch_sweep(MODE_TOTALS, true, 1, a, s, false));
      ar.X = Z;
      ar.Y = Y;
      GW_TRY(launch_sweep(MODE_TOTALS, true, 1, ar, s, false));
    } else {  // symmetric M = A: sigma_max = rho(A)
      a.X = X;
      a.Y = Y;
      GW_TRY(launch_sweep(MODE_TOTALS, true, 1, a, s, false));
    }
    pi_stats_kernel<<<kPiBlocks, 256, 0, s>>>(X, Y, rs, g.n, part);
    pi_finish_kernel<<<1, 32, 0, s>>>(part, st);
    pi_next_kernel<<<grid_for(g.n), 256, 0, s>>>(X, Y, rs, g.n, st, 1e-9);
    GW_KCHECK();
    count_launches(3);
  }
  double h[2];
  GW_CUDA(cudaMemcpyAsync(h, st, sizeof h, cudaMemcpyDeviceToHost, s));
  GW_CUDA(cudaStreamSynchronize(s));
  // rounding of the FP64 sums (at most d_max terms each) stays far below 1e-10 relative
  double up = h[0] * (1.0 + 1e-10), lo = h[1];
  if (g.directed) {
    up = std::sqrt(up);
    lo = std::sqrt(std::max(lo, 0.0));
  }
  if (g.sigma_up == 0.0 || up < g.sigma_up) g.sigma_up = up;
  g.sigma_lo = std::max(g.sigma_lo, lo);
  // cached spectral truncation lengths were found with the old sigma
  g.trunc_cache.erase(std::remove_if(g.trunc_cache.begin(), g.trunc_cache.end(),
                                     [](const Graph::Trunc& t) { return t.kind == GEDWALK_BOUND_SPECTRAL; }),
                      g.trunc_cache.end());
  return GEDWALK_OK;
}

gedwalk_status bound_coef(Graph& g, double alpha, int32_t kind, cudaStream_t s, double* coef) {
  if (kind == GEDWALK_BOUND_SPECTRAL) {
    if (g.sigma_up == 0.0) GW_TRY(power_iteration(g, 300, s));
    if (!(alpha * g.sigma_up < 1.0))
      return fail(GEDWALK_ERR_NOT_CONVERGENT,
                  "alpha * sigma_max = %g >= 1: the spectral bound needs alpha < 1/sigma_max (force L instead)",
                  alpha * g.sigma_up);
    // Lemma spectral-bound: B_l = sqrt(n) alpha sigma / (1 - alpha sigma) * alpha^l W_l
    *coef = std::sqrt(static_cast<double>(g.n)) * alpha * g.sigma_up / (1.0 - alpha * g.sigma_up);
    return GEDWALK_OK;
  }
  if (kind != GEDWALK_BOUND_COMBINATORIAL) return fail(GEDWALK_ERR_INVALID, "unknown bound kind %d", kind);
  if (!(alpha * g.delta < 1.0))
    return fail(GEDWALK_ERR_NOT_CONVERGENT,
                "alpha * d_max = %g >= 1: the combinatorial bound needs alpha < 1/d_max (force L instead)",
                alpha * g.delta);
  *coef = alpha * g.delta / (1.0 - alpha * g.delta);
  return GEDWALK_OK;
}

gedwalk_status truncation_length(Graph& g, double alpha, double eps, int32_t* L, double* bound, cudaStream_t s,
                                 int32_t kind) {
  if (!(alpha > 0.0) || !std::isfinite(alpha)) return fail(GEDWALK_ERR_INVALID, "alpha must be positive");
  if (!(eps > 0.0)) return fail(GEDWALK_ERR_INVALID, "epsilon must be positive");
  double coef = 0.0;
  GW_TRY(bound_coef(g, alpha, kind, s, &coef));
  for (const Graph::Trunc& t : g.trunc_cache)  // L depends only on (graph, alpha, epsilon, bound)
    if (t.alpha == alpha && t.eps == eps && t.kind == kind) {
      *L = t.L;
      if (bound) *bound = t.bound;
      return GEDWALK_OK;
    }
  const int32_t kCap = 4096;
  int32_t rows = std::max(g.tt_alpha == alpha ? g.tt_rows : 0, 4);
  Workspace& ws = g.ws;
  for (;;) {
    GW_TRY(ensure_totals(g, alpha, rows, s));
    GW_TRY(ws.small.ensure(64, s));
    // the stop test reads the row sums where the sweeps' reductions left them
    double* db = ws.small.as<double>();
    int32_t* dl = reinterpret_cast<int32_t*>(db + 1);
    first_crossing_kernel<<<1, 32, 0, s>>>(g.Wa_d.as<double>(), 1, rows, coef, eps, dl, db);
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
      g.trunc_cache.push_back({alpha, eps, hl, hb, kind});
      return GEDWALK_OK;
    }
    if (rows >= kCap) return fail(GEDWALK_ERR_INVALID, "no truncation length <= %d reaches epsilon %g", kCap, eps);
    // B_l = coef W_l shrinks about geometrically once the walks spread: predict the first l below
    // eps from the last ratio W_{l}/W_{l-1}, so that few rows beyond L are computed (each row is
    // one FP64 sweep); without a shrinking ratio, double
    int32_t next = std::min(rows * 2, kCap);
    const double w1 = g.Wa[rows - 1], w0 = g.Wa[rows - 2], b1 = coef * w1;
    if (w0 > 0.0 && w1 > 0.0 && w1 < w0 && b1 > 0.0 && std::isfinite(b1)) {
      const double m = std::ceil(std::log(eps / b1) / std::log(w1 / w0));
      if (m >= 1.0 && m < kCap) next = static_cast<int32_t>(std::min<double>(kCap, rows + m));
    }
    rows = std::max(rows + 1, next);
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
  r->lookahead = p->lookahead;
  r->spec_cols = p->spec_cols;
  if (p->bound != GEDWALK_BOUND_COMBINATORIAL && p->bound != GEDWALK_BOUND_SPECTRAL)
    return fail(GEDWALK_ERR_INVALID, "bound must be GEDWALK_BOUND_COMBINATORIAL or GEDWALK_BOUND_SPECTRAL");
  r->bound_kind = p->bound;
  if (p->L < 0) return fail(GEDWALK_ERR_INVALID, "L must be >= 0");
  if (p->L > 0) {
    if (p->L > 4096) return fail(GEDWALK_ERR_INVALID, "L must be <= 4096");
    r->L = p->L;
    r->bound = NAN;
    double coef = 0.0;
    if (bound_coef(g, r->alpha, p->bound, r->stream, &coef) == GEDWALK_OK) {
      GW_TRY(ensure_totals(g, r->alpha, p->L + 1, r->stream));
      r->bound = coef * g.Wa[p->L];
    }
    return GEDWALK_OK;
  }
  const double eps = eps_override > 0.0 ? eps_override : p->epsilon;
  r->eps = eps;
  return truncation_length(g, r->alpha, eps, &r->L, &r->bound, r->stream, p->bound);
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
  p->bound = GEDWALK_BOUND_COMBINATORIAL;
  p->lookahead = 0;
  p->spec_cols = 0;
  p->reserved = 0;
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

static gedwalk_status upload_impl(const int32_t* row_ptr, const int32_t* col_idx, int32_t n, int64_t nnz,
                                  int32_t flags, bool weighted, const double* vertex_scale, gedwalk_graph_t* out) {
  if (!out) return fail(GEDWALK_ERR_INVALID, "out is NULL");
  if (n < 1) return fail(GEDWALK_ERR_INVALID, "n must be >= 1");
  if (nnz < 0 || nnz >= (int64_t(1) << 31) - 8) return fail(GEDWALK_ERR_INVALID, "nnz must be in [0, 2^31 - 8)");
  if (!row_ptr || (nnz > 0 && !col_idx)) return fail(GEDWALK_ERR_INVALID, "row_ptr/col_idx is NULL");
  const bool directed = (flags & GEDWALK_UPLOAD_DIRECTED) != 0;
  if (directed && weighted) return fail(GEDWALK_ERR_INVALID, "weighted directed graphs are not supported");
  std::string why;
  const bool trusted = (flags & GEDWALK_UPLOAD_TRUSTED) != 0;
  int32_t dmax = 0;  // the largest row length (found while the row pointers are checked)
  // the caller's CSR on the device: validated there, then relabelled there
  DevBuf raw_rp, raw_ci;
  GW_TRY(raw_rp.ensure((static_cast<size_t>(n) + 1) * sizeof(int32_t), 0));
  GW_TRY(raw_ci.ensure(std::max<size_t>(static_cast<size_t>(nnz), 1) * sizeof(int32_t), 0));
  GW_CUDA(cudaMemcpy(raw_rp.p, row_ptr, (static_cast<size_t>(n) + 1) * sizeof(int32_t), cudaMemcpyHostToDevice));
  if (nnz > 0)
    GW_CUDA(cudaMemcpy(raw_ci.p, col_idx, static_cast<size_t>(nnz) * sizeof(int32_t), cudaMemcpyHostToDevice));
  {
    // row_ptr and index ranges are always checked (the plan and the kernels index with
    // them); TRUSTED skips the sortedness, self-loop and symmetry checks
    gedwalk_status vst = GEDWALK_OK;
    const int64_t bad = validate_csr(row_ptr, raw_rp.as<int32_t>(), raw_ci.as<int32_t>(), n, nnz, !trusted, &why,
                                     !directed, &vst, &dmax);
    if (vst != GEDWALK_OK) return vst;
    if (bad >= 0)
      return fail(GEDWALK_ERR_INVALID, "malformed graph at row %lld: %s", static_cast<long long>(bad), why.c_str());
  }
  std::unique_ptr<Graph> g(new Graph());
  GW_CUDA(cudaGetDevice(&g->device));
  g->n = n;
  g->nnz = nnz;
  g->directed = directed;
  // degrees by caller id (weighted and directed graphs): the rows' own lengths; for a directed
  // graph also the reverse (in) degree
  std::vector<int32_t> deg_old, rdeg_old;
  if (weighted || directed) {
    deg_old.resize(n);
    for (int32_t v = 0; v < n; ++v) deg_old[v] = row_ptr[v + 1] - row_ptr[v];
  }
  int32_t rdmax = 0;
  if (directed) {
    rdeg_old.assign(n, 0);
    for (int64_t j = 0; j < nnz; ++j) rdeg_old[col_idx[j]]++;
    for (int32_t v = 0; v < n; ++v) rdmax = std::max(rdmax, rdeg_old[v]);
  }
  g->dmax = dmax;
  // W_{l+1} <= d W_l with d = d_max; on a digraph an l-walk extends at its end along at most
  // max out-degree arcs and at its start along at most max in-degree arcs, so the smaller counts
  g->delta = directed ? std::min(dmax, rdmax) : dmax;
  std::vector<double> scale;  // caller order
  if (weighted) {
    // w(v,u) = s_v s_u; without scales the symmetrically normalised adjacency D^{-1/2} A D^{-1/2}
    // (Section 5.4), s_v = deg(v)^{-1/2} (0 for a vertex without edges, which no walk visits)
    scale.resize(n);
    for (int32_t v = 0; v < n; ++v) {
      if (vertex_scale) {
        if (!(vertex_scale[v] > 0.0) || !std::isfinite(vertex_scale[v]))
          return fail(GEDWALK_ERR_INVALID, "vertex_scale[%d] = %g must be positive and finite", v, vertex_scale[v]);
        scale[v] = vertex_scale[v];
      } else {
        scale[v] = deg_old[v] > 0 ? 1.0 / std::sqrt(static_cast<double>(deg_old[v])) : 0.0;
      }
    }
    // the degree of the combinatorial bound: the largest weighted degree s_v sum_u s_u
    double delta = 0.0;
    for (int32_t v = 0; v < n; ++v) {
      double acc = 0.0;
      for (int64_t j = row_ptr[v]; j < row_ptr[v + 1]; ++j) acc += scale[col_idx[j]];
      delta = std::max(delta, scale[v] * acc);
    }
    g->delta = delta;
    g->weighted = true;
  }
  g->alpha_default = 1.0 / (1.0 + g->delta);
  // relabel: decreasing degree, ties by (directed) decreasing reverse degree, then caller id. A
  // vertex with no arc at all sorts last, so the isolated rows form the tail.
  g->perm.resize(n);
  g->inv.resize(n);
  std::vector<int32_t> rp(static_cast<size_t>(n) + 1);
  GW_TRY(g->rp.ensure(rp.size() * sizeof(int32_t), 0));
  const size_t ci_len = static_cast<size_t>(nnz) + 4;  // 4 zero pad entries for the vector loads at the end
  GW_TRY(g->ci.ensure(ci_len * sizeof(int32_t), 0));
  GW_TRY(g->perm_d.ensure(static_cast<size_t>(n) * sizeof(int32_t), 0));
  DevBuf inv_d;
  GW_TRY(inv_d.ensure(static_cast<size_t>(n) * sizeof(int32_t), 0));
  if (!directed) {
    // on the device: a stable radix sort by degree, the inverse, the new degrees and row pointers
    DevBuf deg_d;
    GW_TRY(deg_d.ensure(static_cast<size_t>(n) * sizeof(int32_t), 0));
    GW_TRY(degree_order(raw_rp.as<int32_t>(), n, dmax, g->perm_d.as<int32_t>(), inv_d.as<int32_t>(),
                        deg_d.as<int32_t>(), g->rp.as<int32_t>()));
    GW_CUDA(cudaMemcpy(g->perm.data(), g->perm_d.p, static_cast<size_t>(n) * sizeof(int32_t), cudaMemcpyDeviceToHost));
    GW_CUDA(cudaMemcpy(g->inv.data(), inv_d.p, static_cast<size_t>(n) * sizeof(int32_t), cudaMemcpyDeviceToHost));
    GW_CUDA(cudaMemcpy(rp.data(), g->rp.p, rp.size() * sizeof(int32_t), cudaMemcpyDeviceToHost));
  } else {
    g->deg.resize(n);
    for (int32_t v = 0; v < n; ++v) g->perm[v] = v;
    std::stable_sort(g->perm.begin(), g->perm.end(), [&](int32_t a, int32_t b) {
      if (deg_old[a] != deg_old[b]) return deg_old[a] > deg_old[b];
      return rdeg_old[a] > rdeg_old[b];
    });
    for (int32_t i = 0; i < n; ++i) g->inv[g->perm[i]] = i;
    rp[0] = 0;
    for (int32_t i = 0; i < n; ++i) {
      g->deg[i] = deg_old[g->perm[i]];
      rp[i + 1] = rp[i] + g->deg[i];
    }
    GW_CUDA(cudaMemcpy(g->rp.p, rp.data(), rp.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    GW_CUDA(cudaMemcpy(g->perm_d.p, g->perm.data(), static_cast<size_t>(n) * sizeof(int32_t), cudaMemcpyHostToDevice));
    GW_CUDA(cudaMemcpy(inv_d.p, g->inv.data(), static_cast<size_t>(n) * sizeof(int32_t), cudaMemcpyHostToDevice));
  }
  // rows from n_active on are isolated: no entry in either direction
  g->n_active = n;
  if (!directed) {
    g->n_active = first_row(0, n, [&](int32_t i) { return rp[i + 1] == rp[i]; });
  } else {
    while (g->n_active > 0 && g->deg[g->n_active - 1] == 0 && rdeg_old[g->perm[g->n_active - 1]] == 0) --g->n_active;
  }
  {
    GW_CUDA(cudaMemset(g->ci.as<int32_t>() + nnz, 0, 4 * sizeof(int32_t)));
    const int64_t blocks = std::min<int64_t>((static_cast<int64_t>(n) * 32 + 255) / 256, 152 * 32);
    relabel_kernel<<<static_cast<int>(blocks), 256>>>(raw_rp.as<int32_t>(), raw_ci.as<int32_t>(), g->rp.as<int32_t>(),
                                                      g->perm_d.as<int32_t>(), inv_d.as<int32_t>(), n,
                                                      g->ci.as<int32_t>());
    GW_KCHECK();
    // sort each row by new id: the rows are ordered by decreasing degree, so the rows above
    // kSortSeg entries (sorted as 1024-entry pieces) are a prefix, and the others are sorted whole
    const int32_t n_long = first_row(0, g->n_active, [&](int32_t i) { return rp[i + 1] - rp[i] <= kSortSeg; });
    std::vector<int2> seg;
    for (int32_t i = 0; i < n_long; ++i)
      for (int32_t b = rp[i]; b < rp[i + 1]; b += kSortSeg) seg.push_back(make_int2(b, std::min(kSortSeg, rp[i + 1] - b)));
    DevBuf seg_d;
    GW_TRY(seg_d.ensure(std::max<size_t>(seg.size(), 1) * sizeof(int2), 0));
    if (!seg.empty())
      GW_CUDA(cudaMemcpy(seg_d.p, seg.data(), seg.size() * sizeof(int2), cudaMemcpyHostToDevice));
    const int64_t work = static_cast<int64_t>(seg.size()) + (g->n_active - n_long);
    if (work > 0) {
      const int64_t sblocks = std::min<int64_t>((work * 32 + 255) / 256, 152 * 32);
      sort_segments_kernel<<<static_cast<int>(sblocks), 256>>>(seg_d.as<int2>(), static_cast<int64_t>(seg.size()),
                                                               g->rp.as<int32_t>(), n_long, g->n_active,
                                                               g->ci.as<int32_t>());
      GW_KCHECK();
    }
    GW_CUDA(cudaDeviceSynchronize());
  }
  raw_ci.release();
  raw_rp.release();
  if (weighted) {
    std::vector<double> sd(n);
    std::vector<float> sf(n);
    for (int32_t i = 0; i < n; ++i) {
      sd[i] = scale[g->perm[i]];
      sf[i] = static_cast<float>(sd[i]);
    }
    GW_TRY(g->rs_d.ensure(static_cast<size_t>(n) * sizeof(double), 0));
    GW_TRY(g->rs_f.ensure(static_cast<size_t>(n) * sizeof(float), 0));
    GW_CUDA(cudaMemcpy(g->rs_d.p, sd.data(), sd.size() * sizeof(double), cudaMemcpyHostToDevice));
    GW_CUDA(cudaMemcpy(g->rs_f.p, sf.data(), sf.size() * sizeof(float), cudaMemcpyHostToDevice));
  }
  GW_TRY(build_plan(g->plan, g->deg, rp, g->n_active, n, true));
  if (directed) {
    // the reverse CSR (row v: the u with an arc u -> v), same ids, rows sorted
    g->deg_r.assign(n, 0);
    for (int32_t i = 0; i < n; ++i) g->deg_r[i] = rdeg_old[g->perm[i]];
    std::vector<int32_t> rpr(static_cast<size_t>(n) + 1, 0);
    for (int32_t i = 0; i < n; ++i) rpr[i + 1] = rpr[i] + g->deg_r[i];
    std::vector<int32_t> cir(static_cast<size_t>(nnz) + 4, 0);
    std::vector<int32_t> fill(rpr.begin(), rpr.end() - 1);
    for (int32_t i = 0; i < n; ++i) {  // rows i in increasing order: every reverse row comes out sorted
      const int32_t v = g->perm[i];
      for (int32_t j = row_ptr[v]; j < row_ptr[v + 1]; ++j) cir[fill[g->inv[col_idx[j]]]++] = i;
    }
    GW_TRY(g->rp_r.ensure(rpr.size() * sizeof(int32_t), 0));
    GW_TRY(g->ci_r.ensure(cir.size() * sizeof(int32_t), 0));
    GW_CUDA(cudaMemcpy(g->rp_r.p, rpr.data(), rpr.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    GW_CUDA(cudaMemcpy(g->ci_r.p, cir.data(), cir.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    GW_TRY(build_plan(g->plan_r, g->deg_r, rpr, g->n_active, n, false));
  }
  *out = reinterpret_cast<gedwalk_graph_t>(g.release());
  return GEDWALK_OK;
}

gedwalk_status gedwalk_graph_upload(const int32_t* row_ptr, const int32_t* col_idx, int32_t n, int64_t nnz,
                                    int32_t flags, gedwalk_graph_t* out) {
  return upload_impl(row_ptr, col_idx, n, nnz, flags, false, nullptr, out);
}

gedwalk_status gedwalk_graph_upload_weighted(const int32_t* row_ptr, const int32_t* col_idx, int32_t n, int64_t nnz,
                                             const double* vertex_scale, int32_t flags, gedwalk_graph_t* out) {
  return upload_impl(row_ptr, col_idx, n, nnz, flags, true, vertex_scale, out);
}

gedwalk_status gedwalk_graph_info_weighted(gedwalk_graph_t h, int32_t* weighted, double* delta) {
  if (!h) return fail(GEDWALK_ERR_INVALID, "graph is NULL");
  Graph* g = G(h);
  if (weighted) *weighted = g->weighted ? 1 : 0;
  if (delta) *delta = g->delta;
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

gedwalk_status gedwalk_truncation_ex(gedwalk_graph_t h, double alpha, double epsilon, int32_t bound_kind, int32_t* L,
                                     double* bound) {
  if (!h || !L) return fail(GEDWALK_ERR_INVALID, "graph or L is NULL");
  Graph* g = G(h);
  std::lock_guard<std::mutex> lk(g->mu);
  GW_CUDA(cudaSetDevice(g->device));
  if (alpha < 0.0 || std::isnan(alpha)) return fail(GEDWALK_ERR_INVALID, "alpha must be positive (0 = default)");
  if (alpha == 0.0) alpha = g->alpha_default;
  double b = 0;
  int32_t l = 0;
  GW_TRY(truncation_length(*g, alpha, epsilon, &l, &b, 0, bound_kind));
  *L = l;
  if (bound) *bound = b;
  return GEDWALK_OK;
}

gedwalk_status gedwalk_sigma_max(gedwalk_graph_t h, int32_t iters, double* upper, double* lower) {
  if (!h) return fail(GEDWALK_ERR_INVALID, "graph is NULL");
  if (iters < 1 || iters > 100000) return fail(GEDWALK_ERR_INVALID, "iters must be in [1, 100000]");
  Graph* g = G(h);
  std::lock_guard<std::mutex> lk(g->mu);
  GW_CUDA(cudaSetDevice(g->device));
  GW_TRY(power_iteration(*g, iters, 0));
  if (upper) *upper = g->sigma_up;
  if (lower) *lower = g->sigma_lo;
  return GEDWALK_OK;
}

}  // extern "C"
