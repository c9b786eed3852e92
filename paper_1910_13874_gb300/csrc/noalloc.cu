// Allocation-free variant of the two-state scoring sweep.
//
// Some callers cannot allocate device memory at all: code that runs after its
// framework has handed every byte of the GPU to its own pool, or embedded services
// that forbid allocation (and its latency or failure) once they are serving. For
// them gedwalk_score_step_noalloc runs one step of the two-state hit/miss
// recurrence on device buffers the caller already owns. The only scratch it needs,
// the per-warp FP64 partial sums of the hit column, lives in the file-scope array
// below, which every GPU that loads this library holds until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "internal.h"

namespace gw {
namespace {

constexpr int kNaWarps = kThreads / 32;
constexpr int kNaRowsPerWarp = 256;
constexpr int kNaRowsPerBlock = kNaRowsPerWarp * kNaWarps;  // 2048
constexpr int kNaMaxBlocks = 8192;
constexpr int kNaSlots = kNaMaxBlocks * kNaWarps;           // 65,536 doubles = 512 KiB
constexpr int64_t kNaMaxRows = int64_t(kNaRowsPerBlock) * kNaMaxBlocks;  // 16,777,216
constexpr int kNaMaxDevices = 64;

// One FP64 partial sum per warp of the largest launch. Shared by every call on a device:
// each call overwrites every slot it reads, so nothing has to start at zero.
static __device__ __align__(256) double g_na_slots[kNaSlots];

std::mutex g_na_mu;
double* g_na_ptr[kNaMaxDevices] = {};  // device address of g_na_slots, per device

// One step of Section 3.1.1 on x = (hit, miss) pairs, one warp per row:
//   hit'(v)  = alpha (sum_{u~v} hit(u) + [v in S] sum_{u~v} miss(u))
//   miss'(v) = alpha [v not in S] sum_{u~v} miss(u)
// Warp w writes sum over its rows of hit'(v) to slots[w].
__global__ void __launch_bounds__(kThreads) na_step(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                                   int32_t n, const uint32_t* __restrict__ mask,
                                                   const float2* __restrict__ x, float2* __restrict__ y, float alpha,
                                                   double* __restrict__ slots) {
  const int lane = threadIdx.x & 31;
  const int warp = blockIdx.x * kNaWarps + (threadIdx.x >> 5);
  const int64_t r0 = int64_t(warp) * kNaRowsPerWarp;
  double cs = 0.0;
  for (int64_t r = r0; r < r0 + kNaRowsPerWarp && r < n; ++r) {
    const int32_t e0 = rp[r], e1 = rp[r + 1];
    float sh = 0.0f, sm = 0.0f;
    for (int32_t j = e0 + lane; j < e1; j += 32) {
      const float2 v = __ldg(x + ci[j]);
      sh += v.x;
      sm += v.y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      sh += __shfl_xor_sync(0xffffffffu, sh, o);
      sm += __shfl_xor_sync(0xffffffffu, sm, o);
    }
    if (lane == 0) {
      const bool inS = (mask[r >> 5] >> (r & 31)) & 1u;
      const float h = alpha * (inS ? sh + sm : sh);
      const float m = inS ? 0.0f : alpha * sm;
      y[r] = make_float2(h, m);
      cs += static_cast<double>(h);
    }
  }
  if (lane == 0) slots[warp] = cs;
}

// out = sum of slots[0..count) in a fixed order (one CTA).
__global__ void __launch_bounds__(kThreads) na_reduce(const double* __restrict__ slots, int32_t count,
                                                     double* __restrict__ out) {
  __shared__ double sm[kNaWarps];
  double v = 0.0;
  for (int i = threadIdx.x; i < count; i += kThreads) v += slots[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = sm[0];
    for (int w = 1; w < kNaWarps; ++w) s += sm[w];
    *out = s;
  }
}

// Device address of the scratch array on the current device; looked up once per device.
gedwalk_status na_scratch(double** out) {
  int dev = 0;
  GW_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNaMaxDevices) return fail(GEDWALK_ERR_INVALID, "device %d not supported", dev);
  std::lock_guard<std::mutex> lk(g_na_mu);
  if (!g_na_ptr[dev]) {
    double* p = nullptr;
    GW_CUDA(cudaGetSymbolAddress(reinterpret_cast<void**>(&p), g_na_slots));
    g_na_ptr[dev] = p;
  }
  *out = g_na_ptr[dev];
  return GEDWALK_OK;
}

}  // namespace
}  // namespace gw

using namespace gw;

extern "C" gedwalk_status gedwalk_score_step_noalloc(const int32_t* d_row_ptr, const int32_t* d_col_idx, int32_t n,
                                                     const uint32_t* d_mask, const float* d_x, float* d_y,
                                                     double alpha, double* d_hit_sum, int64_t stream) {
  if (!d_row_ptr || !d_col_idx || !d_mask || !d_x || !d_y || !d_hit_sum)
    return fail(GEDWALK_ERR_INVALID, "gedwalk_score_step_noalloc: a device pointer is NULL");
  if (n < 1 || int64_t(n) > kNaMaxRows)
    return fail(GEDWALK_ERR_INVALID,
                "gedwalk_score_step_noalloc: n = %d outside [1, %lld]: its fixed scratch holds partial sums for "
                "at most %lld rows",
                n, static_cast<long long>(kNaMaxRows), static_cast<long long>(kNaMaxRows));
  if (!(alpha > 0.0)) return fail(GEDWALK_ERR_INVALID, "gedwalk_score_step_noalloc: alpha must be positive");
  if ((reinterpret_cast<uintptr_t>(d_x) | reinterpret_cast<uintptr_t>(d_y) | reinterpret_cast<uintptr_t>(d_hit_sum)) &
      7u)
    return fail(GEDWALK_ERR_INVALID, "gedwalk_score_step_noalloc: x, y and hit_sum must be 8-byte aligned");
  double* slots = nullptr;
  GW_TRY(na_scratch(&slots));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int blocks = static_cast<int>((int64_t(n) + kNaRowsPerBlock - 1) / kNaRowsPerBlock);
  na_step<<<blocks, kThreads, 0, s>>>(d_row_ptr, d_col_idx, n, d_mask, reinterpret_cast<const float2*>(d_x),
                                      reinterpret_cast<float2*>(d_y), static_cast<float>(alpha), slots);
  GW_KCHECK();
  na_reduce<<<1, kThreads, 0, s>>>(slots, blocks * kNaWarps, d_hit_sum);
  GW_KCHECK();
  return GEDWALK_OK;
}
