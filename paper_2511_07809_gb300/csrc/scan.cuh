// In-place prefix sums of int32 counts on the device: x[0] = 0 stays and
// x[1 .. n] become their inclusive running sums, so a count array stored at
// x[i + 1] turns into offsets.  Three launches: per-block scans (warp shuffles,
// then the warps' totals), the block totals scanned by one thread (int64),
// the block offsets added.  The total comes back in *total (device, int64).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace {

constexpr int kScanThreads = 1024;

__global__ void __launch_bounds__(kScanThreads) k_scan_local(int32_t *x, int n, int64_t *bsum) {
  __shared__ int32_t wsum[kScanThreads / 32];
  const int i = 1 + blockIdx.x * kScanThreads + threadIdx.x, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int32_t v = i <= n ? x[i] : 0;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t y = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += y;
  }
  if (lane == 31) wsum[w] = v;
  __syncthreads();
  if (w == 0) {
    int32_t s = wsum[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    wsum[lane] = s;
  }
  __syncthreads();
  if (w > 0) v += wsum[w - 1];
  if (i <= n) x[i] = v;
  if (threadIdx.x == kScanThreads - 1) bsum[blockIdx.x] = v;
}

__global__ void k_scan_top(int64_t *bsum, int nb, int64_t *total) {
  if (threadIdx.x == 0) {
    int64_t run = 0;
    for (int b = 0; b < nb; ++b) {
      const int64_t v = bsum[b];
      bsum[b] = run;
      run += v;
    }
    *total = run;
  }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_add(int32_t *x, int n, const int64_t *bsum) {
  const int i = 1 + blockIdx.x * kScanThreads + threadIdx.x;
  if (i <= n) x[i] = (int32_t)(x[i] + bsum[blockIdx.x]);
}

// Blocks of int64 scratch a scan of n counts needs (their totals).
inline int scan_blocks(int n) { return (n + kScanThreads - 1) / kScanThreads; }

// Enqueues the scan of x[1 .. n]; bsum: scan_blocks(n) int64, total: 1 int64.
inline void scan_counts(int32_t *x, int n, int64_t *bsum, int64_t *total, cudaStream_t s) {
  const int nb = scan_blocks(n);
  k_scan_local<<<nb, kScanThreads, 0, s>>>(x, n, bsum);
  k_scan_top<<<1, 32, 0, s>>>(bsum, nb, total);
  k_scan_add<<<nb, kScanThreads, 0, s>>>(x, n, bsum);
}

}  // namespace
