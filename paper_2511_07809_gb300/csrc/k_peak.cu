// FP32 CUDA-core throughput probe: the denominator of the "alu" roofline of
// the FP32 plain form.  Each thread runs kChains independent FMA chains
// (enough independent work per warp to cover the FMA latency at full
// occupancy), so the SMs issue FFMA back to back.  The caller times the
// launch with CUDA events on the same stream and divides the flop count this
// entry point reports by the elapsed time.
#include "tlda_internal.h"

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_ffma_probe(int iters, float *sink) {
  float v[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) v[j] = 1.0f + 1e-3f * (float)(threadIdx.x + j);
  // multiplier and addend chosen so the chains neither overflow nor collapse
  // to a constant over ~1e6 steps, and the compiler cannot fold them
  const float m = 0.99999988f + 1e-9f * (float)(blockIdx.x & 7);
  const float c = 1e-7f;
#pragma unroll 1
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int j = 0; j < kChains; ++j) v[j] = fmaf(v[j], m, c);
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += v[j];
  if (s == -1.0f) sink[blockIdx.x] = s;  // never true; keeps the chains live
}

}  // namespace

extern "C" tlda_status tlda_ffma_probe(int32_t iters, float *sink, double *flops_out, void *cuda_stream) {
  if (iters < 1 || !sink || !flops_out) return TLDA_ERR_INVALID;
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ffma_probe, kThreads, 0) != cudaSuccess ||
      per_sm < 1)
    return TLDA_ERR_CUDA;
  const int grid = sms * per_sm;
  k_ffma_probe<<<grid, kThreads, 0, static_cast<cudaStream_t>(cuda_stream)>>>(iters, sink);
  *flops_out = 2.0 * (double)grid * kThreads * (double)iters * kUnroll * kChains;
  return cudaGetLastError() == cudaSuccess ? TLDA_OK : TLDA_ERR_CUDA;
}
