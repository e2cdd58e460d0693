// Document-topic proportions by variational inference with the topics fixed
// (section "Input and Output": the recovered topic-word matrix and weights
// feed a standard VI; the per-document E-step of Blei, Ng and Jordan 2003,
// section 5.2).  One warp per document, the document's K topics spread over
// the lanes (K/32 each, rounded up to a power of two), FP32 throughout.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "tlda.h"
#include "tlda_internal.h"

namespace {

constexpr int kViThreads = 256;

// digamma(x) for x > 0: below 6 the recurrence psi(x) = psi(x + 6) -
// sum_{i<6} 1/(x + i), the six reciprocals summed as one fraction (pairs
// (a, b) -> (a + b, a b)) and divided once; then the asymptotic series
// ln x - 1/(2x) - sum B_2n / (2n x^2n) (Abramowitz and Stegun 6.3.18)
// through the x^-8 term, whose next term is below 2e-10 at x = 6.
__device__ __forceinline__ float digamma_f(float x) {
  float r = 0.f;
  if (x < 6.f) {
    const float a0 = x, a1 = x + 1.f, a2 = x + 2.f, a3 = x + 3.f, a4 = x + 4.f, a5 = x + 5.f;
    const float n01 = a0 + a1, d01 = a0 * a1, n23 = a2 + a3, d23 = a2 * a3, n45 = a4 + a5, d45 = a4 * a5;
    const float n = fmaf(n01, d23, n23 * d01), d = d01 * d23;
    r = -fmaf(n, d45, n45 * d) / (d * d45);
    x += 6.f;
  }
  const float ix = 1.f / x, ix2 = ix * ix;
  const float series = ix2 * (1.f / 12.f - ix2 * (1.f / 120.f - ix2 * (1.f / 252.f - ix2 * (1.f / 240.f))));
  return r + __logf(x) - 0.5f * ix - series;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// KPL topics per lane: topic k = lane + 32 t.  exp(digamma) is taken relative
// to its largest value over the topics, which the per-word normalisation
// cancels, so small gamma never underflows every topic at once.
template <int KPL>
__global__ void __launch_bounds__(kViThreads) k_doc_topics(tlda_csr docs, const float *__restrict__ mu,
                                                          const float *__restrict__ alpha, int K, int n_iter,
                                                          float *__restrict__ theta, float *__restrict__ gamma_out,
                                                          int32_t *err) {
  const int doc = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (doc >= docs.n_docs) return;
  const long long p0 = docs.indptr[doc], p1 = docs.indptr[doc + 1];
  float a[KPL], g[KPL], e[KPL], acc[KPL];
#pragma unroll
  for (int t = 0; t < KPL; ++t) {
    const int k = lane + 32 * t;
    a[t] = k < K ? alpha[k] : 0.f;
  }
  // validation and the document length
  bool bad = p0 < 0 || p1 < p0;
  long long L = 0;
  if (!bad)
    for (long long p = p0 + lane; p < p1; p += 32) {
      const int m = docs.indices[p], f = docs.counts[p];
      if (m < 0 || m >= docs.vocab || f <= 0) bad = true;
      else L += f;
    }
  if (__any_sync(0xffffffffu, bad)) {
    if (lane == 0 && err) atomicOr(err, 1);
#pragma unroll
    for (int t = 0; t < KPL; ++t) {
      const int k = lane + 32 * t;
      if (k < K) {
        theta[(long long)doc * K + k] = __int_as_float(0x7fc00000);
        if (gamma_out) gamma_out[(long long)doc * K + k] = __int_as_float(0x7fc00000);
      }
    }
    return;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) L += __shfl_xor_sync(0xffffffffu, L, o);
  const float l_over_k = (float)L / (float)K;
#pragma unroll
  for (int t = 0; t < KPL; ++t) g[t] = a[t] + l_over_k;

  for (int it = 0; it < n_iter; ++it) {
    float mx = -INFINITY;
#pragma unroll
    for (int t = 0; t < KPL; ++t) {
      const int k = lane + 32 * t;
      e[t] = k < K ? digamma_f(g[t]) : -INFINITY;
      mx = fmaxf(mx, e[t]);
    }
    mx = warp_max(mx);
#pragma unroll
    for (int t = 0; t < KPL; ++t) {
      const int k = lane + 32 * t;
      e[t] = k < K ? __expf(e[t] - mx) : 0.f;
      acc[t] = a[t];
    }
    for (long long q0 = p0; q0 < p1; q0 += 32) {
      const int n = (int)min(32ll, p1 - q0);
      const int mj = lane < n ? docs.indices[q0 + lane] : 0;
      const float fj = lane < n ? (float)docs.counts[q0 + lane] : 0.f;
      for (int i = 0; i < n; ++i) {
        const int m = __shfl_sync(0xffffffffu, mj, i);
        const float f = __shfl_sync(0xffffffffu, fj, i);
        const float *row = mu + (long long)m * K;
        float pv[KPL], s = 0.f;
#pragma unroll
        for (int t = 0; t < KPL; ++t) {
          const int k = lane + 32 * t;
          pv[t] = k < K ? __ldg(row + k) * e[t] : 0.f;
          s += pv[t];
        }
        s = warp_sum(s);
        if (s > 0.f) {
          const float w = __fdividef(f, s);
          if (w <= 3.0e38f) {
#pragma unroll
            for (int t = 0; t < KPL; ++t) acc[t] = fmaf(pv[t], w, acc[t]);
          } else {  // s below f / FLT_MAX (subnormal rows): divide first, pv <= s
#pragma unroll
            for (int t = 0; t < KPL; ++t) acc[t] = fmaf(pv[t] / s, f, acc[t]);
          }
        }
      }
    }
#pragma unroll
    for (int t = 0; t < KPL; ++t) g[t] = acc[t];
  }
  float tot = 0.f;
#pragma unroll
  for (int t = 0; t < KPL; ++t) tot += (lane + 32 * t < K) ? g[t] : 0.f;
  tot = warp_sum(tot);
  const float inv = 1.f / tot;
#pragma unroll
  for (int t = 0; t < KPL; ++t) {
    const int k = lane + 32 * t;
    if (k < K) {
      theta[(long long)doc * K + k] = g[t] * inv;
      if (gamma_out) gamma_out[(long long)doc * K + k] = g[t];
    }
  }
}

template <int KPL>
void launch(const tlda_csr &d, const float *mu, const float *alpha, int K, int n_iter, float *theta, float *gamma,
            int32_t *err, cudaStream_t s) {
  const long long threads = (long long)d.n_docs * 32;
  k_doc_topics<KPL><<<(unsigned)((threads + kViThreads - 1) / kViThreads), kViThreads, 0, s>>>(
      d, mu, alpha, K, n_iter, theta, gamma, err);
}

}  // namespace

extern "C" tlda_status tlda_doc_topics(const tlda_csr *docs, const float *mu, const float *alpha, int32_t K,
                                       int32_t n_iter, float *theta_out, float *gamma_out, int32_t *err_out,
                                       void *cuda_stream) {
  TLDA_RANGE();
  if (!docs || !mu || !alpha || !theta_out || K < 1 || K > tlda::kMaxDim || n_iter < 0 || docs->n_docs < 0 ||
      docs->vocab < 1 || (docs->n_docs > 0 && (!docs->indptr || !docs->indices || !docs->counts)))
    return TLDA_ERR_INVALID;
  if (docs->n_docs == 0) return TLDA_OK;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const int kpl = (K + 31) / 32;
  if (kpl <= 1) launch<1>(*docs, mu, alpha, K, n_iter, theta_out, gamma_out, err_out, s);
  else if (kpl <= 2) launch<2>(*docs, mu, alpha, K, n_iter, theta_out, gamma_out, err_out, s);
  else if (kpl <= 4) launch<4>(*docs, mu, alpha, K, n_iter, theta_out, gamma_out, err_out, s);
  else if (kpl <= 8) launch<8>(*docs, mu, alpha, K, n_iter, theta_out, gamma_out, err_out, s);
  else launch<16>(*docs, mu, alpha, K, n_iter, theta_out, gamma_out, err_out, s);
  return cudaGetLastError() == cudaSuccess ? TLDA_OK : TLDA_ERR_CUDA;
}
