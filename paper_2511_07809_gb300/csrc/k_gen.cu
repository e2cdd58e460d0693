// On-device generation of the seeded synthetic corpora (the simulation
// data-generating process: topic proportions from Dirichlet(alpha0/K) drawn
// as a Polya urn, words from the topics' word distributions).  The definition
// is the one the host generator of the test inputs follows, so a chunk
// generated here equals the host's CSR for the same documents:
//  - counter-based Philox4x32-10 (Salmon, Moraes, Dror and Shaw, SC'11),
//    counter (document lo, document hi, token, tag | refill << 8), key = seed;
//  - lengths by inverting the Poisson table (2^32-scaled CDF), clipped below;
//  - per token a uniform integer by Lemire's multiply-and-reject (2019): the
//    urn weight of topic i is a_num + K a_den n_i, so a draw below K a_num is
//    a fresh topic and the rest copy the topic of an earlier token;
//  - the word by inverting the topic's cumulative table (binary search);
//  - the tokens sorted and merged into strictly ascending (word, count) pairs.
// One warp per document; the urn's copies are resolved by pointer jumping
// within each 32-token chunk.  No arithmetic of the estimation method here.
#include <cuda_runtime.h>

#include <cstdint>

#include "scan.cuh"
#include "tlda.h"
#include "tlda_internal.h"

namespace {

constexpr uint32_t kTagLen = 1u, kTagTok = 2u;
constexpr int kGenMaxLen = 1024;  // longest document (tokens)
constexpr int kGenWarps = 4;

__device__ __forceinline__ void philox10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
    const uint32_t lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
  }
}

// The 32-bit words of one (index, sub, tag) counter; each refill bumps the
// refill field.
struct RStream {
  uint64_t seed, idx;
  uint32_t sub, tag, refill, pos;
  uint32_t b0, b1, b2, b3;
  __device__ void init(uint64_t s, uint64_t i, uint32_t sb, uint32_t tg) {
    seed = s;
    idx = i;
    sub = sb;
    tag = tg;
    refill = 0;
    pos = 4;
  }
  __device__ uint32_t next() {
    if (pos == 4) {
      uint32_t c[4] = {(uint32_t)idx, (uint32_t)(idx >> 32), sub, tag | (refill << 8)};
      philox10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
      b0 = c[0];
      b1 = c[1];
      b2 = c[2];
      b3 = c[3];
      ++refill;
      pos = 0;
    }
    const uint32_t p = pos++;
    return p == 0 ? b0 : p == 1 ? b1 : p == 2 ? b2 : b3;
  }
  // uniform in [0, n), n >= 1
  __device__ uint32_t below(uint32_t n) {
    uint64_t m = (uint64_t)next() * n;
    uint32_t l = (uint32_t)m;
    if (l < n) {
      const uint32_t t = (0u - n) % n;
      while (l < t) {
        m = (uint64_t)next() * n;
        l = (uint32_t)m;
      }
    }
    return (uint32_t)(m >> 32);
  }
};

// first index l with u < cdf[l] (cdf non-decreasing, last entry 2^32 > u)
__device__ __forceinline__ int invert(const uint64_t *cdf, int n, uint64_t u) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (u < __ldg(cdf + mid)) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

struct GenArgs {
  uint64_t seed;
  int V, K;
  const uint64_t *cdf;
  uint32_t a_num, a_den;
  const uint64_t *len_cdf;
  int n_len, min_len;
  int64_t doc0;
  int n_docs;
  int32_t *indptr, *indices, *counts;
  int *err;
};

// pass 1: indptr[d + 1] = distinct words of document d; pass 2: the CSR rows
template <int PASS>
__global__ void __launch_bounds__(kGenWarps * 32) k_gen_docs(GenArgs a) {
  extern __shared__ int gsm[];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int d = blockIdx.x * kGenWarps + wib;
  if (d >= a.n_docs) return;
  int *zs = gsm + wib * 2 * kGenMaxLen, *ws = zs + kGenMaxLen;
  const uint64_t doc = (uint64_t)(a.doc0 + d);
  RStream lr;
  lr.init(a.seed, doc, 0, kTagLen);
  int L = invert(a.len_cdf, a.n_len, lr.next());
  if (L < a.min_len) L = a.min_len;
  if (L > kGenMaxLen) {
    if (lane == 0) atomicOr(a.err, 1);
    return;
  }
  const uint32_t Ka = (uint32_t)a.K * a.a_num, s = (uint32_t)a.K * a.a_den;
  for (int base = 0; base < L; base += 32) {
    const int t = base + lane;
    int z = 0, par = 0;
    bool res = true;
    uint32_t wu = 0;
    if (t < L) {
      RStream r;
      r.init(a.seed, doc, (uint32_t)t, kTagTok);
      const uint32_t u = r.below(Ka + s * (uint32_t)t);
      wu = r.next();
      if (u < Ka) {
        z = (int)(u / a.a_num);
      } else {
        par = (int)((u - Ka) / s);
        if (par < base) z = zs[par];  // an earlier chunk: final
        else res = false;
      }
    }
    // copies within this chunk: pointer jumping (chains are shorter than 32)
#pragma unroll
    for (int step = 0; step < 5; ++step) {
      const int src = res ? lane : par - base;
      const int zz = __shfl_sync(0xffffffffu, z, src);
      const int rr = __shfl_sync(0xffffffffu, (int)res, src);
      const int pp = __shfl_sync(0xffffffffu, par, src);
      if (!res) {
        if (rr) {
          z = zz;
          res = true;
        } else {
          par = pp;
        }
      }
    }
    if (t < L) {
      zs[t] = z;
      ws[t] = invert(a.cdf + (size_t)z * a.V, a.V, (uint64_t)wu);
    }
    __syncwarp();
  }
  // sort the words by rank (ties by token order) into zs
  for (int t = lane; t < L; t += 32) {
    const int w = ws[t];
    int rank = 0;
    for (int u = 0; u < L; ++u) {
      const int x = ws[u];
      rank += (x < w) || (x == w && u < t);
    }
    zs[rank] = w;
  }
  __syncwarp();
  int runs = 0;
  for (int base = 0; base < L; base += 32) {
    const int i = base + lane;
    const bool start = i < L && (i == 0 || zs[i] != zs[i - 1]);
    const unsigned bal = __ballot_sync(0xffffffffu, start);
    if (PASS == 2 && start) {
      int j = i + 1;
      while (j < L && zs[j] == zs[i]) ++j;
      const int o = a.indptr[d] + runs + __popc(bal & ((1u << lane) - 1u));
      a.indices[o] = zs[i];
      a.counts[o] = j - i;
    }
    runs += __popc(bal);
  }
  if (PASS == 1 && lane == 0) {
    a.indptr[d + 1] = runs;
    if (d == 0) a.indptr[0] = 0;
  }
}

}  // namespace

extern "C" tlda_status tlda_generate_docs(uint64_t seed, int32_t V, int32_t K, const uint64_t *topic_cdf,
                                          uint32_t a_num, uint32_t a_den, const uint64_t *len_cdf,
                                          int32_t n_len, int32_t min_len, int64_t doc0, int32_t n_docs,
                                          int32_t *indptr_out, int32_t *indices_out, int32_t *counts_out,
                                          int64_t nnz_cap, int64_t *scratch, int64_t *nnz_out,
                                          void *cuda_stream) {
  TLDA_RANGE();
  if (V < 1 || K < 1 || !topic_cdf || a_num == 0 || a_den == 0 || !len_cdf || n_len < 1 ||
      n_len > kGenMaxLen + 1 || min_len < 0 || min_len > kGenMaxLen || doc0 < 0 || n_docs < 0 || !indptr_out ||
      !scratch || !nnz_out || nnz_cap < 0 || (nnz_cap > 0 && (!indices_out || !counts_out)))
    return TLDA_ERR_INVALID;
  // the urn's integer total must fit in 32 bits for the longest document
  if ((uint64_t)K * a_num + (uint64_t)K * a_den * (uint64_t)kGenMaxLen >= 4294967296ull) return TLDA_ERR_INVALID;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  *nnz_out = 0;
  if (n_docs == 0) {
    return cudaMemsetAsync(indptr_out, 0, sizeof(int32_t), s) == cudaSuccess ? TLDA_OK : TLDA_ERR_CUDA;
  }
  const int nb = scan_blocks(n_docs);
  int64_t *bsum = scratch, *total = scratch + nb;
  int *err = reinterpret_cast<int *>(scratch + nb + 1);
  if (cudaMemsetAsync(err, 0, sizeof(int64_t), s) != cudaSuccess) return TLDA_ERR_CUDA;
  GenArgs a{seed, V, K, topic_cdf, a_num, a_den, len_cdf, n_len, min_len, doc0, n_docs,
            indptr_out, indices_out, counts_out, err};
  const unsigned grid = (unsigned)((n_docs + kGenWarps - 1) / kGenWarps);
  const size_t smem = sizeof(int) * 2 * kGenMaxLen * kGenWarps;
  k_gen_docs<1><<<grid, kGenWarps * 32, smem, s>>>(a);
  scan_counts(indptr_out, n_docs, bsum, total, s);
  int64_t hv[2] = {0, 0};
  if (cudaMemcpyAsync(hv, total, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return TLDA_ERR_CUDA;
  if (hv[1] != 0) return TLDA_ERR_INVALID;  // a document longer than 1024 tokens
  *nnz_out = hv[0];
  if (hv[0] >= 2147483647ll) return TLDA_ERR_OOM;  // int32 offsets
  if (nnz_cap == 0) return TLDA_OK;
  if (hv[0] > nnz_cap) return TLDA_ERR_OOM;
  k_gen_docs<2><<<grid, kGenWarps * 32, smem, s>>>(a);
  return cudaGetLastError() == cudaSuccess ? TLDA_OK : TLDA_ERR_CUDA;
}
