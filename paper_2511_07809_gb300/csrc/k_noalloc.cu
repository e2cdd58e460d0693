// tlda_cp_step_noalloc: one CP-SGD step (FP32 form, same-token correction on)
// that allocates no device memory.  It exists for callers that cannot call
// cudaMalloc: code embedded in a host that owns the whole device-memory budget
// (a framework's caching allocator or a fixed arena that forbids extra
// allocations), and latency-critical loops where cudaMalloc/cudaFree would
// synchronise the device.  Its scratch is one file-scope __device__ array;
// the kernels are the ones the context-based entry points launch.
#include <cstdio>
#include <utility>

#include "tlda_internal.h"

using namespace tlda;

namespace {

// Scratch of every call on a device: 8 MiB, held by each GPU that loads the
// library until the process exits.
constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kNoAllocSplit = 32;
// Largest batch accepted: the scratch cannot hold more documents' rows anyway
// (each takes at least 3 x 64 FP32 of X, Y and Z), and the bound keeps every
// size computation below far from int overflow.
constexpr int kNoAllocMaxDocs = int(kNoAllocScratchBytes / (3 * 64 * sizeof(float)));

// Device address of the scratch array in the current context.  The array's
// name in host code is only a host-side stand-in, and its device address
// belongs to the context that loaded the module: after a device reset, or
// under another (non-primary) context, it can differ.  So it is looked up on
// every call; cudaGetSymbolAddress allocates nothing.
tlda_status scratch_address(unsigned char **out) {
  void *p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return TLDA_ERR_CUDA;
  *out = static_cast<unsigned char *>(p);
  return TLDA_OK;
}

// Carves 256-byte aligned regions off the scratch (or only measures, base == null).
struct Carve {
  unsigned char *base;
  size_t off = 0;
  template <class T>
  T *take(size_t n) {
    off = (off + 255) & ~size_t(255);
    T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
    off += n * sizeof(T);
    return p;
  }
};

// Clears what must start at zero (the scratch keeps the previous call's
// contents, possibly laid out for other sizes) and installs the batch.
__global__ void k_noalloc_reset(DevState *st, BatchDesc b, float *H, long long nH, int *cnt, int V) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = i; e < nH; e += stride) H[e] = 0.f;
  for (long long e = i; e < V; e += stride) cnt[e] = 0;
  if (i == 0) {
    DevState z{};
    z.cur = b;
    *st = z;
  }
}

__global__ void k_noalloc_status(const DevState *st, int32_t *err_out) { *err_out = st->err; }

}  // namespace

extern "C" tlda_status tlda_cp_step_noalloc(const tlda_csr *batch, const float *W, const float *m1,
                                            int32_t dim, int32_t k, double alpha0, float theta,
                                            float *Phi, float lr, float *grad_out, int32_t *err_out,
                                            void *cuda_stream) {
  TLDA_RANGE();
  if (!batch || !W || !m1 || !Phi) return TLDA_ERR_INVALID;
  const int V = batch->vocab, K = k, D = dim > 0 ? dim : k, B = batch->n_docs;
  if (V < 1 || K < 1 || D < K || D > V || B < 0 || B > kNoAllocMaxDocs || !(alpha0 > 0.0) || !(theta > -1.f) ||
      D > kMaxDim || K > kMaxDim || round_up(D, 64) > kMaxDim || round_up(K, 64) > kMaxDim || !batch->indptr ||
      (B > 0 && (!batch->indices || !batch->counts)))
    return TLDA_ERR_INVALID;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  StepArgs a{};
  a.V = V;
  a.D = D;
  a.K = K;
  a.Dp = round_up(D, 64);
  a.Kp = round_up(K, 64);
  a.Bmax = round_up(B > 0 ? B : 1, 128);
  a.nsplit = kNoAllocSplit;
  a.theta = theta;
  a.lr = lr;
  a.c3 = (alpha0 + 1.0) * (alpha0 + 2.0) / 2.0;
  a.same_token = 1;
  a.precision = TLDA_FP32;
  a.Phi = Phi;
  a.grad_out = grad_out;
  a.m1 = m1;
  // layout of the scratch for these sizes; reject what does not fit
  auto layout = [&](unsigned char *base) {
    Carve c{base};
    a.st = c.take<DevState>(1);
    float *U = c.take<float>((size_t)V * a.Dp);
    a.U32 = U;
    a.X32 = c.take<float>((size_t)a.Bmax * a.Dp);
    a.Q32 = c.take<float>((size_t)V * a.Kp);
    a.Y32 = c.take<float>((size_t)a.Bmax * a.Kp);
    a.Z32 = c.take<float>((size_t)a.Bmax * a.Kp);
    a.Zc32 = c.take<float>((size_t)V * a.Kp);
    a.H32 = c.take<float>((size_t)V * a.Kp);
    a.cnt = c.take<int>((size_t)V);
    a.widx = c.take<int>((size_t)V);
    a.Gpart = c.take<float>((size_t)a.nsplit * a.Dp * a.Kp);
    a.Gram = c.take<float>((size_t)a.Kp * a.Kp);
    a.avec = c.take<float>((size_t)a.Kp);
    a.E = c.take<float>((size_t)a.Dp * a.Kp);
    a.G3 = c.take<float>((size_t)a.Dp * a.Kp);
    return std::make_pair(c.off, U);
  };
  const size_t need = layout(nullptr).first;
  if (need > kNoAllocScratchBytes) {
    fprintf(stderr,
            "tlda_cp_step_noalloc: V=%d D=%d K=%d n_docs=%d need %zu bytes of scratch, more than the "
            "%zu-byte static array\n",
            V, D, K, B, need, kNoAllocScratchBytes);
    return TLDA_ERR_OOM;
  }
  unsigned char *base = nullptr;
  tlda_status st = scratch_address(&base);
  if (st != TLDA_OK) return st;
  float *U = layout(base).second;
  BatchDesc b{};
  b.indptr = batch->indptr;
  b.indices = batch->indices;
  b.counts = batch->counts;
  b.nz_base = 0;
  b.n_docs = B;
  k_noalloc_reset<<<64, 256, 0, s>>>(a.st, b, a.H32, (long long)V * a.Kp, a.cnt, V);
  launch_make_u(W, m1, V, D, a.Dp, U, nullptr, s);
  launch_phi_gram(a, s);
  launch_phi_terms(a, s);
  if (B > 0) {
    launch_whiten(a, s, nullptr, true);
    launch_qy_f32(a, s);
    launch_rz(a, s);
    launch_zh_f32(a, s);
    launch_g_f32(a, s);
  }
  launch_reduce_update(a, s);
  if (err_out) k_noalloc_status<<<1, 1, 0, s>>>(a.st, err_out);
  return cudaGetLastError() == cudaSuccess ? TLDA_OK : TLDA_ERR_CUDA;
}
