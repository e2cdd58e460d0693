// Moments and whitening (section "Computing the Centered Cumulants", appendix
// "Uncentered cumulants", section "Online Decomposition of the Second
// Moment") and topic recovery (section "Recovering the Topic Model
// Parameters"), on the device.
//
//  ACCUMULATE  exact integer statistics of each chunk: C_m, T, S2, S3 (int64)
//              and the pair counts P = sum_d (f_d f_d^T - diag f_d), held as a
//              dense V x V FP64 matrix of exact integers (atomic adds of
//              integers below 2^53 are order independent).
//  FINALIZE    M1 = C/T, M2 = (alpha0+1) P/S2 - alpha0 M1 M1^T; top-D
//              eigenpairs by randomised subspace iteration (FP32 products,
//              FP64 CholeskyQR2), FP64 Rayleigh-Ritz with a cyclic Jacobi
//              eigensolver in one block, W = U Lambda^-1/2, m1 = W^T M1.
//  unwhiten    mu_i = ||phi_i||^2 W (W^T W)^-1 phi_i, alpha_i ~ ||phi_i||^-6,
//              clip at 0, normalise (FP64).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "tlda_internal.h"

using namespace tlda;

namespace {

constexpr int kMaxFitV = 65536;

// ------------------------------------------------------------------ scan + pairs
__global__ void k_fit_accumulate(tlda_csr b, int V, double *P, unsigned long long *C,
                                 unsigned long long *TS, int *err) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= b.n_docs) return;
  const int lo = b.indptr[warp], hi = b.indptr[warp + 1];
  if (lo < 0 || hi < lo) {
    if (lane == 0) atomicOr(err, 1);
    return;
  }
  const int u = hi - lo;
  bool bad = false;
  long long L = 0;
  for (int j = lo; j < hi; ++j) {
    const int m = b.indices[j], f = b.counts[j];
    if (m < 0 || m >= V || f <= 0 || (j > lo && m <= b.indices[j - 1])) {
      bad = true;
      continue;
    }
    L += f;
  }
  if (bad) {
    if (lane == 0) atomicOr(err, 1);
    return;
  }
  if (lane == 0) {
    atomicAdd(TS + 0, (unsigned long long)L);
    atomicAdd(TS + 1, (unsigned long long)(L * (L - 1)));
    atomicAdd(TS + 2, (unsigned long long)(L * (L - 1) * (L - 2)));
  }
  for (int j = lo + lane; j < hi; j += 32) atomicAdd(C + b.indices[j], (unsigned long long)b.counts[j]);
  for (int q = lane; q < u * u; q += 32) {
    const int x = q / u, y = q % u;
    const int ma = b.indices[lo + x], mb = b.indices[lo + y];
    const long long fa = b.counts[lo + x], fb = b.counts[lo + y];
    const long long v = fa * fb - (x == y ? fa : 0);
    if (v) atomicAdd(P + (long long)ma * V + mb, (double)v);
  }
}

// ------------------------------------------------------------------ generic GEMMs
// C[M x N] = A[M x Kd] B[Kd x N] (row-major), 64 x 64 tiles, 4 x 4 per thread.
template <class T>
__global__ void __launch_bounds__(256) k_gemm_nn(const T *A, int lda, const T *B, int ldb, T *C, int ldc,
                                                 int M, int N, int Kd) {
  __shared__ T As[16][64 + 1];
  __shared__ T Bs[16][64];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  T acc[4][4];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
  for (int k0 = 0; k0 < Kd; k0 += 16) {
    for (int e = tid; e < 16 * 64; e += 256) {
      const int r = e >> 4, kk = e & 15;  // A: 64 rows x 16
      const int gm = m0 + r, gk = k0 + kk;
      As[kk][r] = (gm < M && gk < Kd) ? A[(long long)gm * lda + gk] : T(0);
      const int kb = e >> 6, nn = e & 63;  // B: 16 x 64
      const int gkb = k0 + kb, gn = n0 + nn;
      Bs[kb][nn] = (gkb < Kd && gn < N) ? B[(long long)gkb * ldb + gn] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      T ar[4], br[4];
      for (int i = 0; i < 4; ++i) ar[i] = As[kk][ty * 4 + i];
      for (int j = 0; j < 4; ++j) br[j] = Bs[kk][tx * 4 + j];
      for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) acc[i][j] += ar[i] * br[j];
    }
    __syncthreads();
  }
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      const int gm = m0 + ty * 4 + i, gn = n0 + tx * 4 + j;
      if (gm < M && gn < N) C[(long long)gm * ldc + gn] = acc[i][j];
    }
}

// C[M x N] += A[Kd x M]^T B[Kd x N] in FP64, split over Kd (atomics into C).
template <class TA, class TB>
__global__ void __launch_bounds__(256) k_gemm_tn64(const TA *A, int lda, const TB *B, int ldb, double *C,
                                                   int ldc, int M, int N, int Kd, int chunk) {
  __shared__ double As[16][64 + 1];
  __shared__ double Bs[16][64];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * 64, n0 = blockIdx.z * 64;
  const int kb = blockIdx.x * chunk, ke = min(Kd, kb + chunk);
  double acc[4][4] = {};
  for (int k0 = kb; k0 < ke; k0 += 16) {
    for (int e = tid; e < 16 * 64; e += 256) {
      const int kk = e >> 6, c = e & 63, gk = k0 + kk;
      As[kk][c] = (gk < ke && m0 + c < M) ? (double)A[(long long)gk * lda + m0 + c] : 0.0;
      Bs[kk][c] = (gk < ke && n0 + c < N) ? (double)B[(long long)gk * ldb + n0 + c] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk)
      for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) acc[i][j] += As[kk][ty * 4 + i] * Bs[kk][tx * 4 + j];
    __syncthreads();
  }
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      const int gm = m0 + ty * 4 + i, gn = n0 + tx * 4 + j;
      if (gm < M && gn < N && acc[i][j] != 0.0) atomicAdd(C + (long long)gm * ldc + gn, acc[i][j]);
    }
}

template <class T>
void gemm_nn(const T *A, int lda, const T *B, int ldb, T *C, int ldc, int M, int N, int Kd, cudaStream_t s) {
  dim3 g((N + 63) / 64, (M + 63) / 64);
  k_gemm_nn<T><<<g, 256, 0, s>>>(A, lda, B, ldb, C, ldc, M, N, Kd);
}

template <class TA, class TB>
void gemm_tn64(const TA *A, int lda, const TB *B, int ldb, double *C, int ldc, int M, int N, int Kd,
               cudaStream_t s) {
  cudaMemsetAsync(C, 0, sizeof(double) * (size_t)M * ldc, s);
  const int chunk = 512;
  dim3 g((Kd + chunk - 1) / chunk, (M + 63) / 64, (N + 63) / 64);
  k_gemm_tn64<TA, TB><<<g, 256, 0, s>>>(A, lda, B, ldb, C, ldc, M, N, Kd, chunk);
}

// ------------------------------------------------------------------ elementwise helpers
__global__ void k_m2_f32(const double *P, const double *M1, int V, double sP, double a0, float *M2) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)V * V) return;
  const int i = (int)(e / V), j = (int)(e % V);
  M2[e] = (float)(sP * P[e] - a0 * M1[i] * M1[j]);
}

__global__ void k_m1(const unsigned long long *C, const unsigned long long *TS, int V, double *M1) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m < V) M1[m] = (double)C[m] / (double)TS[0];
}

__device__ inline unsigned long long splitmix64(unsigned long long x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// Gaussian start block Omega (V x r), Box-Muller on a counter hash.
__global__ void k_gauss(float *O, long long n, unsigned long long seed) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const unsigned long long h1 = splitmix64(seed ^ (2 * e)), h2 = splitmix64(seed ^ (2 * e + 1) ^ 0x5851F42D4C957F2Dull);
  const double u1 = ((h1 >> 11) + 0.5) * (1.0 / 9007199254740992.0);
  const double u2 = (h2 >> 11) * (1.0 / 9007199254740992.0);
  O[e] = (float)(sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2));
}

__global__ void k_f2d(const float *x, double *y, long long n) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) y[e] = x[e];
}

// ------------------------------------------------------------------ small dense FP64 (one block)
// In-place Cholesky G = L L^T (lower triangle of G, global memory), then
// Linv = L^-1.  status[0] = 1 on breakdown (non-positive pivot).
__global__ void k_chol_inv(double *L, int r, double *Linv, int *status) {
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int j = 0; j < r; ++j) {
    if (threadIdx.x == 0) {
      double d = L[j * r + j];
      for (int k = 0; k < j; ++k) d -= L[j * r + k] * L[j * r + k];
      if (!(d > 0.0)) {
        bad = 1;
        d = 1.0;
      }
      L[j * r + j] = sqrt(d);
    }
    __syncthreads();
    for (int i = j + 1 + threadIdx.x; i < r; i += blockDim.x) {
      double v = L[i * r + j];
      for (int k = 0; k < j; ++k) v -= L[i * r + k] * L[j * r + k];
      L[i * r + j] = v / L[j * r + j];
    }
    __syncthreads();
  }
  // column c of L^-1 by forward substitution of L x = e_c (x_i = 0 for i < c)
  for (int c = threadIdx.x; c < r; c += blockDim.x) {
    for (int i = 0; i < r; ++i) {
      double v = (i == c) ? 1.0 : 0.0;
      if (i >= c)
        for (int k = c; k < i; ++k) v -= L[i * r + k] * Linv[k * r + c];
      Linv[i * r + c] = (i < c) ? 0.0 : v / L[i * r + i];
    }
  }
  if (threadIdx.x == 0 && bad) *status = 1;
}

// Transpose r x r (FP64 -> FP32 for the Y Linv^T product).
__global__ void k_transpose_rr(const double *A, int r, float *AT32, double *AT64) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= r * r) return;
  const int i = e / r, j = e % r;
  if (AT32) AT32[j * r + i] = (float)A[e];
  if (AT64) AT64[j * r + i] = A[e];
}

// Cyclic Jacobi for a symmetric r x r FP64 matrix A (r even, global memory,
// overwritten), round-robin ordering so each round applies r/2 disjoint
// rotations in parallel (Golub & Van Loan, "Matrix Computations", sec. 8.5,
// parallel ordering).  Rotation of pair (p, q): tau = (a_qq - a_pp)/(2 a_pq),
// t = sign(tau)/(|tau| + sqrt(1 + tau^2)), c = 1/sqrt(1 + t^2), s = t c, and
// A <- J^T A J, E <- E J.  On return eval[i] = A_ii, columns of Evec are the
// eigenvectors; sweeps stop when the off-diagonal mass is below 1e-30 of the
// total (or after max_sweeps).
__global__ void k_jacobi(double *A, int r, double *Evec, double *eval, int max_sweeps, int *sweeps_out) {
  __shared__ double cs[kMaxDim], sn[kMaxDim];
  __shared__ int pp[kMaxDim], qq[kMaxDim];
  __shared__ double red_o[512], red_t[512];
  const int h = r / 2;
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int i = e / r, j = e % r;
    if (i < j) {
      const double v = 0.5 * (A[i * r + j] + A[j * r + i]);
      A[i * r + j] = v;
      A[j * r + i] = v;
    }
    Evec[e] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    double o = 0.0, t = 0.0;
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
      const double v = A[e] * A[e];
      t += v;
      if (e / r != e % r) o += v;
    }
    red_o[threadIdx.x] = o;
    red_t[threadIdx.x] = t;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if ((int)threadIdx.x < w) {
        red_o[threadIdx.x] += red_o[threadIdx.x + w];
        red_t[threadIdx.x] += red_t[threadIdx.x + w];
      }
      __syncthreads();
    }
    const bool done = red_o[0] <= 1e-30 * red_t[0];
    __syncthreads();
    if (done) break;
    for (int round = 0; round < r - 1; ++round) {
      for (int k = threadIdx.x; k < h; k += blockDim.x) {
        // round-robin pairing: slot 0 holds index 0, the others rotate
        const int sa = k, sb = r - 1 - k;
        int p = sa == 0 ? 0 : 1 + (sa - 1 + round) % (r - 1);
        int q = sb == 0 ? 0 : 1 + (sb - 1 + round) % (r - 1);
        if (p > q) {
          const int tmp = p;
          p = q;
          q = tmp;
        }
        const double apq = A[p * r + q];
        double c = 1.0, sv = 0.0;
        if (apq != 0.0) {
          const double tau = (A[q * r + q] - A[p * r + p]) / (2.0 * apq);
          const double tt = tau >= 0.0 ? 1.0 / (tau + sqrt(1.0 + tau * tau)) : -1.0 / (-tau + sqrt(1.0 + tau * tau));
          c = 1.0 / sqrt(1.0 + tt * tt);
          sv = tt * c;
        }
        cs[k] = c;
        sn[k] = sv;
        pp[k] = p;
        qq[k] = q;
      }
      __syncthreads();
      for (int w = threadIdx.x; w < h * r; w += blockDim.x) {  // rows: A <- J^T A
        const int k = w / r, j = w % r, p = pp[k], q = qq[k];
        const double c = cs[k], sv = sn[k], ap = A[p * r + j], aq = A[q * r + j];
        A[p * r + j] = c * ap - sv * aq;
        A[q * r + j] = sv * ap + c * aq;
      }
      __syncthreads();
      for (int w = threadIdx.x; w < h * r; w += blockDim.x) {  // columns: A <- A J, E <- E J
        const int k = w / r, i = w % r, p = pp[k], q = qq[k];
        const double c = cs[k], sv = sn[k];
        const double ap = A[i * r + p], aq = A[i * r + q];
        A[i * r + p] = c * ap - sv * aq;
        A[i * r + q] = sv * ap + c * aq;
        const double ep = Evec[i * r + p], eq = Evec[i * r + q];
        Evec[i * r + p] = c * ep - sv * eq;
        Evec[i * r + q] = sv * ep + c * eq;
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < r; i += blockDim.x) eval[i] = A[i * r + i];
  if (threadIdx.x == 0) *sweeps_out = sweep;
}

// Z = sP * Z - a0 * M1 (M1^T Q)  (rank-one part of M2 applied to Q), r columns.
__global__ void k_rank1_fix(double *Z, const double *M1, const double *m1q, int V, int r, double sP, double a0) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)V * r) return;
  const int i = (int)(e / r), j = (int)(e % r);
  Z[e] = sP * Z[e] - a0 * M1[i] * m1q[j];
}

// W = U_D Lambda^-1/2 with the sign of each eigenvector fixed so that its
// largest-magnitude entry is positive (lowest index on ties).  One block per column.
__global__ void k_make_w(const double *U, int V, int D, const double *lam, float *W32, double *W64, int *sgn) {
  const int j = blockIdx.x;
  __shared__ double bv[256];
  __shared__ int bi[256];
  double best = -1.0;
  int besti = 0x7fffffff;
  for (int m = threadIdx.x; m < V; m += blockDim.x) {
    const double a = fabs(U[(long long)m * D + j]);
    if (a > best || (a == best && m < besti)) {
      best = a;
      besti = m;
    }
  }
  bv[threadIdx.x] = best;
  bi[threadIdx.x] = besti;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      const double o = bv[threadIdx.x + w];
      const int oi = bi[threadIdx.x + w];
      if (o > bv[threadIdx.x] || (o == bv[threadIdx.x] && oi < bi[threadIdx.x])) {
        bv[threadIdx.x] = o;
        bi[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  const double sg = U[(long long)bi[0] * D + j] < 0 ? -1.0 : 1.0;
  const double sc = sg / sqrt(lam[j]);
  for (int m = threadIdx.x; m < V; m += blockDim.x) {
    const double w = U[(long long)m * D + j] * sc;
    W32[(long long)m * D + j] = (float)w;
    if (W64) W64[(long long)m * D + j] = w;
  }
  if (threadIdx.x == 0 && sgn) sgn[j] = (int)sg;
}

// m1 = W^T M1 (FP64 accumulate), one block per component.
__global__ void k_wtm1(const float *W, const double *M1, int V, int D, float *m1) {
  const int j = blockIdx.x;
  __shared__ double red[256];
  double s = 0.0;
  for (int m = threadIdx.x; m < V; m += blockDim.x) s += (double)W[(long long)m * D + j] * M1[m];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) m1[j] = (float)red[0];
}

// ------------------------------------------------------------------ unwhitening
// T[r][i] = sum_j Ginv[r][j] Phi[j][i] ||phi_i||^2, alpha_i ~ ||phi_i||^-6.
__global__ void k_unwhiten_coef(const float *Phi, int D, int K, const double *Ginv, double *T, double *alpha) {
  __shared__ double nrm2[kMaxDim];
  for (int i = threadIdx.x; i < K; i += blockDim.x) {
    double s = 0.0;
    for (int r = 0; r < D; ++r) s += (double)Phi[r * K + i] * Phi[r * K + i];
    nrm2[i] = s;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < D * K; e += blockDim.x) {
    const int r = e / K, i = e % K;
    double s = 0.0;
    for (int j = 0; j < D; ++j) s += Ginv[r * D + j] * (double)Phi[j * K + i];
    T[e] = s * nrm2[i];
  }
  if (threadIdx.x == 0) {
    double z = 0.0;
    for (int i = 0; i < K; ++i) z += pow(nrm2[i], -3.0);
    for (int i = 0; i < K; ++i) alpha[i] = pow(nrm2[i], -3.0) / z;
  }
}

// clip at 0 and normalise each column of mu (V x K) to sum 1; one block per column.
__global__ void k_clip_norm(double *mu, int V, int K) {
  const int i = blockIdx.x;
  __shared__ double red[256];
  double s = 0.0;
  for (int m = threadIdx.x; m < V; m += blockDim.x) {
    double v = mu[(long long)m * K + i];
    v = v > 0.0 ? v : 0.0;
    mu[(long long)m * K + i] = v;
    s += v;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  const double z = red[0] > 0.0 ? red[0] : 1.0;
  for (int m = threadIdx.x; m < V; m += blockDim.x) mu[(long long)m * K + i] /= z;
}

tlda_status fail(tlda_ctx *c, tlda_status s, const char *msg) {
  if (c) c->err = msg;
  return s;
}

#define CKF(call)                                                                                 \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess) {                                                                      \
      ctx->err = std::string(#call) + ": " + cudaGetErrorString(e_);                              \
      return e_ == cudaErrorMemoryAllocation ? TLDA_ERR_OOM : TLDA_ERR_CUDA;                      \
    }                                                                                             \
  } while (0)

template <class T>
cudaError_t dalloc(T **p, size_t n, bool zero = false) {
  if (n == 0) n = 1;
  cudaError_t e = cudaMalloc(reinterpret_cast<void **>(p), n * sizeof(T));
  if (e == cudaSuccess && zero) e = cudaMemset(*p, 0, n * sizeof(T));
  return e;
}

// Scratch of a FINALIZE or an unwhitening, freed on every exit path.
struct Scratch {
  std::vector<void *> ptrs;
  template <class T>
  cudaError_t get(T **p, size_t n, bool zero = false) {
    cudaError_t e = dalloc(p, n, zero);
    if (e == cudaSuccess) ptrs.push_back(*p);
    return e;
  }
  ~Scratch() {
    for (void *p : ptrs) cudaFree(p);
  }
};

tlda_status finalize(tlda_ctx *ctx) {
  cudaStream_t s = ctx->stream;
  const int V = ctx->V, D = ctx->D;
  int r = round_up(D + 16, 2);
  if (r > V) r = V - (V & 1);
  if (r < D) return fail(ctx, TLDA_ERR_INVALID, "vocabulary too small for the whitening dimension");
  unsigned long long TS[3];
  int ferr = 0;
  CKF(cudaMemcpyAsync(TS, ctx->TS, sizeof TS, cudaMemcpyDeviceToHost, s));
  CKF(cudaMemcpyAsync(&ferr, ctx->fit_err, sizeof ferr, cudaMemcpyDeviceToHost, s));
  CKF(cudaStreamSynchronize(s));
  if (ferr) return fail(ctx, TLDA_ERR_INVALID, "corrupt CSR chunk in fit_moments");
  if (TS[0] == 0 || TS[1] == 0) return fail(ctx, TLDA_ERR_NUMERIC, "no token pairs accumulated");
  const double a0 = ctx->p.alpha0, sP = (a0 + 1.0) / (double)TS[1];
  Scratch sc;
  double *M1 = nullptr, *Q64 = nullptr, *Z64 = nullptr, *G = nullptr, *Linv = nullptr, *LinvT64 = nullptr;
  double *Bm = nullptr, *Ev = nullptr, *ev = nullptr, *m1q = nullptr, *U64 = nullptr, *lam = nullptr, *Ek = nullptr;
  float *M2 = nullptr, *Om = nullptr, *Y = nullptr, *Qf = nullptr, *LinvT32 = nullptr;
  int *status = nullptr;
  const long long VV = (long long)V * V;
  CKF(sc.get(&M1, V));
  CKF(sc.get(&M2, (size_t)VV));
  CKF(sc.get(&Om, (size_t)V * r));
  CKF(sc.get(&Y, (size_t)V * r));
  CKF(sc.get(&Qf, (size_t)V * r));
  CKF(sc.get(&Q64, (size_t)V * r));
  CKF(sc.get(&Z64, (size_t)V * r));
  CKF(sc.get(&G, (size_t)r * r));
  CKF(sc.get(&Linv, (size_t)r * r));
  CKF(sc.get(&LinvT64, (size_t)r * r));
  CKF(sc.get(&LinvT32, (size_t)r * r));
  CKF(sc.get(&Bm, (size_t)r * r));
  CKF(sc.get(&Ev, (size_t)r * r));
  CKF(sc.get(&ev, (size_t)r));
  CKF(sc.get(&Ek, (size_t)r * D));
  CKF(sc.get(&m1q, (size_t)r));
  CKF(sc.get(&U64, (size_t)V * D));
  CKF(sc.get(&lam, (size_t)D));
  CKF(sc.get(&status, 2, true));
  k_m1<<<(V + 255) / 256, 256, 0, s>>>(ctx->Ccnt, ctx->TS, V, M1);
  k_m2_f32<<<(unsigned)((VV + 255) / 256), 256, 0, s>>>(ctx->P64, M1, V, sP, a0, M2);
  k_gauss<<<(unsigned)(((long long)V * r + 255) / 256), 256, 0, s>>>(Om, (long long)V * r, ctx->p.seed * 0x100000001B3ull + 17);
  // one CholeskyQR pass: out = in L^-T with L L^T = in^T in (FP64 Gram)
  auto cholqr_pass = [&](const float *in, float *out) {
    gemm_tn64<float, float>(in, r, in, r, G, r, r, r, V, s);
    k_chol_inv<<<1, 256, 0, s>>>(G, r, Linv, status);
    k_transpose_rr<<<(r * r + 255) / 256, 256, 0, s>>>(Linv, r, LinvT32, nullptr);
    gemm_nn<float>(in, r, LinvT32, r, out, r, V, r, r, s);
  };
  // CholeskyQR2 of Y into Qf (Y is clobbered)
  auto cholqr2 = [&]() {
    cholqr_pass(Y, Qf);
    cholqr_pass(Qf, Y);
    cudaMemcpyAsync(Qf, Y, sizeof(float) * (size_t)V * r, cudaMemcpyDeviceToDevice, s);
  };
  gemm_nn<float>(M2, V, Om, r, Y, r, V, r, V, s);
  cholqr2();
  const int n_iter = 24;
  for (int it = 0; it < n_iter; ++it) {
    gemm_nn<float>(M2, V, Qf, r, Y, r, V, r, V, s);
    cholqr2();
  }
  // FP64 Rayleigh-Ritz on the exact M2 = sP P - a0 M1 M1^T
  k_f2d<<<(unsigned)(((long long)V * r + 255) / 256), 256, 0, s>>>(Qf, Q64, (long long)V * r);
  // one FP64 CholeskyQR pass to make Q64 orthonormal to FP64 accuracy
  gemm_tn64<double, double>(Q64, r, Q64, r, G, r, r, r, V, s);
  k_chol_inv<<<1, 256, 0, s>>>(G, r, Linv, status);
  k_transpose_rr<<<(r * r + 255) / 256, 256, 0, s>>>(Linv, r, nullptr, LinvT64);
  gemm_nn<double>(Q64, r, LinvT64, r, Z64, r, V, r, r, s);
  cudaMemcpyAsync(Q64, Z64, sizeof(double) * (size_t)V * r, cudaMemcpyDeviceToDevice, s);
  gemm_nn<double>(ctx->P64, V, Q64, r, Z64, r, V, r, V, s);
  gemm_tn64<double, double>(M1, 1, Q64, r, m1q, r, 1, r, V, s);
  k_rank1_fix<<<(unsigned)(((long long)V * r + 255) / 256), 256, 0, s>>>(Z64, M1, m1q, V, r, sP, a0);
  gemm_tn64<double, double>(Q64, r, Z64, r, Bm, r, r, r, V, s);
  int *sweeps = status + 1;
  k_jacobi<<<1, 512, 0, s>>>(Bm, r, Ev, ev, 40, sweeps);
  CKF(cudaGetLastError());
  std::vector<double> hev(r), hEv((size_t)r * r);
  int hstat[2];
  CKF(cudaMemcpyAsync(hev.data(), ev, sizeof(double) * r, cudaMemcpyDeviceToHost, s));
  CKF(cudaMemcpyAsync(hEv.data(), Ev, sizeof(double) * r * r, cudaMemcpyDeviceToHost, s));
  CKF(cudaMemcpyAsync(hstat, status, sizeof hstat, cudaMemcpyDeviceToHost, s));
  CKF(cudaStreamSynchronize(s));
  if (hstat[0]) return fail(ctx, TLDA_ERR_NUMERIC, "subspace basis lost rank (CholeskyQR breakdown)");
  // order the Ritz pairs by descending value and keep D of them
  std::vector<int> ord(r);
  for (int i = 0; i < r; ++i) ord[i] = i;
  std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return hev[x] > hev[y]; });
  std::vector<double> hEk((size_t)r * D), hlam(D);
  for (int j = 0; j < D; ++j) {
    hlam[j] = hev[ord[j]];
    for (int i = 0; i < r; ++i) hEk[(size_t)i * D + j] = hEv[(size_t)i * r + ord[j]];
  }
  if (!(hlam[D - 1] > 1e-12 * hlam[0]))
    return fail(ctx, TLDA_ERR_NUMERIC, "M2 has fewer than D positive eigenvalues");
  CKF(cudaMemcpyAsync(Ek, hEk.data(), sizeof(double) * r * D, cudaMemcpyHostToDevice, s));
  CKF(cudaMemcpyAsync(lam, hlam.data(), sizeof(double) * D, cudaMemcpyHostToDevice, s));
  gemm_nn<double>(Q64, r, Ek, D, U64, D, V, D, r, s);
  k_make_w<<<D, 256, 0, s>>>(U64, V, D, lam, ctx->W32, nullptr, nullptr);
  CKF(cudaMemsetAsync(ctx->m1, 0, sizeof(float) * ctx->Dp, s));
  k_wtm1<<<D, 256, 0, s>>>(ctx->W32, M1, V, D, ctx->m1);
  launch_make_u(ctx->W32, ctx->m1, V, D, ctx->Dp, ctx->U32, ctx->U16, s);
  CKF(cudaGetLastError());
  CKF(cudaStreamSynchronize(s));
  ctx->eig = hlam;
  ctx->whitened = true;
  ctx->fitted = true;
  return TLDA_OK;
}

// ------------------------------------------------------------------ fully online mode
// One warp per document of a block of batches (absolute offsets into the
// corpus CSR): validation, L, and the exact counts C_m, T, S2, S3; then the
// document's part of the sketch Z = P Omega of the pair counts,
// Z_m += f_m (f^T Omega - Omega_m) for each of its words (FP64 atomics).  A
// document that fails validation adds nothing and sets *err.
__global__ void __launch_bounds__(256) k_online_acc(const int32_t *indptr, const int32_t *indices,
                                                     const int32_t *counts, int n_docs, int V, int r,
                                                     const double *Om, double *Z, unsigned long long *C,
                                                     unsigned long long *TS, int *err) {
  constexpr int kCols = kMaxDim / 32;
  const int doc = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (doc >= n_docs) return;
  const long long p0 = indptr[doc], p1 = indptr[doc + 1];
  if (p0 < 0 || p1 < p0) {
    if (lane == 0) atomicOr(err, 1);
    return;
  }
  double sv[kCols];
#pragma unroll
  for (int i = 0; i < kCols; ++i) sv[i] = 0.0;
  long long L = 0;
  int prev = -1;
  bool bad = false;
  for (long long p = p0; p < p1; ++p) {  // warp-uniform loop
    const int m = indices[p], f = counts[p];
    if (m < 0 || m >= V || f <= 0 || m <= prev) {
      bad = true;
      break;
    }
    prev = m;
    L += f;
    const double *om = Om + (long long)m * r;
#pragma unroll
    for (int i = 0; i < kCols; ++i) {
      const int col = lane + 32 * i;
      if (col < r) sv[i] += (double)f * om[col];
    }
  }
  if (bad) {
    if (lane == 0) atomicOr(err, 1);
    return;
  }
  for (long long p = p0; p < p1; ++p) {
    const int m = indices[p], f = counts[p];
    const double *om = Om + (long long)m * r;
    double *z = Z + (long long)m * r;
#pragma unroll
    for (int i = 0; i < kCols; ++i) {
      const int col = lane + 32 * i;
      if (col < r) atomicAdd(z + col, (double)f * (sv[i] - om[col]));
    }
    if (lane == 0) atomicAdd(C + m, (unsigned long long)f);
  }
  if (lane == 0 && L > 0) {
    atomicAdd(TS + 0, (unsigned long long)L);
    atomicAdd(TS + 1, (unsigned long long)(L * (L - 1)));
    atomicAdd(TS + 2, (unsigned long long)(L * (L - 1) * (L - 2)));
  }
}

// In-place inverse of an n x n FP64 matrix (row-major) by Gauss-Jordan
// elimination with partial pivoting; false if it is singular.
bool host_inverse(std::vector<double> &A, int n) {
  std::vector<double> I((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) I[(size_t)i * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int i = c + 1; i < n; ++i)
      if (std::fabs(A[(size_t)i * n + c]) > std::fabs(A[(size_t)piv * n + c])) piv = i;
    if (!(std::fabs(A[(size_t)piv * n + c]) > 0.0)) return false;
    if (piv != c)
      for (int j = 0; j < n; ++j) {
        std::swap(A[(size_t)c * n + j], A[(size_t)piv * n + j]);
        std::swap(I[(size_t)c * n + j], I[(size_t)piv * n + j]);
      }
    const double d = A[(size_t)c * n + c];
    for (int j = 0; j < n; ++j) {
      A[(size_t)c * n + j] /= d;
      I[(size_t)c * n + j] /= d;
    }
    for (int i = 0; i < n; ++i) {
      if (i == c) continue;
      const double f = A[(size_t)i * n + c];
      if (f == 0.0) continue;
      for (int j = 0; j < n; ++j) {
        A[(size_t)i * n + j] -= f * A[(size_t)c * n + j];
        I[(size_t)i * n + j] -= f * I[(size_t)c * n + j];
      }
    }
  }
  A.swap(I);
  return true;
}

// Rebuilds the whitening from the online statistics (section "Fully Online
// Implementation", the PCA update): with M1 = C/T, the sketch of
// M2 = (alpha0+1) P/S2 - alpha0 M1 M1^T is Y = (alpha0+1)/S2 Z - alpha0 M1 (M1^T Omega);
// then the single-pass eigendecomposition of Halko, Martinsson and Tropp
// (2011, section 5.5): Q = orth(Y) (FP64 CholeskyQR2), B solves
// B (Q^T Omega) = Q^T Y, B symmetrised, B = E Lambda E^T (Jacobi), U = Q E,
// and W = U_D Lambda_D^-1/2 with the signs of fit_moments, m1 = W^T M1, U.
// The previous W is kept in on_Wold.
tlda_status online_rewhiten(tlda_ctx *ctx) {
  cudaStream_t s = ctx->stream;
  const int V = ctx->V, D = ctx->D, r = ctx->on_r;
  unsigned long long TS[3];
  int ferr = 0;
  CKF(cudaMemcpyAsync(TS, ctx->on_TS, sizeof TS, cudaMemcpyDeviceToHost, s));
  CKF(cudaMemcpyAsync(&ferr, ctx->on_err, sizeof ferr, cudaMemcpyDeviceToHost, s));
  CKF(cudaStreamSynchronize(s));
  if (ferr) return fail(ctx, TLDA_ERR_INVALID, "corrupt CSR batch in the online pass");
  if (TS[0] == 0 || TS[1] == 0) return fail(ctx, TLDA_ERR_NUMERIC, "no token pairs accumulated");
  const double a0 = ctx->p.alpha0, sP = (a0 + 1.0) / (double)TS[1];
  Scratch sc;
  double *M1 = nullptr, *m1q = nullptr, *Y = nullptr, *Q1 = nullptr, *Q2 = nullptr, *G = nullptr;
  double *Linv = nullptr, *LinvT = nullptr, *C1 = nullptr, *C2 = nullptr, *Bm = nullptr, *Ev = nullptr;
  double *ev = nullptr, *Ek = nullptr, *U64 = nullptr, *lam = nullptr;
  int *status = nullptr;
  CKF(sc.get(&M1, V));
  CKF(sc.get(&m1q, r));
  CKF(sc.get(&Y, (size_t)V * r));
  CKF(sc.get(&Q1, (size_t)V * r));
  CKF(sc.get(&Q2, (size_t)V * r));
  CKF(sc.get(&G, (size_t)r * r));
  CKF(sc.get(&Linv, (size_t)r * r));
  CKF(sc.get(&LinvT, (size_t)r * r));
  CKF(sc.get(&C1, (size_t)r * r));
  CKF(sc.get(&C2, (size_t)r * r));
  CKF(sc.get(&Bm, (size_t)r * r));
  CKF(sc.get(&Ev, (size_t)r * r));
  CKF(sc.get(&ev, r));
  CKF(sc.get(&Ek, (size_t)r * D));
  CKF(sc.get(&U64, (size_t)V * D));
  CKF(sc.get(&lam, D));
  CKF(sc.get(&status, 2, true));
  k_m1<<<(V + 255) / 256, 256, 0, s>>>(ctx->on_C, ctx->on_TS, V, M1);
  gemm_tn64<double, double>(M1, 1, ctx->on_Om, r, m1q, r, 1, r, V, s);
  CKF(cudaMemcpyAsync(Y, ctx->on_Z, sizeof(double) * (size_t)V * r, cudaMemcpyDeviceToDevice, s));
  k_rank1_fix<<<(unsigned)(((long long)V * r + 255) / 256), 256, 0, s>>>(Y, M1, m1q, V, r, sP, a0);
  // CholeskyQR2: out = in L^-T with L L^T = in^T in, twice
  auto cholqr_pass = [&](const double *in, double *out) {
    gemm_tn64<double, double>(in, r, in, r, G, r, r, r, V, s);
    k_chol_inv<<<1, 256, 0, s>>>(G, r, Linv, status);
    k_transpose_rr<<<(r * r + 255) / 256, 256, 0, s>>>(Linv, r, nullptr, LinvT);
    gemm_nn<double>(in, r, LinvT, r, out, r, V, r, r, s);
  };
  cholqr_pass(Y, Q1);
  cholqr_pass(Q1, Q2);
  gemm_tn64<double, double>(Q2, r, Y, r, C1, r, r, r, V, s);           // Q^T Y
  gemm_tn64<double, double>(Q2, r, ctx->on_Om, r, C2, r, r, r, V, s);  // Q^T Omega
  CKF(cudaGetLastError());
  std::vector<double> hC1((size_t)r * r), hC2((size_t)r * r);
  int hstat[2];
  CKF(cudaMemcpyAsync(hC1.data(), C1, sizeof(double) * r * r, cudaMemcpyDeviceToHost, s));
  CKF(cudaMemcpyAsync(hC2.data(), C2, sizeof(double) * r * r, cudaMemcpyDeviceToHost, s));
  CKF(cudaMemcpyAsync(hstat, status, sizeof hstat, cudaMemcpyDeviceToHost, s));
  CKF(cudaStreamSynchronize(s));
  if (hstat[0]) return fail(ctx, TLDA_ERR_NUMERIC, "sketch basis lost rank (CholeskyQR breakdown)");
  if (!host_inverse(hC2, r)) return fail(ctx, TLDA_ERR_NUMERIC, "Q^T Omega is singular");
  std::vector<double> hB((size_t)r * r, 0.0);
  for (int i = 0; i < r; ++i)
    for (int k = 0; k < r; ++k) {
      const double c = hC1[(size_t)i * r + k];
      for (int j = 0; j < r; ++j) hB[(size_t)i * r + j] += c * hC2[(size_t)k * r + j];
    }
  for (int i = 0; i < r; ++i)
    for (int j = i + 1; j < r; ++j) {
      const double v = 0.5 * (hB[(size_t)i * r + j] + hB[(size_t)j * r + i]);
      hB[(size_t)i * r + j] = hB[(size_t)j * r + i] = v;
    }
  CKF(cudaMemcpyAsync(Bm, hB.data(), sizeof(double) * r * r, cudaMemcpyHostToDevice, s));
  k_jacobi<<<1, 512, 0, s>>>(Bm, r, Ev, ev, 40, status + 1);
  CKF(cudaGetLastError());
  std::vector<double> hev(r), hEv((size_t)r * r);
  CKF(cudaMemcpyAsync(hev.data(), ev, sizeof(double) * r, cudaMemcpyDeviceToHost, s));
  CKF(cudaMemcpyAsync(hEv.data(), Ev, sizeof(double) * r * r, cudaMemcpyDeviceToHost, s));
  CKF(cudaStreamSynchronize(s));
  std::vector<int> ord(r);
  for (int i = 0; i < r; ++i) ord[i] = i;
  std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return hev[x] > hev[y]; });
  std::vector<double> hEk((size_t)r * D), hlam(D);
  for (int j = 0; j < D; ++j) {
    hlam[j] = hev[ord[j]];
    for (int i = 0; i < r; ++i) hEk[(size_t)i * D + j] = hEv[(size_t)i * r + ord[j]];
  }
  if (!(hlam[D - 1] > 1e-12 * hlam[0]))
    return fail(ctx, TLDA_ERR_NUMERIC, "the sketched M2 has fewer than D positive eigenvalues");
  CKF(cudaMemcpyAsync(Ek, hEk.data(), sizeof(double) * r * D, cudaMemcpyHostToDevice, s));
  CKF(cudaMemcpyAsync(lam, hlam.data(), sizeof(double) * D, cudaMemcpyHostToDevice, s));
  gemm_nn<double>(Q2, r, Ek, D, U64, D, V, D, r, s);
  if (ctx->whitened)
    CKF(cudaMemcpyAsync(ctx->on_Wold, ctx->W32, sizeof(float) * (size_t)V * D, cudaMemcpyDeviceToDevice, s));
  k_make_w<<<D, 256, 0, s>>>(U64, V, D, lam, ctx->W32, nullptr, nullptr);
  CKF(cudaMemsetAsync(ctx->m1, 0, sizeof(float) * ctx->Dp, s));
  k_wtm1<<<D, 256, 0, s>>>(ctx->W32, M1, V, D, ctx->m1);
  launch_make_u(ctx->W32, ctx->m1, V, D, ctx->Dp, ctx->U32, ctx->U16, s);
  CKF(cudaGetLastError());
  CKF(cudaStreamSynchronize(s));
  ctx->eig = hlam;
  return TLDA_OK;
}

// Phi (D x K, device) <- W^T W_old (W_old^T W_old)^-1 Phi: the factors carried
// from the previous whitening (on_Wold) into the current one (W32).
tlda_status online_rotate(tlda_ctx *ctx, float *Phi) {
  cudaStream_t s = ctx->stream;
  const int V = ctx->V, D = ctx->D, K = ctx->K;
  Scratch sc;
  double *A = nullptr, *G = nullptr;
  CKF(sc.get(&A, (size_t)D * D));
  CKF(sc.get(&G, (size_t)D * D));
  gemm_tn64<float, float>(ctx->W32, D, ctx->on_Wold, D, A, D, D, D, V, s);
  gemm_tn64<float, float>(ctx->on_Wold, D, ctx->on_Wold, D, G, D, D, D, V, s);
  CKF(cudaGetLastError());
  std::vector<double> hA((size_t)D * D), hG((size_t)D * D);
  std::vector<float> hP((size_t)D * K);
  CKF(cudaMemcpyAsync(hA.data(), A, sizeof(double) * D * D, cudaMemcpyDeviceToHost, s));
  CKF(cudaMemcpyAsync(hG.data(), G, sizeof(double) * D * D, cudaMemcpyDeviceToHost, s));
  CKF(cudaMemcpyAsync(hP.data(), Phi, sizeof(float) * D * K, cudaMemcpyDeviceToHost, s));
  CKF(cudaStreamSynchronize(s));
  if (!host_inverse(hG, D)) return fail(ctx, TLDA_ERR_NUMERIC, "W^T W of the previous whitening is singular");
  std::vector<double> R((size_t)D * D, 0.0), hN((size_t)D * K, 0.0);
  for (int i = 0; i < D; ++i)
    for (int k = 0; k < D; ++k) {
      const double a = hA[(size_t)i * D + k];
      for (int j = 0; j < D; ++j) R[(size_t)i * D + j] += a * hG[(size_t)k * D + j];
    }
  for (int i = 0; i < D; ++i)
    for (int k = 0; k < D; ++k) {
      const double rr = R[(size_t)i * D + k];
      for (int j = 0; j < K; ++j) hN[(size_t)i * K + j] += rr * hP[(size_t)k * K + j];
    }
  for (size_t e = 0; e < hP.size(); ++e) hP[e] = (float)hN[e];
  CKF(cudaMemcpyAsync(Phi, hP.data(), sizeof(float) * D * K, cudaMemcpyHostToDevice, s));
  CKF(cudaStreamSynchronize(s));
  return TLDA_OK;
}

}  // namespace

extern "C" {

tlda_status tlda_fit_moments(tlda_ctx *ctx, const tlda_csr *chunk, uint32_t flags) {
  if (!ctx) return TLDA_ERR_INVALID;
  if (!(flags & (TLDA_ACCUMULATE | TLDA_FINALIZE))) return fail(ctx, TLDA_ERR_INVALID, "flags must hold ACCUMULATE and/or FINALIZE");
  if (ctx->V > kMaxFitV) return fail(ctx, TLDA_ERR_OOM, "fit_moments keeps a dense V x V pair-count matrix: V <= 65536");
  if (flags & TLDA_ACCUMULATE) {
    if (!chunk) return fail(ctx, TLDA_ERR_INVALID, "chunk is NULL");
    if (chunk->vocab != ctx->V || chunk->n_docs < 0 || !chunk->indptr ||
        (chunk->n_docs > 0 && (!chunk->indices || !chunk->counts)))
      return fail(ctx, TLDA_ERR_INVALID, "bad chunk");
    const size_t V = ctx->V;
    if (!ctx->P64) {
      CKF(dalloc(&ctx->P64, V * V));
      if (!ctx->Ccnt) CKF(dalloc(&ctx->Ccnt, V));
      if (!ctx->TS) CKF(dalloc(&ctx->TS, 3));
      CKF(dalloc(&ctx->fit_err, 1));
    }
    if (!ctx->fit_open) {
      CKF(cudaMemsetAsync(ctx->P64, 0, sizeof(double) * V * V, ctx->stream));
      CKF(cudaMemsetAsync(ctx->Ccnt, 0, sizeof(unsigned long long) * V, ctx->stream));
      CKF(cudaMemsetAsync(ctx->TS, 0, sizeof(unsigned long long) * 3, ctx->stream));
      CKF(cudaMemsetAsync(ctx->fit_err, 0, sizeof(int), ctx->stream));
      ctx->fit_open = true;
    }
    if (chunk->n_docs > 0) {
      const long long threads = (long long)chunk->n_docs * 32;
      k_fit_accumulate<<<(unsigned)((threads + 255) / 256), 256, 0, ctx->stream>>>(*chunk, ctx->V, ctx->P64, ctx->Ccnt,
                                                                                  ctx->TS, ctx->fit_err);
      CKF(cudaGetLastError());
    }
  }
  if (flags & TLDA_FINALIZE) {
    if (!ctx->fit_open) return fail(ctx, TLDA_ERR_STATE, "FINALIZE without any ACCUMULATE");
    ctx->fit_open = false;
    return finalize(ctx);
  }
  return TLDA_OK;
}

tlda_status tlda_get_counts(const tlda_ctx *cctx, int64_t *C, int64_t *T, int64_t *S2, int64_t *S3) {
  tlda_ctx *ctx = const_cast<tlda_ctx *>(cctx);
  if (!ctx) return TLDA_ERR_INVALID;
  if (!ctx->Ccnt || !ctx->TS) return fail(ctx, TLDA_ERR_STATE, "no accumulated statistics");
  unsigned long long ts[3];
  CKF(cudaStreamSynchronize(ctx->stream));
  CKF(cudaMemcpy(ts, ctx->TS, sizeof ts, cudaMemcpyDeviceToHost));
  if (C) CKF(cudaMemcpy(C, ctx->Ccnt, sizeof(int64_t) * ctx->V, cudaMemcpyDeviceToHost));
  if (T) *T = (int64_t)ts[0];
  if (S2) *S2 = (int64_t)ts[1];
  if (S3) *S3 = (int64_t)ts[2];
  return TLDA_OK;
}

tlda_status tlda_unwhiten_topics(tlda_ctx *ctx, const float *Phi, double *mu_out, double *alpha_out, uint32_t flags) {
  if (!ctx || !Phi || !mu_out || !alpha_out) return fail(ctx, TLDA_ERR_INVALID, "NULL argument");
  if (!ctx->whitened) return fail(ctx, TLDA_ERR_STATE, "no whitening: fit or set one first");
  cudaStream_t s = ctx->stream;
  const int V = ctx->V, D = ctx->D, K = ctx->K;
  Scratch sc;
  double *W64 = nullptr, *G = nullptr, *Linv = nullptr, *LinvT = nullptr, *Ginv = nullptr, *T = nullptr;
  double *mu = nullptr, *al = nullptr;
  int *status = nullptr;
  CKF(sc.get(&W64, (size_t)V * D));
  CKF(sc.get(&G, (size_t)D * D));
  CKF(sc.get(&Linv, (size_t)D * D));
  CKF(sc.get(&LinvT, (size_t)D * D));
  CKF(sc.get(&Ginv, (size_t)D * D));
  CKF(sc.get(&T, (size_t)D * K));
  CKF(sc.get(&status, 1, true));
  const bool host = flags & TLDA_HOST_OUTPUT;
  if (host) {
    CKF(sc.get(&mu, (size_t)V * K));
    CKF(sc.get(&al, (size_t)K));
  } else {
    mu = mu_out;
    al = alpha_out;
  }
  k_f2d<<<(unsigned)(((long long)V * D + 255) / 256), 256, 0, s>>>(ctx->W32, W64, (long long)V * D);
  gemm_tn64<double, double>(W64, D, W64, D, G, D, D, D, V, s);         // W^T W
  k_chol_inv<<<1, 256, 0, s>>>(G, D, Linv, status);
  k_transpose_rr<<<(D * D + 255) / 256, 256, 0, s>>>(Linv, D, nullptr, LinvT);
  gemm_nn<double>(LinvT, D, Linv, D, Ginv, D, D, D, D, s);              // (W^T W)^-1 = L^-T L^-1
  k_unwhiten_coef<<<1, 256, 0, s>>>(Phi, D, K, Ginv, T, al);
  gemm_nn<double>(W64, D, T, K, mu, K, V, K, D, s);                     // mu = W (W^T W)^-1 Phi diag(|phi|^2)
  k_clip_norm<<<K, 256, 0, s>>>(mu, V, K);
  CKF(cudaGetLastError());
  int hst = 0;
  CKF(cudaMemcpyAsync(&hst, status, sizeof hst, cudaMemcpyDeviceToHost, s));
  if (host) {
    CKF(cudaMemcpyAsync(mu_out, mu, sizeof(double) * (size_t)V * K, cudaMemcpyDeviceToHost, s));
    CKF(cudaMemcpyAsync(alpha_out, al, sizeof(double) * K, cudaMemcpyDeviceToHost, s));
  }
  CKF(cudaStreamSynchronize(s));
  if (hst) return fail(ctx, TLDA_ERR_NUMERIC, "W^T W is not positive definite");
  return TLDA_OK;
}

tlda_status tlda_online_begin(tlda_ctx *ctx, const double *Omega, int32_t r) {
  if (!ctx) return TLDA_ERR_INVALID;
  if (!Omega || r < ctx->D || r > kMaxDim || (r & 1) || r > ctx->V)
    return fail(ctx, TLDA_ERR_INVALID, "the sketch needs an even r with D <= r <= min(V, 512)");
  const size_t V = ctx->V;
  if (ctx->on_r != r) {
    if (ctx->on_Om) cudaFree(ctx->on_Om);
    if (ctx->on_Z) cudaFree(ctx->on_Z);
    ctx->on_Om = ctx->on_Z = nullptr;
    ctx->on_r = 0;
    CKF(dalloc(&ctx->on_Om, V * r));
    CKF(dalloc(&ctx->on_Z, V * r));
    ctx->on_r = r;
  }
  if (!ctx->on_C) CKF(dalloc(&ctx->on_C, V));
  if (!ctx->on_TS) CKF(dalloc(&ctx->on_TS, 3));
  if (!ctx->on_err) CKF(dalloc(&ctx->on_err, 1));
  if (!ctx->on_Wold) CKF(dalloc(&ctx->on_Wold, V * ctx->D));
  cudaStream_t s = ctx->stream;
  CKF(cudaMemcpyAsync(ctx->on_Om, Omega, sizeof(double) * V * r, cudaMemcpyDeviceToDevice, s));
  CKF(cudaMemsetAsync(ctx->on_Z, 0, sizeof(double) * V * r, s));
  CKF(cudaMemsetAsync(ctx->on_C, 0, sizeof(unsigned long long) * V, s));
  CKF(cudaMemsetAsync(ctx->on_TS, 0, sizeof(unsigned long long) * 3, s));
  CKF(cudaMemsetAsync(ctx->on_err, 0, sizeof(int), s));
  CKF(cudaStreamSynchronize(s));
  ctx->on_active = true;
  return TLDA_OK;
}

tlda_status tlda_online_pass(tlda_ctx *ctx, const tlda_csr *corpus, const int64_t *batch_offsets, int32_t n_batches,
                             float *Phi, float lr, int32_t rewhiten_every, double *loss_out) {
  if (!ctx) return TLDA_ERR_INVALID;
  if (!ctx->on_active) return fail(ctx, TLDA_ERR_STATE, "tlda_online_begin has not been called");
  if (!corpus || corpus->vocab != ctx->V || corpus->n_docs < 0 || !corpus->indptr ||
      (corpus->n_docs > 0 && (!corpus->indices || !corpus->counts)))
    return fail(ctx, TLDA_ERR_INVALID, "bad corpus");
  if (!Phi || !batch_offsets || n_batches < 0 || rewhiten_every < 1)
    return fail(ctx, TLDA_ERR_INVALID, "bad online pass arguments");
  for (int b = 0; b < n_batches; ++b) {
    const int64_t d0 = batch_offsets[b], d1 = batch_offsets[b + 1];
    if (d0 < 0 || d1 < d0 || d1 > corpus->n_docs) return fail(ctx, TLDA_ERR_INVALID, "batch offsets out of range");
  }
  cudaStream_t s = ctx->stream;
  for (int b0 = 0; b0 < n_batches; b0 += rewhiten_every) {
    const int b1 = std::min(n_batches, b0 + rewhiten_every);
    const int64_t d0 = batch_offsets[b0], d1 = batch_offsets[b1];
    const int nd = (int)(d1 - d0);
    if (nd > 0) {
      const long long threads = (long long)nd * 32;
      k_online_acc<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(corpus->indptr + d0, corpus->indices,
                                                                     corpus->counts, nd, ctx->V, ctx->on_r,
                                                                     ctx->on_Om, ctx->on_Z, ctx->on_C,
                                                                     ctx->on_TS, ctx->on_err);
      CKF(cudaGetLastError());
    }
    const bool had = ctx->whitened;  // Phi is carried over from the context's current whitening
    tlda_status st = online_rewhiten(ctx);
    if (st) return st;
    if (had) {
      st = online_rotate(ctx, Phi);
      if (st) return st;
    }
    ctx->whitened = true;
    st = tlda_cp_pass(ctx, corpus, batch_offsets + b0, b1 - b0, Phi, lr, 0, loss_out ? loss_out + b0 : nullptr);
    if (st) return st;
  }
  return TLDA_OK;
}

}  // extern "C"
