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
#include <functional>
#include <vector>

#include "scan.cuh"
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

__global__ void k_d2f(const double *x, float *y, long long n) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) y[e] = (float)x[e];
}

// ------------------------------------------------------------------ small dense FP64
// Transpose r x r (FP64 -> FP32 for the Y Linv^T product).
__global__ void k_transpose_rr(const double *A, int r, float *AT32, double *AT64) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= r * r) return;
  const int i = e / r, j = e % r;
  if (AT32) AT32[j * r + i] = (float)A[e];
  if (AT64) AT64[j * r + i] = A[e];
}

// Control block of the grid-wide Jacobi: the grid barrier's arrival counter,
// an abort flag, the sweep count, and each block's partial sums of the squared
// off-diagonal and total entries (two slots, by sweep parity).
constexpr int kJacThreads = 256, kJacMaxGrid = 256;
struct JacCtl {
  unsigned bar;
  int abort;
  int sweeps;
  int pad;
  double part[2][2][kJacMaxGrid];
};

__device__ __forceinline__ unsigned jac_ld_acquire(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid barrier of a cooperative launch (every block resident): a release
// increment of the arrival counter, then acquire loads until it reaches
// `target`; bounded to about a second; false if it expired here or any block
// flagged an abort.
__device__ bool jac_sync(JacCtl *ctl, unsigned target, int *s_ok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&ctl->bar) : "memory");
    const long long t0 = clock64();
    while (jac_ld_acquire(&ctl->bar) < target) {
      if (*reinterpret_cast<volatile int *>(&ctl->abort)) {
        ok = 0;
        break;
      }
      if (clock64() - t0 > 2000000000ll) {
        atomicExch(&ctl->abort, 1);
        ok = 0;
        break;
      }
    }
    *reinterpret_cast<volatile int *>(s_ok) = ok;
  }
  __syncthreads();
  return *reinterpret_cast<volatile int *>(s_ok) != 0;
}

// Cyclic Jacobi for a symmetric r x r FP64 matrix A (r even, global memory,
// overwritten), round-robin ordering so each round applies r/2 disjoint
// rotations in parallel (Golub & Van Loan, "Matrix Computations", sec. 8.5,
// parallel ordering).  Rotation of pair (p, q): tau = (a_qq - a_pp)/(2 a_pq),
// t = sign(tau)/(|tau| + sqrt(1 + tau^2)), c = 1/sqrt(1 + t^2), s = t c.
// Because the rotations of one round are disjoint, A <- J^T A J is applied in
// one pass over the 2 x 2 blocks (pair k rows, pair l columns), each block
// rotated on the left by pair k and on the right by pair l; the eigenvectors
// are kept as rows, Et <- J^T Et.  The rounds are spread over the whole grid
// (FP64 arithmetic is scarce per SM), one grid barrier per round; every
// block derives the round's rotations itself.  Et starts as I; on return
// eval[i] = A_ii and row i of Et is its eigenvector.
// Sweeps stop when the off-diagonal mass is below 1e-26 r^2 of the total,
// i.e. entries near 1e-13 of the scale (or after max_sweeps).
__global__ void __launch_bounds__(kJacThreads) k_jacobi(double *__restrict__ A, int r, double *__restrict__ Et,
                                                       double *__restrict__ eval, int max_sweeps,
                                                       JacCtl *ctl) {
  __shared__ double cs[kMaxDim / 2], sn[kMaxDim / 2];
  __shared__ int pp[kMaxDim / 2], qq[kMaxDim / 2];
  __shared__ double red_o[kJacThreads / 32], red_t[kJacThreads / 32];
  __shared__ int s_ok, s_done;
  const int G = gridDim.x, tid = threadIdx.x, nt = blockDim.x;
  const int gt = blockIdx.x * nt + tid, gn = G * nt;
  const int h = r / 2, rr = r * r;
  unsigned nbar = 0;
  for (int e = gt; e < rr; e += gn) {
    const int i = e / r, j = e % r;
    if (i < j) {
      const double v = 0.5 * (A[i * r + j] + A[j * r + i]);
      A[i * r + j] = v;
      A[j * r + i] = v;
    }
    Et[e] = (i == j) ? 1.0 : 0.0;
  }
  if (!jac_sync(ctl, ++nbar * G, &s_ok)) return;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    double o = 0.0, t = 0.0;
    for (int e = gt; e < rr; e += gn) {
      const double v = __ldcg(A + e);
      t += v * v;
      if (e / r != e % r) o += v * v;
    }
    for (int m = 16; m > 0; m >>= 1) {
      o += __shfl_xor_sync(0xffffffffu, o, m);
      t += __shfl_xor_sync(0xffffffffu, t, m);
    }
    if ((tid & 31) == 0) {
      red_o[tid >> 5] = o;
      red_t[tid >> 5] = t;
    }
    __syncthreads();
    if (tid == 0) {
      double so = 0.0, st = 0.0;
      for (int w = 0; w < nt / 32; ++w) {
        so += red_o[w];
        st += red_t[w];
      }
      ctl->part[sweep & 1][0][blockIdx.x] = so;
      ctl->part[sweep & 1][1][blockIdx.x] = st;
    }
    if (!jac_sync(ctl, ++nbar * G, &s_ok)) return;
    if (tid == 0) {  // every block sums the partials in the same order
      double so = 0.0, st = 0.0;
      for (int g = 0; g < G; ++g) {
        so += __ldcg(&ctl->part[sweep & 1][0][g]);
        st += __ldcg(&ctl->part[sweep & 1][1][g]);
      }
      s_done = so <= 1e-26 * (double)r * r * st;
    }
    __syncthreads();
    if (s_done) break;
    for (int round = 0; round < r - 1; ++round) {
      for (int k = tid; k < h; k += nt) {
        // round-robin pairing: slot 0 holds index 0, the others rotate
        const int sa = k, sb = r - 1 - k;
        int p = sa == 0 ? 0 : 1 + (sa - 1 + round) % (r - 1);
        int q = sb == 0 ? 0 : 1 + (sb - 1 + round) % (r - 1);
        if (p > q) {
          const int tmp = p;
          p = q;
          q = tmp;
        }
        const double apq = __ldcg(A + p * r + q);
        const double app = __ldcg(A + p * r + p), aqq = __ldcg(A + q * r + q);
        double c = 1.0, sv = 0.0;
        if (apq != 0.0) {
          const double tau = (aqq - app) / (2.0 * apq);
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
      // 2 x 2 blocks, two per thread per iteration (loads before stores)
      const int nb = h * h;
      for (int w0 = gt; w0 < nb; w0 += 2 * gn) {
        double x[2][4];
        int base[2][4];
        bool ok[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int w = w0 + u * gn;
          ok[u] = w < nb;
          const int k = ok[u] ? w / h : 0, l = ok[u] ? w % h : 0;
          const int pk = pp[k], qk = qq[k], pl = pp[l], ql = qq[l];
          base[u][0] = pk * r + pl;
          base[u][1] = pk * r + ql;
          base[u][2] = qk * r + pl;
          base[u][3] = qk * r + ql;
#pragma unroll
          for (int v = 0; v < 4; ++v) x[u][v] = ok[u] ? __ldcg(A + base[u][v]) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          if (!ok[u]) continue;
          const int w = w0 + u * gn, k = w / h, l = w % h;
          const double ck = cs[k], sk = sn[k], cl = cs[l], sl = sn[l];
          const double a1 = ck * x[u][0] - sk * x[u][2], b1 = ck * x[u][1] - sk * x[u][3];
          const double c1 = sk * x[u][0] + ck * x[u][2], d1 = sk * x[u][1] + ck * x[u][3];
          A[base[u][0]] = cl * a1 - sl * b1;
          A[base[u][1]] = (k == l) ? 0.0 : sl * a1 + cl * b1;
          A[base[u][2]] = (k == l) ? 0.0 : cl * c1 - sl * d1;
          A[base[u][3]] = sl * c1 + cl * d1;
        }
      }
      // eigenvector rows: Et[p] <- c Et[p] - s Et[q], Et[q] <- s Et[p] + c Et[q]
      const int ne = h * r;
      for (int w0 = gt; w0 < ne; w0 += 2 * gn) {
        double ep[2], eq[2];
        int ip[2], iq[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int w = w0 + u * gn;
          const int k = w < ne ? w / r : 0, j = w < ne ? w % r : 0;
          ip[u] = pp[k] * r + j;
          iq[u] = qq[k] * r + j;
          ep[u] = w < ne ? __ldcg(Et + ip[u]) : 0.0;
          eq[u] = w < ne ? __ldcg(Et + iq[u]) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int w = w0 + u * gn;
          if (w >= ne) continue;
          const int k = w / r;
          const double c = cs[k], sv = sn[k];
          Et[ip[u]] = c * ep[u] - sv * eq[u];
          Et[iq[u]] = sv * ep[u] + c * eq[u];
        }
      }
      if (!jac_sync(ctl, ++nbar * G, &s_ok)) return;
    }
  }
  for (int i = gt; i < r; i += gn) eval[i] = __ldcg(A + i * r + i);
  if (gt == 0) ctl->sweeps = sweep;
}


// Cholesky factor and inverse of a symmetric positive definite r x r FP64
// matrix A (overwritten): A = L L^T by right-looking elimination (column j:
// l_jj = sqrt(a_jj), l_ij = a_ij / l_jj, then a_ik -= l_ij l_kj for
// j < k <= i), and X = L^-1 by right-looking forward substitution on
// Z = diag(L) X (z_ic -= l_ik / l_kk z_kc for i > k, then x_ic = z_ic / l_ii).
// Spread over the grid, one grid barrier per column of each phase.  L (lower,
// zeros above) and the scratch Z are required; Linv, LinvT64 = L^-T and
// LinvT32 (FP32) are written when given.  status: 1 if a pivot was not
// positive (it is taken as 1), 2 if a grid barrier expired.
__global__ void __launch_bounds__(kJacThreads) k_chol_inv(double *__restrict__ A, int r, double *__restrict__ L,
                                                         double *__restrict__ Z, double *Linv, double *LinvT64,
                                                         float *LinvT32, int *status, JacCtl *ctl) {
  __shared__ int s_ok;
  const int G = gridDim.x, gt = blockIdx.x * blockDim.x + threadIdx.x, gn = G * blockDim.x;
  const int rr = r * r;
  unsigned nbar = 0;
  for (int e = gt; e < rr; e += gn) {
    const int i = e / r, k = e % r;
    Z[e] = (i == k) ? 1.0 : 0.0;
    if (k > i) L[e] = 0.0;
  }
  for (int j = 0; j < r; ++j) {
    double d = __ldcg(A + j * r + j);
    if (!(d > 0.0)) {
      if (gt == 0) atomicMax(status, 1);
      d = 1.0;
    }
    d = sqrt(d);
    const double inv = 1.0 / d;
    const int m = r - j - 1;
    for (int e = gt; e <= m; e += gn) L[(j + e) * r + j] = e == 0 ? d : __ldcg(A + (j + e) * r + j) * inv;
    for (int e = gt; e < m * m; e += gn) {
      const int i = j + 1 + e / m, k = j + 1 + e % m;
      if (k <= i) A[i * r + k] = __ldcg(A + i * r + k) - (__ldcg(A + i * r + j) * inv) * (__ldcg(A + k * r + j) * inv);
    }
    if (!jac_sync(ctl, ++nbar * G, &s_ok)) {
      if (threadIdx.x == 0) atomicMax(status, 2);
      return;
    }
  }
  for (int k = 0; k < r - 1; ++k) {
    const double f = 1.0 / __ldcg(L + k * r + k);
    const int m = r - k - 1, w = k + 1;  // rows k+1 .. r-1, columns 0 .. k
    for (int e = gt; e < m * w; e += gn) {
      const int i = k + 1 + e / w, c = e % w;
      Z[i * r + c] = __ldcg(Z + i * r + c) - __ldcg(L + i * r + k) * f * __ldcg(Z + k * r + c);
    }
    if (!jac_sync(ctl, ++nbar * G, &s_ok)) {
      if (threadIdx.x == 0) atomicMax(status, 2);
      return;
    }
  }
  for (int e = gt; e < rr; e += gn) {
    const int i = e / r, c = e % r;
    const double x = c <= i ? __ldcg(Z + e) / __ldcg(L + i * r + i) : 0.0;
    if (Linv) Linv[e] = x;
    if (LinvT64) LinvT64[c * r + i] = x;
    if (LinvT32) LinvT32[c * r + i] = (float)x;
  }
}

// B = C1 C2^-1 for r x r FP64 matrices (C2 general, row-major): Gauss-Jordan
// elimination with partial pivoting (largest |pivot| among the rows not yet
// used, lowest index on ties) of C2^T B^T = C1^T, spread over the grid, one
// grid barrier per column.  M and R are r x r scratch (the system and its
// right-hand sides, eliminated in place; column j of M is left as it was once
// eliminated, being read no more).  status: 1 if a pivot is zero (C2
// singular), 2 if a grid barrier expired.
__global__ void __launch_bounds__(kJacThreads) k_solve_right(const double *__restrict__ C1,
                                                            const double *__restrict__ C2, int r,
                                                            double *__restrict__ M, double *__restrict__ R,
                                                            double *__restrict__ B, int *status, JacCtl *ctl) {
  __shared__ unsigned char used[kMaxDim];
  __shared__ int piv[kMaxDim];
  __shared__ double red_v[kJacThreads / 32];
  __shared__ int red_i[kJacThreads / 32];
  __shared__ int s_ok, s_p;
  const int G = gridDim.x, tid = threadIdx.x, nt = blockDim.x;
  const int gt = blockIdx.x * nt + tid, gn = G * nt, rr = r * r;
  unsigned nbar = 0;
  for (int e = gt; e < rr; e += gn) {
    const int i = e / r, c = e % r;
    M[e] = C2[c * r + i];
    R[e] = C1[c * r + i];
  }
  for (int i = tid; i < r; i += nt) used[i] = 0;
  if (!jac_sync(ctl, ++nbar * G, &s_ok)) {
    if (tid == 0) atomicMax(status, 2);
    return;
  }
  for (int j = 0; j < r; ++j) {
    double bv = -1.0;
    int bi = r;
    for (int i = tid; i < r; i += nt)
      if (!used[i]) {
        const double v = fabs(__ldcg(M + i * r + j));
        if (v > bv) {
          bv = v;
          bi = i;
        }
      }
    for (int m = 16; m > 0; m >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, bv, m);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, m);
      if (ov > bv || (ov == bv && oi < bi)) {
        bv = ov;
        bi = oi;
      }
    }
    if ((tid & 31) == 0) {
      red_v[tid >> 5] = bv;
      red_i[tid >> 5] = bi;
    }
    __syncthreads();
    if (tid == 0) {
      for (int w = 1; w < nt / 32; ++w)
        if (red_v[w] > bv || (red_v[w] == bv && red_i[w] < bi)) {
          bv = red_v[w];
          bi = red_i[w];
        }
      if (!(bv > 0.0)) {
        if (blockIdx.x == 0) atomicMax(status, 1);
        if (bi >= r)  // no finite candidate: take the first unused row
          for (bi = 0; bi < r && used[bi]; ++bi) {
          }
      }
      used[bi] = 1;
      piv[j] = bi;
      s_p = bi;
    }
    __syncthreads();
    const int p = s_p;
    const double mpj = __ldcg(M + p * r + j);
    const double inv = mpj != 0.0 ? 1.0 / mpj : 0.0;
    const int wm = r - j - 1, width = wm + r;  // columns j+1 .. r-1 of M, then every column of R
    for (int e = gt; e < r * width; e += gn) {
      const int i = e / width, c = e % width;
      if (i == p) continue;
      const double f = __ldcg(M + i * r + j) * inv;
      if (c < wm) {
        const int cc = j + 1 + c;
        M[i * r + cc] = __ldcg(M + i * r + cc) - f * __ldcg(M + p * r + cc);
      } else {
        const int cc = c - wm;
        R[i * r + cc] = __ldcg(R + i * r + cc) - f * __ldcg(R + p * r + cc);
      }
    }
    if (!jac_sync(ctl, ++nbar * G, &s_ok)) {
      if (tid == 0) atomicMax(status, 2);
      return;
    }
  }
  // row j of B^T is the pivot row of column j, divided by its pivot
  for (int e = gt; e < rr; e += gn) {
    const int j = e / r, c = e % r, p = piv[j];
    const double d = __ldcg(M + p * r + j);
    B[c * r + j] = d != 0.0 ? __ldcg(R + p * r + c) / d : 0.0;
  }
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

// Blocks of the grid-wide Jacobi, Cholesky and solve kernels: one per SM, all
// co-resident (cooperative launch).
int coop_grid() {
  static int g = -1;
  if (g >= 0) return g;
  int dev = 0, sms = 0, coop = 0, pj = 0, pc = 0, ps = 0;
  g = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return g;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (!coop || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pj, k_jacobi, kJacThreads, 0) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pc, k_chol_inv, kJacThreads, 0) != cudaSuccess || pj < 1 ||
      pc < 1 || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ps, k_solve_right, kJacThreads, 0) != cudaSuccess ||
      ps < 1)
    return g;
  g = std::min(sms, kJacMaxGrid);
  return g;
}

// The context's control block for those kernels, zeroed on its stream.
tlda_status coop_ctl(tlda_ctx *ctx, JacCtl **out, cudaStream_t s) {
  if (coop_grid() < 1) return fail(ctx, TLDA_ERR_CUDA, "cooperative launch unavailable for the dense FP64 kernels");
  if (!ctx->coop_ctl) CKF(cudaMalloc(&ctx->coop_ctl, sizeof(JacCtl)));
  CKF(cudaMemsetAsync(ctx->coop_ctl, 0, sizeof(JacCtl), s));
  *out = static_cast<JacCtl *>(ctx->coop_ctl);
  return TLDA_OK;
}

// Diagonalises the symmetric r x r matrix A (device, overwritten): eigenvalues
// to ev, eigenvector rows to Et.  Synchronises.
tlda_status run_jacobi(tlda_ctx *ctx, double *A, int r, double *Et, double *ev, cudaStream_t s) {
  JacCtl *ctl = nullptr;
  if (tlda_status st = coop_ctl(ctx, &ctl, s)) return st;
  int ms = 40;
  void *args[] = {&A, &r, &Et, &ev, &ms, &ctl};
  CKF(cudaLaunchCooperativeKernel((const void *)k_jacobi, dim3(coop_grid()), dim3(kJacThreads), args, 0, s));
  int hs[3];
  CKF(cudaMemcpyAsync(hs, &ctl->bar, sizeof hs, cudaMemcpyDeviceToHost, s));
  CKF(cudaStreamSynchronize(s));
  if (hs[1]) return fail(ctx, TLDA_ERR_TIMEOUT, "grid barrier of the Jacobi eigensolver expired");
  ctx->jacobi_sweeps = hs[2];
  return TLDA_OK;
}

// Enqueues k_chol_inv (asynchronous; failures land in *status).
tlda_status run_chol_inv(tlda_ctx *ctx, double *A, int r, double *L, double *Z, double *Linv, double *LinvT64,
                         float *LinvT32, int *status, cudaStream_t s) {
  JacCtl *ctl = nullptr;
  if (tlda_status st = coop_ctl(ctx, &ctl, s)) return st;
  void *args[] = {&A, &r, &L, &Z, &Linv, &LinvT64, &LinvT32, &status, &ctl};
  CKF(cudaLaunchCooperativeKernel((const void *)k_chol_inv, dim3(coop_grid()), dim3(kJacThreads), args, 0, s));
  return TLDA_OK;
}

// Enqueues k_solve_right: B = C1 C2^-1 (asynchronous; failures land in *status).
tlda_status run_solve_right(tlda_ctx *ctx, const double *C1, const double *C2, int r, double *M, double *R,
                            double *B, int *status, cudaStream_t s) {
  JacCtl *ctl = nullptr;
  if (tlda_status st = coop_ctl(ctx, &ctl, s)) return st;
  void *args[] = {&C1, &C2, &r, &M, &R, &B, &status, &ctl};
  CKF(cudaLaunchCooperativeKernel((const void *)k_solve_right, dim3(coop_grid()), dim3(kJacThreads), args, 0, s));
  return TLDA_OK;
}

// Maps the status word of k_chol_inv / k_solve_right to the call's result.
tlda_status chol_status(tlda_ctx *ctx, int st, const char *breakdown) {
  if (st >= 2) return fail(ctx, TLDA_ERR_TIMEOUT, "grid barrier of a dense FP64 kernel expired");
  if (st == 1) return fail(ctx, TLDA_ERR_NUMERIC, breakdown);
  return TLDA_OK;
}

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
  double *Zr = nullptr;
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
  CKF(sc.get(&Zr, (size_t)r * r));
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
  auto cholqr_pass = [&](const float *in, float *out) -> tlda_status {
    gemm_tn64<float, float>(in, r, in, r, G, r, r, r, V, s);
    if (tlda_status st = run_chol_inv(ctx, G, r, Linv, Zr, nullptr, nullptr, LinvT32, status, s)) return st;
    gemm_nn<float>(in, r, LinvT32, r, out, r, V, r, r, s);
    return TLDA_OK;
  };
  // CholeskyQR2 of Y into Qf (Y is clobbered)
  auto cholqr2 = [&]() -> tlda_status {
    if (tlda_status st = cholqr_pass(Y, Qf)) return st;
    if (tlda_status st = cholqr_pass(Qf, Y)) return st;
    CKF(cudaMemcpyAsync(Qf, Y, sizeof(float) * (size_t)V * r, cudaMemcpyDeviceToDevice, s));
    return TLDA_OK;
  };
  gemm_nn<float>(M2, V, Om, r, Y, r, V, r, V, s);
  if (tlda_status st = cholqr2()) return st;
  const int n_iter = 24;
  for (int it = 0; it < n_iter; ++it) {
    gemm_nn<float>(M2, V, Qf, r, Y, r, V, r, V, s);
    if (tlda_status st = cholqr2()) return st;
  }
  // FP64 Rayleigh-Ritz on the exact M2 = sP P - a0 M1 M1^T
  k_f2d<<<(unsigned)(((long long)V * r + 255) / 256), 256, 0, s>>>(Qf, Q64, (long long)V * r);
  // one FP64 CholeskyQR pass to make Q64 orthonormal to FP64 accuracy
  gemm_tn64<double, double>(Q64, r, Q64, r, G, r, r, r, V, s);
  if (tlda_status st = run_chol_inv(ctx, G, r, Linv, Zr, nullptr, LinvT64, nullptr, status, s)) return st;
  gemm_nn<double>(Q64, r, LinvT64, r, Z64, r, V, r, r, s);
  cudaMemcpyAsync(Q64, Z64, sizeof(double) * (size_t)V * r, cudaMemcpyDeviceToDevice, s);
  gemm_nn<double>(ctx->P64, V, Q64, r, Z64, r, V, r, V, s);
  gemm_tn64<double, double>(M1, 1, Q64, r, m1q, r, 1, r, V, s);
  k_rank1_fix<<<(unsigned)(((long long)V * r + 255) / 256), 256, 0, s>>>(Z64, M1, m1q, V, r, sP, a0);
  gemm_tn64<double, double>(Q64, r, Z64, r, Bm, r, r, r, V, s);
  CKF(cudaGetLastError());
  if (tlda_status js = run_jacobi(ctx, Bm, r, Ev, ev, s)) return js;
  std::vector<double> hev(r), hEv((size_t)r * r);
  int hstat[2];
  CKF(cudaMemcpyAsync(hev.data(), ev, sizeof(double) * r, cudaMemcpyDeviceToHost, s));
  CKF(cudaMemcpyAsync(hEv.data(), Ev, sizeof(double) * r * r, cudaMemcpyDeviceToHost, s));
  CKF(cudaMemcpyAsync(hstat, status, sizeof hstat, cudaMemcpyDeviceToHost, s));
  CKF(cudaStreamSynchronize(s));
  if (tlda_status st = chol_status(ctx, hstat[0], "subspace basis lost rank (CholeskyQR breakdown)")) return st;
  // order the Ritz pairs by descending value and keep D of them
  std::vector<int> ord(r);
  for (int i = 0; i < r; ++i) ord[i] = i;
  std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return hev[x] > hev[y]; });
  std::vector<double> hEk((size_t)r * D), hlam(D);
  for (int j = 0; j < D; ++j) {
    hlam[j] = hev[ord[j]];
    for (int i = 0; i < r; ++i) hEk[(size_t)i * D + j] = hEv[(size_t)ord[j] * r + i];
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
// The sketch Z = P Omega of the pair counts P = sum_d (f_d f_d^T - diag f_d),
// taken over a piece of documents at a time as
//   Z += F^T S - diag(c) Omega,   S = F Omega,   c = F^T 1,
// with F the piece's document x word counts.  Row m of F^T S sums f_dm s_d
// over the documents holding word m, which needs the piece's nonzeros grouped
// by word (its transpose).  Per piece:
//   k_sk_rows     one warp per document: validation, the token statistics,
//                 s_d = f_d^T Omega into row d of S, and the number of
//                 nonzeros of each word;
//   scan          those numbers become each word's first slot;
//   k_sk_scatter  one warp per document: each nonzero (document, count) into
//                 a slot of its word;
//   k_sk_z        one warp per run of kSkRun consecutive slots: for each word
//                 met, the run's part of sum_d f_dm (s_d - Omega_m) added to
//                 Z_m and sum_d f_dm to C_m; plainly when all the word's
//                 slots lie in the run, with FP64 atomics when they cross its
//                 ends.
// Precision: the products and the sums within a document (s_d) and within a
// run (at most kSkRun terms) are FP32, from an FP32 copy of Omega; Z
// accumulates the runs in FP64.  (GB300's FP64 rate is 1/64 of its FP32
// rate: with FP64 products the sketch would be bound by them.)
// The per-nonzero work is two row gathers (Omega_m, then s_d) and no atomics
// on Z.  The slots of a word are filled in no fixed order, so Z is not
// bitwise reproducible (its sums are reordered).  A document that fails
// validation adds nothing and sets *err.
constexpr int kSkPieceDocs = 262144;          // documents per piece (rows of S)
constexpr long long kSkPieceNnz = 16ll << 20;  // nonzeros per piece (slots)
constexpr int kSkRun = 128;                    // slots per warp task of k_sk_z

// Workspace of the sketch (one allocation, made by tlda_online_begin).
struct SketchWs {
  float *S;                          // kSkPieceDocs x r
  int32_t *sd, *sf, *sm;             // slots: document (in the piece), count, word
  int32_t *wcnt, *wfill;             // V + 1 (counts, then first slots), V
  int64_t *scan;                     // scan_blocks(V) + 2
  uint8_t *ok;                       // kSkPieceDocs: the document passed validation
  static size_t al(size_t b) { return (b + 255) & ~size_t(255); }
  static size_t bytes(size_t V, size_t r) {
    return al(sizeof(float) * kSkPieceDocs * r) + 3 * al(sizeof(int32_t) * kSkPieceNnz) +
           al(sizeof(int32_t) * (V + 1)) + al(sizeof(int32_t) * V) + al(sizeof(int64_t) * (scan_blocks((int)V) + 2)) +
           al(kSkPieceDocs);
  }
  SketchWs(void *base, size_t V, size_t r) {
    char *p = static_cast<char *>(base);
    S = reinterpret_cast<float *>(p);
    p += al(sizeof(float) * kSkPieceDocs * r);
    int32_t **slot_bufs[] = {&sd, &sf, &sm};
    for (int32_t **b : slot_bufs) {
      *b = reinterpret_cast<int32_t *>(p);
      p += al(sizeof(int32_t) * kSkPieceNnz);
    }
    wcnt = reinterpret_cast<int32_t *>(p);
    p += al(sizeof(int32_t) * (V + 1));
    wfill = reinterpret_cast<int32_t *>(p);
    p += al(sizeof(int32_t) * V);
    scan = reinterpret_cast<int64_t *>(p);
    p += al(sizeof(int64_t) * (scan_blocks((int)V) + 2));
    ok = reinterpret_cast<uint8_t *>(p);
  }
};

struct SkPiece {
  const int32_t *indptr, *indices, *counts;  // indptr of the piece's first document; absolute offsets
  int n_docs, nz_lo, nz_hi;                  // documents; the piece's offsets lie in [nz_lo, nz_hi]
  int V, r;
};

// The r columns are split over gridDim.y warps per document (or run): block
// row y takes columns y 32 KC + lane + 32 c, KC per lane, so that a warp holds
// few registers and many warps are resident; four rows in flight per warp.
template <int KC>
__global__ void __launch_bounds__(256) k_sk_rows(SkPiece q, const float *__restrict__ Om, float *__restrict__ S,
                                                 int32_t *wcnt, uint8_t *ok, unsigned long long *TS, int *err) {
  const int doc = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (doc >= q.n_docs) return;
  const int p0 = q.indptr[doc], p1 = q.indptr[doc + 1];
  bool bad = p0 < q.nz_lo || p1 > q.nz_hi || p1 < p0;
  long long L = 0;
  if (!bad)
    for (int p = p0 + lane; p < p1; p += 32) {
      const int m = q.indices[p], f = q.counts[p];
      const int prev = p > p0 ? q.indices[p - 1] : -1;
      if (m < 0 || m >= q.V || f <= 0 || m <= prev) bad = true;
      else L += f;
    }
  const bool first = blockIdx.y == 0;  // the column group that also counts
  const int cb = blockIdx.y * 32 * KC;
  if (__any_sync(0xffffffffu, bad)) {
    if (lane == 0 && first) {
      ok[doc] = 0;
      atomicOr(err, 1);
    }
    return;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) L += __shfl_xor_sync(0xffffffffu, L, o);
  float sv[KC];
#pragma unroll
  for (int c = 0; c < KC; ++c) sv[c] = 0.f;
  for (int base = p0; base < p1; base += 32) {
    const int n = min(32, p1 - base);
    const int mj = lane < n ? q.indices[base + lane] : 0, fj = lane < n ? q.counts[base + lane] : 0;
    for (int i = 0; i < n; i += 4) {
      int mm[4];
      float ff[4], row[4][KC];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        mm[u] = __shfl_sync(0xffffffffu, mj, (i + u) & 31);
        ff[u] = (float)__shfl_sync(0xffffffffu, fj, (i + u) & 31);
        if (i + u >= n) ff[u] = 0.f;  // lanes past the end hold word 0, count 0
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int c = 0; c < KC; ++c) {
          const int col = cb + lane + 32 * c;
          row[u][c] = col < q.r ? __ldg(Om + (long long)mm[u] * q.r + col) : 0.f;
        }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int c = 0; c < KC; ++c) sv[c] = fmaf(ff[u], row[u][c], sv[c]);
    }
  }
  float *srow = S + (long long)doc * q.r;
#pragma unroll
  for (int c = 0; c < KC; ++c) {
    const int col = cb + lane + 32 * c;
    if (col < q.r) srow[col] = sv[c];
  }
  if (!first) return;
  for (int p = p0 + lane; p < p1; p += 32) atomicAdd(wcnt + q.indices[p] + 1, 1);
  if (lane == 0) {
    ok[doc] = 1;
    if (L > 0) {
      atomicAdd(TS + 0, (unsigned long long)L);
      atomicAdd(TS + 1, (unsigned long long)(L * (L - 1)));
      atomicAdd(TS + 2, (unsigned long long)(L * (L - 1) * (L - 2)));
    }
  }
}

__global__ void __launch_bounds__(256) k_sk_scatter(SkPiece q, const uint8_t *ok, const int32_t *wcnt, int32_t *wfill,
                                                    int32_t *sd, int32_t *sf, int32_t *sm, int *err) {
  const int doc = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (doc >= q.n_docs || !ok[doc]) return;
  const int p0 = q.indptr[doc], p1 = q.indptr[doc + 1];
  for (int p = p0 + lane; p < p1; p += 32) {
    const int m = q.indices[p];
    const long long slot = (long long)wcnt[m] + atomicAdd(wfill + m, 1);
    if (slot < kSkPieceNnz) {  // more slots than the piece's offsets span: overlapping documents
      sd[slot] = doc;
      sf[slot] = q.counts[p];
      sm[slot] = m;
    } else {
      atomicOr(err, 1);
    }
  }
}

template <int KC>
__device__ __forceinline__ void sk_flush(int m, const float (&acc)[KC], long long fs, long long lo, long long hi,
                                         const int32_t *wcnt, int r, int cb, double *Z, unsigned long long *C,
                                         int lane) {
  const bool whole = wcnt[m] >= lo && wcnt[m + 1] <= hi;  // no other run holds word m
  double *z = Z + (long long)m * r;
#pragma unroll
  for (int c = 0; c < KC; ++c) {
    const int col = cb + lane + 32 * c;
    if (col < r) {
      if (whole) z[col] += (double)acc[c];
      else atomicAdd(z + col, (double)acc[c]);
    }
  }
  if (lane == 0 && cb == 0) {
    if (whole) C[m] += (unsigned long long)fs;
    else atomicAdd(C + m, (unsigned long long)fs);
  }
}

template <int KC>
__global__ void __launch_bounds__(256) k_sk_z(const int32_t *__restrict__ wcnt, const int32_t *__restrict__ sd,
                                              const int32_t *__restrict__ sf, const int32_t *__restrict__ sm,
                                              const int64_t *total_p, int r, const float *__restrict__ S,
                                              const float *__restrict__ Om, double *Z, unsigned long long *C,
                                              int *err) {
  const long long total = *total_p;  // valid nonzeros of the piece
  if (total > kSkPieceNnz) {         // k_sk_scatter dropped slots and set *err
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(err, 1);
    return;
  }
  const int lane = threadIdx.x & 31, cb = blockIdx.y * 32 * KC;
  const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
  const long long runs = (total + kSkRun - 1) / kSkRun;
  for (long long t = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < runs; t += nwarps) {
    const long long lo = t * kSkRun, hi = min(total, lo + kSkRun);
    float acc[KC], om[KC];
#pragma unroll
    for (int c = 0; c < KC; ++c) acc[c] = om[c] = 0.f;
    long long fs = 0;
    int cur = -1;
    for (long long base = lo; base < hi; base += 32) {
      const int n = (int)min(32ll, hi - base);
      const bool in = lane < n;
      const int mj = in ? sm[base + lane] : 0, dj = in ? sd[base + lane] : 0, fj = in ? sf[base + lane] : 0;
      for (int i = 0; i < n; i += 4) {
        int mm[4], dd[4], ff[4];
        float row[4][KC];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          mm[u] = __shfl_sync(0xffffffffu, mj, (i + u) & 31);
          dd[u] = __shfl_sync(0xffffffffu, dj, (i + u) & 31);
          ff[u] = __shfl_sync(0xffffffffu, fj, (i + u) & 31);
          if (u > 0 && i + u >= n) {  // past the end: repeat the previous slot with count 0
            mm[u] = mm[u - 1];
            dd[u] = dd[u - 1];
            ff[u] = 0;
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int c = 0; c < KC; ++c) {
            const int col = cb + lane + 32 * c;
            row[u][c] = col < r ? S[(long long)dd[u] * r + col] : 0.f;
          }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (mm[u] != cur) {
            if (cur >= 0) sk_flush<KC>(cur, acc, fs, lo, hi, wcnt, r, cb, Z, C, lane);
            cur = mm[u];
#pragma unroll
            for (int c = 0; c < KC; ++c) {
              const int col = cb + lane + 32 * c;
              acc[c] = 0.f;
              om[c] = col < r ? __ldg(Om + (long long)cur * r + col) : 0.f;
            }
            fs = 0;
          }
          const float fu = (float)ff[u];
#pragma unroll
          for (int c = 0; c < KC; ++c) acc[c] = fmaf(fu, row[u][c] - om[c], acc[c]);
          fs += ff[u];
        }
      }
    }
    if (cur >= 0) sk_flush<KC>(cur, acc, fs, lo, hi, wcnt, r, cb, Z, C, lane);
  }
}

// Workspace of a re-whitening (one FP64 allocation, made by tlda_online_begin).
struct OnlineWs {
  double *Y, *Q1, *Q2, *M1, *U64;               // V x r (three), V, V x D
  double *G, *Z, *LinvT, *L1, *L2, *L1T, *C1, *C2, *Bm, *Et, *Ms, *Rs;  // r x r
  double *m1q, *ev, *Ek, *lam;                  // r, r, r x D, D
  static size_t words(size_t V, size_t r, size_t D) { return 3 * V * r + V + V * D + 12 * r * r + 2 * r + r * D + D; }
  OnlineWs(double *w, size_t V, size_t r, size_t D) {
    double **rr_bufs[] = {&G, &Z, &LinvT, &L1, &L2, &L1T, &C1, &C2, &Bm, &Et, &Ms, &Rs};
    Y = w, Q1 = Y + V * r, Q2 = Q1 + V * r, M1 = Q2 + V * r, U64 = M1 + V;
    w = U64 + V * D;
    for (double **b : rr_bufs) {
      *b = w;
      w += r * r;
    }
    m1q = w, ev = m1q + r, Ek = ev + r, lam = Ek + r * D;
  }
};

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
  OnlineWs w(ctx->on_ws, V, r, D);
  int *status = ctx->on_status;
  CKF(cudaMemsetAsync(status, 0, 2 * sizeof(int), s));
  k_m1<<<(V + 255) / 256, 256, 0, s>>>(ctx->on_C, ctx->on_TS, V, w.M1);
  gemm_tn64<double, double>(w.M1, 1, ctx->on_Om, r, w.m1q, r, 1, r, V, s);
  CKF(cudaMemcpyAsync(w.Y, ctx->on_Z, sizeof(double) * (size_t)V * r, cudaMemcpyDeviceToDevice, s));
  k_rank1_fix<<<(unsigned)(((long long)V * r + 255) / 256), 256, 0, s>>>(w.Y, w.M1, w.m1q, V, r, sP, a0);
  // CholeskyQR2: out = in L^-T with L L^T = in^T in, twice; Y = Q2 (L1 L2)^T
  auto cholqr_pass = [&](const double *in, double *out, double *Lf) -> tlda_status {
    gemm_tn64<double, double>(in, r, in, r, w.G, r, r, r, V, s);
    if (tlda_status st = run_chol_inv(ctx, w.G, r, Lf, w.Z, nullptr, w.LinvT, nullptr, status, s)) return st;
    gemm_nn<double>(in, r, w.LinvT, r, out, r, V, r, r, s);
    return TLDA_OK;
  };
  if (tlda_status st = cholqr_pass(w.Y, w.Q1, w.L1)) return st;
  if (tlda_status st = cholqr_pass(w.Q1, w.Q2, w.L2)) return st;
  gemm_tn64<double, double>(w.Q2, r, ctx->on_Om, r, w.C2, r, r, r, V, s);  // Q^T Omega
  // Q^T Y = R = (L1 L2)^T = L2^T L1^T
  k_transpose_rr<<<(r * r + 255) / 256, 256, 0, s>>>(w.L1, r, nullptr, w.L1T);
  gemm_tn64<double, double>(w.L2, r, w.L1T, r, w.C1, r, r, r, r, s);
  // B = (Q^T Y)(Q^T Omega)^-1, symmetrised by the eigensolver
  if (tlda_status st = run_solve_right(ctx, w.C1, w.C2, r, w.Ms, w.Rs, w.Bm, status + 1, s)) return st;
  CKF(cudaGetLastError());
  int hstat[2];
  CKF(cudaMemcpyAsync(hstat, status, sizeof hstat, cudaMemcpyDeviceToHost, s));
  CKF(cudaStreamSynchronize(s));
  if (tlda_status st = chol_status(ctx, hstat[0], "sketch basis lost rank (CholeskyQR breakdown)")) return st;
  if (tlda_status st = chol_status(ctx, hstat[1], "Q^T Omega is singular")) return st;
  if (tlda_status js = run_jacobi(ctx, w.Bm, r, w.Et, w.ev, s)) return js;
  std::vector<double> hev(r), hEv((size_t)r * r);
  CKF(cudaMemcpyAsync(hev.data(), w.ev, sizeof(double) * r, cudaMemcpyDeviceToHost, s));
  CKF(cudaMemcpyAsync(hEv.data(), w.Et, sizeof(double) * r * r, cudaMemcpyDeviceToHost, s));
  CKF(cudaStreamSynchronize(s));
  std::vector<int> ord(r);
  for (int i = 0; i < r; ++i) ord[i] = i;
  std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return hev[x] > hev[y]; });
  std::vector<double> hEk((size_t)r * D), hlam(D);
  for (int j = 0; j < D; ++j) {
    hlam[j] = hev[ord[j]];
    for (int i = 0; i < r; ++i) hEk[(size_t)i * D + j] = hEv[(size_t)ord[j] * r + i];
  }
  if (!(hlam[D - 1] > 1e-12 * hlam[0]))
    return fail(ctx, TLDA_ERR_NUMERIC, "the sketched M2 has fewer than D positive eigenvalues");
  CKF(cudaMemcpyAsync(w.Ek, hEk.data(), sizeof(double) * r * D, cudaMemcpyHostToDevice, s));
  CKF(cudaMemcpyAsync(w.lam, hlam.data(), sizeof(double) * D, cudaMemcpyHostToDevice, s));
  gemm_nn<double>(w.Q2, r, w.Ek, D, w.U64, D, V, D, r, s);
  if (ctx->whitened)
    CKF(cudaMemcpyAsync(ctx->on_Wold, ctx->W32, sizeof(float) * (size_t)V * D, cudaMemcpyDeviceToDevice, s));
  k_make_w<<<D, 256, 0, s>>>(w.U64, V, D, w.lam, ctx->W32, nullptr, nullptr);
  CKF(cudaMemsetAsync(ctx->m1, 0, sizeof(float) * ctx->Dp, s));
  k_wtm1<<<D, 256, 0, s>>>(ctx->W32, w.M1, V, D, ctx->m1);
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
  OnlineWs w(ctx->on_ws, V, ctx->on_r, D);  // r x r buffers hold the D x D ones (D <= r)
  int *status = ctx->on_status;
  CKF(cudaMemsetAsync(status, 0, sizeof(int), s));
  gemm_tn64<float, float>(ctx->W32, D, ctx->on_Wold, D, w.C1, D, D, D, V, s);
  gemm_tn64<float, float>(ctx->on_Wold, D, ctx->on_Wold, D, w.C2, D, D, D, V, s);
  // R = (W^T W_old)(W_old^T W_old)^-1
  if (tlda_status st = run_solve_right(ctx, w.C1, w.C2, D, w.Ms, w.Rs, w.Bm, status, s)) return st;
  CKF(cudaGetLastError());
  std::vector<double> R((size_t)D * D);
  std::vector<float> hP((size_t)D * K);
  int hst = 0;
  CKF(cudaMemcpyAsync(R.data(), w.Bm, sizeof(double) * D * D, cudaMemcpyDeviceToHost, s));
  CKF(cudaMemcpyAsync(hP.data(), Phi, sizeof(float) * D * K, cudaMemcpyDeviceToHost, s));
  CKF(cudaMemcpyAsync(&hst, status, sizeof hst, cudaMemcpyDeviceToHost, s));
  CKF(cudaStreamSynchronize(s));
  if (tlda_status st = chol_status(ctx, hst, "W^T W of the previous whitening is singular")) return st;
  std::vector<double> hN((size_t)D * K, 0.0);
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

// Documents [d0, d0 + nd) of `corpus` into the online statistics and sketch,
// in pieces of at most kSkPieceDocs documents and kSkPieceNnz nonzeros (the
// piece offsets are read back once; validation errors land in on_err).
tlda_status online_accumulate(tlda_ctx *ctx, const tlda_csr *corpus, int64_t d0, int nd) {
  if (nd <= 0) return TLDA_OK;
  cudaStream_t s = ctx->stream;
  // columns per lane: 4 up to r = 128, else 8, in ny column groups of 32 kc
  const int V = ctx->V, r = ctx->on_r, kc = r <= 128 ? 4 : 8, ny = (r + 32 * kc - 1) / (32 * kc);
  SketchWs w(ctx->on_sk, V, r);
  int64_t *total = w.scan + scan_blocks(V);
  auto piece = [&](int64_t a, int n, int32_t lo, int32_t hi) -> tlda_status {
    const SkPiece q{corpus->indptr + a, corpus->indices, corpus->counts, n, lo, hi, V, r};
    CKF(cudaMemsetAsync(w.wcnt, 0, sizeof(int32_t) * (V + 1), s));
    CKF(cudaMemsetAsync(w.wfill, 0, sizeof(int32_t) * V, s));
    const unsigned g = (unsigned)(((long long)n * 32 + 255) / 256);
    const dim3 gr(g, ny);
    if (kc == 4) k_sk_rows<4><<<gr, 256, 0, s>>>(q, ctx->on_Om32, w.S, w.wcnt, w.ok, ctx->on_TS, ctx->on_err);
    else k_sk_rows<8><<<gr, 256, 0, s>>>(q, ctx->on_Om32, w.S, w.wcnt, w.ok, ctx->on_TS, ctx->on_err);
    scan_counts(w.wcnt, V, w.scan, total, s);
    k_sk_scatter<<<g, 256, 0, s>>>(q, w.ok, w.wcnt, w.wfill, w.sd, w.sf, w.sm, ctx->on_err);
    const long long span = std::max<long long>(1, (long long)hi - lo);
    const dim3 zg((unsigned)std::min<long long>((span + 8ll * kSkRun - 1) / (8ll * kSkRun), 8ll * ctx->num_sms / ny), ny);
    if (kc == 4) k_sk_z<4><<<zg, 256, 0, s>>>(w.wcnt, w.sd, w.sf, w.sm, total, r, w.S, ctx->on_Om32, ctx->on_Z, ctx->on_C, ctx->on_err);
    else k_sk_z<8><<<zg, 256, 0, s>>>(w.wcnt, w.sd, w.sf, w.sm, total, r, w.S, ctx->on_Om32, ctx->on_Z, ctx->on_C, ctx->on_err);
    CKF(cudaGetLastError());
    return TLDA_OK;
  };
  // a piece whose offsets span more than kSkPieceNnz slots is halved
  std::function<tlda_status(int64_t, int64_t, int32_t, int32_t)> run = [&](int64_t a, int64_t b, int32_t lo,
                                                                          int32_t hi) -> tlda_status {
    if ((long long)hi - lo <= kSkPieceNnz) return piece(a, (int)(b - a), lo, hi);
    if (b - a == 1) return fail(ctx, TLDA_ERR_OOM, "a document with more than 16M nonzeros");
    const int64_t mid = a + (b - a) / 2;
    int32_t hm = 0;
    CKF(cudaMemcpyAsync(&hm, corpus->indptr + mid, sizeof hm, cudaMemcpyDeviceToHost, s));
    CKF(cudaStreamSynchronize(s));
    if (tlda_status st = run(a, mid, lo, hm)) return st;
    return run(mid, b, hm, hi);
  };
  const int np = (nd + kSkPieceDocs - 1) / kSkPieceDocs;
  std::vector<int32_t> h(np + 1);
  CKF(cudaMemcpy2DAsync(h.data(), sizeof(int32_t), corpus->indptr + d0, sizeof(int32_t) * kSkPieceDocs,
                        sizeof(int32_t), np, cudaMemcpyDeviceToHost, s));
  CKF(cudaMemcpyAsync(h.data() + np, corpus->indptr + d0 + nd, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  CKF(cudaStreamSynchronize(s));
  for (int i = 0; i < np; ++i) {
    const int64_t a = d0 + (int64_t)i * kSkPieceDocs, b = std::min<int64_t>(a + kSkPieceDocs, d0 + nd);
    if (tlda_status st = run(a, b, h[i], h[i + 1])) return st;
  }
  return TLDA_OK;
}

// Rebuild the whitening; carry Phi (if given) from the previous one.
tlda_status online_whiten(tlda_ctx *ctx, float *Phi) {
  const bool had = ctx->whitened;
  if (tlda_status st = online_rewhiten(ctx)) return st;
  if (had && Phi)
    if (tlda_status st = online_rotate(ctx, Phi)) return st;
  ctx->whitened = true;
  return TLDA_OK;
}

}  // namespace

extern "C" {

tlda_status tlda_fit_moments(tlda_ctx *ctx, const tlda_csr *chunk, uint32_t flags) {
  TLDA_RANGE();
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
  TLDA_RANGE();
  if (!ctx || !Phi || !mu_out || !alpha_out) return fail(ctx, TLDA_ERR_INVALID, "NULL argument");
  if (!ctx->whitened) return fail(ctx, TLDA_ERR_STATE, "no whitening: fit or set one first");
  cudaStream_t s = ctx->stream;
  const int V = ctx->V, D = ctx->D, K = ctx->K;
  Scratch sc;
  double *W64 = nullptr, *G = nullptr, *Linv = nullptr, *LinvT = nullptr, *Ginv = nullptr, *T = nullptr;
  double *Lf = nullptr, *Zs = nullptr;
  double *mu = nullptr, *al = nullptr;
  int *status = nullptr;
  CKF(sc.get(&W64, (size_t)V * D));
  CKF(sc.get(&G, (size_t)D * D));
  CKF(sc.get(&Linv, (size_t)D * D));
  CKF(sc.get(&LinvT, (size_t)D * D));
  CKF(sc.get(&Ginv, (size_t)D * D));
  CKF(sc.get(&Lf, (size_t)D * D));
  CKF(sc.get(&Zs, (size_t)D * D));
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
  if (tlda_status st = run_chol_inv(ctx, G, D, Lf, Zs, Linv, LinvT, nullptr, status, s)) return st;
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
  if (tlda_status st = chol_status(ctx, hst, "W^T W is not positive definite")) return st;
  return TLDA_OK;
}

tlda_status tlda_online_begin(tlda_ctx *ctx, const double *Omega, int32_t r) {
  TLDA_RANGE();
  if (!ctx) return TLDA_ERR_INVALID;
  if (!Omega || r < ctx->D || r > kMaxDim || (r & 1) || r > ctx->V)
    return fail(ctx, TLDA_ERR_INVALID, "the sketch needs an even r with D <= r <= min(V, 512)");
  const size_t V = ctx->V;
  if (ctx->on_r != r) {
    if (ctx->on_Om) cudaFree(ctx->on_Om);
    if (ctx->on_Z) cudaFree(ctx->on_Z);
    if (ctx->on_ws) cudaFree(ctx->on_ws);
    if (ctx->on_sk) cudaFree(ctx->on_sk);
    if (ctx->on_Om32) cudaFree(ctx->on_Om32);
    ctx->on_Om = ctx->on_Z = ctx->on_ws = nullptr;
    ctx->on_sk = nullptr;
    ctx->on_Om32 = nullptr;
    ctx->on_r = 0;
    CKF(dalloc(&ctx->on_Om, V * r));
    CKF(dalloc(&ctx->on_Z, V * r));
    CKF(dalloc(&ctx->on_ws, OnlineWs::words(V, r, ctx->D)));
    CKF(dalloc(reinterpret_cast<char **>(&ctx->on_sk), SketchWs::bytes(V, r)));
    CKF(dalloc(&ctx->on_Om32, V * r));
    ctx->on_r = r;
  }
  if (!ctx->on_C) CKF(dalloc(&ctx->on_C, V));
  if (!ctx->on_TS) CKF(dalloc(&ctx->on_TS, 3));
  if (!ctx->on_err) CKF(dalloc(&ctx->on_err, 1));
  if (!ctx->on_status) CKF(dalloc(&ctx->on_status, 2));
  if (!ctx->on_Wold) CKF(dalloc(&ctx->on_Wold, V * ctx->D));
  cudaStream_t s = ctx->stream;
  CKF(cudaMemcpyAsync(ctx->on_Om, Omega, sizeof(double) * V * r, cudaMemcpyDeviceToDevice, s));
  k_d2f<<<(unsigned)((V * r + 255) / 256), 256, 0, s>>>(ctx->on_Om, ctx->on_Om32, (long long)(V * r));
  CKF(cudaGetLastError());
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
  TLDA_RANGE();
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
  for (int b0 = 0; b0 < n_batches; b0 += rewhiten_every) {
    const int b1 = std::min(n_batches, b0 + rewhiten_every);
    const int64_t d0 = batch_offsets[b0], d1 = batch_offsets[b1];
    if (tlda_status st = online_accumulate(ctx, corpus, d0, (int)(d1 - d0))) return st;
    if (tlda_status st = online_whiten(ctx, Phi)) return st;
    tlda_status st = tlda_cp_pass(ctx, corpus, batch_offsets + b0, b1 - b0, Phi, lr, 0,
                                  loss_out ? loss_out + b0 : nullptr);
    if (st) return st;
  }
  return TLDA_OK;
}

tlda_status tlda_online_accumulate(tlda_ctx *ctx, const tlda_csr *corpus) {
  TLDA_RANGE();
  if (!ctx) return TLDA_ERR_INVALID;
  if (!ctx->on_active) return fail(ctx, TLDA_ERR_STATE, "tlda_online_begin has not been called");
  if (!corpus || corpus->vocab != ctx->V || corpus->n_docs < 0 || !corpus->indptr ||
      (corpus->n_docs > 0 && (!corpus->indices || !corpus->counts)))
    return fail(ctx, TLDA_ERR_INVALID, "bad corpus");
  return online_accumulate(ctx, corpus, 0, corpus->n_docs);
}

tlda_status tlda_online_whiten(tlda_ctx *ctx, float *Phi) {
  TLDA_RANGE();
  if (!ctx) return TLDA_ERR_INVALID;
  if (!ctx->on_active) return fail(ctx, TLDA_ERR_STATE, "tlda_online_begin has not been called");
  return online_whiten(ctx, Phi);
}

tlda_status tlda_online_get_sketch(tlda_ctx *ctx, double *Z_out, int64_t *C_out, int64_t *TS_out) {
  TLDA_RANGE();
  if (!ctx) return TLDA_ERR_INVALID;
  if (!ctx->on_active) return fail(ctx, TLDA_ERR_STATE, "tlda_online_begin has not been called");
  const size_t V = ctx->V, r = ctx->on_r;
  cudaStream_t s = ctx->stream;
  int herr = 0;
  if (Z_out) CKF(cudaMemcpyAsync(Z_out, ctx->on_Z, sizeof(double) * V * r, cudaMemcpyDefault, s));
  if (C_out) CKF(cudaMemcpyAsync(C_out, ctx->on_C, sizeof(int64_t) * V, cudaMemcpyDefault, s));
  if (TS_out) CKF(cudaMemcpyAsync(TS_out, ctx->on_TS, sizeof(int64_t) * 3, cudaMemcpyDefault, s));
  CKF(cudaMemcpyAsync(&herr, ctx->on_err, sizeof herr, cudaMemcpyDeviceToHost, s));
  CKF(cudaStreamSynchronize(s));
  if (herr) return fail(ctx, TLDA_ERR_INVALID, "a corrupt document was met since tlda_online_begin");
  return TLDA_OK;
}

tlda_status tlda_online_set_sketch(tlda_ctx *ctx, const double *Z, const int64_t *C, const int64_t *TS) {
  TLDA_RANGE();
  if (!ctx) return TLDA_ERR_INVALID;
  if (!ctx->on_active) return fail(ctx, TLDA_ERR_STATE, "tlda_online_begin has not been called");
  if (!Z || !C || !TS) return fail(ctx, TLDA_ERR_INVALID, "Z, C and TS are required");
  const size_t V = ctx->V, r = ctx->on_r;
  cudaStream_t s = ctx->stream;
  CKF(cudaMemcpyAsync(ctx->on_Z, Z, sizeof(double) * V * r, cudaMemcpyDefault, s));
  CKF(cudaMemcpyAsync(ctx->on_C, C, sizeof(int64_t) * V, cudaMemcpyDefault, s));
  CKF(cudaMemcpyAsync(ctx->on_TS, TS, sizeof(int64_t) * 3, cudaMemcpyDefault, s));
  CKF(cudaMemsetAsync(ctx->on_err, 0, sizeof(int), s));
  CKF(cudaStreamSynchronize(s));
  return TLDA_OK;
}

}  // extern "C"
