// Hot-path kernels of the online Tensor LDA CP step (eq. vec_deriv and the SGD
// update of section "Online Learning of the Third Moment"), plain FP32 form,
// plus the pieces both precisions share: batch scan + whitening, the
// touched-word compaction, the Phi-only terms and the final reduction/update.
//
// Per step, with U = W - 1 m1^T (V x D), X = F U, Y = X Phi, Q = U Phi:
//   a1  L_d, S3, c_m = sum_d f_dm, CSR validation,
//       touched words {m : c_m > 0}                        k_scan_whiten
//   a2  X = F U (= F W - L m1^T)                           k_scan_whiten
//   a3  Y = X Phi;  a4 Q = U Phi (touched rows)            k_qy_f32
//   a4  R_d = sum_m f_dm Q_m^2,  Z = Y*Y - R;  H = F^T Y   k_rz
//   a6  Zc_m = Q_m * (2 c_m Q_m - 2 H_m)                   k_zh_f32
//   a5+a6  G1 + G2 = X^T Z + U^T Zc (split reduction)      k_g_f32
//   a7/a8  G3, P = Phi (Phi^T Phi * Phi^T Phi)             k_phi_gram, k_phi_terms
//   a9  grad = E - 3 c3/S3 (G1 + G2), Phi -= lr grad       k_reduce_update
// where E = 3(1+theta) P - 3 G3.  Words a batch does not touch have c_m = 0
// and H_m = 0, so they contribute nothing to G2 and are skipped.
#include <cstdio>

#include "tlda_internal.h"

namespace tlda {

__device__ __forceinline__ float4 f4(float x) { return make_float4(x, x, x, x); }
__device__ __forceinline__ float4 fma4(float s, float4 a, float4 c) {
  return make_float4(fmaf(s, a.x, c.x), fmaf(s, a.y, c.y), fmaf(s, a.z, c.z), fmaf(s, a.w, c.w));
}

// ------------------------------------------------------------ batch descriptor
__global__ void k_set_desc(DevState *st, BatchDesc b) { st->cur = b; }

__global__ void k_begin_pass(DevState *st, const BatchDesc *descs, int n) {
  st->descs = descs;
  st->n_descs = n;
  st->pass_pos = 1;
  st->cur = descs[0];
}

void launch_set_desc(DevState *st, const BatchDesc &b, cudaStream_t s) {
  k_set_desc<<<1, 1, 0, s>>>(st, b);
}
void launch_begin_pass(DevState *st, const BatchDesc *descs, int n, cudaStream_t s) {
  k_begin_pass<<<1, 1, 0, s>>>(st, descs, n);
}

// ------------------------------------------------------------ U = W - 1 m1^T
__global__ void k_make_u(const float *W, const float *m1, int V, int D, int Dp, float *U32,
                         __nv_bfloat16 *U16) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)V * Dp) return;
  const int m = (int)(e / Dp), i = (int)(e % Dp);
  const float u = i < D ? W[(long long)m * D + i] - m1[i] : 0.f;
  U32[e] = u;
  if (U16) U16[e] = __float2bfloat16_rn(u);
}

void launch_make_u(const float *W, const float *m1, int V, int D, int Dp, float *U32,
                   __nv_bfloat16 *U16, cudaStream_t s) {
  const long long n = (long long)V * Dp;
  k_make_u<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(W, m1, V, D, Dp, U32, U16);
}

// ------------------------------------------------------------ a1 + a2: scan and whiten
// Nonzeros of one document, 32 at a time: lane j holds nonzero base + j (word,
// count), checked in place; invalid entries get weight 0 on row 0.
struct NzChunk {
  int m, f;      // word (0 if invalid) and count (0 if invalid)
  bool in;       // lane holds a nonzero of this chunk
  bool bad;      // lane's nonzero breaks the CSR rules
  int n;         // nonzeros in this chunk (same in all lanes)
};

__device__ __forceinline__ NzChunk load_chunk(const BatchDesc &b, int V, int base, int hi, int lane, int prev) {
  NzChunk c;
  const int j = base + lane;
  c.in = j < hi;
  c.n = min(32, hi - base);
  int m = -1, f = 0;
  if (c.in) {
    m = __ldg(b.indices + ((long long)j - b.nz_base));
    f = __ldg(b.counts + ((long long)j - b.nz_base));
  }
  int mp = __shfl_up_sync(0xffffffffu, m, 1);
  if (lane == 0) mp = prev;
  const bool valid = c.in && m >= 0 && m < V && f > 0;
  c.bad = c.in && (!valid || m <= mp);
  c.m = valid ? m : 0;
  c.f = valid ? f : 0;
  return c;
}

// One warp per document: validates the row, accumulates L_d and
// x_d = sum_m f_dm u_m (FP32) four U rows in flight at a time, and (stats)
// adds c_m, appends first-seen words to the touched list, adds the block's
// share of S3.  TC=true also writes X in BF16 row-major (X16), whole rows.
template <int NV, bool TC>
__global__ void __launch_bounds__(32 * kDocsPerBlock)
    k_scan_whiten(StepArgs a, float *X_out, int stats) {
  const BatchDesc b = a.st->cur;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int d0 = blockIdx.x * kDocsPerBlock;
  if (d0 >= (TC ? round_up(b.n_docs, 64) : b.n_docs)) return;
  const int d = d0 + warp;
  __shared__ unsigned long long s3;
  if (threadIdx.x == 0) s3 = 0;
  __syncthreads();
  float4 acc[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) acc[v] = f4(0.f);
  if (d < b.n_docs) {
    const int lo = b.indptr[d], hi = b.indptr[d + 1];
    bool bad = (lo < b.nz_base) || (hi < lo);
    long long lsum = 0;
    int prev = -1;
    if (!bad) {
      for (int base = lo; base < hi; base += 32) {
        const NzChunk c = load_chunk(b, a.V, base, hi, lane, prev);
        if (__any_sync(0xffffffffu, c.bad)) bad = true;
        prev = __shfl_sync(0xffffffffu, c.in ? c.m : -1, c.n - 1);
        lsum += c.f;
        if (stats && a.same_token) {
          bool fresh = false;
          if (c.f > 0) fresh = atomicAdd(a.cnt + c.m, c.f) == 0;
          const unsigned nm = __ballot_sync(0xffffffffu, fresh);
          if (nm) {
            int t0 = 0;
            if (lane == 0) t0 = atomicAdd(&a.st->n_touched, __popc(nm));
            t0 = __shfl_sync(0xffffffffu, t0, 0);
            if (fresh) a.widx[t0 + __popc(nm & ((1u << lane) - 1u))] = c.m;
          }
        }
        for (int q = 0; q < c.n; q += 4) {
          int mm[4];
          float ff[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            mm[u] = __shfl_sync(0xffffffffu, c.m, (q + u) & 31);
            ff[u] = (float)__shfl_sync(0xffffffffu, c.f, (q + u) & 31);
            if (q + u >= c.n) ff[u] = 0.f;
          }
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            const int col = v * 128 + lane * 4;
            if (col < a.Dp) {
              float4 r[4];
#pragma unroll
              for (int u = 0; u < 4; ++u)
                r[u] = __ldg(reinterpret_cast<const float4 *>(a.U32 + (long long)mm[u] * a.Dp + col));
#pragma unroll
              for (int u = 0; u < 4; ++u) acc[v] = fma4(ff[u], r[u], acc[v]);
            }
          }
        }
      }
    }
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    const long long L = lsum;
    if (bad && lane == 0) atomicOr(&a.st->err, kErrCsr);
    if (stats && lane == 0 && L >= 3) atomicAdd(&s3, (unsigned long long)(L * (L - 1) * (L - 2)));
    if (X_out) {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const int col = v * 128 + lane * 4;
        const float c[4] = {acc[v].x, acc[v].y, acc[v].z, acc[v].w};
        for (int q = 0; q < 4; ++q)
          if (col + q < a.D) X_out[(long long)d * a.D + col + q] = c[q];
      }
    } else if (!TC) {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const int col = v * 128 + lane * 4;
        if (col < a.Dp) *reinterpret_cast<float4 *>(a.X32 + (long long)d * a.Dp + col) = acc[v];
      }
    }
  }
  if constexpr (TC) {
    if (!X_out && d < round_up(b.n_docs, 64)) {
      // row-major BF16 copy: the A operand of Y = X Phi and of G1 = X^T Z (rows
      // past the batch, up to the next multiple of 64, are written as zeros)
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const int col = v * 128 + lane * 4;
        if (col < a.Dp) {
          __nv_bfloat162 p[2] = {__floats2bfloat162_rn(acc[v].x, acc[v].y), __floats2bfloat162_rn(acc[v].z, acc[v].w)};
          *reinterpret_cast<uint2 *>(a.X16 + (long long)d * a.Dp + col) = *reinterpret_cast<const uint2 *>(p);
        }
      }
    }
  }
  __syncthreads();
  if (stats && threadIdx.x == 0 && s3) atomicAdd(&a.st->S3, s3);
}

void launch_whiten(const StepArgs &a, cudaStream_t s, float *X_out, bool stats) {
  const bool tc = a.precision == TLDA_BF16 && X_out == nullptr;
  const int grid = round_up(a.Bmax, 64) / kDocsPerBlock;
  const int nv = (a.Dp + 127) / 128;
#define TLDA_WHITEN(NVv)                                                                        \
  if (nv == NVv) {                                                                              \
    if (tc) k_scan_whiten<NVv, true><<<grid, 32 * kDocsPerBlock, 0, s>>>(a, X_out, stats);     \
    else k_scan_whiten<NVv, false><<<grid, 32 * kDocsPerBlock, 0, s>>>(a, X_out, stats);       \
    return;                                                                                     \
  }
  TLDA_WHITEN(1) TLDA_WHITEN(2) TLDA_WHITEN(3) TLDA_WHITEN(4)
#undef TLDA_WHITEN
}

// ------------------------------------------------------------ a7/a8: Phi-only terms
// Gram = Phi^T Phi (Kp x Kp, zero padded) in 32 x 32 tiles over 64-row slabs
// of Phi held in shared memory; the extra block row forms a = m1^T Phi.
__global__ void __launch_bounds__(256) k_phi_gram(StepArgs a) {
  const int bx = blockIdx.x, by = blockIdx.y, tid = threadIdx.x;
  if (by == (int)gridDim.y - 1) {
    if (tid < 32) {
      const int j = bx * 32 + tid;
      float s = 0.f;
      if (j < a.K) {
#pragma unroll 8
        for (int r = 0; r < a.D; ++r) s = fmaf(a.m1[r], a.Phi[(long long)r * a.K + j], s);
      }
      if (j < a.Kp) a.avec[j] = s;
    }
    return;
  }
  __shared__ float Pi[64][33], Pj[64][33];
  const int ii = tid >> 3, jj = (tid & 7) * 4;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (int r0 = 0; r0 < a.D; r0 += 64) {
#pragma unroll
    for (int e = tid; e < 64 * 32; e += 256) {
      const int r = e >> 5, c = e & 31, gr = r0 + r;
      const int ci = by * 32 + c, cj = bx * 32 + c;
      Pi[r][c] = (gr < a.D && ci < a.K) ? a.Phi[(long long)gr * a.K + ci] : 0.f;
      Pj[r][c] = (gr < a.D && cj < a.K) ? a.Phi[(long long)gr * a.K + cj] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int r = 0; r < 64; ++r) {
      const float x = Pi[r][ii];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = fmaf(x, Pj[r][jj + q], acc[q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) a.Gram[(by * 32 + ii) * a.Kp + bx * 32 + jj + q] = acc[q];
}

// P = Phi (Gram * Gram) in 32 x 32 tiles (rows r of Phi, columns i), then per
// entry G3 = 2 phi_ri a_i + m1_r |phi_i|^2 - 2 m1_r a_i^2 and
// E = 3(1+theta) P - 3 G3.  Block (0, 0) also forms the Phi-only loss part.
__global__ void __launch_bounds__(256) k_phi_terms(StepArgs a) {
  const int bx = blockIdx.x, by = blockIdx.y, tid = threadIdx.x;
  __shared__ float Pr[32][65], G2[64][33];
  const int rr = tid >> 3, ic = (tid & 7) * 4;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (int j0 = 0; j0 < a.K; j0 += 64) {
#pragma unroll
    for (int e = tid; e < 32 * 64; e += 256) {
      const int r = e >> 6, j = e & 63, gr = by * 32 + r, gj = j0 + j;
      Pr[r][j] = (gr < a.D && gj < a.K) ? a.Phi[(long long)gr * a.K + gj] : 0.f;
      const int jb = e >> 5, c = e & 31, gjb = j0 + jb, gi = bx * 32 + c;
      const float g = (gjb < a.K && gi < a.K) ? a.Gram[gjb * a.Kp + gi] : 0.f;
      G2[jb][c] = g * g;
    }
    __syncthreads();
#pragma unroll 8
    for (int j = 0; j < 64; ++j) {
      const float x = Pr[rr][j];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = fmaf(x, G2[j][ic + q], acc[q]);
    }
    __syncthreads();
  }
  const int r = by * 32 + rr;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = bx * 32 + ic + q;
    if (r < a.D && i < a.K) {
      const float ai = a.avec[i], n2 = a.Gram[i * a.Kp + i], mr = a.m1[r];
      const float g3 = 2.f * a.Phi[(long long)r * a.K + i] * ai + mr * n2 - 2.f * mr * ai * ai;
      a.G3[r * a.Kp + i] = g3;
      a.E[r * a.Kp + i] = 3.f * (1.f + a.theta) * acc[q] - 3.f * g3;
    }
  }
  if (bx == 0 && by == 0 && a.want_loss) {
    __shared__ double red[256];
    double s = 0.0;
    for (int q = tid; q < a.K * a.K; q += blockDim.x) {
      const double g = a.Gram[(q / a.K) * a.Kp + (q % a.K)];
      s += 0.5 * (1.0 + a.theta) * g * g * g;
    }
    for (int i = tid; i < a.K; i += blockDim.x) {
      const double ai = a.avec[i], n2 = a.Gram[i * a.Kp + i];
      s -= 3.0 * ai * n2 - 2.0 * ai * ai * ai;
    }
    red[tid] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if (tid < w) red[tid] += red[tid + w];
      __syncthreads();
    }
    if (tid == 0) a.st->loss_phi = red[0];
  }
}

void launch_phi_gram(const StepArgs &a, cudaStream_t s) {
  dim3 g(a.Kp / 32, a.Kp / 32 + 1);
  k_phi_gram<<<g, 256, 0, s>>>(a);
}

void launch_phi_terms(const StepArgs &a, cudaStream_t s) {
  dim3 g(a.Kp / 32, a.Dp / 32);
  k_phi_terms<<<g, 256, 0, s>>>(a);
}

// ------------------------------------------------------------ Phi^T image (BF16 forms)
__global__ void k_phi_img(StepArgs a) { phi_img_groups(a, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x); }

void launch_phi_img(const StepArgs &a, cudaStream_t s) { k_phi_img<<<16, 256, 0, s>>>(a); }

// ------------------------------------------------------------ a3/a4: Q and Y (FP32)
// Rows t < n_touched: Q[widx[t]] = U[widx[t]] Phi; then Y[d] = X[d] Phi.
// 64 x 64 output tile per block, 4 x 4 per thread, Phi read with bounds
// straight from the caller's D x K layout (zero padding).
__global__ void __launch_bounds__(256) k_qy_f32(StepArgs a) {
  const int nt = a.same_token ? a.st->n_touched : 0;
  const int rows = nt + a.st->cur.n_docs;
  const int r0 = blockIdx.x * 64;
  if (r0 >= rows) return;
  const int n0 = blockIdx.y * 64;
  __shared__ __align__(16) float As[32][68];
  __shared__ __align__(16) float Bs[32][64];
  __shared__ const float *arow[64];
  __shared__ float *orow[64];
  const int tid = threadIdx.x;
  if (tid < 64) {
    const int r = r0 + tid;
    const float *ap = nullptr;
    float *op = nullptr;
    if (r < nt) {
      const int m = a.widx[r];
      ap = a.U32 + (long long)m * a.Dp;
      op = a.Q32 + (long long)m * a.Kp;
    } else if (r < rows) {
      const int d = r - nt;
      ap = a.X32 + (long long)d * a.Dp;
      op = a.Y32 + (long long)d * a.Kp;
    }
    arow[tid] = ap;
    orow[tid] = op;
  }
  __syncthreads();
  const int tx = tid & 15, ty = tid >> 4;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  for (int k0 = 0; k0 < a.Dp; k0 += 32) {
    {
      const int r = tid >> 2, kk = (tid & 3) * 8;
      const float *ap = arow[r];
      float4 v0 = f4(0.f), v1 = f4(0.f);
      if (ap) {
        v0 = *reinterpret_cast<const float4 *>(ap + k0 + kk);
        v1 = *reinterpret_cast<const float4 *>(ap + k0 + kk + 4);
      }
      As[kk + 0][r] = v0.x; As[kk + 1][r] = v0.y; As[kk + 2][r] = v0.z; As[kk + 3][r] = v0.w;
      As[kk + 4][r] = v1.x; As[kk + 5][r] = v1.y; As[kk + 6][r] = v1.z; As[kk + 7][r] = v1.w;
    }
    for (int e = tid; e < 32 * 64; e += 256) {
      const int kk = e >> 6, n = e & 63, gi = k0 + kk, gn = n0 + n;
      Bs[kk][n] = (gi < a.D && gn < a.K) ? a.Phi[(long long)gi * a.K + gn] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < 32; ++kk) {
      const float4 av = *reinterpret_cast<const float4 *>(&As[kk][ty * 4]);
      const float4 bv = *reinterpret_cast<const float4 *>(&Bs[kk][tx * 4]);
      const float ar[4] = {av.x, av.y, av.z, av.w}, br[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(ar[i], br[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    float *op = orow[ty * 4 + i];
    if (op) *reinterpret_cast<float4 *>(op + n0 + tx * 4) = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
  }
}

// ------------------------------------------------------------ a4 + a6 scatter: R, Z, H
// One warp per document (8 per block: small blocks keep more warps resident
// per SM): r_d = sum_m f_dm q_m^2 over gathered Q rows (four in flight),
// z_d = y_d^2 - r_d, H_m += f_dm y_d (vector atomics), and the document part
// of the loss.  TC=true writes Z as whole BF16 rows (Z16), zero rows past the
// batch up to the next multiple of 64.
template <int NK, bool TC>
__global__ void __launch_bounds__(256) k_rz(StepArgs a) {
  const BatchDesc b = a.st->cur;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int d0 = blockIdx.x * 8, d = d0 + warp;
  if (d0 >= (TC ? round_up(b.n_docs, 64) : b.n_docs)) return;
  float4 y[NK], r[NK];
#pragma unroll
  for (int v = 0; v < NK; ++v) {
    const int col = v * 128 + lane * 4;
    y[v] = (d < b.n_docs && col < a.Kp) ? *reinterpret_cast<const float4 *>(a.Y32 + (long long)d * a.Kp + col)
                                         : f4(0.f);
    r[v] = f4(0.f);
  }
  if (a.same_token && d < b.n_docs) {
    const int lo = b.indptr[d], hi = b.indptr[d + 1];
    if (lo >= b.nz_base) {
      for (int base = lo; base < hi; base += 32) {
        const NzChunk c = load_chunk(b, a.V, base, hi, lane, -1);
        for (int q = 0; q < c.n; q += 4) {
          int mm[4];
          float ff[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            mm[u] = __shfl_sync(0xffffffffu, c.m, (q + u) & 31);
            ff[u] = (float)__shfl_sync(0xffffffffu, c.f, (q + u) & 31);
            if (q + u >= c.n) ff[u] = 0.f;
          }
          // all NK x 4 row pieces are requested before the first H atomic (loads
          // are not moved across the atomics by the compiler)
          float4 qv[NK][4];
#pragma unroll
          for (int v = 0; v < NK; ++v) {
            const int col = v * 128 + lane * 4;
#pragma unroll
            for (int u = 0; u < 4; ++u)
              qv[v][u] = col < a.Kp ? *reinterpret_cast<const float4 *>(a.Q32 + (long long)mm[u] * a.Kp + col)
                                    : f4(0.f);
          }
#pragma unroll
          for (int v = 0; v < NK; ++v) {
            const int col = v * 128 + lane * 4;
            if (col < a.Kp) {
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                const float ff2 = ff[u];
                r[v].x = fmaf(ff2 * qv[v][u].x, qv[v][u].x, r[v].x);
                r[v].y = fmaf(ff2 * qv[v][u].y, qv[v][u].y, r[v].y);
                r[v].z = fmaf(ff2 * qv[v][u].z, qv[v][u].z, r[v].z);
                r[v].w = fmaf(ff2 * qv[v][u].w, qv[v][u].w, r[v].w);
                if (ff2 != 0.f)
                  atomicAdd(reinterpret_cast<float4 *>(a.H32 + (long long)mm[u] * a.Kp + col),
                            make_float4(ff2 * y[v].x, ff2 * y[v].y, ff2 * y[v].z, ff2 * y[v].w));
              }
            }
          }
        }
      }
    }
  }
  float ls = 0.f;
#pragma unroll
  for (int v = 0; v < NK; ++v) {
    const int col = v * 128 + lane * 4;
    if (col < a.Kp) {
      const float4 z = make_float4(y[v].x * y[v].x - r[v].x, y[v].y * y[v].y - r[v].y,
                                   y[v].z * y[v].z - r[v].z, y[v].w * y[v].w - r[v].w);
      if constexpr (TC) {
        if (d < round_up(b.n_docs, 64)) {
          __nv_bfloat162 p[2] = {__floats2bfloat162_rn(z.x, z.y), __floats2bfloat162_rn(z.z, z.w)};
          *reinterpret_cast<uint2 *>(a.Z16 + (long long)d * a.Kp + col) = *reinterpret_cast<const uint2 *>(p);
        }
      } else {
        if (d < b.n_docs) *reinterpret_cast<float4 *>(a.Z32 + (long long)d * a.Kp + col) = z;
      }
      if (a.want_loss)
        ls += y[v].x * (y[v].x * y[v].x - 3.f * r[v].x) + y[v].y * (y[v].y * y[v].y - 3.f * r[v].y) +
              y[v].z * (y[v].z * y[v].z - 3.f * r[v].z) + y[v].w * (y[v].w * y[v].w - 3.f * r[v].w);
    }
  }
  if (a.want_loss) {
    for (int o = 16; o > 0; o >>= 1) ls += __shfl_xor_sync(0xffffffffu, ls, o);
    if (lane == 0 && ls != 0.f) atomicAdd(&a.st->loss_data, (double)ls);
  }
}

// ------------------------------------------------------------ a6: Zc rows
// One warp per touched word (compact slot t): Zc_t = q * (2 c q - 2 H_m); then
// H_m and c_m are cleared for the next batch (this warp is their only reader).
template <int NK>
__global__ void __launch_bounds__(256) k_zh_f32(StepArgs a) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = blockIdx.x * 8 + warp;
  if (t >= a.st->n_touched) return;
  const int m = a.widx[t];
  const float c = (float)a.cnt[m];
  float ls = 0.f;
#pragma unroll
  for (int v = 0; v < NK; ++v) {
    const int col = v * 128 + lane * 4;
    if (col < a.Kp) {
      float4 *hp = reinterpret_cast<float4 *>(a.H32 + (long long)m * a.Kp + col);
      const float4 q = *reinterpret_cast<const float4 *>(a.Q32 + (long long)m * a.Kp + col);
      const float4 h = *hp;
      const float4 z = make_float4(q.x * (2.f * c * q.x - 2.f * h.x), q.y * (2.f * c * q.y - 2.f * h.y),
                                   q.z * (2.f * c * q.z - 2.f * h.z), q.w * (2.f * c * q.w - 2.f * h.w));
      *reinterpret_cast<float4 *>(a.Zc32 + (long long)t * a.Kp + col) = z;
      *hp = f4(0.f);
      ls += q.x * q.x * q.x + q.y * q.y * q.y + q.z * q.z * q.z + q.w * q.w * q.w;
    }
  }
  if (a.want_loss) {
    for (int o = 16; o > 0; o >>= 1) ls += __shfl_xor_sync(0xffffffffu, ls, o);
    if (lane == 0) atomicAdd(&a.st->loss_data, 2.0 * (double)c * (double)ls);
  }
  __syncwarp();
  if (lane == 0) a.cnt[m] = 0;
}

// ------------------------------------------------------------ a5 + a6: G1 + G2 (FP32)
// Split reduction over the rows [docs: (X, Z)] ++ [touched words: (U, Zc)]:
// block (s, ti, tn) sums rows of split s into the 64 x 64 tile (ti, tn) of
// partial s, 4 x 4 outputs per thread.
__global__ void __launch_bounds__(256) k_g_f32(StepArgs a) {
  const int nd = a.st->cur.n_docs, nt = a.same_token ? a.st->n_touched : 0;
  const int R = nd + nt;
  const int s = blockIdx.x, i0 = blockIdx.y * 64, n0 = blockIdx.z * 64;
  const int rb = (int)((long long)R * s / a.nsplit), re = (int)((long long)R * (s + 1) / a.nsplit);
  __shared__ __align__(16) float As[32][64];
  __shared__ __align__(16) float Bs[32][64];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  for (int r0 = rb; r0 < re; r0 += 32) {
    {
      const int rr = tid >> 3, cc = (tid & 7) * 8, r = r0 + rr;
      float4 a0 = f4(0.f), a1 = f4(0.f), b0 = f4(0.f), b1 = f4(0.f);
      if (r < re) {
        const float *ap, *bp;
        if (r < nd) {
          ap = a.X32 + (long long)r * a.Dp;
          bp = a.Z32 + (long long)r * a.Kp;
        } else {
          const int t = r - nd;
          ap = a.U32 + (long long)a.widx[t] * a.Dp;
          bp = a.Zc32 + (long long)t * a.Kp;
        }
        a0 = *reinterpret_cast<const float4 *>(ap + i0 + cc);
        a1 = *reinterpret_cast<const float4 *>(ap + i0 + cc + 4);
        b0 = *reinterpret_cast<const float4 *>(bp + n0 + cc);
        b1 = *reinterpret_cast<const float4 *>(bp + n0 + cc + 4);
      }
      *reinterpret_cast<float4 *>(&As[rr][cc]) = a0;
      *reinterpret_cast<float4 *>(&As[rr][cc + 4]) = a1;
      *reinterpret_cast<float4 *>(&Bs[rr][cc]) = b0;
      *reinterpret_cast<float4 *>(&Bs[rr][cc + 4]) = b1;
    }
    __syncthreads();
#pragma unroll 8
    for (int rr = 0; rr < 32; ++rr) {
      const float4 av = *reinterpret_cast<const float4 *>(&As[rr][ty * 4]);
      const float4 bv = *reinterpret_cast<const float4 *>(&Bs[rr][tx * 4]);
      const float ar[4] = {av.x, av.y, av.z, av.w}, br[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(ar[i], br[j], acc[i][j]);
    }
    __syncthreads();
  }
  float *gp = a.Gpart + (long long)s * a.Dp * a.Kp;
#pragma unroll
  for (int i = 0; i < 4; ++i)
    *reinterpret_cast<float4 *>(gp + (long long)(i0 + ty * 4 + i) * a.Kp + n0 + tx * 4) =
        make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
}

void launch_qy_f32(const StepArgs &a, cudaStream_t s) {
  dim3 g((a.V + a.Bmax + 63) / 64, a.Kp / 64);
  k_qy_f32<<<g, 256, 0, s>>>(a);
}

void launch_rz(const StepArgs &a, cudaStream_t s) {
  const int nk = (a.Kp + 127) / 128;
  const bool tc = a.precision == TLDA_BF16;
#define TLDA_RZ(NKv)                                                                      \
  if (nk == NKv) {                                                                        \
    if (tc) k_rz<NKv, true><<<round_up(a.Bmax, 64) / 8, 256, 0, s>>>(a);                 \
    else k_rz<NKv, false><<<round_up(a.Bmax, 64) / 8, 256, 0, s>>>(a);                   \
    return;                                                                               \
  }
  TLDA_RZ(1) TLDA_RZ(2) TLDA_RZ(3) TLDA_RZ(4)
#undef TLDA_RZ
}

void launch_zh_f32(const StepArgs &a, cudaStream_t s) {
  const int nk = (a.Kp + 127) / 128;
  if (nk == 1) k_zh_f32<1><<<(a.V + 7) / 8, 256, 0, s>>>(a);
  else if (nk == 2) k_zh_f32<2><<<(a.V + 7) / 8, 256, 0, s>>>(a);
  else if (nk == 3) k_zh_f32<3><<<(a.V + 7) / 8, 256, 0, s>>>(a);
  else k_zh_f32<4><<<(a.V + 7) / 8, 256, 0, s>>>(a);
}

void launch_g_f32(const StepArgs &a, cudaStream_t s) {
  dim3 g(a.nsplit, a.Dp / 64, a.Kp / 64);
  k_g_f32<<<g, 256, 0, s>>>(a);
}

// ------------------------------------------------------------ a9: reduce + update
// 32 entries (i, n) per block, the partial sums split over 8 warps:
// g = sum over partials; grad = E - 3 c3/S3 g; Phi -= lr grad (skipped on a
// sticky error or S3 = 0); the BF16 Phi^T image follows Phi.
__global__ void __launch_bounds__(256) k_reduce_update(StepArgs a) {
  DevState *st = a.st;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int e = blockIdx.x * 32 + lane;
  const unsigned long long S3 = st->S3;
  const int err = st->err;
  const double scale = S3 ? a.c3 / (double)S3 : 0.0;
  const bool live = e < a.D * a.K;
  const int i = live ? e / a.K : 0, n = live ? e % a.K : 0;
  const long long off = (long long)i * a.Kp + n, stride = (long long)a.Dp * a.Kp;
  float part = 0.f;
  if (live) {  // eight partials in flight per iteration
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    int s = w;
    for (; s + 56 < a.nsplit; s += 64) {
#pragma unroll
      for (int u = 0; u < 8; ++u) acc[u] += a.Gpart[(s + 8 * u) * stride + off];
    }
    for (; s < a.nsplit; s += 8) acc[0] += a.Gpart[s * stride + off];
#pragma unroll
    for (int u = 0; u < 8; ++u) part += acc[u];
  }
  __shared__ float red[8][32];
  red[w][lane] = part;
  __syncthreads();
  if (w == 0 && live) {
    float g = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) g += red[q][lane];
    if (a.mode == 1) {
      a.gdata_out[e] = S3 ? (float)(scale * (double)g) + a.G3[off] : 0.f;
    } else {
      const float grad = S3 ? a.E[off] - (float)(3.0 * scale * (double)g) : 0.f;
      if (a.grad_out) a.grad_out[e] = grad;
      float phi = a.Phi[e];
      if (!err && S3) {
        phi -= a.lr * grad;
        a.Phi[e] = phi;
      }
      if (a.PhiImg) a.PhiImg[phi_img_index(n, i, a.Kp)] = __float2bfloat16_rn(phi);
    }
  }
}

// End of a step (one warp, after the reduction): the step's loss, the
// per-step sums cleared for the next batch, the step counter, and the next
// batch descriptor of a pass.
__global__ void k_step_end(StepArgs a) {
  DevState *st = a.st;
  if (threadIdx.x != 0) return;
  const unsigned long long S3 = st->S3;
  const double scale = S3 ? a.c3 / (double)S3 : 0.0;
  st->loss = S3 ? st->loss_phi - scale * st->loss_data : 0.0;
  st->last_S3 = S3;
  st->S3 = 0;
  st->loss_data = 0.0;
  st->n_touched = 0;
  st->step += 1;
  if (st->descs && st->pass_pos < st->n_descs) st->cur = st->descs[st->pass_pos++];
}

void launch_reduce_update(const StepArgs &a, cudaStream_t s) {
  k_reduce_update<<<(a.D * a.K + 31) / 32, 256, 0, s>>>(a);
  k_step_end<<<1, 32, 0, s>>>(a);
}

}  // namespace tlda
