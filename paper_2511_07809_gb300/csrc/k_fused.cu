// Fused BF16 tensor-core CP-step data term for D, K in (64, 128] (padded to
// 128).  One persistent CTA per SM walks 32-document tiles of the batch and
// accumulates G1 + G2 (eq. vec_deriv's data term with the same-token terms of
// distinct-token triples) in TMEM, without any V-sized intermediate.
//
// With q_j = u_{m_j} Phi for the tile's nonzeros j (word m_j, count f_j,
// document d_j), the per-document quantities are sums over nonzeros:
//   y_d = sum_{j in d} f_j q_j          (= x_d Phi, x_d = sum f u)
//   r_d = sum_{j in d} f_j q_j^2
// and the data term is one reduction over nonzeros:
//   G1 + G2 = sum_d x_d z_d^T + sum_m u_m [q_m (2 c_m q_m - 2 H_m)]^T
//           = sum_j u_{m_j} [f_j (z_{d_j} + 2 q_j^2 - 2 q_j y_{d_j})]^T,
//   z_d = y_d^2 - r_d.
// Per tile (chunks of 128 nonzeros, U rows gathered with cp.async):
//   pass 1: Q = U Phi (tcgen05, U K-major); Y^T += Q^T F^T, R^T += (Q*Q)^T F^T
//           (tcgen05, MN-major; F^T holds f_j at column d_j)
//   then    y, z = y^2 - r into shared memory (FP32)
//   pass 2: Q = U Phi again; B''_j = f_j (z + 2 q^2 - 2 q y); G += U^T B''
//           (tcgen05, both MN-major: the gathered U tile read the other way)
// Each CTA writes its 128 x 128 partial; the reduction kernel sums them.
#include "tc_ptx.cuh"

namespace tlda {
namespace {
using namespace tc;

constexpr int kT = 32;        // documents per tile
constexpr int kChunk = 128;   // nonzeros per chunk
constexpr int kFusedThreads = 256;

// shared-memory map (bytes from the 1024-aligned base)
constexpr int kOffPhi = 0;          // Phi^T image 2 x [128 x 64] BF16               32 KB
constexpr int kOffU0 = 32768;       // U chunk     2 x [128 x 64] BF16 (buffer 0)    32 KB
constexpr int kOffU1 = 65536;       //                               (buffer 1)    32 KB
constexpr int kOffQ = 98304;        // Q chunk (pass 1) / B'' chunk (pass 2)        32 KB
constexpr int kOffQ2 = 131072;      // Q*Q chunk                                    32 KB
constexpr int kOffF = 163840;       // F^T chunk   [128 x 64 documents] BF16        16 KB
constexpr int kOffY = 180224;       // y tile FP32 32 x 128                         16 KB
constexpr int kOffZ = 196608;       // z tile FP32 32 x 128                         16 KB
constexpr int kWin = 1024;          // nonzeros whose metadata sit in shared memory
constexpr int kOffMeta = 212992;    // window metadata m, f, d (12 KB), indptr slice, L
constexpr int kOffBar = kOffMeta + 3 * kWin * 4 + 512;  // 4 mbarriers + TMEM slot
constexpr int kFusedSmem = 1024 + kOffBar + 64;

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_one() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// 4 consecutive values (col multiple of 4, < 128) of row `row` of a
// 2 x [rows x 64] BF16 tile in the 128-byte swizzle layout.
__device__ __forceinline__ void st_bf16x4(unsigned char *tile, int sub_bytes, int row, int col, float a, float b,
                                          float c, float d) {
  __nv_bfloat162 lo = __floats2bfloat162_rn(a, b), hi = __floats2bfloat162_rn(c, d);
  uint2 pk;
  pk.x = *reinterpret_cast<uint32_t *>(&lo);
  pk.y = *reinterpret_cast<uint32_t *>(&hi);
  *reinterpret_cast<uint2 *>(tile + (col >> 6) * sub_bytes + sw_chunk(row, (col & 63) >> 3) + ((col & 7) << 1)) = pk;
}

__global__ void __launch_bounds__(kFusedThreads, 1) k_fused(StepArgs a) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char *sm = align1024(smem_raw);
  unsigned char *sPhi = sm + kOffPhi, *sQ = sm + kOffQ, *sQ2 = sm + kOffQ2, *sF = sm + kOffF;
  float *sY = reinterpret_cast<float *>(sm + kOffY), *sZ = reinterpret_cast<float *>(sm + kOffZ);
  int *s_m = reinterpret_cast<int *>(sm + kOffMeta);        // kWin raw word indices (-1 past the end)
  float *s_f = reinterpret_cast<float *>(s_m + kWin);       // kWin weights (0 if invalid)
  int *s_d = reinterpret_cast<int *>(s_f + kWin);           // kWin local documents
  int *s_ptr = s_d + kWin;                                  // kT + 1 absolute offsets
  int *s_L = s_ptr + 64;                                    // kT token counts
  uint64_t *bars = reinterpret_cast<uint64_t *>(sm + kOffBar);  // 0: Phi, 1: Y/R and G, 2-3: Q buffers
  uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 4);
  __shared__ int failed, s_bad, s_mlast;
  __shared__ float s_red[kFusedThreads / 32];

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int quad = warp & 3, half = warp >> 2;
  const BatchDesc b = a.st->cur;
  const int nd = b.n_docs;
  const int ntiles = (nd + kT - 1) / kT;
  float *gp = a.Gpart + (long long)blockIdx.x * a.Dp * a.Kp;

  if (tid == 0) {
    for (int i = 0; i < 4; ++i) mbar_init(&bars[i], 1);
    fence_mbar_init();
    failed = 0;
  }
  if (warp == 0) tmem_alloc(tslot, 512);
  // F^T tile starts (and is kept) at zero; entries are written and cleared per chunk
  for (int e = tid; e < 16384 / 16; e += kFusedThreads) reinterpret_cast<uint4 *>(sF)[e] = make_uint4(0u, 0u, 0u, 0u);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  // TMEM columns: Q (two buffers, chunk parity), Y^T, R^T, G
  const uint32_t colQ0 = tmem, colYt = tmem + 256, colRt = tmem + 320, colG = tmem + 384;
  const bool has_work = ntiles > (int)blockIdx.x;
  if (has_work && tid == 0) {
    mbar_arrive_expect_tx(&bars[0], 32768);
    bulk_load(sPhi, a.PhiImg, 32768, &bars[0]);
  }
  if (has_work && !mbar_wait(&bars[0], 0)) failed = 1;
  __syncthreads();
  uint32_t mph = 0;        // completed phases of barrier 1 (Y/R and G products)
  uint32_t qph[2] = {0, 0};  // completed phases of barriers 2, 3 (Q products)
  bool g_init = false;     // G accumulator holds data (uniform across the CTA)
  const uint32_t idQ = idesc_bf16(128, 128);
  const uint32_t idYR = idesc_bf16(128, 64) | (1u << 15) | (1u << 16);
  const uint32_t idG = idesc_bf16(128, 128) | (1u << 15) | (1u << 16);

  auto mma_wait = [&]() {
    const bool ok = mbar_wait(&bars[1], mph & 1);
    ++mph;
    if (!ok) failed = 1;
    tc_fence_after();
  };
  auto q_wait = [&](int buf) {
    const bool ok = mbar_wait(&bars[2 + buf], qph[buf] & 1);
    ++qph[buf];
    if (!ok) failed = 1;
    tc_fence_after();
  };

  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    if (failed) break;
    const int d0 = tile * kT, Te = min(kT, nd - d0);
    if (tid <= Te) s_ptr[tid] = b.indptr[d0 + tid];
    if (tid < kT) s_L[tid] = 0;
    if (tid == 0) {
      s_bad = 0;
      s_mlast = -1;
    }
    __syncthreads();
    if (tid < Te && (s_ptr[tid + 1] < s_ptr[tid] || s_ptr[tid] < b.nz_base)) s_bad = 1;
    const int nz0 = s_ptr[0];
    const int nnz = max(0, s_ptr[Te] - nz0);
    const int nch = (nnz + kChunk - 1) / kChunk;
    const int nwin = (nnz + kWin - 1) / kWin;

    // metadata of nonzeros [w0, w0 + kWin) of the tile; pass 1 also validates
    // the entries and adds the documents' token counts
    auto load_window = [&](int w0, bool check) {
      constexpr int kPer = kWin / kFusedThreads;
      int mr[kPer], fr[kPer];
#pragma unroll
      for (int u = 0; u < kPer; ++u) {  // all loads in flight first
        const int j = w0 + tid + u * kFusedThreads;
        mr[u] = -1;
        fr[u] = 0;
        if (j < nnz) {
          mr[u] = __ldg(b.indices + ((long long)(nz0 + j) - b.nz_base));
          fr[u] = __ldg(b.counts + ((long long)(nz0 + j) - b.nz_base));
        }
      }
#pragma unroll
      for (int u = 0; u < kPer; ++u) {
        const int t = tid + u * kFusedThreads, j = w0 + t;
        int dd = 0;
        float f = 0.f;
        if (j < nnz) {
          const int p = nz0 + j;
          int lo = 0, hi = Te - 1;  // last document whose range starts at or before p
          while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_ptr[mid] <= p) lo = mid;
            else hi = mid - 1;
          }
          dd = lo;
          const bool valid = mr[u] >= 0 && mr[u] < a.V && fr[u] > 0;
          f = valid ? (float)fr[u] : 0.f;
          if (check) {
            if (!valid) s_bad = 1;
            else atomicAdd(s_L + dd, fr[u]);
          }
        }
        s_m[t] = mr[u];
        s_f[t] = f;
        s_d[t] = dd;
      }
      __syncthreads();
      if (check) {  // words strictly ascending within a document
        for (int t = tid; t < kWin; t += kFusedThreads) {
          const int j = w0 + t;
          if (j < nnz && nz0 + j > s_ptr[s_d[t]]) {
            const int mp = t > 0 ? s_m[t - 1] : s_mlast;
            if (s_m[t] <= mp) s_bad = 1;
          }
        }
        __syncthreads();
        if (tid == 0) s_mlast = s_m[kWin - 1];
      }
    };
    // cp.async gather of the BF16 U rows of window chunk c into buffer buf
    auto gather = [&](int c, int buf) {
      unsigned char *sU = sm + (buf ? kOffU1 : kOffU0);
      for (int pce = tid; pce < kChunk * 16; pce += kFusedThreads) {
        const int r = pce >> 4, pc = pce & 15;
        const int m = s_m[c * kChunk + r];
        unsigned char *dst = sU + (pc >> 3) * 16384 + sw_chunk(r, pc & 7);
        if (m >= 0 && m < a.V) cp_async16(dst, a.U16 + (long long)m * a.Dp + pc * 8);
        else *reinterpret_cast<uint4 *>(dst) = make_uint4(0u, 0u, 0u, 0u);
      }
      cp_async_commit();
    };
    // Q chunk = U chunk Phi (rows = nonzeros) into TMEM buffer buf; committed
    // to barrier 2 + buf
    auto issue_q = [&](int buf) {
      if (tid == 0) {
        const uint32_t ub = smem_u32(sm + (buf ? kOffU1 : kOffU0)), pb = smem_u32(sPhi);
#pragma unroll
        for (int kk = 0; kk < 8; ++kk)
          mma_bf16(colQ0 + buf * 128, sdesc_sw128(ub + (kk >> 2) * 16384 + (kk & 3) * 32),
                   sdesc_sw128(pb + (kk >> 2) * 16384 + (kk & 3) * 32), idQ, kk > 0 ? 1u : 0u);
        mma_commit(&bars[2 + buf]);
      }
    };
    // 64 consecutive FP32 columns (4 loads in flight, one wait) of this warp's lanes
    auto tmem_ld64 = [&](uint32_t taddr, float (&v)[64]) {
      uint32_t r[64];
#pragma unroll
      for (int p = 0; p < 4; ++p)
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(r[p * 16 + 0]), "=r"(r[p * 16 + 1]), "=r"(r[p * 16 + 2]), "=r"(r[p * 16 + 3]),
              "=r"(r[p * 16 + 4]), "=r"(r[p * 16 + 5]), "=r"(r[p * 16 + 6]), "=r"(r[p * 16 + 7]),
              "=r"(r[p * 16 + 8]), "=r"(r[p * 16 + 9]), "=r"(r[p * 16 + 10]), "=r"(r[p * 16 + 11]),
              "=r"(r[p * 16 + 12]), "=r"(r[p * 16 + 13]), "=r"(r[p * 16 + 14]), "=r"(r[p * 16 + 15])
            : "r"(taddr + p * 16)
            : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int i = 0; i < 64; ++i) v[i] = __uint_as_float(r[i]);
    };
    float lacc = 0.f;

    // ---------------- pass 1: y and r over all chunks (buffer of global chunk g = g & 1).
    // The Q product of chunk c+1 runs while chunk c's Q rows are read out.
    auto put_f = [&](int c, bool on) {  // F^T row r: f_r at the column of its document
      if (tid < kChunk) {
        const int t = c * kChunk + tid, dd = s_d[t];
        *reinterpret_cast<__nv_bfloat16 *>(sF + sw_chunk(tid, dd >> 3) + ((dd & 7) << 1)) =
            __float2bfloat16_rn(on ? s_f[t] : 0.f);
      }
    };
    for (int w = 0; w < nwin && !failed; ++w) {
      const int w0 = w * kWin, wch = min(kWin, nnz - w0 + kChunk - 1) / kChunk, gb = w0 / kChunk;
      load_window(w0, true);
      gather(0, gb & 1);
      if (wch > 1) gather(1, (gb + 1) & 1);
      if (wch > 1) cp_async_wait_one();
      else cp_async_wait_all();
      put_f(0, true);
      fence_proxy_async();
      __syncthreads();
      issue_q(gb & 1);
      for (int c = 0; c < wch; ++c) {
        const int g = gb + c, buf = g & 1;
        if (c + 1 < wch) {  // chunk c+1's rows have landed: start its Q product now
          cp_async_wait_all();
          fence_proxy_async();
          tc_fence_before();
          __syncthreads();
          tc_fence_after();
          issue_q(buf ^ 1);
        }
        q_wait(buf);
        if (__syncthreads_or(failed)) break;
        if (c + 2 < wch) gather(c + 2, buf);  // this buffer's Q product is done
        {  // Q and Q*Q rows (BF16) for the MN-major reductions over nonzeros
          const int row = quad * 32 + lane;
          float q[64];
          tmem_ld64(colQ0 + buf * 128 + (static_cast<uint32_t>(quad * 32) << 16) + half * 64, q);
#pragma unroll
          for (int i = 0; i < 64; i += 4) {
            const int c0 = half * 64 + i;
            st_bf16x4(sQ, 16384, row, c0, q[i], q[i + 1], q[i + 2], q[i + 3]);
            st_bf16x4(sQ2, 16384, row, c0, q[i] * q[i], q[i + 1] * q[i + 1], q[i + 2] * q[i + 2],
                      q[i + 3] * q[i + 3]);
          }
        }
        fence_proxy_async();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid == 0) {  // Y^T += Q^T F^T, R^T += (Q*Q)^T F^T  (M = topics, N = 64 documents)
          const uint32_t qb = smem_u32(sQ), q2b = smem_u32(sQ2), fb = smem_u32(sF);
#pragma unroll
          for (int kk = 0; kk < 8; ++kk) {
            mma_bf16(colYt, sdesc_mn_sw128(qb + kk * 2048, 16384), sdesc_mn_sw128(fb + kk * 2048, 16384), idYR,
                     (g > 0 || kk > 0) ? 1u : 0u);
            mma_bf16(colRt, sdesc_mn_sw128(q2b + kk * 2048, 16384), sdesc_mn_sw128(fb + kk * 2048, 16384), idYR,
                     (g > 0 || kk > 0) ? 1u : 0u);
          }
          mma_commit(&bars[1]);
        }
        mma_wait();
        put_f(c, false);                     // these products are done: clear c's entries
        if (c + 1 < wch) put_f(c + 1, true);  // and place c+1's
        fence_proxy_async();
        if (__syncthreads_or(failed)) break;
      }
    }
    cp_async_wait_all();
    if (__syncthreads_or(failed)) break;
    // ---------------- y, z = y^2 - r (FP32, [document][topic]); S3 and validation
    {
      const int topic = quad * 32 + lane;
      float yv[16], rv[16];
      if (nch > 0) {
        tmem_ld16(colYt + (static_cast<uint32_t>(quad * 32) << 16) + half * 16, yv);
        tmem_ld16(colRt + (static_cast<uint32_t>(quad * 32) << 16) + half * 16, rv);
      } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) yv[i] = rv[i] = 0.f;
      }
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int dd = half * 16 + i;
        const float y = dd < Te ? yv[i] : 0.f;
        const float r = (dd < Te && a.same_token) ? rv[i] : 0.f;
        sY[dd * 128 + topic] = y;
        sZ[dd * 128 + topic] = y * y - r;
        lacc += y * (y * y - 3.f * r);
      }
    }
    if (warp == 0) {
      const long long L = lane < Te ? s_L[lane] : 0;
      unsigned long long s3 = L >= 3 ? (unsigned long long)(L * (L - 1) * (L - 2)) : 0ull;
      for (int o = 16; o > 0; o >>= 1) s3 += __shfl_xor_sync(0xffffffffu, s3, o);
      if (lane == 0) {
        if (s3) atomicAdd(&a.st->S3, s3);
        if (s_bad) atomicOr(&a.st->err, kErrCsr);
      }
    }
    __syncthreads();
    // ---------------- pass 2 in reverse chunk order: the last two chunks of
    // pass 1 are still in their buffers; earlier ones are gathered again.
    // The Q product of the next (lower) chunk runs during this chunk's B''.
    for (int w = nwin - 1; w >= 0 && !failed; --w) {
      const int w0 = w * kWin, wch = min(kWin, nnz - w0 + kChunk - 1) / kChunk, gb = w0 / kChunk;
      if (nwin > 1) load_window(w0, false);
      auto resident = [&](int c) { return nwin == 1 && c >= wch - 2; };
      if (!resident(wch - 1)) gather(wch - 1, (gb + wch - 1) & 1);
      if (wch > 1 && !resident(wch - 2)) gather(wch - 2, (gb + wch - 2) & 1);
      if (wch > 1 && !resident(wch - 2) && !resident(wch - 1)) cp_async_wait_one();
      else cp_async_wait_all();
      fence_proxy_async();
      tc_fence_before();
      __syncthreads();
      tc_fence_after();
      issue_q((gb + wch - 1) & 1);
      for (int c = wch - 1; c >= 0; --c) {
        const int g = gb + c, buf = g & 1;
        if (c > 0) {  // chunk c-1's rows are in: start its Q product now
          cp_async_wait_all();
          fence_proxy_async();
          tc_fence_before();
          __syncthreads();
          tc_fence_after();
          issue_q(buf ^ 1);
        }
        q_wait(buf);
        if (__syncthreads_or(failed)) break;
        {
          const int row = quad * 32 + lane, t = c * kChunk + row;
          const int dd = s_d[t];
          const float f = s_f[t];
          const float4 *yr = reinterpret_cast<const float4 *>(sY + dd * 128 + half * 64);
          const float4 *zr = reinterpret_cast<const float4 *>(sZ + dd * 128 + half * 64);
          float q[64];
          tmem_ld64(colQ0 + buf * 128 + (static_cast<uint32_t>(quad * 32) << 16) + half * 64, q);
#pragma unroll
          for (int i4 = 0; i4 < 16; ++i4) {
            const float4 y4 = yr[i4], z4 = zr[i4];
            const float ys[4] = {y4.x, y4.y, y4.z, y4.w}, zs[4] = {z4.x, z4.y, z4.z, z4.w};
            float bb[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const float qi = q[i4 * 4 + u];
              if (a.same_token) {
                bb[u] = f * (zs[u] + 2.f * qi * qi - 2.f * qi * ys[u]);
                lacc += 2.f * f * qi * qi * qi;
              } else {
                bb[u] = f * zs[u];
              }
            }
            st_bf16x4(sQ, 16384, row, half * 64 + i4 * 4, bb[0], bb[1], bb[2], bb[3]);
          }
        }
        fence_proxy_async();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid == 0) {  // G += U_chunk^T B''_chunk (M = features, N = topics)
          const uint32_t ub = smem_u32(sm + (buf ? kOffU1 : kOffU0)), bq = smem_u32(sQ);
#pragma unroll
          for (int kk = 0; kk < 8; ++kk)
            mma_bf16(colG, sdesc_mn_sw128(ub + kk * 2048, 16384), sdesc_mn_sw128(bq + kk * 2048, 16384), idG,
                     (g_init || kk > 0) ? 1u : 0u);
          mma_commit(&bars[1]);
        }
        g_init = true;
        mma_wait();
        if (__syncthreads_or(failed)) break;
        if (c > 1 && !resident(c - 2)) gather(c - 2, buf);  // this buffer's products are done
      }
    }
    cp_async_wait_all();
    if (a.want_loss) {
      for (int o = 16; o > 0; o >>= 1) lacc += __shfl_xor_sync(0xffffffffu, lacc, o);
      if (lane == 0) s_red[warp] = lacc;
      __syncthreads();
      if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < kFusedThreads / 32; ++w) t += s_red[w];
        atomicAdd(&a.st->loss_data, t);
      }
    }
    if (__syncthreads_or(failed)) break;
  }
  cp_async_wait_all();
  // ---------------- partial G of this CTA -> Gpart[blockIdx.x] (rows = features)
  if (failed) {
    if (tid == 0) atomicOr(&a.st->err, kErrTimeout);
  } else {
    const int row = quad * 32 + lane;
#pragma unroll 1
    for (int p = 0; p < 4; ++p) {
      const int c0 = half * 64 + p * 16;
      float v[16];
      if (g_init) tmem_ld16(colG + (static_cast<uint32_t>(quad * 32) << 16) + c0, v);
      else
        for (int i = 0; i < 16; ++i) v[i] = 0.f;
#pragma unroll
      for (int q = 0; q < 16; q += 4)
        *reinterpret_cast<float4 *>(gp + (long long)row * a.Kp + c0 + q) = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 512);
}

}  // namespace

bool fused_supported(int Dp, int Kp) { return Dp == 128 && Kp == 128; }

void launch_fused(const StepArgs &a, cudaStream_t s, int grid) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, kFusedSmem);
    attr = true;
  }
  k_fused<<<grid, kFusedThreads, kFusedSmem, s>>>(a);
}

}  // namespace tlda
