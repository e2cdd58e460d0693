// Fused BF16 tensor-core CP-step data term for D, K in (64, 128] (padded to
// 128), and the persistent kernel that runs a whole online pass with it.
//
// Data term.  With q_j = u_{m_j} Phi for the nonzeros j of a tile of
// documents (word m_j, count f_j, document d_j), the per-document sums
//   y_d = sum_{j in d} f_j q_j          (= x_d Phi, x_d = sum f u)
//   r_d = sum_{j in d} f_j q_j^2
// give G1 + G2 of eq. vec_deriv (with the same-token terms of distinct-token
// triples) as one reduction over nonzeros:
//   G1 + G2 = sum_d x_d z_d^T + sum_m u_m [q_m (2 c_m q_m - 2 H_m)]^T
//           = sum_j u_{m_j} [f_j (z_{d_j} + 2 q_j^2 - 2 q_j y_{d_j})]^T,
//   z_d = y_d^2 - r_d.
// Per tile (chunks of 128 nonzeros, U rows gathered with cp.async):
//   pass 1: Q = U Phi (tcgen05, U K-major); Y^T += Q^T F^T, R^T += (Q*Q)^T F^T
//           (tcgen05, MN-major; F^T holds f_j at column d_j)
//   then    y, z = y^2 - r into shared memory (FP32)
//   pass 2: Q = U Phi again; B''_j = f_j (z + 2 q^2 - 2 q y); G += U^T B''
//           (tcgen05, both MN-major: the gathered U tile read the other way)
// G stays in TMEM across a block's tiles; each block then writes its
// 128 x 128 partial.
//
// k_fused runs the data term of one step (the reduction and the update are
// separate kernels).  k_pass runs steps [s0, s1) of a pass in one cooperative
// launch, each step in two phases separated by grid barriers:
//   A  the data blocks (all but the last few): the data term of the step's
//      batch over a range of documents equal in nonzeros (split points from
//      k_pass_prep), in tiles of at most the batch's tuned size; the last
//      blocks: the Phi-only terms E = 3(1+theta) P - 3 G3
//      (P = Phi (Phi^T Phi * Phi^T Phi)) and their loss parts, in jobs of
//      kPassPhiCols columns dealt round-robin;
//   B  block b: its slice of the entries of Phi: the partials summed,
//      grad = E - 3 c3/S3 (G1 + G2), Phi -= lr grad, and the BF16 Phi^T
//      image the next step's MMAs read.
// Between its arrival at the mid-step barrier and its wait, a block that has
// documents in the next step requests that step's first tile, and a Phi-only
// block brings the CSR of the step after next into L2.
// Every wait (mbarrier or grid barrier) is bounded; an expired wait sets an
// abort flag that ends every block's loop and is reported as a timeout.
#include <algorithm>

#include "tc_ptx.cuh"

namespace tlda {
namespace {
using namespace tc;

constexpr int kT = kPassTileDocs;  // documents per tile, at most
constexpr int kChunk = 128;   // nonzeros per chunk
constexpr int kFusedThreads = 256;
constexpr int kMinPassGrid = 128;  // at least one block per Phi column (K <= 128)
constexpr int kPhiCols = kPassPhiCols;

// shared-memory map (bytes from the 1024-aligned base)
constexpr int kOffPhi = 0;          // Phi^T image 2 x [128 x 64] BF16               32 KB
constexpr int kOffU0 = 32768;       // U chunk     2 x [128 x 64] BF16 (buffer 0)    32 KB
constexpr int kOffU1 = 65536;       //                               (buffer 1)    32 KB
constexpr int kOffQ = 98304;        // Q chunk (pass 1) / B'' chunk (pass 2)        32 KB
constexpr int kOffQ2 = 131072;      // Q*Q chunk                                    32 KB
constexpr int kOffF = 163840;       // F^T chunk   [128 x 64 documents] BF16        16 KB
// y and z rows of one document are kYP floats apart: the 4-float pad moves
// each document's row by four banks, so the lanes of one warp, which read
// rows of a few different documents at the same topic, do not collide
constexpr int kYP = 132;
constexpr int kOffY = 180224;       // y tile FP32 32 x kYP                         16.5 KB
constexpr int kOffZ = kOffY + 32 * kYP * 4;  // z tile FP32 32 x kYP                16.5 KB
constexpr int kWin = 1024;          // nonzeros whose metadata sit in shared memory
constexpr int kOffMeta = kOffZ + 32 * kYP * 4;  // window metadata m, f, d (12 KB), indptr slice, L
constexpr int kOffBar = kOffMeta + 3 * kWin * 4 + 512;  // 4 mbarriers, TMEM slot, flags
constexpr int kFusedSmem = 1024 + kOffBar + 64;

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Named block barrier over the n threads (a multiple of 32) that use barrier
// `id`; id 0 with every thread of the block is __syncthreads().  The _or form
// also returns whether any of them passed a true `v`.
__device__ __forceinline__ void bar_sync_n(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }
__device__ __forceinline__ bool bar_or_n(int id, int n, bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.or.pred q, %2, %3, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"(static_cast<uint32_t>(v)), "r"(id), "r"(n)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void cp_async_wait_one() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// 8 consecutive values (col multiple of 8, < 128) of row `row` of a
// 2 x [rows x 64] BF16 tile in the 128-byte swizzle layout: one whole
// 16-byte chunk, so the 32 rows a warp writes at once (8 rows per XOR
// pattern) fill every bank once per 128 bytes.
__device__ __forceinline__ void st_bf16x8(unsigned char *tile, int sub_bytes, int row, int col, const float *v) {
  uint4 pk;
  __nv_bfloat162 h;
  h = __floats2bfloat162_rn(v[0], v[1]);
  pk.x = *reinterpret_cast<uint32_t *>(&h);
  h = __floats2bfloat162_rn(v[2], v[3]);
  pk.y = *reinterpret_cast<uint32_t *>(&h);
  h = __floats2bfloat162_rn(v[4], v[5]);
  pk.z = *reinterpret_cast<uint32_t *>(&h);
  h = __floats2bfloat162_rn(v[6], v[7]);
  pk.w = *reinterpret_cast<uint32_t *>(&h);
  *reinterpret_cast<uint4 *>(tile + (col >> 6) * sub_bytes + sw_chunk(row, (col & 63) >> 3)) = pk;
}

// One row of B'' = f (z + 2 q^2 - 2 q y) (same-token correction on) or f z
// (off), 64 topics from col0, staged as BF16 into `tile`; y and z rows of the
// row's document from shared memory.  Groups of 8 topics that start at or
// past `ncols` (padding topics, whose G columns are never read) are neither
// computed nor stored.  With kLoss the row's loss part 2 f sum q^3 is added
// to lacc (skipped when the caller wants no loss).
template <bool kSame, bool kLoss>
__device__ __forceinline__ void b2_row(const float (&q)[64], const float4 *yr, const float4 *zr, float f,
                                       unsigned char *tile, int row, int col0, int ncols, float &lacc) {
#pragma unroll
  for (int i8 = 0; i8 < 8; ++i8) {
    if (i8 * 8 >= ncols) break;
    float bb[8];
#pragma unroll
    for (int h4 = 0; h4 < 2; ++h4) {
      const float4 z4 = zr[i8 * 2 + h4];
      const float zs[4] = {z4.x, z4.y, z4.z, z4.w};
      if (kSame) {
        const float4 y4 = yr[i8 * 2 + h4];
        const float ys[4] = {y4.x, y4.y, y4.z, y4.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float qi = q[i8 * 8 + h4 * 4 + u];
          bb[h4 * 4 + u] = f * (zs[u] + 2.f * qi * (qi - ys[u]));
          if (kLoss) lacc += 2.f * f * qi * qi * qi;
        }
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) bb[h4 * 4 + u] = f * zs[u];
      }
    }
    st_bf16x8(tile, 16384, row, col0 + i8 * 8, bb);
  }
}

__device__ __forceinline__ void b2_row_any(bool same, bool loss, const float (&q)[64], const float4 *yr,
                                           const float4 *zr, float f, unsigned char *tile, int row, int col0,
                                           int ncols, float &lacc) {
  if (same) {
    if (loss) b2_row<true, true>(q, yr, zr, f, tile, row, col0, ncols, lacc);
    else b2_row<true, false>(q, yr, zr, f, tile, row, col0, ncols, lacc);
  } else {
    b2_row<false, false>(q, yr, zr, f, tile, row, col0, ncols, lacc);
  }
}

// 64 consecutive FP32 TMEM columns of this warp's lanes (4 loads in flight, one wait).
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, float (&v)[64]) {
  uint32_t r[64];
#pragma unroll
  for (int p = 0; p < 4; ++p)
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[p * 16 + 0]), "=r"(r[p * 16 + 1]), "=r"(r[p * 16 + 2]), "=r"(r[p * 16 + 3]), "=r"(r[p * 16 + 4]),
          "=r"(r[p * 16 + 5]), "=r"(r[p * 16 + 6]), "=r"(r[p * 16 + 7]), "=r"(r[p * 16 + 8]), "=r"(r[p * 16 + 9]),
          "=r"(r[p * 16 + 10]), "=r"(r[p * 16 + 11]), "=r"(r[p * 16 + 12]), "=r"(r[p * 16 + 13]),
          "=r"(r[p * 16 + 14]), "=r"(r[p * 16 + 15])
        : "r"(taddr + p * 16)
        : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 64; ++i) v[i] = __uint_as_float(r[i]);
}

// Block sum of one float per thread (every thread calls; the result is valid
// in thread 0).
__device__ __forceinline__ float block_sum(float v, float *red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  float t = 0.f;
  if (threadIdx.x == 0)
    for (int w = 0; w < kFusedThreads / 32; ++w) t += red[w];
  return t;
}

// One block's tile engine: shared-memory views, TMEM columns and the phases
// of its mbarriers (0: Phi image, 1: Y/R and G products, 2-3: Q buffers).
struct NoPre {
  __device__ bool operator()() const { return true; }
};

struct Fused {
  unsigned char *sm, *sPhi, *sQ, *sQ2, *sF;
  float *sY, *sZ;
  int *s_m, *s_d, *s_ptr, *s_L;
  float *s_f;
  uint64_t *bars;
  int *sh;                       // [0] failed, [1] bad tile, [2] last word of the previous window
  uint32_t tmem, colQ0, colYt, colRt, colG;
  uint32_t mph, qph0, qph1, pph;
  int tid, warp, lane, quad, half;

  __device__ bool failed() const { return *reinterpret_cast<volatile int *>(sh) != 0; }
  __device__ void fail() { *reinterpret_cast<volatile int *>(sh) = 1; }

  __device__ void init(unsigned char *raw) {
    sm = align1024(raw);
    sPhi = sm + kOffPhi;
    sQ = sm + kOffQ;
    sQ2 = sm + kOffQ2;
    sF = sm + kOffF;
    sY = reinterpret_cast<float *>(sm + kOffY);
    sZ = reinterpret_cast<float *>(sm + kOffZ);
    s_m = reinterpret_cast<int *>(sm + kOffMeta);   // kWin raw word indices (-1 past the end)
    s_f = reinterpret_cast<float *>(s_m + kWin);    // kWin weights (0 if invalid)
    s_d = reinterpret_cast<int *>(s_f + kWin);      // kWin local documents
    s_ptr = s_d + kWin;                             // kT + 1 absolute offsets
    s_L = s_ptr + 64;                               // kT token counts
    bars = reinterpret_cast<uint64_t *>(sm + kOffBar);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 4);
    sh = reinterpret_cast<int *>(bars + 5);
    tid = threadIdx.x;
    warp = tid >> 5;
    lane = tid & 31;
    quad = warp & 3;
    half = warp >> 2;
    mph = qph0 = qph1 = pph = 0;
    if (tid == 0) {
      for (int i = 0; i < 4; ++i) mbar_init(&bars[i], 1);
      fence_mbar_init();
      sh[0] = sh[1] = 0;
      sh[2] = -1;
    }
    if (warp == 0) tmem_alloc(tslot, 512);
    // the F^T tile starts (and is kept) at zero; entries are written and cleared per chunk
    for (int e = tid; e < 16384 / 16; e += kFusedThreads)
      reinterpret_cast<uint4 *>(sF)[e] = make_uint4(0u, 0u, 0u, 0u);
    // the Q and Q*Q tiles start at zero: their padding-topic columns are
    // never written by the staging, so they only ever hold finite values
    for (int e = tid; e < 65536 / 16; e += kFusedThreads)
      reinterpret_cast<uint4 *>(sQ)[e] = make_uint4(0u, 0u, 0u, 0u);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    tmem = *tslot;
    // TMEM columns: Q (two buffers, chunk parity), Y^T, R^T, G
    colQ0 = tmem;
    colYt = tmem + 256;
    colRt = tmem + 320;
    colG = tmem + 384;
  }

  __device__ void finish() {
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 512);
  }

  // Phi^T image into shared memory by bulk copy (image written by an earlier kernel).
  __device__ void phi_bulk(const __nv_bfloat16 *img) {
    if (tid == 0) {
      mbar_arrive_expect_tx(&bars[0], 32768);
      bulk_load(sPhi, img, 32768, &bars[0]);
    }
  }
  __device__ void phi_wait() {
    if (!mbar_wait(&bars[0], pph & 1)) fail();
    ++pph;
  }

  // Partial G (rows = features) -> dst (rows < D, columns < K rounded up to
  // 16, row pitch Kp, FP32); zeros if no tile added to it.
  __device__ void write_g(float *dst, int D, int K, int Kp, bool g_init) {
    const int row = quad * 32 + lane;
    tc_fence_after();
#pragma unroll 1
    for (int p = 0; p < 4; ++p) {
      const int c0 = half * 64 + p * 16;
      if (c0 >= K) break;  // warp-uniform
      float v[16];
      if (g_init) tmem_ld16(colG + (static_cast<uint32_t>(quad * 32) << 16) + c0, v);
      else
        for (int i = 0; i < 16; ++i) v[i] = 0.f;
      if (row < D) {
#pragma unroll
        for (int q = 0; q < 16; q += 4)
          *reinterpret_cast<float4 *>(dst + (long long)row * Kp + c0 + q) = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
      }
    }
    tc_fence_before();
  }

  // Partial G in the slice-blocked layout of the pass kernel: entry e = i K + n
  // of this block's partial goes to dst[(e / per) G + blk][e % per], so the
  // partials of one slice of entries are contiguous across blocks.
  __device__ void write_g_sliced(float *dst, int D, int K, int G, int blk, int per, bool g_init) {
    const int row = quad * 32 + lane;
    tc_fence_after();
    if ((K & 3) == 0) {
      // staged row-major in the U buffers (free once the tiles are done),
      // then copied out slice by slice: each slice's `per` entries are one
      // contiguous run in global memory, so the stores are whole lines
      float *stage = reinterpret_cast<float *>(sm + kOffU0);
      if (half * 64 < K) {  // warp-uniform: this warp's 64 columns, one TMEM wait
        float v[64];
        if (g_init) tmem_ld64(colG + (static_cast<uint32_t>(quad * 32) << 16) + half * 64, v);
        else
          for (int i = 0; i < 64; ++i) v[i] = 0.f;
        if (row < D) {
#pragma unroll
          for (int q = 0; q < 64; q += 4)
            if (half * 64 + q < K)
              *reinterpret_cast<float4 *>(stage + row * K + half * 64 + q) = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
        }
      }
      __syncthreads();
      const int n4 = D * K / 4;
      for (int v4 = tid; v4 < n4; v4 += kFusedThreads) {
        const int e = v4 * 4, sl = e / per;  // per is a multiple of 4: a float4 never straddles slices
        *reinterpret_cast<float4 *>(dst + ((long long)sl * G + blk) * per + (e - sl * per)) =
            *reinterpret_cast<const float4 *>(stage + e);
      }
    } else {
#pragma unroll 1
      for (int p = 0; p < 4; ++p) {
        const int c0 = half * 64 + p * 16;
        if (c0 >= K) break;  // warp-uniform
        float v[16];
        if (g_init) tmem_ld16(colG + (static_cast<uint32_t>(quad * 32) << 16) + c0, v);
        else
          for (int i = 0; i < 16; ++i) v[i] = 0.f;
        if (row < D) {
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            if (c0 + q < K) {
              const int e = row * K + c0 + q, sl = e / per;
              dst[((long long)sl * G + blk) * per + (e - sl * per)] = v[q];
            }
          }
        }
      }
    }
    tc_fence_before();
  }

  // Tile header: the row offsets of documents [d0, d0 + Te) into s_ptr
  // (checked), the token counts and the window state cleared.
  // Run by threads gt = 0 .. gn - 1 (gn >= 64) that share barrier `bid`.
  __device__ void tile_head(const BatchDesc &b, int d0, int Te, int gt = -1, int gn = kFusedThreads, int bid = 0) {
    if (gt < 0) gt = tid;
    if (gt <= Te) s_ptr[gt] = b.indptr[d0 + gt];
    if (gt < kT) s_L[gt] = 0;
    if (gt == 0) {
      sh[1] = 0;
      sh[2] = -1;
    }
    bar_sync_n(bid, gn);
    if (gt < Te && (s_ptr[gt + 1] < s_ptr[gt] || s_ptr[gt] < b.nz_base)) sh[1] = 1;
  }

  // Metadata of nonzeros [w0, w0 + kWin) of the tile (nonzeros nz0 .. nz0 +
  // nnz of Te documents); pass 1 (check) also validates the entries and adds
  // the documents' token counts.  In two halves: window_loads requests the
  // words and counts of nonzeros nz0 + j, j < lim, into registers (all in
  // flight together); window_fill files them with their documents (needs
  // s_ptr) into shared memory, nonzeros past nnz as empty.
  template <int kGn = kFusedThreads>
  __device__ void window_loads(const BatchDesc &b, long long nz0, int lim, int w0, int gt, int (&mr)[kWin / kGn],
                               int (&fr)[kWin / kGn]) {
#pragma unroll
    for (int u = 0; u < kWin / kGn; ++u) {
      const int j = w0 + gt + u * kGn;
      mr[u] = -1;
      fr[u] = 0;
      if (j < lim) {
        mr[u] = __ldg(b.indices + (nz0 + j - b.nz_base));
        fr[u] = __ldg(b.counts + (nz0 + j - b.nz_base));
      }
    }
  }
  template <int kGn = kFusedThreads>
  __device__ void load_window(const StepArgs &a, const BatchDesc &b, int nz0, int nnz, int Te, int w0, bool check,
                              int gt = -1, int bid = 0) {
    if (gt < 0) gt = tid;
    int mr[kWin / kGn], fr[kWin / kGn];
    window_loads<kGn>(b, nz0, nnz, w0, gt, mr, fr);
    window_fill<kGn>(a, nz0, nnz, Te, w0, check, gt, bid, mr, fr);
  }
  template <int kGn = kFusedThreads>
  __device__ void window_fill(const StepArgs &a, int nz0, int nnz, int Te, int w0, bool check, int gt, int bid,
                              const int (&mr)[kWin / kGn], const int (&fr)[kWin / kGn]) {
    constexpr int kPer = kWin / kGn;
    int dds[kPer], ms[kPer];  // kept for the order check below
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const int t = gt + u * kGn, j = w0 + t;
      int dd = 0, m = -1;
      float f = 0.f;
      if (j < nnz) {
        const int p = nz0 + j;
        // last document whose range starts at or before p: a fixed
        // five-step search (Te <= kT = 32), so a thread's searches overlap
        int lo = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1)
          if (lo + step < Te && s_ptr[lo + step] <= p) lo += step;
        dd = lo;
        m = mr[u];
        const bool valid = m >= 0 && m < a.V && fr[u] > 0;
        f = valid ? (float)fr[u] : 0.f;
        if (check) {
          if (!valid) sh[1] = 1;
          else atomicAdd(s_L + dd, fr[u]);
        }
      }
      s_m[t] = m;
      s_f[t] = f;
      s_d[t] = dd;
      dds[u] = dd;
      ms[u] = m;
    }
    bar_sync_n(bid, kGn);
    if (check) {  // words strictly ascending within a document
#pragma unroll
      for (int u = 0; u < kPer; ++u) {
        const int t = gt + u * kGn, j = w0 + t;
        if (j < nnz && nz0 + j > s_ptr[dds[u]]) {
          const int mp = t > 0 ? s_m[t - 1] : sh[2];
          if (ms[u] <= mp) sh[1] = 1;
        }
      }
      bar_sync_n(bid, kGn);
      if (gt == 0) sh[2] = s_m[kWin - 1];
    }
  }

  // cp.async gather of the BF16 U rows of window chunk c into buffer buf.
  __device__ void gather(const StepArgs &a, int c, int buf, int gt = -1, int gn = kFusedThreads) {
    unsigned char *sU = sm + (buf ? kOffU1 : kOffU0);
    if (gt < 0) gt = tid;
    for (int pce = gt; pce < kChunk * 16; pce += gn) {
      const int r = pce >> 4, pc = pce & 15;
      const int m = s_m[c * kChunk + r];
      unsigned char *dst = sU + (pc >> 3) * 16384 + sw_chunk(r, pc & 7);
      if (m >= 0 && m < a.V) cp_async16(dst, a.U16 + (long long)m * a.Dp + pc * 8);
      else *reinterpret_cast<uint4 *>(dst) = make_uint4(0u, 0u, 0u, 0u);
    }
    cp_async_commit();
  }

  // The first tile of batch b (tiles of td documents) requested ahead, by
  // every thread: its header, its first window's metadata and the U rows of
  // its first two chunks (still in flight on return).  A later
  // tiles(..., prefetched = true) on the same batch starts from them.  Uses
  // s_ptr, the window metadata and both U buffers.
  // nzh is the offset of the tile's first nonzero as the split rows give it,
  // lim the nonzeros of the batch from there on (at most kWin): the window's
  // words and counts are requested together with the header's offsets, not
  // after them (a header that disagrees, only possible for a corrupt batch,
  // falls back to the plain order).
  // Run by the 128 threads gt = 0 .. 127 that share barrier `bid` (the
  // rest of the block may do other work meanwhile).
  __device__ void prefetch(const StepArgs &a, const BatchDesc &b, int td, int gt, int bid, long long nzh, int lim) {
    if (b.n_docs <= 0) return;
    const int Te = min(td, b.n_docs);
    int mr[kWin / 128], fr[kWin / 128];
    window_loads<128>(b, nzh, lim, 0, gt, mr, fr);
    tile_head(b, 0, Te, gt, 128, bid);
    const int nz0 = s_ptr[0], nnz = max(0, s_ptr[Te] - nz0);
    if (nnz == 0) return;
    const int wch = min(kWin, nnz + kChunk - 1) / kChunk;
    if (nz0 == nzh && min(nnz, kWin) <= lim) window_fill<128>(a, nz0, nnz, Te, 0, true, gt, bid, mr, fr);
    else load_window<128>(a, b, nz0, nnz, Te, 0, true, gt, bid);
    gather(a, 0, 0, gt, 128);
    if (wch > 1) gather(a, 1, 1, gt, 128);
  }

  // The data term of tiles tile0, tile0 + tstride, ... of batch b (td <= kT
  // documents each), added to the G columns.  S3 and validation bits go to
  // S3_dst and err_dst, the per-document loss parts to lacc.  Expects the Phi
  // image in shared memory, or (phi_pending) pre() to bring it there: pre()
  // then runs once, by every thread, after the first window's CSR slice and
  // U rows are requested and before the first MMA (it waits for whatever the
  // image waits for and copies it in; false if that failed).  With
  // `prefetched`, prefetch(a, b, td) has already requested tile tile0's
  // header, first window and first U rows.  tsplit > 0 (tile0 = 0, tstride = 1)
  // makes two tiles, documents [0, tsplit) and [tsplit, nd), instead of
  // tiles of td.  Returns false on an expired wait.
  template <class Pre = NoPre>
  __device__ bool tiles(const StepArgs &a, const BatchDesc &b, int tile0, int tstride, int td, float &lacc,
                        bool &g_init, unsigned long long *S3_dst, int *err_dst, bool phi_pending = false,
                        Pre pre = Pre(), bool prefetched = false, int tsplit = 0) {
    const int nd = b.n_docs;
    const int ntiles = tsplit > 0 ? 2 : nd > 0 ? (nd + td - 1) / td : 0;
    const uint32_t idQ = idesc_bf16(128, 128);
    const uint32_t idYR = idesc_bf16(128, 64) | (1u << 15) | (1u << 16);
    const uint32_t idG = idesc_bf16(128, 128) | (1u << 15) | (1u << 16);
    const uint32_t lane_off = static_cast<uint32_t>(quad * 32) << 16;

    auto mma_wait = [&]() {
      if (!mbar_wait(&bars[1], mph & 1)) fail();
      ++mph;
      tc_fence_after();
    };
    auto q_wait = [&](int buf) {
      uint32_t &ph = buf ? qph1 : qph0;
      if (!mbar_wait(&bars[2 + buf], ph & 1)) fail();
      ++ph;
      tc_fence_after();
    };

    for (int tile = tile0; tile < ntiles; tile += tstride) {
      if (failed()) break;
      const int d0 = tsplit > 0 ? (tile ? tsplit : 0) : tile * td;
      const int Te = tsplit > 0 ? (tile ? nd - tsplit : tsplit) : min(td, nd - d0);
      const bool pf = prefetched && tile == tile0;  // header, first window and U rows requested already
      if (!pf) tile_head(b, d0, Te);
      const int nz0 = s_ptr[0];
      const int nnz = max(0, s_ptr[Te] - nz0);
      const int nch = (nnz + kChunk - 1) / kChunk;
      const int nwin = (nnz + kWin - 1) / kWin;
      auto load_window = [&](int w0, bool check) { this->load_window(a, b, nz0, nnz, Te, w0, check); };
      auto gather = [&](int c, int buf) { this->gather(a, c, buf); };
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
      auto put_f = [&](int c, bool on) {  // F^T row r: f_r at the column of its document
        if (tid < kChunk) {
          const int t = c * kChunk + tid, dd = s_d[t];
          *reinterpret_cast<__nv_bfloat16 *>(sF + sw_chunk(tid, dd >> 3) + ((dd & 7) << 1)) =
              __float2bfloat16_rn(on ? s_f[t] : 0.f);
        }
      };

      // ---------------- pass 1: y and r over all chunks (buffer of global chunk g = g & 1).
      // The Q product of chunk c+1 runs while chunk c's Q rows are read out.
      for (int w = 0; w < nwin && !failed(); ++w) {
        const int w0 = w * kWin, wch = min(kWin, nnz - w0 + kChunk - 1) / kChunk, gb = w0 / kChunk;
        if (!(pf && w == 0)) {
          load_window(w0, true);
          gather(0, gb & 1);
          if (wch > 1) gather(1, (gb + 1) & 1);
        }
        if (wch > 1) cp_async_wait_one();
        else cp_async_wait_all();
        put_f(0, true);
        fence_proxy_async();
        if (phi_pending) {  // the Phi^T image: pre() brings it into shared memory
          if (!pre()) fail();
          phi_pending = false;
        }
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
          q_wait(buf);  // each thread waits itself: the buffer and Q(c) are free to use
          if (c + 2 < wch) gather(c + 2, buf);  // this buffer's Q product is done
          {  // Q and Q*Q rows (BF16) for the MN-major reductions over nonzeros
            const int row = quad * 32 + lane;
            float q[64];
            tmem_ld64(colQ0 + buf * 128 + lane_off + half * 64, q);
#pragma unroll
            for (int i = 0; i < 64; i += 8) {
              if (half * 64 + i >= a.K) break;  // padding topics: their Y, R rows are never read
              float q2[8];
#pragma unroll
              for (int u = 0; u < 8; ++u) q2[u] = q[i + u] * q[i + u];
              st_bf16x8(sQ, 16384, row, half * 64 + i, q + i);
              st_bf16x8(sQ2, 16384, row, half * 64 + i, q2);
            }
          }
          fence_proxy_async();
          tc_fence_before();
          if (__syncthreads_or(failed())) break;  // also orders the previous chunk's F^T entries
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
          if (c + 1 < wch) put_f(c + 1, true);  // and place c+1's (read after the next staging barrier)
          fence_proxy_async();
        }
      }
      cp_async_wait_all();
      if (__syncthreads_or(failed())) break;
      // ---------------- y, z = y^2 - r (FP32, [document][topic]); S3 and validation
      {
        const int topic = quad * 32 + lane;
        float yv[16], rv[16];
        if (nch > 0) {
          tmem_ld16(colYt + lane_off + half * 16, yv);
          tmem_ld16(colRt + lane_off + half * 16, rv);
        } else {
#pragma unroll
          for (int i = 0; i < 16; ++i) yv[i] = rv[i] = 0.f;
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int dd = half * 16 + i;
          const float y = dd < Te ? yv[i] : 0.f;
          const float r = (dd < Te && a.same_token) ? rv[i] : 0.f;
          sY[dd * kYP + topic] = y;
          sZ[dd * kYP + topic] = y * y - r;
          if (a.want_loss && topic < a.K) lacc += y * (y * y - 3.f * r);
        }
      }
      if (warp == 0) {
        const long long L = lane < Te ? s_L[lane] : 0;
        unsigned long long s3 = L >= 3 ? (unsigned long long)(L * (L - 1) * (L - 2)) : 0ull;
        for (int o = 16; o > 0; o >>= 1) s3 += __shfl_xor_sync(0xffffffffu, s3, o);
        if (lane == 0) {
          if (s3) atomicAdd(S3_dst, s3);
          if (sh[1]) atomicOr(err_dst, kErrCsr);
        }
      }
      __syncthreads();
      // ---------------- pass 2 in reverse chunk order: the last two chunks of
      // pass 1 are still in their buffers (rows in shared memory, Q in TMEM);
      // earlier ones are gathered again.  The Q product of the next (lower)
      // chunk runs during this chunk's B''.
      for (int w = nwin - 1; w >= 0 && !failed(); --w) {
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
        // a resident chunk's Q is also still in its TMEM buffer from pass 1
        if (!resident(wch - 1)) issue_q((gb + wch - 1) & 1);
        for (int c = wch - 1; c >= 0; --c) {
          const int g = gb + c, buf = g & 1;
          if (c > 0) {  // chunk c-1's rows are in: start its Q product now
            cp_async_wait_all();
            fence_proxy_async();
            tc_fence_before();
            __syncthreads();
            tc_fence_after();
            if (!resident(c - 1)) issue_q(buf ^ 1);
          }
          if (!resident(c)) q_wait(buf);
          else tc_fence_after();
          {
            const int row = quad * 32 + lane, t = c * kChunk + row;
            const int dd = s_d[t];
            const float f = s_f[t];
            const float4 *yr = reinterpret_cast<const float4 *>(sY + dd * kYP + half * 64);
            const float4 *zr = reinterpret_cast<const float4 *>(sZ + dd * kYP + half * 64);
            float q[64];
            tmem_ld64(colQ0 + buf * 128 + lane_off + half * 64, q);
            b2_row_any(a.same_token, a.want_loss, q, yr, zr, f, sQ, row, half * 64, a.K - half * 64, lacc);
          }
          fence_proxy_async();
          tc_fence_before();
          if (__syncthreads_or(failed())) break;
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
          mma_wait();  // each thread waits itself: the B'' tile and this U buffer are free
          if (c > 1 && !resident(c - 2)) gather(c - 2, buf);  // this buffer's products are done
        }
      }
      cp_async_wait_all();
      if (__syncthreads_or(failed())) break;
    }
    cp_async_wait_all();
    if (phi_pending) {  // no tile reached an MMA: still run pre() (the grid barrier's wait)
      if (!pre()) fail();
    }
    __syncthreads();
    return !failed();
  }
};

__global__ void __launch_bounds__(kFusedThreads, 1) k_fused(StepArgs a) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ float s_red[kFusedThreads / 32];
  Fused f;
  f.init(smem_raw);
  const BatchDesc b = a.st->cur;
  const int ntiles = (b.n_docs + kT - 1) / kT;
  const bool has_work = b.n_docs > 0 && ntiles > (int)blockIdx.x;
  if (has_work) {
    f.phi_bulk(a.PhiImg);
    f.phi_wait();
  }
  __syncthreads();
  float lacc = 0.f;
  bool g_init = false;
  if (has_work) f.tiles(a, b, blockIdx.x, gridDim.x, kT, lacc, g_init, &a.st->S3, &a.st->err);
  if (a.want_loss) {
    const float t = block_sum(lacc, s_red);
    if (f.tid == 0 && t != 0.f) atomicAdd(&a.st->loss_data, (double)t);
  }
  if (f.failed()) {
    if (f.tid == 0) atomicOr(&a.st->err, kErrTimeout);
  } else {
    f.write_g(a.Gpart + (long long)blockIdx.x * a.Dp * a.Kp, a.D, a.K, a.Kp, g_init);
  }
  f.finish();
}

// ------------------------------------------------------------ persistent pass
__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid barrier (every block is resident: cooperative launch) in two halves:
// grid_arrive is a release increment of the launch's monotone arrival
// counter, grid_wait polls it with acquire loads until it reaches `target`
// and checks the abort flag and the bound every 16th poll (bounded; false if
// it expired here, or if any block flagged an abort).  Work that needs
// nothing from the other blocks can run between the two.
__device__ void grid_arrive(PassCtl *ctl) {
  __syncthreads();
  // release: this block's writes (ordered before by the block barrier)
  if (threadIdx.x == 0) asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&ctl->bar) : "memory");
}

__device__ bool grid_wait(PassCtl *ctl, unsigned target, int *s_ok) {
  if (threadIdx.x == 0) {
    int ok = 1;
    const long long t0 = clock64();
    unsigned polls = 0;
    while (ld_acquire(&ctl->bar) < target) {
      if ((++polls & 15u) != 0u) continue;
      if (*reinterpret_cast<volatile int *>(&ctl->abort)) {
        ok = 0;
        break;
      }
      if (clock64() - t0 > kWaitCycles) {
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

// Self-test of the bounded grid barrier: block 0 never arrives, so every
// block waits the bound out (or sees the abort flag the first one raises) and
// counts itself in S3[0].  Ends in about one second.
__global__ void k_barrier_selftest(PassCtl *ctl) {
  __shared__ int s_ok;
  if (blockIdx.x != 0) grid_arrive(ctl);
  const bool ok = grid_wait(ctl, gridDim.x, &s_ok);
  if (threadIdx.x == 0 && !ok) atomicAdd(&ctl->S3[0], 1ull);
}

// What a block of the pass needs to know of one step before it starts: the
// batch's descriptor and the block's entries of the step's split row (its
// documents [d_lo, d_hi), indptr at d_lo, the batch's nonzeros [lo, hi), the
// documents of its first tile when it takes two).
struct StepPlan {
  BatchDesc d;
  int w[6];
};

__global__ void __launch_bounds__(kFusedThreads, 1) k_pass(StepArgs a, PassArgs p) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ float s_red[kFusedThreads / 32];
  __shared__ float s_am[kPhiCols];
  __shared__ int s_ok, s_stop;
  Fused f;
  f.init(smem_raw);
  if (threadIdx.x == 0) s_stop = 0;
  PassCtl *ctl = p.ctl;
  DevState *st = a.st;
  const int G = gridDim.x, blk = blockIdx.x, tid = f.tid;
  const int D = a.D, K = a.K, Kp = a.Kp, DK = a.D * a.K;
  // phase B: this block's entries of Phi (row-major D x K), a multiple of 4
  // per block (16-byte slices for the bulk copies)
  const int per = ((DK + G - 1) / G + 3) & ~3;
  const int e0 = min(DK, blk * per), e1 = min(DK, e0 + per);
  // phase A: Phi (D x K FP32, rows padded to K + 1 floats against bank
  // conflicts) in the U-buffer and Q region, free until the tiles start
  float *sPh = reinterpret_cast<float *>(f.sm + kOffU0);
  const int ldp = K + 1;
  __shared__ float s_m1[128];
  if (tid < 128) s_m1[tid] = tid < D ? a.m1[tid] : 0.f;
  // the steps' plans in shared memory, three slots (step s in slot
  // (s - s0) mod 3): the first two now, each later one two steps ahead (by
  // the second warp group after the mid-step arrival), so that neither the
  // step's start nor the next step's first-tile request waits for them
  __shared__ __align__(16) StepPlan s_plan[3];
  auto request_plan = [&](int s, int t) {  // by threads t = 0 .. 10 (cp.async)
    if (s >= p.s1 || t < 0 || t >= 11) return;
    StepPlan *pl = &s_plan[(s - p.s0) % 3];
    if (t < 5) {
      cp_async8(reinterpret_cast<char *>(&pl->d) + 8 * t, reinterpret_cast<const char *>(p.descs + s) + 8 * t);
    } else {
      const int k = t - 5;
      const int off = k < 2 ? blk + k : k == 2 ? G + 1 + blk : k < 5 ? p.split_stride - 2 + (k - 3) : 2 * G + 2 + blk;
      cp_async4(&pl->w[k], p.splits + (long long)s * p.split_stride + off);
    }
  };
  request_plan(p.s0, tid);
  request_plan(p.s0 + 1, tid - 11);
  cp_async_commit();
  cp_async_wait_all();
  __syncthreads();
  unsigned nbar = 0;
  bool bar_pending = false;
  double last_loss = 0.0;
  unsigned long long last_S3 = 0;

  // this block's documents of step s: [d_lo, d_hi), an equal share of the
  // batch's nonzeros, in tiles of td <= cap documents; false for a block
  // without documents (the last blocks take only the Phi-only columns)
  // (ts > 0: two tiles, the first of ts documents, as the split rows give them)
  auto block_range = [&](int s, BatchDesc &bs, int &td, int &ts) -> bool {
    const StepPlan &pl = s_plan[(s - p.s0) % 3];
    const BatchDesc b = pl.d;
    const int nd = b.n_docs;
    const int cap = p.tile_cap > 0 ? p.tile_cap : (b.tile_cap > 0 ? b.tile_cap : 32);
    const int nwork = nd > 0 ? pass_data_blocks(p, G, nd) : 0;
    bs = b;
    td = 1;
    ts = 0;
    if (blk >= nwork) return false;
    const int d_lo = pl.w[0], d_hi = pl.w[1];
    bs.indptr = b.indptr + d_lo;
    bs.n_docs = max(0, d_hi - d_lo);
    const int nt = (bs.n_docs + cap - 1) / cap;
    td = nt > 0 ? (bs.n_docs + nt - 1) / nt : 1;
    const int t1 = pl.w[5];
    if (nt == 2 && t1 > 0 && t1 < bs.n_docs && t1 <= min(cap, kT) && bs.n_docs - t1 <= min(cap, kT)) ts = t1;
    return true;
  };
  bool prefetched = false;  // this step's first tile requested during the previous step

  for (int s = p.s0; s < p.s1; ++s) {
    const int slot = s & 1;
    const int nd = s_plan[(s - p.s0) % 3].d.n_docs;
    // the last e_blocks blocks take no tiles: they start on the Phi-only
    // columns as soon as the step begins
    const int Gd = pass_data_blocks(p, G, nd);
    const int nwork = nd > 0 ? Gd : 0;
    BatchDesc bs;
    int td, ts;
    const bool has = block_range(s, bs, td, ts);

    // ---------------- phase A: the data term of this block's tiles.  The
    // first tile's CSR slice and U rows are requested before the wait for the
    // previous step's barrier (they need nothing from phase B); then the Phi^T
    // image (written by every block in that phase B) comes in 16-byte cp.async
    // pieces (plain global reads, so its writers need no proxy fence).
    auto pre = [&]() -> bool {
      if (bar_pending) {
        bar_pending = false;
        if (!grid_wait(ctl, nbar * G, &s_ok)) return false;
      }
      const uint4 *src = reinterpret_cast<const uint4 *>(a.PhiImg);
      uint4 *dstp = reinterpret_cast<uint4 *>(f.sPhi);
      for (int e = tid; e < 32768 / 16; e += kFusedThreads) cp_async16(dstp + e, src + e);
      cp_async_commit();
      cp_async_wait_all();
      fence_proxy_async();  // read by the tensor cores
      return true;
    };
    if (has) {
      float lacc = 0.f;
      bool g_init = false;
      f.tiles(a, bs, 0, 1, td, lacc, g_init, &ctl->S3[slot], &st->err, true, pre, prefetched, ts);
      if (a.want_loss) {
        const float t = block_sum(lacc, s_red);
        if (tid == 0 && t != 0.f) atomicAdd(&ctl->loss_data[slot], (double)t);
      }
      if (!f.failed()) f.write_g_sliced(a.Gpart, D, K, G, blk, per, g_init);
      __syncthreads();
    }
    if (bar_pending) {  // no tiles here: wait before the Phi-only columns
      bar_pending = false;
      if (!grid_wait(ctl, nbar * G, &s_ok)) break;
    }
    // the Phi-only terms, kPhiCols columns per job: the dedicated blocks take
    // the jobs round-robin (job j to dedicated block j mod n), a fixed
    // assignment with no counter round trip; with no dedicated blocks every
    // block takes them the same way.  Phi is staged once per block (in the U
    // slots; rows padded to K + 1 floats against bank conflicts).
    const int e_idx = G > Gd ? blk - Gd : blk;  // < 0: a data block, no columns
    const int e_cnt = G > Gd ? G - Gd : G;
    bool staged = false;
    constexpr int kEC = kPhiCols;  // columns per job (a multiple of 4, at most 16)
    constexpr int kEC4 = kEC / 4;
    for (int job = 0; e_idx >= 0; ++job) {
      const int n0 = (e_idx + job * e_cnt) * kEC;
      if (n0 >= K) break;
      if (!staged) {
        constexpr int kRows = 128 / (kFusedThreads / 32);  // rows of Phi per warp (16)
        float ph[kRows][4];
#pragma unroll
        for (int i = 0; i < kRows; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int r = f.warp + 8 * i, n = f.lane + 32 * j;
            ph[i][j] = (r < D && n < K) ? __ldcg(a.Phi + r * K + n) : 0.f;
          }
#pragma unroll
        for (int i = 0; i < kRows; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int r = f.warp + 8 * i, n = f.lane + 32 * j;
            if (r < D && n < K) sPh[r * ldp + n] = ph[i][j];
          }
        __syncthreads();
        staged = true;
      }
      // columns n = n0 .. n0+kEC-1 (those < K): G_{b,n} = phi_b . phi_n for
      // all b (Phi^T Phi is symmetric), a_n = m1 . phi_n, then for every row r
      //   P_rn = sum_b Phi_rb G_{b,n}^2,
      //   G3_rn = 2 Phi_rn a_n + m1_r |phi_n|^2 - 2 m1_r a_n^2,
      //   E_rn = 3(1+theta) P_rn - 3 G3_rn,
      // and the columns' loss part (1+theta)/2 sum_b G^3 - (3 a |phi|^2 - 2 a^3).
      // The job's columns are staged [row][kEC] (float4-aligned, read as
      // broadcasts), so each step of the two reductions is one load of the
      // thread's own entry, kEC/4 float4 loads and kEC FMAs.  The y and z
      // tiles (free in these blocks) hold the staging and the sums.
      float *sC = f.sY;                 // 128 x kEC: Phi columns n0.. (zero past K)
      float *sGh = sC + 128 * kEC;      // 2 x 128 x kEC: half sums
      float *sGc = sGh + 2 * 128 * kEC; // 128 x kEC: the Gram columns
      for (int i = tid; i < 128 * kEC; i += kFusedThreads) {
        const int r = i / kEC, k = i % kEC;
        sC[i] = (r < D && n0 + k < K) ? sPh[r * ldp + n0 + k] : 0.f;
      }
      __syncthreads();
      {
        const int b = tid & 127, rh = tid >> 7;
        float g[kEC];
#pragma unroll
        for (int k = 0; k < kEC; ++k) g[k] = 0.f;
        if (b < K) {
          const int r0 = rh ? (D + 1) / 2 : 0, r1 = rh ? D : (D + 1) / 2;
#pragma unroll 2
          for (int r = r0; r < r1; ++r) {
            const float x = sPh[r * ldp + b];
#pragma unroll
            for (int q = 0; q < kEC4; ++q) {
              const float4 c = reinterpret_cast<const float4 *>(sC)[r * kEC4 + q];
              g[4 * q] = fmaf(x, c.x, g[4 * q]);
              g[4 * q + 1] = fmaf(x, c.y, g[4 * q + 1]);
              g[4 * q + 2] = fmaf(x, c.z, g[4 * q + 2]);
              g[4 * q + 3] = fmaf(x, c.w, g[4 * q + 3]);
            }
          }
        }
        float4 *dst = reinterpret_cast<float4 *>(sGh + (rh * 128 + b) * kEC);
#pragma unroll
        for (int q = 0; q < kEC4; ++q) dst[q] = make_float4(g[4 * q], g[4 * q + 1], g[4 * q + 2], g[4 * q + 3]);
        for (int k = f.warp; k < kEC; k += kFusedThreads / 32) {  // a for column n0 + k
          float am = 0.f;
          for (int r = f.lane; r < D; r += 32) am = fmaf(s_m1[r], sC[r * kEC + k], am);
          for (int o = 16; o > 0; o >>= 1) am += __shfl_xor_sync(0xffffffffu, am, o);
          if (f.lane == 0) s_am[k] = am;
        }
        __syncthreads();
        for (int i = tid; i < 128 * kEC; i += kFusedThreads)
          sGc[i] = i / kEC < K ? sGh[i] + sGh[128 * kEC + i] : 0.f;
        __syncthreads();
      }
      {
        const int r = tid & 127, bh = tid >> 7;
        float pv[kEC];
#pragma unroll
        for (int k = 0; k < kEC; ++k) pv[k] = 0.f;
        if (r < D) {
          const int b0 = bh ? (K + 1) / 2 : 0, b1 = bh ? K : (K + 1) / 2;
#pragma unroll 2
          for (int bb = b0; bb < b1; ++bb) {
            const float x = sPh[r * ldp + bb];
#pragma unroll
            for (int q = 0; q < kEC4; ++q) {
              const float4 gq = reinterpret_cast<const float4 *>(sGc)[bb * kEC4 + q];
              pv[4 * q] = fmaf(x, gq.x * gq.x, pv[4 * q]);
              pv[4 * q + 1] = fmaf(x, gq.y * gq.y, pv[4 * q + 1]);
              pv[4 * q + 2] = fmaf(x, gq.z * gq.z, pv[4 * q + 2]);
              pv[4 * q + 3] = fmaf(x, gq.w * gq.w, pv[4 * q + 3]);
            }
          }
        }
        float4 *dst = reinterpret_cast<float4 *>(sGh + (bh * 128 + r) * kEC);  // the half sums are free again
#pragma unroll
        for (int q = 0; q < kEC4; ++q) dst[q] = make_float4(pv[4 * q], pv[4 * q + 1], pv[4 * q + 2], pv[4 * q + 3]);
        __syncthreads();
        if (tid < D) {
          const float mr = s_m1[tid];
#pragma unroll
          for (int k = 0; k < kEC; ++k) {
            if (n0 + k < K) {
              const float P = sGh[tid * kEC + k] + sGh[(128 + tid) * kEC + k];
              const float am = s_am[k];
              const float n2 = sGc[(n0 + k) * kEC + k];
              const float g3 = 2.f * sC[tid * kEC + k] * am + mr * n2 - 2.f * mr * am * am;
              a.E[tid * Kp + n0 + k] = 3.f * (1.f + a.theta) * P - 3.f * g3;
            }
          }
        }
      }
      if (a.want_loss) {
        float v = 0.f;
        if (tid < K) {
#pragma unroll
          for (int k = 0; k < kEC; ++k) {
            const float gk = sGc[tid * kEC + k];
            if (n0 + k < K) v += 0.5f * (1.f + a.theta) * gk * gk * gk;
          }
        }
        if (tid < kEC && n0 + tid < K) {
          const float am = s_am[tid];
          const float n2 = sGc[(n0 + tid) * kEC + tid];
          v -= 3.f * am * n2 - 2.f * am * am * am;
        }
        const float t = block_sum(v, s_red);
        if (tid == 0) atomicAdd(&ctl->loss_phi[slot], (double)t);
      }
      __syncthreads();
    }
    if (f.failed() && tid == 0) atomicExch(&ctl->abort, 1);
    cp_async_wait_all();  // the plan requested a step ago (blocks without tiles wait nowhere else)
    grid_arrive(ctl);
    ++nbar;
    // Between the arrival and phase B the block splits in two groups of four
    // warps.  Warps 4..7 do what needs nothing of this step's other blocks:
    // the plan of the step after next, the next step's first tile (header,
    // first window, first U rows) and, in a Phi-only block, the CSR of the
    // step after next into L2.  Warps 0..3 wait for the barrier, run phase B
    // (partial slices in the Q buffers, so the two do not touch the same
    // shared memory) and make the end-of-step arrival.  The groups join after
    // that; a failure is carried past the join in s_stop.
    BatchDesc bn;
    int tdn = 1, tsn = 0;
    const bool pf_next = s + 1 < p.s1 && !f.failed() && block_range(s + 1, bn, tdn, tsn);
    if (tid >= 128) {
      const int gt = tid - 128;
      request_plan(s + 2, gt);
      cp_async_commit();
      if (blk >= Gd && s + 2 < p.s1) {
        // lines dealt round-robin over this step's Phi-only blocks, so that
        // the first-tile requests of batch s + 2 meet L2, not HBM
        const BatchDesc b2 = p.descs[s + 2];
        const int *nz2 = p.splits + (long long)(s + 2) * p.split_stride + p.split_stride - 2;
        const long long lo = nz2[0], hi = nz2[1];
        if (b2.n_docs > 0 && lo >= 0 && hi > lo) {
          const int e_i = blk - Gd, e_n = G - Gd;
          l2_prefetch_lines(b2.indptr, (long long)(b2.n_docs + 1) * 4, e_i, e_n, gt, 128);
          l2_prefetch_lines(b2.indices + lo, (hi - lo) * 4, e_i, e_n, gt, 128);
          l2_prefetch_lines(b2.counts + lo, (hi - lo) * 4, e_i, e_n, gt, 128);
        }
      }
      if (pf_next) {
        // the first nonzero of this block's range and the batch's nonzeros
        // from there on bound the window requested with the header
        const StepPlan &pn = s_plan[(s + 1 - p.s0) % 3];
        const long long nzh = pn.w[2];
        const long long lo = bn.nz_base + max(0, pn.w[3]), hi = bn.nz_base + pn.w[4];
        const int lim = nzh >= lo && nzh < hi ? (int)min((long long)kWin, hi - nzh) : 0;
        f.prefetch(a, bn, tsn > 0 ? tsn : tdn, gt, 1, nzh, lim);  // the first tile's documents
      }
    } else {
      // ---------------- phase B (warps 0..3): sum the partials of this
      // block's entries, grad = E - 3 c3/S3 (G1 + G2), Phi -= lr grad, the
      // Phi^T image
      bool ok = true;
      if (tid == 0) {
        const long long t0 = clock64();
        unsigned polls = 0;
        while (ld_acquire(&ctl->bar) < nbar * G) {
          if ((++polls & 15u) != 0u) continue;
          if (*reinterpret_cast<volatile int *>(&ctl->abort) || clock64() - t0 > kWaitCycles) {
            atomicExch(&ctl->abort, 1);
            ok = false;
            break;
          }
        }
      }
      float E_own = 0.f, phi_own = 0.f;
      // the other threads of the group learn the barrier's outcome here
      if (bar_or_n(2, 128, tid == 0 && !ok)) {
        if (tid == 0) s_stop = 1;
      } else {
        const unsigned long long S3g = *reinterpret_cast<volatile unsigned long long *>(&ctl->S3[slot]);
        const int err = *reinterpret_cast<volatile int *>(&st->err);
        const double scale = S3g ? a.c3 / (double)S3g : 0.0;
        if (tid < e1 - e0) {  // this thread's entry: loads in flight during the copy
          const int e = e0 + tid;
          E_own = __ldcg(a.E + (e / K) * Kp + e % K);
          phi_own = __ldcg(a.Phi + e);
        }
        if (e1 > e0 && nwork > 0) {  // this slice of every partial, in 16-byte cp.async pieces
          const int n16 = nwork * per / 4;
          const float4 *src = reinterpret_cast<const float4 *>(a.Gpart + (long long)blk * G * per);
          float4 *dst = reinterpret_cast<float4 *>(f.sm + kOffQ);  // the Q and Q*Q buffers: 64 KB
          for (int e = tid; e < n16; e += 128) cp_async16(dst + e, src + e);
          cp_async_commit();
          cp_async_wait_all();
        }
        if (bar_or_n(2, 128, f.failed())) {
          if (tid == 0) {
            atomicExch(&ctl->abort, 1);
            s_stop = 1;
          }
        } else {
          if (tid < e1 - e0) {
            const float *sG = reinterpret_cast<const float *>(f.sm + kOffQ);
            float g4[4] = {0.f, 0.f, 0.f, 0.f};
            int c = 0;
            for (; c + 3 < nwork; c += 4) {
#pragma unroll
              for (int u = 0; u < 4; ++u) g4[u] += sG[(c + u) * per + tid];
            }
            for (; c < nwork; ++c) g4[0] += sG[c * per + tid];
            const float g = (g4[0] + g4[1]) + (g4[2] + g4[3]);
            const int e = e0 + tid, i = e / K, n = e % K;
            const float grad = S3g ? E_own - (float)(3.0 * scale * (double)g) : 0.f;
            float phi = phi_own;
            if (!err && S3g) {
              phi -= a.lr * grad;
              a.Phi[e] = phi;
            }
            a.PhiImg[phi_img_index(n, i, Kp)] = __float2bfloat16_rn(phi);
          }
          if (blk == 0 && tid == 0) {
            last_S3 = S3g;
            last_loss = 0.0;
            if (S3g) {
              const double lp = *reinterpret_cast<volatile double *>(&ctl->loss_phi[slot]);
              const double ld = *reinterpret_cast<volatile double *>(&ctl->loss_data[slot]);
              last_loss = lp - scale * ld;
            }
            if (p.losses) p.losses[s] = last_loss;
            ctl->S3[slot ^ 1] = 0;
            ctl->loss_data[slot ^ 1] = 0.0;
            ctl->loss_phi[slot ^ 1] = 0.0;
          }
          // the end-of-step arrival: only this group wrote what the other
          // blocks need (Phi, its image, the step's sums), so it arrives
          // without waiting for the request of warps 4..7
          if (s + 1 < p.s1) {
            bar_sync_n(2, 128);  // orders the group's writes before the release
            if (tid == 0) asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&ctl->bar) : "memory");
          }
        }
      }
    }
    __syncthreads();  // the two groups join
    if (s_stop) break;
    prefetched = pf_next;
    if (s + 1 < p.s1) {  // waited for in the next step (the arrival is above)
      ++nbar;
      bar_pending = true;
    } else if (p.record && blk == 0 && tid == 0) {
      st->step += p.s1 - p.s0;
      st->last_S3 = last_S3;
      st->loss = last_loss;
    }
  }
  if (tid == 0 && (f.failed() || *reinterpret_cast<volatile int *>(&ctl->abort))) atomicOr(&st->err, kErrTimeout);
  cp_async_wait_all();  // a prefetch left in flight by an early exit
  f.finish();
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

int pass_grid() {
  int dev = 0, sms = 0, coop = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) return 0;
  if (cudaFuncSetAttribute(k_pass, cudaFuncAttributeMaxDynamicSharedMemorySize, kFusedSmem) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pass, kFusedThreads, kFusedSmem) != cudaSuccess)
    return 0;
  return (per_sm >= 1 && sms >= kMinPassGrid) ? sms : 0;
}

cudaError_t launch_barrier_selftest(PassCtl *ctl, cudaStream_t s, int grid) {
  void *args[] = {&ctl};
  return cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(k_barrier_selftest), dim3(grid), dim3(32), args,
                                     0, s);
}

cudaError_t launch_pass(const StepArgs &a, const PassArgs &p, cudaStream_t s, int grid) {
  // phase B copies its slice of every data block's partial into the Q and
  // Q*Q buffers (64 KB)
  const int per = ((a.D * a.K + grid - 1) / grid + 3) & ~3;
  const int most = std::max(pass_data_blocks(p, grid, 0), pass_data_blocks(p, grid, p.e_small_docs + 1));
  if ((long long)most * per * 4 > 65536) return cudaErrorInvalidValue;
  StepArgs aa = a;
  PassArgs pp = p;
  void *args[] = {&aa, &pp};
  return cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(k_pass), dim3(grid), dim3(kFusedThreads), args,
                                     kFusedSmem, s);
}

}  // namespace tlda
