// BF16 tensor-core form of the CP-step contractions on sm_103a: tcgen05 MMAs
// issued by one thread, operands staged in shared memory (TMA for the large
// operands, 128-byte swizzle, K-major), FP32 accumulators in TMEM read back
// with tcgen05.ld.
//
//   k_qy_tc  [Q; Y] = [U; X] Phi   (eq. vec_deriv: Y = X Phi; the same-token
//            term needs Q = U Phi).  M = 128 rows of [U; X] per CTA, N = Kp,
//            K = Dp in 64-feature chunks.  A by TMA from the BF16 copy UX16;
//            B from the swizzled BF16 image of Phi^T.
//   k_g_tc   G1 + G2 = [X; U_t]^T [Z; Zc] as a split reduction over 64-row
//            chunks (the batch's documents, then its touched words): both
//            operands are read MN-major straight from their row-major BF16
//            copies (X16, Z16 and the [Zc | U_t] rows of ZU16) through a TMA
//            ring; each CTA accumulates a 128-feature x Kp tile in TMEM, then
//            writes its rows of the partial.  D and K up to 512.
//   k_zc_tc  Zc rows of the touched words with their U rows (BF16).
// Every wait on an mbarrier is bounded (about one second of clock cycles);
// on expiry the kernel sets the context's timeout bit and leaves.
#include <cstdio>

#include "tc_ptx.cuh"

namespace tlda {
namespace {
using namespace tc;

// Operands stream in 64-feature chunks through a ring of NST stages (A by
// TMA, B as one bulk copy or TMA boxes).  N = KP is one MMA up to 256 columns,
// two halves of KP/2 above that (each <= 256, a multiple of 16), accumulated
// side by side in TMEM.
__host__ __device__ constexpr int tc_stages(int kp) { return kp <= 256 ? 4 : kp <= 448 ? 3 : 2; }
__host__ __device__ constexpr int tc_stage_bytes(int kp) { return 128 * 128 + kp * 128; }

// ------------------------------------------------------------------ Q and Y
template <int KP>
__global__ void __launch_bounds__(128) k_qy_tc(StepArgs a, const __grid_constant__ CUtensorMap tmA) {
  constexpr int NST = tc_stages(KP), NH = KP > 256 ? 2 : 1, NN = KP / NH;
  constexpr int A_BYTES = 128 * 128, B_BYTES = KP * 128, STAGE = A_BYTES + B_BYTES;
  extern __shared__ unsigned char smem_raw[];
  unsigned char *smem = align1024(smem_raw);
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + NST * STAGE);
  uint64_t *empty = full + NST;
  uint64_t *done = empty + NST;
  uint32_t *tslot = reinterpret_cast<uint32_t *>(done + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nd = a.st->cur.n_docs;
  const int rows = a.V + nd;
  const int r0 = blockIdx.x * 128;
  if (r0 >= rows) return;
  const int KA = a.Dp / 64;
  if (tid == 0) {
    for (int i = 0; i < NST; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    mbar_init(done, 1);
    fence_mbar_init();
  }
  if (warp == 0) tmem_alloc(tslot, tmem_cols(KP));
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  __shared__ int failed;
  if (tid == 0) failed = 0;
  __syncthreads();
  if (tid == 0) {  // producer: A rows by TMA, B = the Phi^T image chunk (K-major, swizzled) by bulk copy
    fence_proxy_async();
    for (int i = 0; i < KA; ++i) {
      const int st = i % NST;
      if (i >= NST && !mbar_wait(&empty[st], ((i / NST) - 1) & 1)) {
        failed = 1;
        break;
      }
      unsigned char *sa = smem + st * STAGE, *sb = sa + A_BYTES;
      mbar_arrive_expect_tx(&full[st], STAGE);
      tma_load_2d(sa, &tmA, &full[st], i * 64, r0);
      bulk_load(sb, a.PhiImg + (long long)i * KP * 64, B_BYTES, &full[st]);
    }
  } else if (tid == 32) {  // MMA issuer
    for (int i = 0; i < KA; ++i) {
      const int st = i % NST;
      if (!mbar_wait(&full[st], (i / NST) & 1)) {
        failed = 1;
        break;
      }
      tc_fence_after();
      const uint32_t aBase = smem_u32(smem + st * STAGE), bBase = aBase + A_BYTES;
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)
#pragma unroll
        for (int h = 0; h < NH; ++h)
          mma_bf16(tmem + h * NN, sdesc_sw128(aBase + kk * 32), sdesc_sw128(bBase + h * NN * 128 + kk * 32),
                   idesc_bf16(128, NN), (i > 0 || kk > 0) ? 1u : 0u);
      mma_commit(&empty[st]);
    }
    mma_commit(done);
  }
  __syncthreads();
  // warp-uniform decision: tcgen05.ld below is .sync.aligned
  const bool ok = __all_sync(0xffffffffu, !failed && mbar_wait(done, 0));
  if (ok) {
    // each warp's 32 rows x 32 columns pass through shared memory (the ring is
    // free once every MMA is done), so that a store covers four rows of 128
    // bytes rather than 32 rows of 16
    tc_fence_after();
    float *stg = reinterpret_cast<float *>(smem) + warp * (32 * 33);
    const int rbase = r0 + warp * 32;
#pragma unroll 1
    for (int c0 = 0; c0 < KP; c0 += 32) {
      float v[16], w[16];
      tmem_ld16(tmem + (static_cast<uint32_t>(warp * 32) << 16) + c0, v);
      tmem_ld16(tmem + (static_cast<uint32_t>(warp * 32) << 16) + c0 + 16, w);
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        stg[lane * 33 + j] = v[j];
        stg[lane * 33 + 16 + j] = w[j];
      }
      __syncwarp();
#pragma unroll
      for (int it = 0; it < 8; ++it) {
        const int rr = it * 4 + (lane >> 3), c4 = (lane & 7) * 4, row = rbase + rr;
        float *out = row < a.V ? a.Q32 + (long long)row * a.Kp
                               : (row < rows ? a.Y32 + (long long)(row - a.V) * a.Kp : nullptr);
        if (out)
          *reinterpret_cast<float4 *>(out + c0 + c4) =
              make_float4(stg[rr * 33 + c4], stg[rr * 33 + c4 + 1], stg[rr * 33 + c4 + 2], stg[rr * 33 + c4 + 3]);
      }
      __syncwarp();
    }
  } else if (lane == 0) {
    atomicOr(&a.st->err, kErrTimeout);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, tmem_cols(KP));
}

// ------------------------------------------------------------------ G1 + G2
// Block (s, mt): split s of the 64-row reduction chunks, feature rows
// mt*128 .. mt*128+127.  A chunk's A tile is two TMA boxes of 64 rows x 64
// features of X16 (documents) or of the U_t columns of ZU16 (touched words),
// its B tile Kp/64 boxes of 64 rows x 64 topics of Z16 or of the Zc columns of
// ZU16; every box lands as 64 rows of 128 swizzled bytes, which is the
// MN-major operand layout (64-element blocks 8 KB apart).  Rows past the
// batch's documents (up to the next multiple of 64) are zero in X16 and Z16,
// and features past Dp read as zero.  N is one MMA up to 256 topics, else
// 256 + (Kp - 256) side by side in TMEM.
template <int KP>
__global__ void __launch_bounds__(128) k_g_tc(StepArgs a, const __grid_constant__ CUtensorMap tmX,
                                              const __grid_constant__ CUtensorMap tmU,
                                              const __grid_constant__ CUtensorMap tmZ,
                                              const __grid_constant__ CUtensorMap tmC) {
  constexpr int NST = tc_stages(KP), N0 = KP > 256 ? 256 : KP, N1 = KP - N0;
  constexpr int A_BYTES = 128 * 128, B_BYTES = KP * 128, STAGE = A_BYTES + B_BYTES;
  constexpr uint32_t kMN = (1u << 15) | (1u << 16);  // A and B MN-major
  extern __shared__ unsigned char smem_raw[];
  unsigned char *smem = align1024(smem_raw);
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + NST * STAGE);
  uint64_t *empty = full + NST;
  uint64_t *done = empty + NST;
  uint32_t *tslot = reinterpret_cast<uint32_t *>(done + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nd = a.st->cur.n_docs, nt = a.same_token ? a.st->n_touched : 0;
  const int cB = (nd + 63) / 64, cT = (nt + 63) / 64, C = cB + cT;
  const int s = blockIdx.x, m0 = blockIdx.y * 128;
  const int c0 = (int)((long long)C * s / a.nsplit), c1 = (int)((long long)C * (s + 1) / a.nsplit);
  const int n = c1 - c0;
  float *gp = a.Gpart + (long long)s * a.Dp * a.Kp;
  if (n <= 0) {
    for (int e = tid; e < 128 * a.Kp; e += 128) {
      const int row = m0 + e / a.Kp;
      if (row < a.Dp) gp[(long long)row * a.Kp + e % a.Kp] = 0.f;
    }
    return;
  }
  if (tid == 0) {
    for (int i = 0; i < NST; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    mbar_init(done, 1);
    fence_mbar_init();
  }
  if (warp == 0) tmem_alloc(tslot, tmem_cols(KP));
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  __shared__ int failed;
  if (tid == 0) failed = 0;
  __syncthreads();
  if (tid == 0) {  // TMA producer
    for (int i = 0; i < n; ++i) {
      const int st = i % NST;
      if (i >= NST && !mbar_wait(&empty[st], ((i / NST) - 1) & 1)) {
        failed = 1;
        break;
      }
      const int c = c0 + i;
      unsigned char *sa = smem + st * STAGE, *sb = sa + A_BYTES;
      mbar_arrive_expect_tx(&full[st], STAGE);
      if (c < cB) {
        const int row = c * 64;
        tma_load_2d(sa, &tmX, &full[st], m0, row);
        tma_load_2d(sa + 8192, &tmX, &full[st], m0 + 64, row);
#pragma unroll
        for (int j = 0; j < KP / 64; ++j) tma_load_2d(sb + j * 8192, &tmZ, &full[st], j * 64, row);
      } else {
        const int row = (c - cB) * 64;
        tma_load_2d(sa, &tmU, &full[st], m0, row);
        tma_load_2d(sa + 8192, &tmU, &full[st], m0 + 64, row);
#pragma unroll
        for (int j = 0; j < KP / 64; ++j) tma_load_2d(sb + j * 8192, &tmC, &full[st], j * 64, row);
      }
    }
  } else if (tid == 32) {  // MMA issuer: 16 reduction rows (2 KB of each tile) per MMA
    for (int i = 0; i < n; ++i) {
      const int st = i % NST;
      if (!mbar_wait(&full[st], (i / NST) & 1)) {
        failed = 1;
        break;
      }
      tc_fence_after();
      const uint32_t aBase = smem_u32(smem + st * STAGE), bBase = aBase + A_BYTES;
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const uint64_t ad = sdesc_mn_sw128(aBase + kk * 2048, 8192);
        const uint32_t acc = (i > 0 || kk > 0) ? 1u : 0u;
        mma_bf16(tmem, ad, sdesc_mn_sw128(bBase + kk * 2048, 8192), idesc_bf16(128, N0) | kMN, acc);
        if constexpr (N1 > 0)
          mma_bf16(tmem + N0, ad, sdesc_mn_sw128(bBase + (N0 / 64) * 8192 + kk * 2048, 8192),
                   idesc_bf16(128, N1) | kMN, acc);
      }
      mma_commit(&empty[st]);
    }
    mma_commit(done);
  }
  __syncthreads();
  const bool ok = __all_sync(0xffffffffu, !failed && mbar_wait(done, 0));
  if (ok) {
    tc_fence_after();
    const int row = m0 + warp * 32 + lane;
#pragma unroll
    for (int q0 = 0; q0 < KP; q0 += 16) {
      float v[16];
      tmem_ld16(tmem + (static_cast<uint32_t>(warp * 32) << 16) + q0, v);
      if (row < a.Dp) {
#pragma unroll
        for (int q = 0; q < 16; q += 4)
          *reinterpret_cast<float4 *>(gp + (long long)row * a.Kp + q0 + q) =
              make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
      }
    }
  } else if (tid == 0) {
    atomicOr(&a.st->err, kErrTimeout);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, tmem_cols(KP));
}

// ------------------------------------------------------------------ Zc (BF16, transposed)
// k_zc_tc: one warp per compact slot t (8 per block): row t of ZU16 takes
// [Zc_t | U_m] in BF16, Zc_t = q (2 c_m q - 2 H_m) with m = widx[t].  Slots
// in [n_touched, round_up(n_touched, 64)) get zero rows (chunk padding);
// k_g_tc reads the rows directly.  k_h_clear then clears H_m and c_m for the
// next batch: a warp that loads an H row and then stores to it (an L2 miss
// followed by a write to the pending line) ran about six times slower than
// the load or the store alone.
template <int NK>
__global__ void __launch_bounds__(256) k_zc_tc(StepArgs a) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = blockIdx.x * 8 + warp, nt = a.st->n_touched;
  if (t >= round_up(nt, 64)) return;  // per warp: no block barrier follows
  const int m = t < nt ? a.widx[t] : -1;
  const float c = m >= 0 ? (float)a.cnt[m] : 0.f;
  __nv_bfloat16 *row = a.ZU16 + (long long)t * (a.Kp + a.Dp);
  float ls = 0.f;
#pragma unroll
  for (int v = 0; v < NK; ++v) {
    const int col = v * 128 + lane * 4;
    if (col < a.Kp) {
      float z[4] = {0.f, 0.f, 0.f, 0.f};
      if (m >= 0) {
        const float4 *hp = reinterpret_cast<const float4 *>(a.H32 + (long long)m * a.Kp + col);
        const float4 q = *reinterpret_cast<const float4 *>(a.Q32 + (long long)m * a.Kp + col);
        const float4 h = *hp;
        z[0] = q.x * (2.f * c * q.x - 2.f * h.x);
        z[1] = q.y * (2.f * c * q.y - 2.f * h.y);
        z[2] = q.z * (2.f * c * q.z - 2.f * h.z);
        z[3] = q.w * (2.f * c * q.w - 2.f * h.w);
        ls += q.x * q.x * q.x + q.y * q.y * q.y + q.z * q.z * q.z + q.w * q.w * q.w;
      }
      __nv_bfloat162 p[2] = {__floats2bfloat162_rn(z[0], z[1]), __floats2bfloat162_rn(z[2], z[3])};
      *reinterpret_cast<uint2 *>(row + col) = *reinterpret_cast<const uint2 *>(p);
    }
  }
  for (int i = lane * 8; i < a.Dp; i += 256) {
    uint4 u = make_uint4(0u, 0u, 0u, 0u);
    if (m >= 0) u = *reinterpret_cast<const uint4 *>(a.U16 + (long long)m * a.Dp + i);
    *reinterpret_cast<uint4 *>(row + a.Kp + i) = u;
  }
  if (a.want_loss && m >= 0) {
    for (int o = 16; o > 0; o >>= 1) ls += __shfl_xor_sync(0xffffffffu, ls, o);
    if (lane == 0) atomicAdd(&a.st->loss_data, 2.0 * (double)c * (double)ls);
  }
}

template <int NK>
__global__ void __launch_bounds__(256) k_h_clear(StepArgs a) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = blockIdx.x * 8 + warp;
  if (t >= a.st->n_touched) return;
  const int m = a.widx[t];
#pragma unroll
  for (int v = 0; v < NK; ++v) {
    const int col = v * 128 + lane * 4;
    if (col < a.Kp) *reinterpret_cast<float4 *>(a.H32 + (long long)m * a.Kp + col) = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  if (lane == 0) a.cnt[m] = 0;
}

// ------------------------------------------------------------------ host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// 2D BF16 tensor [outer x inner] (row pitch in bytes), box [box_outer x 64],
// 128-byte swizzle.
bool make_map(CUtensorMap *m, const void *base, uint64_t inner, uint64_t outer, uint64_t pitch_bytes,
              uint32_t box_outer) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {pitch_bytes};
  cuuint32_t box[2] = {64, box_outer};
  cuuint32_t estr[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

struct TcMaps {
  CUtensorMap ux;  // UX16: (V + Bmax) x Dp, box 128 rows x 64
  CUtensorMap gx;  // X16: Bmax x Dp, box 64 rows x 64 (features past Dp read as zero)
  CUtensorMap gu;  // U_t columns of ZU16: round_up(V, 64) x Dp, box 64 x 64
  CUtensorMap gz;  // Z16: Bmax x Kp, box 64 x 64
  CUtensorMap gc;  // Zc columns of ZU16: round_up(V, 64) x Kp, box 64 x 64
};

template <int KP>
int tc_smem() {
  return 1024 + tc_stages(KP) * tc_stage_bytes(KP) + 128;
}

template <int KP>
void qy_launch(const StepArgs &a, const TcMaps &m, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_qy_tc<KP>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc_smem<KP>());
    attr = true;
  }
  k_qy_tc<KP><<<(a.V + a.Bmax + 127) / 128, 128, tc_smem<KP>(), s>>>(a, m.ux);
}

template <int KP>
void g_launch(const StepArgs &a, const TcMaps &m, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_g_tc<KP>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc_smem<KP>());
    attr = true;
  }
  k_g_tc<KP><<<dim3(a.nsplit, (a.Dp + 127) / 128), 128, tc_smem<KP>(), s>>>(a, m.gx, m.gu, m.gz, m.gc);
}

}  // namespace

bool tc_supported(int Dp, int Kp) { return Dp <= 512 && Kp <= 512; }

void *tc_make_maps(const __nv_bfloat16 *UX16, const __nv_bfloat16 *ZU16, const __nv_bfloat16 *Z16, int V, int Bmax,
                   int Dp, int Kp) {
  TcMaps *m = new TcMaps();
  const uint64_t Vr = (uint64_t)(V + 63) / 64 * 64, ldzu = (uint64_t)(Kp + Dp) * 2;
  bool ok = make_map(&m->ux, UX16, Dp, (uint64_t)V + Bmax, (uint64_t)Dp * 2, 128) &&
            make_map(&m->gx, UX16 + (size_t)V * Dp, Dp, (uint64_t)Bmax, (uint64_t)Dp * 2, 64) &&
            make_map(&m->gu, ZU16 + Kp, Dp, Vr, ldzu, 64) &&
            make_map(&m->gz, Z16, Kp, (uint64_t)Bmax, (uint64_t)Kp * 2, 64) &&
            make_map(&m->gc, ZU16, Kp, Vr, ldzu, 64);
  if (!ok) {
    delete m;
    return nullptr;
  }
  return m;
}

void tc_free_maps(void *p) { delete static_cast<TcMaps *>(p); }

#define TLDA_KP_DISPATCH(F)                                       \
  switch (a.Kp) {                                                 \
    case 64: return F<64>(a, m, s);                               \
    case 128: return F<128>(a, m, s);                             \
    case 192: return F<192>(a, m, s);                             \
    case 256: return F<256>(a, m, s);                             \
    case 320: return F<320>(a, m, s);                             \
    case 384: return F<384>(a, m, s);                             \
    case 448: return F<448>(a, m, s);                             \
    default: return F<512>(a, m, s);                              \
  }

void launch_qy_tc(const StepArgs &a, cudaStream_t s) {
  const TcMaps &m = *static_cast<const TcMaps *>(a.tc_maps);
  TLDA_KP_DISPATCH(qy_launch)
}

void launch_g_tc(const StepArgs &a, cudaStream_t s) {
  const TcMaps &m = *static_cast<const TcMaps *>(a.tc_maps);
  TLDA_KP_DISPATCH(g_launch)
}
#undef TLDA_KP_DISPATCH

void launch_zh_tc(const StepArgs &a, cudaStream_t s) {
  const int nk = (a.Kp + 127) / 128;
  const unsigned grid = (unsigned)(round_up(a.V, 64) / 8);
  if (nk == 1) {
    k_zc_tc<1><<<grid, 256, 0, s>>>(a);
    k_h_clear<1><<<grid, 256, 0, s>>>(a);
  } else if (nk == 2) {
    k_zc_tc<2><<<grid, 256, 0, s>>>(a);
    k_h_clear<2><<<grid, 256, 0, s>>>(a);
  } else if (nk == 3) {
    k_zc_tc<3><<<grid, 256, 0, s>>>(a);
    k_h_clear<3><<<grid, 256, 0, s>>>(a);
  } else {
    k_zc_tc<4><<<grid, 256, 0, s>>>(a);
    k_h_clear<4><<<grid, 256, 0, s>>>(a);
  }
}

}  // namespace tlda
