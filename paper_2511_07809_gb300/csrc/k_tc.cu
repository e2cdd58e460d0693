// BF16 tensor-core form of the CP-step contractions on sm_103a: tcgen05 MMAs
// issued by one thread, operands staged in shared memory (TMA for the large
// operands, 128-byte swizzle, K-major), FP32 accumulators in TMEM read back
// with tcgen05.ld.
//
//   k_qy_tc  [Q; Y] = [U; X] Phi   (eq. vec_deriv: Y = X Phi; the same-token
//            term needs Q = U Phi).  M = 128 rows of [U; X] per CTA, N = Kp,
//            K = Dp in 64-feature chunks.  A by TMA from the BF16 copy UX16;
//            B from the swizzled BF16 image of Phi^T.
//   k_g_tc   G1 + G2 = [X; U_t]^T [Z; Zc] as a split reduction over the
//            reduction-major copies AT16 (Dp x ldT) and BT16 (Kp x ldT):
//            each CTA streams 64-column chunks through a TMA ring and
//            accumulates a 128-feature x Kp tile in TMEM, then writes its
//            rows of the partial.  D and K up to 512.
//   k_zh_tc  Zc rows of the touched words, written transposed (BF16) next to
//            the touched words' U^T columns.
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
    tc_fence_after();
    const int row = r0 + warp * 32 + lane;
    float *out = nullptr;
    if (row < a.V) out = a.Q32 + (long long)row * a.Kp;
    else if (row < rows) out = a.Y32 + (long long)(row - a.V) * a.Kp;
#pragma unroll
    for (int c0 = 0; c0 < KP; c0 += 16) {
      float v[16];
      tmem_ld16(tmem + (static_cast<uint32_t>(warp * 32) << 16) + c0, v);
      if (out) {
#pragma unroll
        for (int q = 0; q < 16; q += 4)
          *reinterpret_cast<float4 *>(out + c0 + q) = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
      }
    }
  } else if (lane == 0) {
    atomicOr(&a.st->err, kErrTimeout);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, tmem_cols(KP));
}

// ------------------------------------------------------------------ G1 + G2
// Block (s, mt): split s of the reduction chunks, feature rows mt*128 ..
template <int KP>
__global__ void __launch_bounds__(128) k_g_tc(StepArgs a, const __grid_constant__ CUtensorMap tmA,
                                              const __grid_constant__ CUtensorMap tmB) {
  constexpr int NST = tc_stages(KP), NH = KP > 256 ? 2 : 1, NN = KP / NH;
  constexpr int A_BYTES = 128 * 128, B_BYTES = KP * 128, STAGE = A_BYTES + B_BYTES;
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
      const int col = c < cB ? c * 64 : a.Bmax + (c - cB) * 64;
      unsigned char *sa = smem + st * STAGE, *sb = sa + A_BYTES;
      mbar_arrive_expect_tx(&full[st], STAGE);
      tma_load_2d(sa, &tmA, &full[st], col, m0);
#pragma unroll
      for (int h = 0; h < NH; ++h) tma_load_2d(sb + h * NN * 128, &tmB, &full[st], col, h * NN);
    }
  } else if (tid == 32) {  // MMA issuer
    for (int i = 0; i < n; ++i) {
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
// One block per 64 compact slots t0 .. t0+63 (touched words m = widx[t]).  It
// walks the Kp + Dp output rows in tiles of 64: rows k < Kp of BT16 take
// Zc_t[k] = q_mk (2 c_m q_mk - 2 H_mk) (H_mk is cleared), rows i of AT16 take
// U_m[i].  Each tile is staged transposed in shared memory and written as 64
// rows of 128 bytes (whole lines) into columns Bmax + t0 .. t0+63, so a block
// has the pages of 64 rows in flight at a time rather than those of all
// Kp + Dp rows.  Slots in [n_touched, round_up(n_touched, 64)) write zero
// columns (chunk padding); the slots' c_m are cleared at the end.
constexpr int kZhSlots = 64;
constexpr int kZhPitch = 66;  // staged row: 64 slots + 2 (33 words: conflict-free reads)

__global__ void __launch_bounds__(512) k_zh_tc(StepArgs a) {
  __shared__ __align__(16) __nv_bfloat16 zt[64 * kZhPitch];  // [row of the tile][slot]
  __shared__ int ms[kZhSlots];
  __shared__ float cs[kZhSlots];
  __shared__ double lsum[16];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int t0 = blockIdx.x * kZhSlots, nt = a.st->n_touched;
  if (t0 >= round_up(nt, 64)) return;  // uniform over the block
  if (tid < kZhSlots) {
    const int t = t0 + tid;
    const int m = t < nt ? a.widx[t] : -1;
    ms[tid] = m;
    cs[tid] = m >= 0 ? (float)a.cnt[m] : 0.f;
  }
  __syncthreads();
  double ls = 0.0;
  const long long colT = (long long)a.Bmax + t0;
  for (int r0 = 0; r0 < a.Kp + a.Dp; r0 += 64) {  // Kp and Dp are multiples of 64
    const bool isB = r0 < a.Kp;
    if (isB) {
      for (int e = tid; e < kZhSlots * 16; e += 512) {  // slot, four columns
        const int sl = e >> 4, c4 = (e & 15) * 4, m = ms[sl];
        float z[4] = {0.f, 0.f, 0.f, 0.f};
        if (m >= 0) {
          float4 *hp = reinterpret_cast<float4 *>(a.H32 + (long long)m * a.Kp + r0 + c4);
          const float4 q = *reinterpret_cast<const float4 *>(a.Q32 + (long long)m * a.Kp + r0 + c4);
          const float4 h = *hp;
          const float c = cs[sl];
          z[0] = q.x * (2.f * c * q.x - 2.f * h.x);
          z[1] = q.y * (2.f * c * q.y - 2.f * h.y);
          z[2] = q.z * (2.f * c * q.z - 2.f * h.z);
          z[3] = q.w * (2.f * c * q.w - 2.f * h.w);
          *hp = make_float4(0.f, 0.f, 0.f, 0.f);
          if (a.want_loss)
            ls += 2.0 * (double)c * (double)(q.x * q.x * q.x + q.y * q.y * q.y + q.z * q.z * q.z + q.w * q.w * q.w);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) zt[(c4 + k) * kZhPitch + sl] = __float2bfloat16_rn(z[k]);
      }
    } else {
      const int i0 = r0 - a.Kp;
      for (int e = tid; e < kZhSlots * 8; e += 512) {  // slot, eight columns
        const int sl = e >> 3, c8 = (e & 7) * 8, m = ms[sl];
        uint4 u = make_uint4(0u, 0u, 0u, 0u);
        if (m >= 0) u = *reinterpret_cast<const uint4 *>(a.U16 + (long long)m * a.Dp + i0 + c8);
        const __nv_bfloat16 *uv = reinterpret_cast<const __nv_bfloat16 *>(&u);
#pragma unroll
        for (int k = 0; k < 8; ++k) zt[(c8 + k) * kZhPitch + sl] = uv[k];
      }
    }
    __syncthreads();
    {
      const int row = tid >> 3, j = tid & 7;  // 64 rows x 8 pieces of 16 bytes
      const uint32_t *src = reinterpret_cast<const uint32_t *>(zt + row * kZhPitch + 8 * j);
      const uint4 v = make_uint4(src[0], src[1], src[2], src[3]);
      __nv_bfloat16 *dst = isB ? a.BT16 + (long long)(r0 + row) * a.ldT : a.AT16 + (long long)(r0 - a.Kp + row) * a.ldT;
      *reinterpret_cast<uint4 *>(dst + colT + 8 * j) = v;
    }
    __syncthreads();
  }
  if (a.want_loss) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ls += __shfl_xor_sync(0xffffffffu, ls, o);
    if (lane == 0) lsum[warp] = ls;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < 16; ++w) t += lsum[w];
      if (t != 0.0) atomicAdd(&a.st->loss_data, t);
    }
  }
  if (tid < kZhSlots && ms[tid] >= 0) a.cnt[ms[tid]] = 0;
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
// 128-byte swizzle (box_outer = 1 for tile::gather4 row gathers).
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
  CUtensorMap ug;  // U16: V x Dp, box 1 row x 64 (row gathers)
  CUtensorMap ux;  // UX16: (V + Bmax) x Dp, box 128 rows x 64
  CUtensorMap at;  // AT16: Dp x ldT, box 128 rows x 64 (rows >= Dp read as zero)
  CUtensorMap bt;  // BT16: Kp x ldT, box Kp rows x 64
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
  k_g_tc<KP><<<dim3(a.nsplit, (a.Dp + 127) / 128), 128, tc_smem<KP>(), s>>>(a, m.at, m.bt);
}

}  // namespace

bool tc_supported(int Dp, int Kp) { return Dp <= 512 && Kp <= 512; }

void *tc_make_maps(const __nv_bfloat16 *UX16, const __nv_bfloat16 *AT16, const __nv_bfloat16 *BT16, int V,
                   int Bmax, int Dp, int Kp, int ldT) {
  TcMaps *m = new TcMaps();
  bool ok = make_map(&m->ug, UX16, Dp, (uint64_t)V, (uint64_t)Dp * 2, 1) &&
            make_map(&m->ux, UX16, Dp, (uint64_t)V + Bmax, (uint64_t)Dp * 2, 128) &&
            make_map(&m->at, AT16, ldT, Dp, (uint64_t)ldT * 2, 128) &&
            make_map(&m->bt, BT16, ldT, Kp, (uint64_t)ldT * 2, Kp > 256 ? Kp / 2 : Kp);
  if (!ok) {
    delete m;
    return nullptr;
  }
  return m;
}

void tc_free_maps(void *p) { delete static_cast<TcMaps *>(p); }

const void *tc_gather_map(const void *maps) { return &static_cast<const TcMaps *>(maps)->ug; }

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
  k_zh_tc<<<round_up(a.V, 64) / kZhSlots, 512, 0, s>>>(a);
}

}  // namespace tlda
