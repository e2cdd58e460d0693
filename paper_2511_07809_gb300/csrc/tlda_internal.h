// Internal declarations of libtlda: device-side state, batch descriptors,
// the context workspace and the kernel launchers shared by the .cu files.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "tlda.h"

#include <nvtx3/nvToolsExt.h>

namespace tlda {

constexpr int kMaxDim = 512;     // D and K are padded to multiples of 64, at most 512
constexpr int kErrCsr = 1;       // sticky device error bits
constexpr int kErrTimeout = 2;
constexpr int kDocsPerBlock = 16; // whitening: one warp per document

__host__ __device__ inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

// One batch of documents as the kernels see it.  Nonzero j of the batch (an
// absolute offset read from indptr) lives at indices[j - nz_base].
struct BatchDesc {
  const int32_t *indptr;
  const int32_t *indices;
  const int32_t *counts;
  long long nz_base;
  int32_t n_docs;
  int32_t tile_cap;              // documents per tile of this batch in the pass kernel (0: 32)
};

// Bands of batch sizes with a tile size of their own: band b holds the
// batches of (512 b, 512 (b + 1)] documents, the last one everything above.
constexpr int kCapBands = 16;
inline int cap_band(int n_docs) { return n_docs <= 0 ? 0 : (n_docs - 1) / 512 < kCapBands ? (n_docs - 1) / 512 : kCapBands - 1; }

// Device-resident per-context state of the CP step.  Every step kernel reads
// the current batch from `cur`, so one step sequence (or a captured graph of
// it) can be replayed over a whole pass: the last block of the reduction
// kernel advances `cur` to descs[pass_pos] and clears the per-step sums.
struct DevState {
  BatchDesc cur;
  const BatchDesc *descs;        // pass descriptors (device) or null
  int32_t n_descs;
  int32_t pass_pos;              // next descriptor of the pass
  int32_t step;                  // steps completed on this context
  int32_t err;                   // sticky error bits (kErr*)
  int32_t n_touched;             // distinct words of the current batch
  unsigned long long S3;         // sum_d L(L-1)(L-2) of the current batch
  unsigned long long last_S3;    // S3 of the last completed step
  double loss_data;              // sum_d sum_i (y^3 - 3 y r) + 2 sum_m c_m sum_i q^3
  double loss_phi;               // (1+theta)/2 sum G^3 - sum_i (3 a_i |phi_i|^2 - 2 a_i^3)
  double loss;                   // loss of the last completed step
};

// Control block of one persistent-pass launch (zeroed before the launch).
// Per-step sums live in slot (step & 1): a slot is cleared during the
// update phase of the step before its next use.
struct PassCtl {
  unsigned int bar;              // grid-barrier arrivals
  int abort;                     // set by a block whose bounded wait expired
  unsigned long long S3[2];
  double loss_data[2];
  double loss_phi[2];
};

// Steps [s0, s1) of a pass of the persistent kernel.
struct PassArgs {
  const BatchDesc *descs;        // all batches of the pass (device)
  int s0, s1;
  int tile_cap;                  // most documents per tile (0: each batch's own)
  double *losses;                // per-step loss (device, indexed by step) or null
  PassCtl *ctl;
  int record;                    // 1: advance the context's step state (0 for tuning runs)
  int e_blocks;                  // blocks that take only the Phi-only columns (no data tiles),
  int e_blocks_small;            //   e_blocks_small of them for a batch of at most
  int e_small_docs;              //   e_small_docs documents (pass_data_blocks)
  const int *splits;             // per step, split_stride entries (pass_split_stride): the data
  int split_stride;              //   blocks' document ranges, equal in nonzeros; the offset of
                                 //   each range's first nonzero; the first tile of each range
                                 //   that takes two; the batch's nonzeros [lo, hi) relative to
                                 //   nz_base (launch_pass_prep)
};

// Row of one step in PassArgs::splits for a pass of `grid` blocks: entries
// 0..grid the split documents, grid+1..2 grid+1 indptr at those documents
// (absolute offsets), 2 grid+2..3 grid+1 the documents of each range's first
// tile (0: tiles of equal size), then lo and hi.
inline int pass_split_stride(int grid) { return 3 * grid + 4; }
constexpr int kPassTileDocs = 32;  // most documents in one tile of the pass kernel

// Element (topic n, feature k) of the B operand Phi^T in the shared-memory
// layout of the tensor-core kernels: (Dp/64) sub-tiles of [Kp rows x 64]
// BF16, 16-byte chunk c of row n stored at chunk c ^ (n mod 8).
__host__ __device__ inline long long phi_img_index(int n, int k, int Kp) {
  const int sub = k >> 6, kc = k & 63;
  return (long long)sub * Kp * 64 + n * 64 + ((((kc >> 3) ^ (n & 7)) & 7) << 3) + (kc & 7);
}

// Kernel-side view of the workspace for one CP step.
struct StepArgs {
  int V, D, K, Dp, Kp, Bmax;
  int nsplit;                    // partial sums of the data-term reduction
  float theta, lr;
  double c3;
  int same_token, want_loss, mode;   // mode 0: update Phi; 1: data term only
  DevState *st;
  // whitening (U = W - 1 m1^T, padded to Dp columns)
  const float *U32;              // V x Dp
  const float *m1;               // Dp
  // FP32 work
  float *X32;                    // Bmax x Dp
  float *Q32;                    // V x Kp   (rows of the batch's words only)
  float *Y32;                    // Bmax x Kp
  float *Z32;                    // Bmax x Kp: Y*Y - R
  float *Zc32;                   // V x Kp: compact rows Q*(2cQ - 2H) of the touched words
  float *H32;                    // V x Kp, zero between steps
  int *cnt;                      // V, zero between steps (c_m = sum_d f_dm)
  int *widx;                     // V: touched words of the batch, compact
  float *Gpart;                  // nsplit x Dp x Kp
  float *Gram;                   // Kp x Kp: Phi^T Phi
  float *avec;                   // Kp: m1^T Phi
  float *E;                      // Dp x Kp: 3(1+theta) P - 3 G3
  float *G3;                     // Dp x Kp
  // BF16 tensor-core work
  const __nv_bfloat16 *U16;      // V x Dp
  __nv_bfloat16 *X16;            // Bmax x Dp
  __nv_bfloat16 *ZU16;           // round_up(V, 64) x (Kp + Dp): [Zc | U] rows of the touched words
  __nv_bfloat16 *Z16;            // Bmax x Kp: Z rows of the documents (BF16)
  int precision;
  const void *tc_maps;           // host pointer to the TMA tensor maps (BF16 form)
  __nv_bfloat16 *PhiImg;         // shared-memory image of Phi^T (BF16 form, Kp x Dp, swizzled)
  // caller buffers
  float *Phi;                    // D x K (user layout), updated in place
  float *grad_out;               // D x K or null
  float *gdata_out;              // D x K or null (mode 1)
};

#ifdef __CUDACC__
// Lines first, first + stride, ... (128 bytes each, line 0 at p) of the
// `bytes` bytes at p into L2, spread over threads t = 0 .. nt - 1.  Every
// address lies inside [p, p + bytes).
__device__ inline void l2_prefetch_lines(const void *p, long long bytes, int first, int stride, int t, int nt) {
  const char *c = static_cast<const char *>(p);
  for (long long off = (long long)(first + (long long)t * stride) * 128; off < bytes;
       off += (long long)stride * 128 * nt)
    asm volatile("prefetch.global.L2 [%0];" ::"l"(c + off));
}

// Groups g = g0, g0 + gs, ... of the BF16 Phi^T image: group g holds the 8
// features kc*8 .. kc*8+7 of topic n (g = kc*Kp + n) as one 16-byte chunk
// (zero outside D x K).
__device__ inline void phi_img_groups(const StepArgs &a, int g0, int gs) {
  const int groups = a.Kp * (a.Dp / 8);
  for (int g = g0; g < groups; g += gs) {
    const int n = g % a.Kp, kc = g / a.Kp;
    __align__(16) __nv_bfloat16 v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int k = kc * 8 + q;
      v[q] = __float2bfloat16_rn((k < a.D && n < a.K) ? a.Phi[(long long)k * a.K + n] : 0.f);
    }
    *reinterpret_cast<uint4 *>(a.PhiImg + phi_img_index(n, kc * 8, a.Kp)) = *reinterpret_cast<const uint4 *>(v);
  }
}
#endif

// An NVTX range around one C-ABI call (named by the function; free when no
// profiler is attached).
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};
#define TLDA_RANGE() ::tlda::NvtxRange tlda_nvtx_range_(__func__)

}  // namespace tlda

struct tlda_ctx {
  int V = 0, D = 0, K = 0, Dp = 0, Kp = 0, Bmax = 0;
  tlda_params p{};
  cudaStream_t stream = nullptr, side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  int device = 0, num_sms = 0;
  std::string err;
  bool whitened = false;
  // whitening state
  float *W32 = nullptr;          // V x D (as set/fitted)
  float *m1 = nullptr;           // Dp (zero padded)
  float *U32 = nullptr;          // V x Dp
  __nv_bfloat16 *U16 = nullptr;  // V x Dp
  std::vector<double> eig;       // D eigenvalues (host copy)
  // step workspace
  float *X32 = nullptr, *Q32 = nullptr, *Y32 = nullptr, *Z32 = nullptr, *Zc32 = nullptr;
  float *H32 = nullptr;
  int *cnt = nullptr, *widx = nullptr;
  float *Gpart = nullptr, *Gram = nullptr, *avec = nullptr, *E = nullptr, *G3 = nullptr;
  int nsplit = 0, nsplit_tc = 0;
  bool fused = false;            // BF16 form through the fused kernel
  int fused_grid = 0;            // its persistent CTAs (SMs minus those left to the side stream)
  __nv_bfloat16 *UX16 = nullptr, *X16 = nullptr, *ZU16 = nullptr, *Z16 = nullptr;
  void *tc_maps = nullptr;
  __nv_bfloat16 *PhiImg = nullptr;
  tlda::DevState *st = nullptr;
  tlda::DevState *st_host = nullptr;   // pinned mirror for reads
  tlda::BatchDesc *descs = nullptr;    // pass descriptors (device)
  int descs_cap = 0;
  int *splits = nullptr;               // per pass step, the data blocks' document ranges (device)
  tlda::BatchDesc *descs_pin = nullptr;  // pinned staging of the persistent pass's descriptors
  int descs_pin_cap = 0;
  bool descs_pin_busy = false;          // its last upload may still be in flight
  // fit state
  double *P64 = nullptr;               // V x V pair counts (allocated on first ACCUMULATE)
  unsigned long long *Ccnt = nullptr;  // V word totals
  unsigned long long *TS = nullptr;    // T, S2, S3 of the fit
  int *fit_err = nullptr;
  bool fit_open = false, fitted = false;
  // fully online mode: exact counts and the sketch Z = P Omega of the pair counts
  int on_r = 0;
  bool on_active = false;
  double *on_Om = nullptr, *on_Z = nullptr;           // V x r
  unsigned long long *on_C = nullptr, *on_TS = nullptr;  // V; T, S2, S3
  int *on_err = nullptr;
  float *on_Wold = nullptr;            // V x D: the whitening before the last rebuild
  double *on_ws = nullptr;             // workspace of a re-whitening (V x r x 3 + r x r x 12 + ...)
  void *on_sk = nullptr;               // workspace of the sketch (per-piece S and word slots)
  float *on_Om32 = nullptr;            // V x r: FP32 copy of Omega for the sketch's products
  int *on_status = nullptr;            // its device status words
  int jacobi_sweeps = 0;               // sweeps of the last symmetric eigensolve
  void *coop_ctl = nullptr;            // control block of the grid-wide FP64 kernels (k_fit.cu)
  // pass staging (host input)
  int32_t *stage[2] = {nullptr, nullptr};
  long long stage_cap = 0;
  // pass stream and the cached graph of one step (keyed by the baked arguments)
  cudaStream_t pstream = nullptr;
  cudaEvent_t ev_pass0 = nullptr, ev_pass1 = nullptr;
  cudaGraphExec_t step_exec = nullptr;
  // persistent pass kernel (BF16 fused form)
  int pass_grid = 0;                   // its blocks (0: not available)
  int tile_cap = 32;                   // most documents per tile (tuned on the first pass)
  int cap_band[tlda::kCapBands] = {32, 32, 32, 32, 32, 32, 32, 32, 32, 32, 32, 32, 32, 32, 32, 32};  // per size band
  bool tuned = false;
  tlda::PassCtl *ctl = nullptr;
  tlda::DevState *st_tune = nullptr;   // device state of tuning runs (kept apart from st)
  double *dlosses = nullptr;           // per-step losses of a pass (device)
  int dlosses_cap = 0;
  float *phi_scratch = nullptr;        // D x K: tuning runs on a copy of Phi
  cudaStream_t cstream = nullptr;      // host-input copies of the pass
  cudaEvent_t ev_seg[4] = {nullptr, nullptr, nullptr, nullptr};
  float g_lr = 0.f;
  const float *g_phi = nullptr;
  int g_loss = -1;
  // event profiler: kernels whose bit is set in prof_mask are bracketed by events
  uint32_t prof_mask = 0;
  struct ProfRec { int id; cudaEvent_t a, b; };
  std::vector<ProfRec> prof_pending;
  std::vector<cudaEvent_t> prof_pool;
  long long prof_launches[16] = {};
  double prof_ms[16] = {};
};

namespace tlda {
// Kernels of one CP step, in launch order (ids used by the event profiler).
enum KernelId {
  kWhiten = 0, kQY, kRZ, kZH, kG, kReduceUpdate, kPhiGram, kPhiTerms, kFused, kPass, kNumKernels
};
extern const char *const kKernelNames[kNumKernels];

// k_step.cu
void launch_set_desc(DevState *st, const BatchDesc &b, cudaStream_t s);
void launch_begin_pass(DevState *st, const BatchDesc *descs, int n, cudaStream_t s);
void launch_whiten(const StepArgs &a, cudaStream_t s, float *X_out, bool stats);
void launch_qy_f32(const StepArgs &a, cudaStream_t s);
void launch_rz(const StepArgs &a, cudaStream_t s);
void launch_zh_f32(const StepArgs &a, cudaStream_t s);
void launch_g_f32(const StepArgs &a, cudaStream_t s);
void launch_phi_gram(const StepArgs &a, cudaStream_t s);
void launch_phi_terms(const StepArgs &a, cudaStream_t s);
void launch_reduce_update(const StepArgs &a, cudaStream_t s);
void launch_make_u(const float *W, const float *m1, int V, int D, int Dp, float *U32,
                   __nv_bfloat16 *U16, cudaStream_t s);
void launch_phi_img(const StepArgs &a, cudaStream_t s);
// k_fused.cu (BF16 fused tensor-core data term)
bool fused_supported(int Dp, int Kp);
void launch_fused(const StepArgs &a, cudaStream_t s, int grid);
int pass_grid();                                  // co-resident blocks of the pass kernel (0: none)
cudaError_t launch_pass(const StepArgs &a, const PassArgs &p, cudaStream_t s, int grid);
// Document ranges of the data blocks of steps [s0, s1): for step s, entries
// s * p.split_stride + i, i = 0..n (n = pass_data_blocks of the step's batch),
// with range i = [split_i, split_{i+1}) equal in nonzeros (lower bounds of
// i nnz / n), non-decreasing; entry grid + 1 + i is indptr[split_i], the
// offset of range i's first nonzero; entry 2 grid + 2 + i, for a range that
// takes two tiles, the documents of its first tile (the boundary with the
// fewest 128-nonzero chunks in the two), else 0.  max_docs: the largest batch
// among the steps (sizes the shared-memory offsets).
// The descriptors of a short pass, handed to the prologue kernel in its
// launch parameters (no separate upload); the kernel writes them to
// PassArgs::descs for the pass kernel.  n = 0: they are there already.
constexpr int kInlineDescs = 64;
struct InlineDescs {
  int n;
  BatchDesc d[kInlineDescs];
};
cudaError_t launch_pass_prep(const StepArgs &a, bool image, const PassArgs &p, int grid, int max_docs,
                             const InlineDescs &inl,
                               cudaStream_t s);

constexpr int kPassPhiCols = 8;  // Phi-only columns per job of the pass kernel (a multiple of 4, <= 16)

// Data blocks of a pass step over a batch of n_docs documents (the other
// blocks of the grid take only the Phi-only columns).
__host__ __device__ inline int pass_data_blocks(const PassArgs &p, int grid, int n_docs) {
  const int eb = n_docs <= p.e_small_docs ? p.e_blocks_small : p.e_blocks;
  return grid - (eb < 0 ? 0 : eb > grid / 2 ? grid / 2 : eb);
}
cudaError_t launch_barrier_selftest(PassCtl *ctl, cudaStream_t s, int grid);
// k_tc.cu (BF16 tensor-core form)
bool tc_supported(int Dp, int Kp);
void *tc_make_maps(const __nv_bfloat16 *UX16, const __nv_bfloat16 *ZU16, const __nv_bfloat16 *Z16, int V, int Bmax,
                   int Dp, int Kp);
void tc_free_maps(void *maps);
void launch_qy_tc(const StepArgs &a, cudaStream_t s);
void launch_zh_tc(const StepArgs &a, cudaStream_t s);
void launch_g_tc(const StepArgs &a, cudaStream_t s);
}  // namespace tlda
