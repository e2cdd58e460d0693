// C ABI of libtlda (declared in include/tlda.h): context and workspace
// management, argument checks, and the orchestration of the per-batch kernel
// chain on the context's stream.
#include <algorithm>
#include <cstdarg>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <vector>

#include "tlda_internal.h"

using namespace tlda;

namespace tlda {
const char *const kKernelNames[kNumKernels] = {"scan_whiten", "qy", "rz", "zh", "g_reduce",
                                                "reduce_update", "phi_gram", "phi_terms", "fused",
                                                "pass"};
}

namespace {

tlda_status fail(tlda_ctx *c, tlda_status s, const char *fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    c->err = buf;
  }
  return s;
}

#define CK(call)                                                                             \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? TLDA_ERR_OOM : TLDA_ERR_CUDA,       \
                  "%s: %s", #call, cudaGetErrorString(e_));                                  \
  } while (0)

#define CKL()                                                                                \
  do {                                                                                       \
    cudaError_t e_ = cudaGetLastError();                                                     \
    if (e_ != cudaSuccess)                                                                   \
      return fail(ctx, TLDA_ERR_CUDA, "kernel launch: %s", cudaGetErrorString(e_));          \
  } while (0)

template <class T>
cudaError_t dalloc(T **p, size_t n, bool zero = false) {
  if (n == 0) n = 1;
  cudaError_t e = cudaMalloc(reinterpret_cast<void **>(p), n * sizeof(T));
  if (e == cudaSuccess && zero) e = cudaMemset(*p, 0, n * sizeof(T));
  return e;
}

template <class T>
void dfree(T *&p) {
  if (p) cudaFree(p);
  p = nullptr;
}

StepArgs make_args(tlda_ctx *c) {
  StepArgs a{};
  a.V = c->V;
  a.D = c->D;
  a.K = c->K;
  a.Dp = c->Dp;
  a.Kp = c->Kp;
  a.Bmax = c->Bmax;
  a.nsplit = c->nsplit;
  a.theta = c->p.theta;
  a.lr = 0.f;
  a.c3 = (c->p.alpha0 + 1.0) * (c->p.alpha0 + 2.0) / 2.0;
  a.same_token = c->p.same_token_correction ? 1 : 0;
  a.want_loss = 0;
  a.mode = 0;
  a.st = c->st;
  a.U32 = c->U32;
  a.m1 = c->m1;
  a.X32 = c->X32;
  a.Q32 = c->Q32;
  a.Y32 = c->Y32;
  a.Z32 = c->Z32;
  a.Zc32 = c->Zc32;
  a.H32 = c->H32;
  a.cnt = c->cnt;
  a.widx = c->widx;
  a.Gpart = c->Gpart;
  a.Gram = c->Gram;
  a.avec = c->avec;
  a.E = c->E;
  a.G3 = c->G3;
  a.U16 = c->U16;
  a.X16 = c->X16;
  a.ZU16 = c->ZU16;
  a.Z16 = c->Z16;
  a.precision = c->p.precision;
  a.tc_maps = c->tc_maps;
  a.PhiImg = c->PhiImg;
  if (a.precision == TLDA_BF16) a.nsplit = c->fused ? c->fused_grid : c->nsplit_tc;
  return a;
}

tlda_status check_csr(tlda_ctx *ctx, const tlda_csr *b, bool allow_empty_ptrs = false) {
  if (!b) return fail(ctx, TLDA_ERR_INVALID, "batch is NULL");
  if (b->vocab != ctx->V) return fail(ctx, TLDA_ERR_INVALID, "batch vocab %d != context V %d", b->vocab, ctx->V);
  if (b->n_docs < 0) return fail(ctx, TLDA_ERR_INVALID, "n_docs < 0");
  if (!allow_empty_ptrs && (!b->indptr || (b->n_docs > 0 && (!b->indices || !b->counts))))
    return fail(ctx, TLDA_ERR_INVALID, "NULL CSR array");
  return TLDA_OK;
}

BatchDesc desc_of(const tlda_csr *b) {
  BatchDesc d{};
  d.indptr = b->indptr;
  d.indices = b->indices;
  d.counts = b->counts;
  d.nz_base = 0;
  d.n_docs = b->n_docs;
  return d;
}

// Event bracket around one kernel launch when its profiler bit is set.
struct Prof {
  tlda_ctx *c;
  int id;
  cudaStream_t s;
  cudaEvent_t a = nullptr, b = nullptr;
  Prof(tlda_ctx *c_, int id_, cudaStream_t s_) : c(c_), id(id_), s(s_) {
    if (!(c->prof_mask & (1u << id))) return;
    for (cudaEvent_t *e : {&a, &b}) {
      if (!c->prof_pool.empty()) {
        *e = c->prof_pool.back();
        c->prof_pool.pop_back();
      } else if (cudaEventCreate(e) != cudaSuccess) {
        *e = nullptr;
      }
    }
    if (a) cudaEventRecord(a, s);
  }
  ~Prof() {
    if (!a || !b) return;
    cudaEventRecord(b, s);
    c->prof_pending.push_back({id, a, b});
  }
};

// Enqueues one CP step on ctx->stream for the batch in st->cur: the Phi-only
// terms on the side stream, the data-term chain on the main stream, then the
// reduction and update once both are done.
tlda_status enqueue_step(tlda_ctx *ctx, const StepArgs &a, cudaStream_t main) {
  const bool tc = a.precision == TLDA_BF16;
  CK(cudaEventRecord(ctx->ev_fork, main));
  CK(cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0));
  { Prof p(ctx, kPhiGram, ctx->side); launch_phi_gram(a, ctx->side); }
  { Prof p(ctx, kPhiTerms, ctx->side); launch_phi_terms(a, ctx->side); }
  CKL();
  CK(cudaEventRecord(ctx->ev_join, ctx->side));
  if (tc && ctx->fused) {
    // the fused kernel fills its SMs' shared memory: it leaves kPhiSMs SMs
    // free so the side stream's Phi-only kernels run beside it
    Prof p(ctx, kFused, main);
    launch_fused(a, main, ctx->fused_grid);
  } else {
    { Prof p(ctx, kWhiten, main); launch_whiten(a, main, nullptr, true); }
    { Prof p(ctx, kQY, main); if (tc) launch_qy_tc(a, main); else launch_qy_f32(a, main); }
    { Prof p(ctx, kRZ, main); launch_rz(a, main); }
    if (a.same_token) { Prof p(ctx, kZH, main); if (tc) launch_zh_tc(a, main); else launch_zh_f32(a, main); }
    { Prof p(ctx, kG, main); if (tc) launch_g_tc(a, main); else launch_g_f32(a, main); }
  }
  CKL();
  CK(cudaStreamWaitEvent(main, ctx->ev_join, 0));
  { Prof p(ctx, kReduceUpdate, main); launch_reduce_update(a, main); }
  CKL();
  return TLDA_OK;
}

// Folds finished event brackets into the per-kernel totals (synchronises).
tlda_status harvest_profile(tlda_ctx *ctx) {
  if (ctx->prof_pending.empty()) return TLDA_OK;
  CK(cudaDeviceSynchronize());
  for (auto &r : ctx->prof_pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      ctx->prof_ms[r.id] += ms;
      ctx->prof_launches[r.id] += 1;
    }
    ctx->prof_pool.push_back(r.a);
    ctx->prof_pool.push_back(r.b);
  }
  ctx->prof_pending.clear();
  return TLDA_OK;
}

tlda_status read_state(tlda_ctx *ctx) {
  CK(cudaMemcpyAsync(ctx->st_host, ctx->st, sizeof(DevState), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return TLDA_OK;
}

tlda_status take_sticky(tlda_ctx *ctx) {
  const int e = ctx->st_host->err;
  if (e) {
    const int zero = 0;
    CK(cudaMemcpy(&ctx->st->err, &zero, sizeof(int), cudaMemcpyHostToDevice));
    if (e & kErrTimeout) return fail(ctx, TLDA_ERR_TIMEOUT, "a bounded device wait expired");
    return fail(ctx, TLDA_ERR_INVALID, "corrupt CSR batch (indptr, index, order or count)");
  }
  return TLDA_OK;
}

// ------------------------------------------------------------ persistent pass
constexpr long long kStageWords = 1ll << 23;  // int32 words per host-input staging buffer (32 MB)
constexpr long long kFirstStageWords = 1ll << 18;  // int32 words of a host-input pass's first segment (1 MB)
constexpr int kTuneBatches = 128;
// Blocks of the persistent pass that compute only the Phi-only columns
// (P, G3 and their loss parts); more of them for small batches, whose data
// blocks finish early.
constexpr int kPassEBlocks = 8;
constexpr int kPassSmallDocs = 2560;

// Capacity, in steps, of the descriptor, split-point and pinned staging
// buffers: at least kDescsMin on first use, then doubled, so that a pass
// longer than the one before rarely reallocates (cudaMalloc, cudaFree and
// cudaMallocHost synchronise with the device).
constexpr int kDescsMin = 4096;
int desc_capacity(int have, int n) {
  const int grown = have > (1 << 29) ? n : 2 * have;
  return std::max(n, std::max(kDescsMin, grown));
}

tlda_status ensure_descs(tlda_ctx *ctx, int n) {
  if (ctx->descs_cap < n) {
    const int cap = desc_capacity(ctx->descs_cap, n);
    dfree(ctx->descs);
    dfree(ctx->splits);
    ctx->descs_cap = 0;
    CK(dalloc(&ctx->descs, (size_t)cap));
    CK(dalloc(&ctx->splits, (size_t)cap * pass_split_stride(ctx->pass_grid)));
    ctx->descs_cap = cap;
  }
  return TLDA_OK;
}

// One cooperative launch: steps [s0, s1) of the descriptors in ctx->descs,
// after the launch that computes their split points, clears the control block
// and (when `image`) writes the Phi^T image from a.Phi.
tlda_status pass_launch(tlda_ctx *ctx, const StepArgs &a, int s0, int s1, int cap, double *dl, int record,
                        bool image, cudaStream_t ps, const InlineDescs *inl = nullptr) {
  PassArgs pa{};
  pa.descs = ctx->descs;
  pa.s0 = s0;
  pa.s1 = s1;
  pa.tile_cap = cap;
  pa.losses = dl;
  pa.ctl = ctx->ctl;
  pa.record = record;
  pa.e_blocks = kPassEBlocks;
  // for small batches, one block per job of Phi-only columns (one round)
  pa.e_blocks_small = std::max(kPassEBlocks, (ctx->K + kPassPhiCols - 1) / kPassPhiCols);
  pa.e_small_docs = kPassSmallDocs;
  pa.splits = ctx->splits;
  pa.split_stride = pass_split_stride(ctx->pass_grid);
  static const InlineDescs kNone{};  // n = 0: the descriptors are in ctx->descs
  CK(launch_pass_prep(a, image, pa, ctx->pass_grid, ctx->Bmax, inl ? *inl : kNone, ps));
  Prof pr(ctx, kPass, ps);
  CK(launch_pass(a, pa, ps, ctx->pass_grid));
  return TLDA_OK;
}

// Times each candidate tile size on the batches of each size band among hd
// (the first batches of a pass; at least 8 steps per timing, repeating the
// band's batches), on a scratch copy of Phi (lr = 0) and a scratch device
// state (a corrupt batch is left for the real pass to report), and keeps the
// fastest per band.  A band without batches takes the size of the nearest
// band that has some.  The best size depends on the batch size: it sets how
// many 128-nonzero chunks a tile spans and how many tiles each block takes.
// ctx->descs serves as scratch (a pass uploads its own descriptors after).
tlda_status tune_tiles(tlda_ctx *ctx, const float *Phi, const std::vector<BatchDesc> &hd, cudaStream_t ps) {
  StepArgs a = make_args(ctx);
  a.Phi = ctx->phi_scratch;
  a.st = ctx->st_tune;
  CK(cudaMemsetAsync(ctx->st_tune, 0, sizeof(DevState), ps));
  CK(cudaMemcpyAsync(ctx->phi_scratch, Phi, sizeof(float) * ctx->D * ctx->K, cudaMemcpyDeviceToDevice, ps));
  launch_phi_img(a, ps);
  CKL();
  std::vector<BatchDesc> band[kCapBands];
  for (const BatchDesc &d : hd) band[cap_band(d.n_docs)].push_back(d);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  const int cands[] = {8, 14, 16, 18, 20, 24, 28, 32};
  bool have[kCapBands] = {};
  tlda_status s = TLDA_OK;
  for (int bb = 0; bb < kCapBands && s == TLDA_OK; ++bb) {
    if (band[bb].empty()) continue;
    std::vector<BatchDesc> v = band[bb];
    while (v.size() < 8) v.insert(v.end(), band[bb].begin(), band[bb].end());
    const int n = (int)v.size();
    s = ensure_descs(ctx, n);
    if (s) break;
    if (cudaMemcpyAsync(ctx->descs, v.data(), sizeof(BatchDesc) * n, cudaMemcpyHostToDevice, ps) != cudaSuccess ||
        cudaStreamSynchronize(ps) != cudaSuccess) {  // v is pageable
      s = fail(ctx, TLDA_ERR_CUDA, "tile tuning: descriptor upload");
      break;
    }
    int best = 32;
    float best_ms = 0.f;
    for (int c : cands) {
      float ms = 0.f;
      for (int rep = 0; rep < 2 && s == TLDA_OK; ++rep) {  // the first run is a warm-up
        cudaEventRecord(e0, ps);
        s = pass_launch(ctx, a, 0, n, c, nullptr, 0, false, ps);
        cudaEventRecord(e1, ps);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
          s = fail(ctx, TLDA_ERR_CUDA, "tile tuning: %s", cudaGetErrorString(cudaGetLastError()));
      }
      if (s) break;
      if (best_ms == 0.f || ms < best_ms) {
        best_ms = ms;
        best = c;
      }
    }
    ctx->cap_band[bb] = best;
    have[bb] = true;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s) return s;
  for (int bb = 0; bb < kCapBands; ++bb) {
    if (have[bb]) continue;
    for (int dd = 1; dd < kCapBands; ++dd) {
      if (bb - dd >= 0 && have[bb - dd]) {
        ctx->cap_band[bb] = ctx->cap_band[bb - dd];
        break;
      }
      if (bb + dd < kCapBands && have[bb + dd]) {
        ctx->cap_band[bb] = ctx->cap_band[bb + dd];
        break;
      }
    }
  }
  ctx->tile_cap = hd.empty() ? ctx->tile_cap : ctx->cap_band[cap_band(hd[0].n_docs)];
  ctx->tuned = true;
  return TLDA_OK;
}

// The whole pass through the persistent kernel on the pass stream.  Device
// input: one launch.  Host input: the batches are cut into segments that fit
// a staging buffer; segment g is copied on the copy stream into buffer g & 1
// (after the kernel of segment g - 2 is done with it) while the kernel of
// segment g - 1 runs.
tlda_status cp_pass_persistent(tlda_ctx *ctx, const tlda_csr *corpus, const int64_t *off, int nb, float *Phi,
                               float lr, bool host, double *loss_out, bool no_wait) {
  std::vector<int> seg{0};
  std::vector<BatchDesc> hd(nb);
  if (host) {
    const int32_t *ip = corpus->indptr;
    auto need = [&](int b0, int b1) {
      return (long long)(off[b1] - off[b0] + 1) + 2ll * ((long long)ip[off[b1]] - ip[off[b0]]);
    };
    long long max_need = 0;
    for (int b = 0; b < nb; ++b) {
      if (ip[off[b + 1]] < ip[off[b]] || ip[off[b]] < 0)
        return fail(ctx, TLDA_ERR_INVALID, "host indptr not monotone at batch %d", b);
      max_need = std::max(max_need, need(b, b + 1));
    }
    // the staging buffers take a whole segment's size on first use, so a later
    // pass with more batches does not reallocate them (cudaFree synchronises)
    const long long cap = std::max(max_need, kStageWords);
    if (ctx->stage_cap < cap) {
      dfree(ctx->stage[0]);
      dfree(ctx->stage[1]);
      ctx->stage_cap = 0;
      CK(dalloc(&ctx->stage[0], (size_t)cap));
      CK(dalloc(&ctx->stage[1], (size_t)cap));
      ctx->stage_cap = cap;
    }
    // the first segment small (about 1 MB), so that the kernels start while
    // the next segment is still being copied; then whole staging buffers
    for (int b0 = 0; b0 < nb;) {
      const long long lim = b0 == 0 ? std::min(ctx->stage_cap, kFirstStageWords) : ctx->stage_cap;
      int b1 = b0 + 1;
      while (b1 < nb && need(b0, b1 + 1) <= lim) ++b1;
      seg.push_back(b1);
      b0 = b1;
    }
    for (size_t g = 0; g + 1 < seg.size(); ++g) {
      const int b0 = seg[g], b1 = seg[g + 1];
      const long long d0 = off[b0], nds = off[b1] - d0, lo = ip[d0], nnz = ip[off[b1]] - lo;
      int32_t *sg = ctx->stage[g & 1];
      for (int b = b0; b < b1; ++b) {
        BatchDesc &d = hd[b];
        d.indptr = sg + (off[b] - d0);
        d.indices = sg + nds + 1;
        d.counts = sg + nds + 1 + nnz;
        d.nz_base = lo;
        d.n_docs = (int32_t)(off[b + 1] - off[b]);
      }
    }
  } else {
    seg.push_back(nb);
    for (int b = 0; b < nb; ++b) {
      BatchDesc &d = hd[b];
      d.indptr = corpus->indptr + off[b];
      d.indices = corpus->indices;
      d.counts = corpus->counts;
      d.nz_base = 0;
      d.n_docs = (int32_t)(off[b + 1] - off[b]);
    }
  }
  tlda_status s = TLDA_OK;
  if (loss_out && !no_wait && ctx->dlosses_cap < nb) {  // grown like the descriptor buffers
    const int cap = desc_capacity(ctx->dlosses_cap, nb);
    dfree(ctx->dlosses);
    ctx->dlosses_cap = 0;
    CK(dalloc(&ctx->dlosses, (size_t)cap));
    ctx->dlosses_cap = cap;
  }
  // a device-input pass runs on the context's stream; a host-input pass on
  // the pass stream, so that the copy stream's staging overlaps its kernels
  cudaStream_t ps = host ? ctx->pstream : ctx->stream;
  if (host) {
    CK(cudaEventRecord(ctx->ev_pass0, ctx->stream));
    CK(cudaStreamWaitEvent(ps, ctx->ev_pass0, 0));
  }
  if (!ctx->tuned && !host) {
    s = tune_tiles(ctx, Phi, std::vector<BatchDesc>(hd.begin(), hd.begin() + std::min(nb, kTuneBatches)), ps);
    if (s) return s;
  }
  for (BatchDesc &d : hd) d.tile_cap = ctx->cap_band[cap_band(d.n_docs)];
  s = ensure_descs(ctx, nb);
  if (s) return s;
  // staged through pinned memory, so the upload needs no host wait before
  // the launch.  The pinned copy is rewritten only once the previous pass's
  // upload is done: known once that pass synchronised at its end, waited for
  // here after a pass that returned before it did
  // A short device-input pass hands its descriptors to the prologue kernel
  // in the launch parameters instead.
  // each launch (one per staged segment with host input) of at most
  // kInlineDescs steps takes its descriptors in the prologue's parameters
  bool inline_descs = true;
  for (size_t g = 0; g + 1 < seg.size(); ++g)
    if (seg[g + 1] - seg[g] > kInlineDescs) inline_descs = false;
  InlineDescs inl;
  inl.n = 0;
  if (!inline_descs && ctx->descs_pin_busy) {
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaStreamSynchronize(ctx->pstream));
    ctx->descs_pin_busy = false;
  }
  if (!inline_descs && ctx->descs_pin_cap < nb) {
    const int cap = desc_capacity(ctx->descs_pin_cap, nb);
    if (ctx->descs_pin) cudaFreeHost(ctx->descs_pin);
    ctx->descs_pin = nullptr;
    ctx->descs_pin_cap = 0;
    CK(cudaMallocHost(&ctx->descs_pin, sizeof(BatchDesc) * (size_t)cap));
    ctx->descs_pin_cap = cap;
  }
  if (!inline_descs) {
    std::memcpy(ctx->descs_pin, hd.data(), sizeof(BatchDesc) * (size_t)nb);
    CK(cudaMemcpyAsync(ctx->descs, ctx->descs_pin, sizeof(BatchDesc) * nb, cudaMemcpyHostToDevice, ps));
    ctx->descs_pin_busy = true;
  }
  StepArgs a = make_args(ctx);
  a.lr = lr;
  a.Phi = Phi;
  a.want_loss = loss_out ? 1 : 0;
  for (size_t g = 0; g + 1 < seg.size() && s == TLDA_OK; ++g) {
    const int b0 = seg[g], b1 = seg[g + 1];
    if (host) {
      cudaStream_t cs = ctx->cstream;
      const int32_t *ip = corpus->indptr;
      const long long d0 = off[b0], d1 = off[b1], lo = ip[d0], hi = ip[d1];
      const long long nds = d1 - d0;
      int32_t *sg = ctx->stage[g & 1];
      if (g >= 2) CK(cudaStreamWaitEvent(cs, ctx->ev_seg[2 + (g & 1)], 0));
      CK(cudaMemcpyAsync(sg, ip + d0, sizeof(int32_t) * (nds + 1), cudaMemcpyHostToDevice, cs));
      if (hi > lo) {
        CK(cudaMemcpyAsync(sg + nds + 1, corpus->indices + lo, sizeof(int32_t) * (hi - lo), cudaMemcpyHostToDevice, cs));
        CK(cudaMemcpyAsync(sg + nds + 1 + (hi - lo), corpus->counts + lo, sizeof(int32_t) * (hi - lo),
                           cudaMemcpyHostToDevice, cs));
      }
      CK(cudaEventRecord(ctx->ev_seg[g & 1], cs));
      CK(cudaStreamWaitEvent(ps, ctx->ev_seg[g & 1], 0));
    }
    // each batch's own tile size; the Phi^T image before the first segment
    // (each pass launch keeps it current)
    if (inline_descs) {
      inl.n = b1 - b0;
      std::memcpy(inl.d, hd.data() + b0, sizeof(BatchDesc) * (size_t)inl.n);
    }
    s = pass_launch(ctx, a, b0, b1, 0, no_wait ? loss_out : loss_out ? ctx->dlosses : nullptr, 1, g == 0, ps,
                    inline_descs ? &inl : nullptr);
    if (host && s == TLDA_OK) CK(cudaEventRecord(ctx->ev_seg[2 + (g & 1)], ps));
  }
  if (s == TLDA_OK && loss_out && !no_wait)
    CK(cudaMemcpyAsync(loss_out, ctx->dlosses, sizeof(double) * nb, cudaMemcpyDeviceToHost, ps));
  if (host) {
    CK(cudaEventRecord(ctx->ev_pass1, ps));
    CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_pass1, 0));
  }
  if (s) return s;
  // TLDA_NO_WAIT: no wait here (losses, if asked for, went to device
  // memory); the device status goes to the next tlda_sync, and a pinned
  // descriptor buffer in use stays marked busy (the next pass that needs it
  // waits for this one first)
  if (no_wait) return TLDA_OK;
  s = read_state(ctx);  // synchronises the context's stream, which follows the pass
  if (s == TLDA_OK) ctx->descs_pin_busy = false;
  if (s == TLDA_OK) s = take_sticky(ctx);
  return s;
}

const uint32_t kStateMagic = 0x41444C54u;  // "TLDA"
const uint32_t kStateVersion = 1;

uint32_t crc32_update(uint32_t crc, const void *data, size_t n) {
  const unsigned char *p = static_cast<const unsigned char *>(data);
  crc = ~crc;
  for (size_t i = 0; i < n; ++i) {
    crc ^= p[i];
    for (int b = 0; b < 8; ++b) crc = (crc >> 1) ^ (0xEDB88320u & (0u - (crc & 1u)));
  }
  return ~crc;
}

}  // namespace

// ============================================================================ ABI

extern "C" {

void tlda_default_params(tlda_params *p, int32_t k) {
  if (!p) return;
  std::memset(p, 0, sizeof *p);
  p->k = k;
  p->dim = 0;
  p->alpha0 = 1.0;
  p->theta = 0.f;
  p->precision = TLDA_FP32;
  p->same_token_correction = 1;
  p->seed = 0;
  p->max_batch = 8192;
}

const char *tlda_last_error(const tlda_ctx *ctx) { return ctx ? ctx->err.c_str() : "NULL context"; }

int32_t tlda_eig_sweeps(const tlda_ctx *ctx) { return ctx ? ctx->jacobi_sweeps : -1; }

tlda_status tlda_selftest_barrier(void *cuda_stream, int32_t *blocks_out, int32_t *gave_up_out) {
  const int grid = pass_grid();
  if (blocks_out) *blocks_out = grid;
  if (gave_up_out) *gave_up_out = 0;
  if (grid <= 0) return TLDA_ERR_UNIMPLEMENTED;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  PassCtl *ctl = nullptr;
  if (cudaMalloc(&ctl, sizeof(PassCtl)) != cudaSuccess) return TLDA_ERR_OOM;
  PassCtl h{};
  tlda_status st = TLDA_ERR_CUDA;
  if (cudaMemsetAsync(ctl, 0, sizeof(PassCtl), s) == cudaSuccess &&
      launch_barrier_selftest(ctl, s, grid) == cudaSuccess &&
      cudaMemcpyAsync(&h, ctl, sizeof(PassCtl), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
      cudaStreamSynchronize(s) == cudaSuccess) {
    if (gave_up_out) *gave_up_out = (int32_t)h.S3[0];
    st = (h.abort && (int)h.S3[0] == grid) ? TLDA_ERR_TIMEOUT : TLDA_ERR_CUDA;
  }
  cudaFree(ctl);
  return st;
}

tlda_status tlda_create(tlda_ctx **out, int32_t vocab, const tlda_params *p, void *cuda_stream) {
  TLDA_RANGE();
  if (!out || !p) return TLDA_ERR_INVALID;
  *out = nullptr;
  const int K = p->k, D = p->dim > 0 ? p->dim : p->k;
  if (vocab < 1 || K < 1 || D < K || round_up(D, 64) > kMaxDim || round_up(K, 64) > kMaxDim ||
      D > vocab || !(p->alpha0 > 0.0) || !(p->theta > -1.f) ||
      (p->precision != TLDA_FP32 && p->precision != TLDA_BF16) || p->max_batch < 0 ||
      p->max_batch > (1 << 20))
    return TLDA_ERR_INVALID;
  if (p->precision == TLDA_BF16 && !tc_supported(round_up(D, 64), round_up(K, 64))) return TLDA_ERR_UNIMPLEMENTED;
  tlda_ctx *ctx = new tlda_ctx();
  ctx->p = *p;
  ctx->p.dim = D;
  if (ctx->p.max_batch == 0) ctx->p.max_batch = 8192;
  ctx->V = vocab;
  ctx->D = D;
  ctx->K = K;
  ctx->Dp = round_up(D, 64);
  ctx->Kp = round_up(K, 64);
  ctx->Bmax = round_up(ctx->p.max_batch, 128);
  ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  auto bail = [&](tlda_status s, const char *what, cudaError_t e) {
    fprintf(stderr, "tlda_create: %s: %s\n", what, cudaGetErrorString(e));
    tlda_destroy(ctx);
    return s;
  };
  cudaError_t e;
#define CA(call)                                                                            \
  if ((e = (call)) != cudaSuccess)                                                          \
    return bail(e == cudaErrorMemoryAllocation ? TLDA_ERR_OOM : TLDA_ERR_CUDA, #call, e);
  CA(cudaGetDevice(&ctx->device));
  CA(cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device));
  CA(cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking));
  CA(cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming));
  CA(cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming));
  CA(cudaStreamCreateWithFlags(&ctx->pstream, cudaStreamNonBlocking));
  CA(cudaEventCreateWithFlags(&ctx->ev_pass0, cudaEventDisableTiming));
  CA(cudaEventCreateWithFlags(&ctx->ev_pass1, cudaEventDisableTiming));
  const size_t V = vocab, Dp = ctx->Dp, Kp = ctx->Kp, Bm = ctx->Bmax;
  const int tiles = (ctx->Dp / 64) * (ctx->Kp / 64);
  ctx->nsplit = std::max(8, std::min(256, 2 * ctx->num_sms / tiles));
  // k_g_tc: one block per (split, 128-feature tile); as many splits as fill the SMs once
  ctx->nsplit_tc = std::max(8, std::min(64, ctx->num_sms / ((ctx->Dp + 127) / 128)));
  ctx->fused = p->precision == TLDA_BF16 && fused_supported(ctx->Dp, ctx->Kp) && !getenv("TLDA_NO_FUSED");
  ctx->fused_grid = std::max(1, ctx->num_sms - 8);
  CA(dalloc(&ctx->W32, V * D, true));
  CA(dalloc(&ctx->m1, Dp, true));
  CA(dalloc(&ctx->U32, V * Dp, true));
  CA(dalloc(&ctx->X32, Bm * Dp, true));
  CA(dalloc(&ctx->Q32, V * Kp, true));
  CA(dalloc(&ctx->Y32, Bm * Kp, true));
  CA(dalloc(&ctx->Z32, Bm * Kp, true));
  CA(dalloc(&ctx->Zc32, V * Kp, true));
  CA(dalloc(&ctx->H32, V * Kp, true));
  CA(dalloc(&ctx->cnt, V, true));
  CA(dalloc(&ctx->widx, V, true));
  // partial sums; the pass kernel's slice-blocked layout needs up to
  // blocks x (D K + 4 blocks) floats
  CA(dalloc(&ctx->Gpart, (size_t)std::max({ctx->nsplit, ctx->nsplit_tc, ctx->num_sms}) * Dp * Kp +
                             4 * (size_t)ctx->num_sms * ctx->num_sms, true));
  CA(dalloc(&ctx->Gram, Kp * Kp, true));
  CA(dalloc(&ctx->avec, Kp, true));
  CA(dalloc(&ctx->E, Dp * Kp, true));
  CA(dalloc(&ctx->G3, Dp * Kp, true));
  CA(dalloc(&ctx->st, 1, true));
  CA(cudaMallocHost(reinterpret_cast<void **>(&ctx->st_host), sizeof(DevState)));
  std::memset(ctx->st_host, 0, sizeof(DevState));
  if (p->precision == TLDA_BF16) {
    // U rows then X rows in one BF16 matrix: one TMA map covers [U; X]
    CA(dalloc(&ctx->UX16, (V + Bm) * Dp, true));
    ctx->U16 = ctx->UX16;
    ctx->X16 = ctx->UX16 + V * Dp;
    CA(dalloc(&ctx->ZU16, (size_t)round_up(V, 64) * (Kp + Dp), true));
    CA(dalloc(&ctx->Z16, (size_t)Bm * Kp, true));
    CA(dalloc(&ctx->PhiImg, Dp * Kp, true));
    ctx->tc_maps = tc_make_maps(ctx->UX16, ctx->ZU16, ctx->Z16, vocab, ctx->Bmax, ctx->Dp, ctx->Kp);
    if (!ctx->tc_maps) return bail(TLDA_ERR_CUDA, "cuTensorMapEncodeTiled", cudaErrorUnknown);
  }
  if (ctx->fused && !getenv("TLDA_NO_PASS")) ctx->pass_grid = pass_grid();
  if (ctx->pass_grid > 0) {
    CA(dalloc(&ctx->ctl, 1, true));
    CA(dalloc(&ctx->st_tune, 1, true));
    CA(dalloc(&ctx->phi_scratch, (size_t)D * K, true));
    CA(cudaStreamCreateWithFlags(&ctx->cstream, cudaStreamNonBlocking));
    for (cudaEvent_t &ev : ctx->ev_seg) CA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  }
#undef CA
  CK(cudaDeviceSynchronize());
  *out = ctx;
  return TLDA_OK;
}

tlda_status tlda_destroy(tlda_ctx *ctx) {
  if (!ctx) return TLDA_ERR_INVALID;
  if (ctx->stream || ctx->side) cudaDeviceSynchronize();
  dfree(ctx->W32); dfree(ctx->m1); dfree(ctx->U32); dfree(ctx->UX16);
  ctx->U16 = nullptr;
  if (ctx->tc_maps) tc_free_maps(ctx->tc_maps);
  dfree(ctx->X32); dfree(ctx->Q32); dfree(ctx->Y32); dfree(ctx->Z32); dfree(ctx->Zc32);
  dfree(ctx->H32); dfree(ctx->cnt); dfree(ctx->widx); dfree(ctx->Gpart); dfree(ctx->Gram);
  dfree(ctx->avec); dfree(ctx->E); dfree(ctx->G3); dfree(ctx->ZU16); dfree(ctx->Z16); dfree(ctx->PhiImg);
  dfree(ctx->st); dfree(ctx->descs); dfree(ctx->splits); dfree(ctx->P64); dfree(ctx->Ccnt);
  dfree(ctx->TS); dfree(ctx->fit_err); dfree(ctx->stage[0]); dfree(ctx->stage[1]);
  dfree(ctx->ctl); dfree(ctx->st_tune); dfree(ctx->dlosses); dfree(ctx->phi_scratch);
  dfree(ctx->on_Om); dfree(ctx->on_Z); dfree(ctx->on_C); dfree(ctx->on_TS); dfree(ctx->on_err);
  dfree(ctx->on_Wold); dfree(ctx->on_ws); dfree(ctx->on_status); dfree(ctx->on_sk); dfree(ctx->on_Om32);
  if (ctx->coop_ctl) cudaFree(ctx->coop_ctl);
  if (ctx->cstream) cudaStreamDestroy(ctx->cstream);
  for (cudaEvent_t ev : ctx->ev_seg)
    if (ev) cudaEventDestroy(ev);
  if (ctx->st_host) cudaFreeHost(ctx->st_host);
  if (ctx->descs_pin) cudaFreeHost(ctx->descs_pin);
  for (auto &r : ctx->prof_pending) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (cudaEvent_t e : ctx->prof_pool) cudaEventDestroy(e);
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
  if (ctx->side) cudaStreamDestroy(ctx->side);
  if (ctx->step_exec) cudaGraphExecDestroy(ctx->step_exec);
  if (ctx->pstream) cudaStreamDestroy(ctx->pstream);
  if (ctx->ev_pass0) cudaEventDestroy(ctx->ev_pass0);
  if (ctx->ev_pass1) cudaEventDestroy(ctx->ev_pass1);
  delete ctx;
  return TLDA_OK;
}

tlda_status tlda_sync(tlda_ctx *ctx) {
  if (!ctx) return TLDA_ERR_INVALID;
  tlda_status s = read_state(ctx);
  if (s != TLDA_OK) return s;
  return take_sticky(ctx);
}

tlda_status tlda_set_whitening(tlda_ctx *ctx, const float *W, const float *m1) {
  if (!ctx || !W || !m1) return fail(ctx, TLDA_ERR_INVALID, "NULL argument");
  CK(cudaMemcpyAsync(ctx->W32, W, sizeof(float) * (size_t)ctx->V * ctx->D, cudaMemcpyDeviceToDevice,
                     ctx->stream));
  CK(cudaMemsetAsync(ctx->m1, 0, sizeof(float) * ctx->Dp, ctx->stream));
  CK(cudaMemcpyAsync(ctx->m1, m1, sizeof(float) * ctx->D, cudaMemcpyDeviceToDevice, ctx->stream));
  launch_make_u(ctx->W32, ctx->m1, ctx->V, ctx->D, ctx->Dp, ctx->U32, ctx->U16, ctx->stream);
  CKL();
  ctx->eig.assign(ctx->D, 0.0);
  ctx->whitened = true;
  return TLDA_OK;
}

tlda_status tlda_get_whitening(const tlda_ctx *cctx, float *W, float *m1, double *eigvals) {
  tlda_ctx *ctx = const_cast<tlda_ctx *>(cctx);
  if (!ctx) return TLDA_ERR_INVALID;
  if (!ctx->whitened) return fail(ctx, TLDA_ERR_STATE, "no whitening: fit or set one first");
  if (W) CK(cudaMemcpyAsync(W, ctx->W32, sizeof(float) * (size_t)ctx->V * ctx->D, cudaMemcpyDeviceToDevice, ctx->stream));
  if (m1) CK(cudaMemcpyAsync(m1, ctx->m1, sizeof(float) * ctx->D, cudaMemcpyDeviceToDevice, ctx->stream));
  if (eigvals) std::memcpy(eigvals, ctx->eig.data(), sizeof(double) * ctx->D);
  CK(cudaStreamSynchronize(ctx->stream));
  return TLDA_OK;
}

tlda_status tlda_whiten_batch(tlda_ctx *ctx, const tlda_csr *batch, float *X_out) {
  TLDA_RANGE();
  if (!ctx) return TLDA_ERR_INVALID;
  tlda_status s = check_csr(ctx, batch);
  if (s) return s;
  if (!X_out && batch->n_docs > 0) return fail(ctx, TLDA_ERR_INVALID, "X_out is NULL");
  if (!ctx->whitened) return fail(ctx, TLDA_ERR_STATE, "no whitening: fit or set one first");
  if (batch->n_docs > ctx->Bmax) return fail(ctx, TLDA_ERR_INVALID, "n_docs %d > max_batch %d", batch->n_docs, ctx->Bmax);
  if (batch->n_docs == 0) return TLDA_OK;
  launch_set_desc(ctx->st, desc_of(batch), ctx->stream);
  StepArgs a = make_args(ctx);
  launch_whiten(a, ctx->stream, X_out, false);
  CKL();
  return TLDA_OK;
}

static tlda_status step_common(tlda_ctx *ctx, const tlda_csr *batch, float *Phi, float lr,
                               float *grad_out, double *loss_out, int mode, float *gdata_out,
                               int64_t *S3_out) {
  if (!ctx) return TLDA_ERR_INVALID;
  tlda_status s = check_csr(ctx, batch);
  if (s) return s;
  if (!Phi) return fail(ctx, TLDA_ERR_INVALID, "Phi is NULL");
  if (!ctx->whitened) return fail(ctx, TLDA_ERR_STATE, "no whitening: fit or set one first");
  if (batch->n_docs > ctx->Bmax) return fail(ctx, TLDA_ERR_INVALID, "n_docs %d > max_batch %d", batch->n_docs, ctx->Bmax);
  StepArgs a = make_args(ctx);
  a.lr = lr;
  a.Phi = Phi;
  a.grad_out = grad_out;
  a.gdata_out = gdata_out;
  a.mode = mode;
  a.want_loss = loss_out ? 1 : 0;
  launch_set_desc(ctx->st, desc_of(batch), ctx->stream);
  if (a.PhiImg) launch_phi_img(a, ctx->stream);
  CKL();
  s = enqueue_step(ctx, a, ctx->stream);
  if (s) return s;
  if (loss_out || mode == 1) {
    s = read_state(ctx);
    if (s) return s;
    if (loss_out) *loss_out = ctx->st_host->loss;
    if (S3_out) *S3_out = (int64_t)ctx->st_host->last_S3;
    return take_sticky(ctx);
  }
  return TLDA_OK;
}

tlda_status tlda_cp_step(tlda_ctx *ctx, const tlda_csr *batch, float *Phi, float lr, float *grad_out,
                         double *loss_out) {
  TLDA_RANGE();
  return step_common(ctx, batch, Phi, lr, grad_out, loss_out, 0, nullptr, nullptr);
}

tlda_status tlda_cp_data_term(tlda_ctx *ctx, const tlda_csr *batch, const float *Phi, float *G_data_out,
                              int64_t *S3_out) {
  TLDA_RANGE();
  if (ctx && !G_data_out) return fail(ctx, TLDA_ERR_INVALID, "G_data_out is NULL");
  return step_common(ctx, batch, const_cast<float *>(Phi), 0.f, nullptr, nullptr, 1, G_data_out, S3_out);
}

tlda_status tlda_cp_pass(tlda_ctx *ctx, const tlda_csr *corpus, const int64_t *batch_offsets,
                         int32_t n_batches, float *Phi, float lr, uint32_t flags, double *loss_out) {
  TLDA_RANGE();
  if (!ctx) return TLDA_ERR_INVALID;
  tlda_status s = check_csr(ctx, corpus);
  if (s) return s;
  if (!Phi || !batch_offsets || n_batches < 0) return fail(ctx, TLDA_ERR_INVALID, "bad pass arguments");
  if (!ctx->whitened) return fail(ctx, TLDA_ERR_STATE, "no whitening: fit or set one first");
  if (n_batches == 0) return TLDA_OK;
  const bool host = flags & TLDA_HOST_INPUT, no_wait = flags & TLDA_NO_WAIT;
  if (no_wait && host) return fail(ctx, TLDA_ERR_INVALID, "TLDA_NO_WAIT needs device input");
  for (int b = 0; b < n_batches; ++b) {
    const int64_t d0 = batch_offsets[b], d1 = batch_offsets[b + 1];
    if (d0 < 0 || d1 < d0 || d1 > corpus->n_docs) return fail(ctx, TLDA_ERR_INVALID, "batch_offsets[%d] out of range", b);
    if (d1 - d0 > ctx->Bmax) return fail(ctx, TLDA_ERR_INVALID, "batch %d has %lld docs > max_batch", b, (long long)(d1 - d0));
  }
  if (ctx->pass_grid > 0 && (ctx->prof_mask & ~(1u << kPass)) == 0)
    return cp_pass_persistent(ctx, corpus, batch_offsets, n_batches, Phi, lr, host, loss_out, no_wait);
  // descriptors
  {
    const tlda_status es = ensure_descs(ctx, n_batches);
    if (es) return es;
  }
  std::vector<BatchDesc> hd(n_batches);
  long long max_nnz = 0;
  if (host) {
    for (int b = 0; b < n_batches; ++b) {
      const int64_t d0 = batch_offsets[b], d1 = batch_offsets[b + 1];
      const long long lo = corpus->indptr[d0], hi = corpus->indptr[d1];
      if (lo < 0 || hi < lo) return fail(ctx, TLDA_ERR_INVALID, "host indptr not monotone at batch %d", b);
      max_nnz = std::max(max_nnz, hi - lo);
    }
    const long long need = (long long)(ctx->Bmax + 1) + 2 * max_nnz;
    if (ctx->stage_cap < need) {
      dfree(ctx->stage[0]);
      dfree(ctx->stage[1]);
      CK(dalloc(&ctx->stage[0], (size_t)need));
      CK(dalloc(&ctx->stage[1], (size_t)need));
      ctx->stage_cap = need;
    }
  }
  for (int b = 0; b < n_batches; ++b) {
    const int64_t d0 = batch_offsets[b], d1 = batch_offsets[b + 1];
    BatchDesc d{};
    d.n_docs = (int32_t)(d1 - d0);
    if (host) {
      int32_t *sg = ctx->stage[b & 1];
      d.indptr = sg;
      d.indices = sg + (ctx->Bmax + 1);
      d.counts = sg + (ctx->Bmax + 1) + max_nnz;
      d.nz_base = corpus->indptr[d0];
    } else {
      d.indptr = corpus->indptr + d0;
      d.indices = corpus->indices;
      d.counts = corpus->counts;
      d.nz_base = 0;
    }
    hd[b] = d;
  }
  // the pass runs on the context's own non-blocking stream, ordered after
  // and before the caller's stream by events (graph capture needs a stream
  // other than the legacy default one)
  cudaStream_t ps = ctx->pstream;
  CK(cudaEventRecord(ctx->ev_pass0, ctx->stream));
  CK(cudaStreamWaitEvent(ps, ctx->ev_pass0, 0));
  CK(cudaMemcpyAsync(ctx->descs, hd.data(), sizeof(BatchDesc) * n_batches, cudaMemcpyHostToDevice, ps));
  CK(cudaStreamSynchronize(ps));  // hd is pageable: keep it alive until copied
  StepArgs a = make_args(ctx);
  a.lr = lr;
  a.Phi = Phi;
  a.want_loss = loss_out ? 1 : 0;
  double *losses = nullptr;
  if (loss_out && !no_wait) CK(cudaMallocHost(reinterpret_cast<void **>(&losses), sizeof(double) * n_batches));
  launch_begin_pass(ctx->st, ctx->descs, n_batches, ps);
  if (a.PhiImg) launch_phi_img(a, ps);
  CKL();
  // one captured step, replayed per batch (not while the event profiler is on)
  const bool use_graph = ctx->prof_mask == 0;
  if (use_graph && !(ctx->step_exec && ctx->g_lr == lr && ctx->g_phi == Phi && ctx->g_loss == a.want_loss)) {
    if (ctx->step_exec) {
      cudaGraphExecDestroy(ctx->step_exec);
      ctx->step_exec = nullptr;
    }
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(ps, cudaStreamCaptureModeThreadLocal));
    tlda_status cs = enqueue_step(ctx, a, ps);
    cudaError_t ce = cudaStreamEndCapture(ps, &g);
    if (cs) {
      if (g) cudaGraphDestroy(g);
      return cs;
    }
    CK(ce);
    ce = cudaGraphInstantiate(&ctx->step_exec, g, 0);
    cudaGraphDestroy(g);
    CK(ce);
    ctx->g_lr = lr;
    ctx->g_phi = Phi;
    ctx->g_loss = a.want_loss;
  }
  for (int b = 0; b < n_batches && s == TLDA_OK; ++b) {
    if (host) {
      // the slot was last read by step b-2, earlier on the same stream
      const int64_t d0 = batch_offsets[b], d1 = batch_offsets[b + 1];
      const long long lo = corpus->indptr[d0], hi = corpus->indptr[d1];
      const BatchDesc &d = hd[b];
      CK(cudaMemcpyAsync(const_cast<int32_t *>(d.indptr), corpus->indptr + d0, sizeof(int32_t) * (d1 - d0 + 1),
                         cudaMemcpyHostToDevice, ps));
      if (hi > lo) {
        CK(cudaMemcpyAsync(const_cast<int32_t *>(d.indices), corpus->indices + lo, sizeof(int32_t) * (hi - lo),
                           cudaMemcpyHostToDevice, ps));
        CK(cudaMemcpyAsync(const_cast<int32_t *>(d.counts), corpus->counts + lo, sizeof(int32_t) * (hi - lo),
                           cudaMemcpyHostToDevice, ps));
      }
    }
    if (use_graph) CK(cudaGraphLaunch(ctx->step_exec, ps));
    else s = enqueue_step(ctx, a, ps);
    if (loss_out && s == TLDA_OK)
      CK(cudaMemcpyAsync(no_wait ? loss_out + b : losses + b, &ctx->st->loss, sizeof(double),
                         no_wait ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ps));
  }
  CK(cudaEventRecord(ctx->ev_pass1, ps));
  CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_pass1, 0));
  if (s) {
    if (losses) cudaFreeHost(losses);
    return s;
  }
  if (no_wait) return TLDA_OK;  // the device status goes to the next tlda_sync
  s = read_state(ctx);
  if (s == TLDA_OK) {
    if (loss_out) std::memcpy(loss_out, losses, sizeof(double) * n_batches);
    s = take_sticky(ctx);
  }
  if (losses) cudaFreeHost(losses);
  return s;
}

tlda_status tlda_fit_batched(tlda_ctx *ctx, const tlda_csr *corpus, const int64_t *batch_offsets,
                             int32_t n_batches, int32_t epochs, int32_t n_starts, float *Phi, float lr,
                             uint32_t flags, double *loss_out) {
  TLDA_RANGE();
  if (!ctx) return TLDA_ERR_INVALID;
  if (!corpus || !batch_offsets || !Phi || n_batches < 1 || epochs < 1 || n_starts < 1)
    return fail(ctx, TLDA_ERR_INVALID, "bad batched-fit arguments");
  if (flags & TLDA_REUSE_WHITENING) {
    if (!ctx->whitened) return fail(ctx, TLDA_ERR_STATE, "TLDA_REUSE_WHITENING without a whitening");
  } else if (tlda_status s = tlda_fit_moments(ctx, corpus, TLDA_ACCUMULATE | TLDA_FINALIZE)) {
    return s;
  }
  const size_t DK = (size_t)ctx->D * ctx->K;
  std::vector<double> last(n_batches);
  int best = -1;
  double best_loss = 0.0;
  for (int st = 0; st < n_starts; ++st) {
    float *P = Phi + st * DK;
    for (int e = 0; e < epochs; ++e) {
      tlda_status s = tlda_cp_pass(ctx, corpus, batch_offsets, n_batches, P, lr, 0,
                                   e + 1 == epochs ? last.data() : nullptr);
      if (s) return s;
    }
    double m = 0.0;
    for (double v : last) m += v;
    m /= n_batches;
    if (loss_out) loss_out[st] = m;
    if (m == m && (best < 0 || m < best_loss)) {
      best = st;
      best_loss = m;
    }
  }
  if (best > 0) {
    CK(cudaMemcpyAsync(Phi, Phi + best * DK, sizeof(float) * DK, cudaMemcpyDeviceToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  return TLDA_OK;
}

tlda_status tlda_autotune(tlda_ctx *ctx, const tlda_csr *corpus, const int64_t *batch_offsets, int32_t n_batches,
                          const float *Phi, int32_t fixed_cap, int32_t *tile_cap_out) {
  TLDA_RANGE();
  if (!ctx) return TLDA_ERR_INVALID;
  if (ctx->pass_grid <= 0) return fail(ctx, TLDA_ERR_UNIMPLEMENTED, "no persistent pass kernel on this context");
  if (fixed_cap < 0 || fixed_cap > 32) return fail(ctx, TLDA_ERR_INVALID, "tile size %d not in 1..32", fixed_cap);
  if (fixed_cap > 0) {
    ctx->tile_cap = fixed_cap;
    for (int &c : ctx->cap_band) c = fixed_cap;
    ctx->tuned = true;
  } else {
    if (!ctx->whitened) return fail(ctx, TLDA_ERR_STATE, "no whitening: fit or set one first");
    tlda_status s = check_csr(ctx, corpus);
    if (s) return s;
    if (!Phi || !batch_offsets || n_batches < 1) return fail(ctx, TLDA_ERR_INVALID, "bad tuning arguments");
    const int n = std::min<int>(n_batches, kTuneBatches);
    std::vector<BatchDesc> hd(n);
    for (int b = 0; b < n; ++b) {
      const int64_t d0 = batch_offsets[b], d1 = batch_offsets[b + 1];
      if (d0 < 0 || d1 < d0 || d1 > corpus->n_docs) return fail(ctx, TLDA_ERR_INVALID, "batch_offsets[%d] out of range", b);
      if (d1 - d0 > ctx->Bmax) return fail(ctx, TLDA_ERR_INVALID, "batch %d has %lld docs > max_batch", b, (long long)(d1 - d0));
      hd[b] = BatchDesc{corpus->indptr + d0, corpus->indices, corpus->counts, 0, (int32_t)(d1 - d0), 0};
    }
    cudaStream_t ps = ctx->pstream;
    CK(cudaEventRecord(ctx->ev_pass0, ctx->stream));
    CK(cudaStreamWaitEvent(ps, ctx->ev_pass0, 0));
    s = tune_tiles(ctx, Phi, hd, ps);
    CK(cudaEventRecord(ctx->ev_pass1, ps));
    CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_pass1, 0));
    if (s) return s;
  }
  if (tile_cap_out) *tile_cap_out = ctx->tile_cap;
  return TLDA_OK;
}

tlda_status tlda_profile(tlda_ctx *ctx, uint32_t mask) {
  if (!ctx) return TLDA_ERR_INVALID;
  tlda_status s = harvest_profile(ctx);
  if (s) return s;
  ctx->prof_mask = mask & ((1u << kNumKernels) - 1u);
  for (int i = 0; i < 16; ++i) {
    ctx->prof_ms[i] = 0.0;
    ctx->prof_launches[i] = 0;
  }
  return TLDA_OK;
}

tlda_status tlda_profile_read(tlda_ctx *ctx, int32_t kernel, const char **name, int64_t *launches,
                              double *total_ms) {
  if (!ctx) return TLDA_ERR_INVALID;
  if (kernel < 0 || kernel >= kNumKernels) return fail(ctx, TLDA_ERR_INVALID, "no kernel %d", kernel);
  tlda_status s = harvest_profile(ctx);
  if (s) return s;
  if (name) *name = kKernelNames[kernel];
  if (launches) *launches = ctx->prof_launches[kernel];
  if (total_ms) *total_ms = ctx->prof_ms[kernel];
  return TLDA_OK;
}

tlda_status tlda_save_state(const tlda_ctx *cctx, const char *path) {
  TLDA_RANGE();
  tlda_ctx *ctx = const_cast<tlda_ctx *>(cctx);
  if (!ctx || !path) return TLDA_ERR_INVALID;
  if (!ctx->whitened) return fail(ctx, TLDA_ERR_STATE, "nothing to save: no whitening");
  std::vector<float> W((size_t)ctx->V * ctx->D), m1(ctx->D);
  std::vector<unsigned long long> C(ctx->V, 0), TS(3, 0);
  CK(cudaStreamSynchronize(ctx->stream));
  CK(cudaMemcpy(W.data(), ctx->W32, sizeof(float) * W.size(), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(m1.data(), ctx->m1, sizeof(float) * ctx->D, cudaMemcpyDeviceToHost));
  if (ctx->Ccnt) CK(cudaMemcpy(C.data(), ctx->Ccnt, sizeof(unsigned long long) * ctx->V, cudaMemcpyDeviceToHost));
  if (ctx->TS) CK(cudaMemcpy(TS.data(), ctx->TS, sizeof(unsigned long long) * 3, cudaMemcpyDeviceToHost));
  FILE *f = fopen(path, "wb");
  if (!f) return fail(ctx, TLDA_ERR_INVALID, "cannot open %s for writing", path);
  uint32_t hdr[4] = {kStateMagic, kStateVersion, (uint32_t)ctx->V, (uint32_t)ctx->D};
  uint32_t crc = 0;
  auto put = [&](const void *p, size_t n) {
    fwrite(p, 1, n, f);
    crc = crc32_update(crc, p, n);
  };
  put(hdr, sizeof hdr);
  put(W.data(), sizeof(float) * W.size());
  put(m1.data(), sizeof(float) * m1.size());
  put(ctx->eig.data(), sizeof(double) * ctx->D);
  put(C.data(), sizeof(unsigned long long) * C.size());
  put(TS.data(), sizeof(unsigned long long) * 3);
  fwrite(&crc, sizeof crc, 1, f);
  const bool ok = fflush(f) == 0;
  fclose(f);
  return ok ? TLDA_OK : fail(ctx, TLDA_ERR_INVALID, "write to %s failed", path);
}

tlda_status tlda_load_state(tlda_ctx *ctx, const char *path) {
  TLDA_RANGE();
  if (!ctx || !path) return TLDA_ERR_INVALID;
  FILE *f = fopen(path, "rb");
  if (!f) return fail(ctx, TLDA_ERR_INVALID, "cannot open %s", path);
  std::vector<unsigned char> buf;
  unsigned char tmp[65536];
  size_t n;
  while ((n = fread(tmp, 1, sizeof tmp, f)) > 0) buf.insert(buf.end(), tmp, tmp + n);
  fclose(f);
  const size_t nW = (size_t)ctx->V * ctx->D;
  const size_t body = 16 + 4 * nW + 4 * ctx->D + 8 * ctx->D + 8 * (size_t)ctx->V + 24;
  if (buf.size() != body + 4) return fail(ctx, TLDA_ERR_INVALID, "state file size mismatch");
  uint32_t hdr[4], crc;
  std::memcpy(hdr, buf.data(), 16);
  std::memcpy(&crc, buf.data() + body, 4);
  if (hdr[0] != kStateMagic || hdr[1] != kStateVersion) return fail(ctx, TLDA_ERR_INVALID, "not a tlda state file");
  if ((int)hdr[2] != ctx->V || (int)hdr[3] != ctx->D) return fail(ctx, TLDA_ERR_INVALID, "state V/D mismatch");
  if (crc32_update(0, buf.data(), body) != crc) return fail(ctx, TLDA_ERR_INVALID, "state CRC mismatch");
  const unsigned char *p = buf.data() + 16;
  float *dW = nullptr, *dm = nullptr;
  CK(dalloc(&dW, nW));
  CK(dalloc(&dm, ctx->D));
  CK(cudaMemcpy(dW, p, 4 * nW, cudaMemcpyHostToDevice));
  p += 4 * nW;
  CK(cudaMemcpy(dm, p, 4 * ctx->D, cudaMemcpyHostToDevice));
  p += 4 * ctx->D;
  tlda_status s = tlda_set_whitening(ctx, dW, dm);
  CK(cudaStreamSynchronize(ctx->stream));
  cudaFree(dW);
  cudaFree(dm);
  if (s) return s;
  std::memcpy(ctx->eig.data(), p, 8 * ctx->D);
  p += 8 * ctx->D;
  if (!ctx->Ccnt) CK(dalloc(&ctx->Ccnt, ctx->V, true));
  if (!ctx->TS) CK(dalloc(&ctx->TS, 3, true));
  CK(cudaMemcpy(ctx->Ccnt, p, 8 * (size_t)ctx->V, cudaMemcpyHostToDevice));
  p += 8 * (size_t)ctx->V;
  CK(cudaMemcpy(ctx->TS, p, 24, cudaMemcpyHostToDevice));
  ctx->fitted = true;
  return TLDA_OK;
}

}  // extern "C"
