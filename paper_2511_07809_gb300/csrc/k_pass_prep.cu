// Prologue of a persistent pass launch (split points of every step's data
// blocks, the BF16 Phi^T image, the control block), one kernel before the
// cooperative launch of k_pass.
#include "tlda_internal.h"

namespace tlda {
namespace {

__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
               "l"(src)
               : "memory");
}

// What a pass launch needs before it starts, in one launch:
// * blocks [0, s1 - s0): per step, the n_blocks + 1 split points of its
//   documents.  split_i is the first document whose start offset reaches
//   i nnz / n_blocks (a lower bound by binary search on indptr), made
//   non-decreasing by a running maximum, so the ranges partition
//   [0, n_docs) even when indptr is corrupt (the tiles' validation then sees
//   every document once).  Beside each split point goes indptr there, the
//   offset of the range's first nonzero (the pass requests a range's first
//   window of metadata together with its offsets).  The batch's offsets are read into shared memory
//   first (4-byte cp.async copies, all of a thread's in flight together)
//   when they fit `cap` entries;
//   For a range that takes two tiles, the documents of the first go beside
//   them (the boundary with the fewest 128-nonzero chunks in the two).
//   The last two entries of a step's row take the batch's nonzeros [lo, hi)
//   relative to nz_base, and the blocks of the first two steps bring those
//   nonzeros' indices and counts into L2;
// * the blocks after them (when `image`): the BF16 Phi^T image from Phi;
// * block 0 also clears the pass's control block;
// * with inline descriptors (a short pass), each step's block takes its
//   batch's descriptor from the launch parameters and stores it for k_pass.
constexpr int kSplitThreads = 256;
constexpr int kPrepImgBlocks = 8;
__global__ void __launch_bounds__(kSplitThreads) k_pass_prep(StepArgs a, int image, PassArgs p, int grid, int *splits,
                                                            int cap, InlineDescs inl) {
  extern __shared__ int s_ip[];
  __shared__ int s_wmax[kSplitThreads / 32];
  const int n_steps = p.s1 - p.s0;
  if (blockIdx.x == 0) {
    unsigned int *w = reinterpret_cast<unsigned int *>(p.ctl);
    for (int i = threadIdx.x; i < (int)(sizeof(PassCtl) / sizeof(unsigned int)); i += kSplitThreads) w[i] = 0u;
  }
  if ((int)blockIdx.x >= n_steps) {
    if (image) phi_img_groups(a, (blockIdx.x - n_steps) * kSplitThreads + threadIdx.x, kPrepImgBlocks * kSplitThreads);
    return;
  }
  const int s = p.s0 + blockIdx.x;
  const BatchDesc b = inl.n > 0 ? inl.d[blockIdx.x] : p.descs[s];
  if (inl.n > 0 && threadIdx.x == 0) const_cast<BatchDesc *>(p.descs)[s] = b;  // for the pass kernel
  const int nd = b.n_docs;
  const int n_blocks = pass_data_blocks(p, grid, nd), stride = p.split_stride;
  const bool in_smem = nd + 1 <= cap;
  if (in_smem) {
    for (int d = threadIdx.x; d <= nd; d += kSplitThreads) cp_async4(s_ip + d, b.indptr + d);
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
  }
  __syncthreads();
  auto ip = [&](int d) -> long long { return in_smem ? s_ip[d] : b.indptr[d]; };
  const long long base = nd > 0 ? ip(0) : 0;
  const long long nnz = nd > 0 ? ip(nd) - base : 0;
  if (threadIdx.x == 0) {  // the batch's nonzeros, relative to nz_base
    splits[(long long)s * stride + stride - 2] = (int)(base - b.nz_base);
    splits[(long long)s * stride + stride - 1] = (int)(base + nnz - b.nz_base);
  }
  if (blockIdx.x < 2 && nd > 0 && nnz > 0 && base >= b.nz_base) {
    // the first two steps' CSR into L2 (later steps: the pass's Phi-only
    // blocks, two steps ahead)
    l2_prefetch_lines(b.indices + (base - b.nz_base), nnz * 4, 0, 1, threadIdx.x, blockDim.x);
    l2_prefetch_lines(b.counts + (base - b.nz_base), nnz * 4, 0, 1, threadIdx.x, blockDim.x);
  }
  __shared__ int s_spl[kSplitThreads + 1];
  int carry = 0;  // running maximum of the earlier rounds
  for (int i0 = 0; i0 <= n_blocks; i0 += kSplitThreads) {
    const int i = i0 + threadIdx.x;
    int v = 0;
    if (i <= n_blocks) {
      v = nd;
      if (i == 0) {
        v = 0;
      } else if (i < n_blocks && nnz > 0) {
        const long long target = base + nnz * i / n_blocks;
        int lo = 0, hi = nd;
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (ip(mid) < target) lo = mid + 1;
          else hi = mid;
        }
        v = lo;
      }
      v = min(v, nd);
    }
    // inclusive running maximum over this round (warp shuffles, then the warps)
    int m = max(v, carry);
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, m, o);
      if ((threadIdx.x & 31) >= o) m = max(m, t);
    }
    if ((threadIdx.x & 31) == 31) s_wmax[threadIdx.x >> 5] = m;
    __syncthreads();
    for (int w = 0; w < (int)(threadIdx.x >> 5); ++w) m = max(m, s_wmax[w]);
    if (i <= n_blocks) {
      const int v_i = i == n_blocks ? nd : m;
      splits[(long long)s * stride + i] = v_i;
      splits[(long long)s * stride + grid + 1 + i] = nd > 0 ? (int)ip(v_i) : 0;  // its first nonzero
      if (i <= kSplitThreads) s_spl[i] = v_i;
    }
    __syncthreads();
    carry = s_wmax[0];
    for (int w = 1; w < kSplitThreads / 32; ++w) carry = max(carry, s_wmax[w]);
    __syncthreads();
  }
  // Repair of the range boundaries where a range would need one more
  // 128-nonzero chunk (or a second tile) than its neighbours: when the
  // batch averages at most one tile per block, each inner boundary may move
  // by up to two documents to lower the larger chunk count of its two
  // ranges (ranges of more than cap documents count as eight more); odd
  // boundaries first, then even ones (boundaries of one parity share no
  // range), twice.
  const int r_cap = min(p.tile_cap > 0 ? p.tile_cap : (b.tile_cap > 0 ? b.tile_cap : kPassTileDocs), kPassTileDocs);
  if (in_smem && nd > 0 && n_blocks > 1 && n_blocks < kSplitThreads && nd <= (long long)n_blocks * r_cap) {
    auto cost = [&](int da, int db) -> int {
      const long long z = ip(db) - ip(da);
      return (int)((z > 0 ? z : 0) + 127) / 128 + (db - da > r_cap ? 8 : 0);
    };
    for (int round = 0; round < 4; ++round) {
      const int j = 2 * threadIdx.x + 1 + (round & 1);  // boundary j between ranges j - 1 and j
      if (j < n_blocks) {
        const int lo_b = s_spl[j - 1], hi_b = s_spl[j + 1], cur = s_spl[j];
        int best = max(cost(lo_b, cur), cost(cur, hi_b)), at = cur;
        for (int dlt = -2; dlt <= 2; ++dlt) {
          const int c = cur + dlt;
          if (dlt == 0 || c <= lo_b || c >= hi_b) continue;  // ranges stay non-empty
          const int v = max(cost(lo_b, c), cost(c, hi_b));
          if (v < best) {
            best = v;
            at = c;
          }
        }
        s_spl[j] = at;
      }
      __syncthreads();
    }
    for (int i = threadIdx.x; i <= n_blocks; i += kSplitThreads) {
      splits[(long long)s * stride + i] = s_spl[i];
      splits[(long long)s * stride + grid + 1 + i] = (int)ip(s_spl[i]);
    }
    __syncthreads();
  }
  // A range of more than cap documents (at most 2 cap) takes two tiles.  The
  // pass processes a tile in chunks of 128 nonzeros, so the boundary between
  // them is the one with the fewest chunks in the two (then the most even),
  // rather than the middle document.  0: tiles of equal size.
  const int b_cap = p.tile_cap > 0 ? p.tile_cap : (b.tile_cap > 0 ? b.tile_cap : kPassTileDocs);
  const int cap2 = min(b_cap, kPassTileDocs);
  const bool pick = in_smem && nd > 0 && n_blocks < kSplitThreads;
  for (int i = threadIdx.x; i < n_blocks; i += kSplitThreads) {
    int t1 = 0;
    if (pick) {
      const int da = s_spl[i], D = s_spl[i + 1] - da;
      if (D > cap2 && D <= 2 * cap2) {
        const long long za = ip(da), zb = ip(da + D);
        int best = 1 << 30, even = 1 << 30;
        for (int m1 = max(1, D - cap2); m1 <= min(D - 1, cap2); ++m1) {
          const long long zm = ip(da + m1);
          const long long n1 = zm > za ? zm - za : 0, n2 = zb > zm ? zb - zm : 0;
          const int c = (int)((n1 + 127) / 128 + (n2 + 127) / 128), e = abs(2 * m1 - D);
          if (c < best || (c == best && e < even)) {
            best = c;
            even = e;
            t1 = m1;
          }
        }
      }
    }
    splits[(long long)s * stride + 2 * grid + 2 + i] = t1;
  }
}

}  // namespace

cudaError_t launch_pass_prep(const StepArgs &a, bool image, const PassArgs &p, int grid, int max_docs,
                             const InlineDescs &inl, cudaStream_t s) {
  if (p.s1 <= p.s0) return cudaSuccess;
  if (grid < 2 || p.split_stride < pass_split_stride(grid)) return cudaErrorInvalidValue;
  if (inl.n != 0 && inl.n != p.s1 - p.s0) return cudaErrorInvalidValue;  // one inline descriptor per step
  // the offsets of batches up to 11,999 documents go through shared memory
  // (at most 48,000 bytes: within the default dynamic shared-memory limit)
  const int cap = max_docs + 1 <= 12000 ? max_docs + 1 : 0;
  const int blocks = (p.s1 - p.s0) + (image ? kPrepImgBlocks : 0);
  k_pass_prep<<<blocks, kSplitThreads, (size_t)cap * sizeof(int), s>>>(a, image ? 1 : 0, p, grid,
                                                                      const_cast<int *>(p.splits), cap, inl);
  return cudaGetLastError();
}

}  // namespace tlda
