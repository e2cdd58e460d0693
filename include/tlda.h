/*
 * tlda.h — C ABI of the GB300 online Tensor LDA library (libtlda).
 *
 * The library runs the data-parallel hot path of online Tensor LDA
 * (Kangaslahti et al., "Analyzing Political Text at Scale with Online Tensor
 * LDA"): demean and whiten bag-of-words minibatches into D dimensions, take the
 * implicit third-order-moment CP gradient (eq. vec_deriv) and apply the SGD
 * factor update (section "Online Learning of the Third Moment").  The moments
 * (M1, M2, whitening W) and the recovery of topics (section "Recovering the
 * Topic Model Parameters") sit on either side of that loop.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Plain pointers and sizes only.  "device" pointers address CUDA global
 *    memory of the context's device; "host" pointers address CPU memory.
 *  - Ownership: every array is owned by the caller; the context owns only its
 *    workspace.  No call keeps a pointer after it returns.
 *  - Streams: work is enqueued on the context's stream (tlda_create) and is
 *    asynchronous unless the entry point says it synchronises.
 *  - Errors: no exception crosses the ABI.  Each call returns a tlda_status;
 *    tlda_last_error() gives a message for the last failure on that context.
 *    Device-side validation failures (a corrupt CSR batch, a bounded wait
 *    that expired) are sticky: they stop later updates of Phi and are
 *    reported by the next synchronising call (tlda_sync, or any call that
 *    documents that it synchronises), which also clears them.
 *  - A context is used by one host thread at a time.
 *
 * Notation: V vocabulary size, D whitening dimension (D >= K), K topics,
 * B documents in a batch.  Matrices are row-major with the stated shape.
 */
#ifndef TLDA_H
#define TLDA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tlda_ctx tlda_ctx;

typedef enum {
  TLDA_OK = 0,
  TLDA_ERR_INVALID = 1,        /* bad argument, or a corrupt CSR batch          */
  TLDA_ERR_CUDA = 2,           /* a CUDA runtime call failed                    */
  TLDA_ERR_NUMERIC = 3,        /* e.g. M2 has fewer than D positive eigenvalues */
  TLDA_ERR_TIMEOUT = 4,        /* a bounded device-side wait expired            */
  TLDA_ERR_OOM = 5,            /* workspace allocation failed / size limit      */
  TLDA_ERR_STATE = 6,          /* call out of order (e.g. cp_step before fit)   */
  TLDA_ERR_UNIMPLEMENTED = 7
} tlda_status;

typedef enum { TLDA_FP32 = 0, TLDA_BF16 = 1 } tlda_precision;

/* A batch (or chunk) of documents as a count CSR, the document-term matrix F
 * of section "Computing the Centered Cumulants" restricted to these rows.
 * Row d holds the distinct words indices[indptr[d] .. indptr[d+1]) with their
 * counts.  indptr entries are absolute offsets into indices/counts, so a batch
 * may be a view into a larger corpus CSR: indptr must be non-decreasing with
 * indptr[0] >= 0.  Within a row indices are strictly ascending and in [0, V);
 * counts are > 0.  Documents with fewer than three tokens are legal: they
 * carry no ordered triple of distinct tokens and contribute nothing to the
 * third moment (pooled normalisation by S3 = sum_d L_d(L_d-1)(L_d-2)).
 * All three arrays are DEVICE pointers unless an entry point says otherwise. */
typedef struct {
  int32_t n_docs;
  int32_t vocab;               /* must equal the context's V */
  const int32_t *indptr;       /* n_docs + 1 */
  const int32_t *indices;
  const int32_t *counts;
} tlda_csr;

/* Method parameters (section "Hyperparameter Tuning"; D from section
 * "Online Decomposition of the Second Moment"). */
typedef struct {
  int32_t k;                   /* topics K (>= 1)                                  */
  int32_t dim;                 /* whitening dimension D (0 means D = K; D >= K)    */
  double alpha0;               /* topic mixing alpha0 > 0                          */
  float theta;                 /* orthogonality penalty theta (> -1)               */
  int32_t precision;           /* tlda_precision of the CP-step contractions       */
  int32_t same_token_correction; /* 1: triples of distinct tokens (default);
                                    0: drop the same-token terms                   */
  uint64_t seed;               /* seed of the randomised subspace start (fit)      */
  int32_t max_batch;           /* largest n_docs of a cp_step / whiten call;
                                  0 means 8192 (sizes the workspace)               */
} tlda_params;

/* Fills *p with defaults: k=K given, D=K, alpha0=1, theta=0, FP32, correction
 * on, seed 0, max_batch 8192. */
void tlda_default_params(tlda_params *p, int32_t k);

/* Creates a context for vocabulary size `vocab` on the current CUDA device,
 * with all work enqueued on `cuda_stream` (a cudaStream_t; NULL = the legacy
 * default stream).  Allocates the workspace (device memory linear in V and
 * max_batch).  D and K are padded to multiples of 64, at most 512, in both
 * forms.  The BF16 form takes the fused tensor-core kernels for D, K in
 * (64, 128] and the multi-kernel tensor-core form otherwise.  Two
 * environment variables, read here, pin the form for comparisons (the results
 * agree within the BF16 tolerance): TLDA_NO_FUSED set takes the multi-kernel
 * tensor-core form at every size; TLDA_NO_PASS set keeps the fused per-step
 * kernel but not the persistent pass kernel of tlda_cp_pass.  Returns
 * TLDA_ERR_INVALID for bad sizes/parameters, TLDA_ERR_OOM if the workspace
 * cannot be allocated. */
tlda_status tlda_create(tlda_ctx **out, int32_t vocab, const tlda_params *p, void *cuda_stream);

/* Frees the context and its workspace (synchronises the stream first). */
tlda_status tlda_destroy(tlda_ctx *ctx);

/* Message of the last failure on ctx ("" if none).  Owned by ctx. */
const char *tlda_last_error(const tlda_ctx *ctx);

/* Sweeps the symmetric eigensolver (cyclic Jacobi, stopped once off-diagonal
 * entries are near 1e-13 of the matrix scale, at most 40) took in the last
 * whitening built on ctx (tlda_fit_moments' finalisation or an online
 * re-whitening); 0 before any, -1 for a NULL context.  Diagnostic. */
int32_t tlda_eig_sweeps(const tlda_ctx *ctx);

/* Synchronises the context's stream and returns (then clears) any sticky
 * device-side status: TLDA_ERR_INVALID for a corrupt batch, TLDA_ERR_TIMEOUT
 * for an expired bounded wait. */
tlda_status tlda_sync(tlda_ctx *ctx);

/* ---------------------------------------------------------------- moments */
#define TLDA_ACCUMULATE 1u
#define TLDA_FINALIZE 2u

/* Moment estimation (section "Computing the Centered Cumulants" and appendix
 * "Uncentered cumulants"; whitening of section "Online Decomposition of the
 * Second Moment", read as W^T M2 W = I with the uncentred M2).
 * With TLDA_ACCUMULATE, adds `chunk` (device CSR) to the running integer
 * statistics: word totals C_m, T = sum L, S2 = sum L(L-1), S3, and the exact
 * pair counts P = sum_d (f_d f_d^T - diag f_d) (a V x V FP64 accumulator held
 * on the device; V <= 65536).  With TLDA_FINALIZE (chunk may be NULL), forms
 * M1 = C/T and M2 = (alpha0+1) P/S2 - alpha0 M1 M1^T, finds the top-D
 * eigenpairs by randomised subspace iteration (FP32 products, FP64
 * orthonormalisation, FP64 Rayleigh-Ritz with a Jacobi eigensolver on the
 * device), and sets W = U_D Lambda_D^-1/2 and m1 = W^T M1.  FINALIZE
 * synchronises and returns TLDA_ERR_NUMERIC if lambda_D <= 1e-12 lambda_1,
 * TLDA_ERR_INVALID if any accumulated chunk was corrupt.  Both flags may be
 * given together.  A later ACCUMULATE after FINALIZE starts a new fit. */
tlda_status tlda_fit_moments(tlda_ctx *ctx, const tlda_csr *chunk, uint32_t flags);

/* Copies the whitening out: W (V x D FP32, device), m1 = W^T M1 (D FP32,
 * device), eigenvalues lambda_1 >= ... >= lambda_D (D FP64, host).  Any
 * pointer may be NULL.  Synchronises.  TLDA_ERR_STATE before a fit. */
tlda_status tlda_get_whitening(const tlda_ctx *ctx, float *W, float *m1, double *eigvals);

/* Integer statistics of the accumulated fit (host outputs, any may be NULL):
 * C (V int64 word totals), T, S2, S3.  Synchronises. */
tlda_status tlda_get_counts(const tlda_ctx *ctx, int64_t *C, int64_t *T, int64_t *S2, int64_t *S3);

/* Installs a whitening instead of fitting one: W (V x D FP32, device) and
 * m1 (D FP32, device).  The CP step uses whitened M2 = I by definition, so its
 * arithmetic does not depend on how W was obtained. */
tlda_status tlda_set_whitening(tlda_ctx *ctx, const float *W, const float *m1);

/* ------------------------------------------------------------- hot path */

/* Whitened, centred counts of a batch (section "Online Decomposition of the
 * Second Moment", x = W (f - M1) in the paper's notation):
 *   X[d,:] = sum_m f_dm W[m,:] - L_d m1,   L_d = sum_m f_dm,
 * i.e. X = F U with U = W - 1 m1^T; the demeaned counts are never densified.
 * X_out: B x D FP32, device, caller-allocated.  Asynchronous; a corrupt batch
 * is reported by tlda_sync.  TLDA_ERR_STATE without a whitening. */
tlda_status tlda_whiten_batch(tlda_ctx *ctx, const tlda_csr *batch, float *X_out);

/* One stochastic tensor gradient step on one minibatch (eq. vec_deriv and
 * the update Phi_{t+1} = Phi_t - beta dL/dPhi), in place on Phi (D x K FP32,
 * device), with lr = beta.  The gradient is
 *   grad = 3(1+theta) Phi (Phi^T Phi * Phi^T Phi) - 3 [c3/S3 (G1 + G2) + G3],
 *   c3 = (alpha0+1)(alpha0+2)/2, X = F U, Y = X Phi, Q = U Phi,
 *   G1 = X^T (Y*Y - F(Q*Q)),  G2 = U^T [Q * (2 c*Q - 2 F^T Y)], c = F^T 1,
 *   G3_i = 2 phi_i (m1.phi_i) + m1 ||phi_i||^2 - 2 m1 (m1.phi_i)^2,
 * the gradient of (1+theta)/2 ||sum phi_i^3||^2 - <sum phi_i^3, T_B> for the
 * batch's whitened third moment written in centred form through Theorem 1
 * (distinct-token triples; G2 and the F(Q*Q) term are the same-token terms,
 * dropped when same_token_correction = 0).  lr = 0 gives the gradient only.
 * grad_out (D x K FP32, device) may be NULL.  loss_out (host) may be NULL;
 * when given, the call synchronises, writes the loss
 *   (1+theta)/2 sum_ij (phi_i.phi_j)^3 - sum_i T_B(phi_i, phi_i, phi_i)
 * at the incoming Phi and returns any sticky status.  A batch with S3 = 0
 * leaves Phi unchanged (grad 0, loss 0).  A corrupt batch leaves Phi
 * unchanged.  TLDA_ERR_STATE without a whitening; TLDA_ERR_INVALID if
 * n_docs > max_batch. */
tlda_status tlda_cp_step(tlda_ctx *ctx, const tlda_csr *batch, float *Phi, float lr,
                         float *grad_out, double *loss_out);

/* The data term of the same step without the update (diagnostics and
 * parity): G_data = c3/S3 (G1 + G2) + G3 (D x K FP32, device) at Phi, and
 * S3 (host, may be NULL).  Synchronises. */
tlda_status tlda_cp_data_term(tlda_ctx *ctx, const tlda_csr *batch, const float *Phi,
                              float *G_data_out, int64_t *S3_out);

#define TLDA_HOST_INPUT 1u     /* corpus arrays are in host memory (pinned for overlap) */
#define TLDA_NO_WAIT 4u        /* tlda_cp_pass: return without waiting; loss_out in device memory */

/* One online pass (section "Fully Online Implementation", with W fixed):
 * batch b is documents [batch_offsets[b], batch_offsets[b+1]) of `corpus`;
 * one CP step per batch, in order, on Phi (D x K FP32, device).
 * batch_offsets: host, n_batches + 1 non-decreasing document offsets.
 * With TLDA_HOST_INPUT the corpus CSR is in host memory and is copied to
 * the device inside the call (double-buffered, each copy overlapped with the
 * compute of the batches before it); otherwise it is in device memory.
 * loss_out (host, n_batches doubles) may be NULL; if given, it receives each
 * step's loss.  An empty batch (equal offsets) is a step with S3 = 0: Phi
 * unchanged, loss 0.  Synchronises at the end and returns any sticky status.
 * With TLDA_NO_WAIT (device input only, else TLDA_ERR_INVALID) the call
 * returns once the pass is enqueued, without waiting for it; loss_out, if
 * not NULL, is then device memory.  The sticky status (a corrupt batch, an
 * expired wait) is returned by the next tlda_sync, and Phi and loss_out are
 * ready when the context's stream has passed the call.
 * A device-input pass runs on the context's stream; a host-input pass runs
 * on internal streams, after the context stream's earlier work and before
 * its later work.
 *
 * In the BF16 form with D, K in (64, 128] the whole pass runs in one
 * persistent cooperative kernel (host input: one launch per staged
 * segment), with the tile size of tlda_autotune; a first device-input pass
 * on a context with no tile size runs the tuner on its first batches.
 * Otherwise each step is one replay of a captured CUDA graph. */
tlda_status tlda_cp_pass(tlda_ctx *ctx, const tlda_csr *corpus, const int64_t *batch_offsets,
                         int32_t n_batches, float *Phi, float lr, uint32_t flags,
                         double *loss_out);

#define TLDA_REUSE_WHITENING 2u /* tlda_fit_batched: keep the context's whitening */

/* The batched mode (section "Batched Implementation Enables Arbitrary
 * Scaling"): the corpus is read once for the moments, then looped over for
 * the third-moment decomposition.
 *  1. Unless flags hold TLDA_REUSE_WHITENING, tlda_fit_moments(ACCUMULATE |
 *     FINALIZE) runs on the whole `corpus` (device CSR): M1, then M2 and its
 *     whitening.
 *  2. For each of n_starts initial factor matrices, `epochs` passes of
 *     tlda_cp_pass over the batches (batch_offsets: host, n_batches + 1
 *     document offsets).  Phi is device memory holding n_starts consecutive
 *     D x K FP32 matrices, each updated in place.
 *  3. The start whose last epoch has the lowest mean step loss is copied
 *     into the first matrix of Phi.  NaN losses never win.  Several starts
 *     guard against the spurious stationary points of the unconstrained CP
 *     objective: one collapsed component, or two components sharing one
 *     topic.
 * loss_out (host, n_starts doubles) may be NULL; it receives each start's
 * mean last-epoch loss.  Synchronises.  Errors as tlda_fit_moments and
 * tlda_cp_pass; TLDA_ERR_STATE with TLDA_REUSE_WHITENING and no whitening. */
tlda_status tlda_fit_batched(tlda_ctx *ctx, const tlda_csr *corpus, const int64_t *batch_offsets,
                             int32_t n_batches, int32_t epochs, int32_t n_starts, float *Phi, float lr,
                             uint32_t flags, double *loss_out);

/* Tile size of the persistent pass kernel: the most documents per tile,
 * 1..32 (each batch is split into ceil(n_docs / SMs) document tiles up to
 * this size).  The size is kept per band of batch sizes (512-document bands,
 * the last one open), since the best one depends on how many 128-nonzero
 * chunks a tile spans and how many tiles each block takes.  With
 * fixed_cap > 0 every band gets fixed_cap and nothing runs (corpus may be
 * NULL).  With fixed_cap = 0 the candidates 8, 14, 16, 18, 20, 24, 28 and 32
 * are timed on the batches of each band among up to the first 128 batches of
 * `corpus` (device CSR, batches as in tlda_cp_pass; at least 8 steps per
 * timing), stepping a scratch copy of Phi (D x K FP32, device; Phi itself and
 * the context's step and error state are left unchanged: a corrupt batch
 * among them is reported by the pass that steps it), and the fastest is kept
 * per band; a band without batches takes the nearest tuned band's size.  A
 * device-input tlda_cp_pass on an untuned context tunes this way on its own
 * first batches.  *tile_cap_out (may be NULL) receives the size of the first
 * batch's band.  Synchronises.  TLDA_ERR_UNIMPLEMENTED on a context without
 * the persistent pass kernel; TLDA_ERR_STATE without a whitening. */
tlda_status tlda_autotune(tlda_ctx *ctx, const tlda_csr *corpus, const int64_t *batch_offsets,
                          int32_t n_batches, const float *Phi, int32_t fixed_cap,
                          int32_t *tile_cap_out);

/* ------------------------------------------------------- fully online mode */

/* Starts the fully online mode (section "Fully Online Implementation"): the
 * context keeps exact token statistics (C, T, S2, S3) and a one-pass sketch
 * Z = P Omega of the pair counts P = sum_d (f_d f_d^T - diag f_d), with the
 * caller's test matrix Omega (V x r FP64, device, row-major, typically
 * Gaussian or random signs; r even, D <= r <= min(V, 512)).  Omega is
 * copied and the statistics are cleared; the context's whitening, if any, is
 * kept.  The sketch's products use the FP32 values of Omega and sum in FP32
 * within a document and within a run of at most 128 nonzeros of a word, then
 * in FP64 (Z stays FP64): with +-1 entries every such sum is an integer, so Z
 * is exact while those sums stay below 2^24 in magnitude.
 * Synchronises.  TLDA_ERR_INVALID for bad sizes. */
tlda_status tlda_online_begin(tlda_ctx *ctx, const double *Omega, int32_t r);

/* One fully online pass: batch b is documents [batch_offsets[b],
 * batch_offsets[b+1]) of `corpus` (device CSR, indptr absolute), taken in
 * blocks of `rewhiten_every` batches.  For each block, its documents first
 * update the statistics and the sketch; then the whitening is rebuilt from
 * them: M1 = C/T, Y = (alpha0+1)/S2 Z - alpha0 M1 (M1^T Omega) (the sketch
 * of M2), Q = orth(Y), B solves B (Q^T Omega) = Q^T Y, B = E Lambda E^T
 * (symmetrised), U = Q E, W = U_D Lambda_D^-1/2 with the sign convention of
 * tlda_fit_moments (Halko, Martinsson and Tropp 2011, section 5.5).  If the
 * context already had a whitening W_old, Phi (D x K FP32, device) is carried
 * into the new basis, Phi <- W^T W_old (W_old^T W_old)^-1 Phi, so that the
 * topics it encodes stay put.  Then the block's CP steps run as in
 * tlda_cp_pass.  rewhiten_every = 1 is the paper's per-batch order: update
 * M1, update the PCA, then take the gradient step.  loss_out (host,
 * n_batches doubles) may be NULL.  Synchronises.  TLDA_ERR_STATE before
 * tlda_online_begin; TLDA_ERR_INVALID for a corrupt batch (the statistics
 * then hold part of it: begin again); TLDA_ERR_NUMERIC if the sketched M2
 * has fewer than D positive eigenvalues. */
tlda_status tlda_online_pass(tlda_ctx *ctx, const tlda_csr *corpus, const int64_t *batch_offsets,
                             int32_t n_batches, float *Phi, float lr, int32_t rewhiten_every,
                             double *loss_out);

/* The online statistics alone: adds every document of `corpus` (device CSR)
 * to the token statistics and the sketch, as tlda_online_pass does for a
 * block, without re-whitening or CP steps.  With tlda_online_whiten this
 * gives the one-pass sketch of a corpus read in chunks before its CP pass.
 * The corpus is taken in pieces of up to 262,144 documents and 16M nonzeros
 * (Z += F^T (F Omega) - diag(F^T 1) Omega per piece, F its counts); the
 * call reads the piece offsets back (a short synchronisation) and enqueues
 * the rest.  A corrupt document (a decreasing indptr, an offset outside the
 * piece's, a word outside [0, V) or not ascending, a count <= 0) adds
 * nothing and is reported by the next tlda_online_whiten or
 * tlda_online_get_sketch (TLDA_ERR_INVALID).  TLDA_ERR_OOM for a document
 * of more than 16M nonzeros; TLDA_ERR_STATE before tlda_online_begin. */
tlda_status tlda_online_accumulate(tlda_ctx *ctx, const tlda_csr *corpus);

/* Rebuilds the whitening from the statistics accumulated so far, exactly as
 * tlda_online_pass does before a block's CP steps.  If the context already
 * had a whitening and Phi (D x K FP32, device) is not NULL, Phi is carried
 * into the new basis.  Synchronises.  Errors as tlda_online_pass. */
tlda_status tlda_online_whiten(tlda_ctx *ctx, float *Phi);

/* Checkpoint of the online statistics: copies out the sketch Z = P Omega
 * (V x r FP64, row-major), the word counts C (V int64) and T, S2, S3 (3
 * int64), each to a host or device pointer (any may be NULL).  Synchronises.
 * TLDA_ERR_INVALID, after the copies, if a corrupt document was met since
 * tlda_online_begin; TLDA_ERR_STATE before tlda_online_begin. */
tlda_status tlda_online_get_sketch(tlda_ctx *ctx, double *Z_out, int64_t *C_out, int64_t *TS_out);

/* Resume: replaces the online statistics with saved ones (same shapes, host
 * or device pointers, all required) and clears the corrupt-document flag.
 * The test matrix is the one given to tlda_online_begin, which must have
 * been called with the Omega and r of the saved run.  Synchronises. */
tlda_status tlda_online_set_sketch(tlda_ctx *ctx, const double *Z, const int64_t *C, const int64_t *TS);

/* --------------------------------------------------------------- recovery */
#define TLDA_HOST_OUTPUT 1u    /* mu_out / alpha_out are host pointers */

/* Topic recovery (section "Recovering the Topic Model Parameters"), in FP64
 * on the device: with lambda_i = ||phi_i||^3, v_i = phi_i/||phi_i||,
 *   mu_i = lambda_i (W^T)^dagger v_i,  (W^T)^dagger = W (W^T W)^-1,
 *   alpha_i proportional to lambda_i^-2, normalised to sum 1,
 * then each mu_i is clipped at 0 and normalised to sum 1.  No "+ M1"
 * re-centring: the whitening is by the uncentred M2, so the CP factors are
 * already the uncentred topics (Theorem 1).  Phi: D x K FP32, device.
 * mu_out: V x K FP64 (column i = topic i); alpha_out: K FP64.  Device
 * pointers, or host with TLDA_HOST_OUTPUT (then the call synchronises). */
tlda_status tlda_unwhiten_topics(tlda_ctx *ctx, const float *Phi, double *mu_out,
                                 double *alpha_out, uint32_t flags);

/* ------------------------------------------------------- allocation-free */

/* The paper has no counterpart of this entry point: it serves callers that
 * cannot allocate device memory.  Examples are code embedded in a host that
 * owns the whole device-memory budget (a framework's caching allocator, a
 * fixed arena that forbids further cudaMalloc), and latency-critical loops
 * where cudaMalloc/cudaFree would synchronise the device.
 *
 * It computes one CP-SGD step with the same arithmetic as tlda_cp_step (FP32
 * form, same-token correction on), without a context.  Inputs:
 *   batch (host struct of device CSR pointers; V = batch->vocab),
 *   W (V x D FP32), m1 = W^T M1 (D FP32), Phi (D x K FP32, updated in place),
 *   grad_out (D x K FP32, may be NULL), err_out (one int32, may be NULL),
 *   all device pointers, dim = D (0 means K), k = K, alpha0, theta, lr = beta.
 * The work is enqueued on cuda_stream and the call returns without waiting.
 * If err_out is given, it receives the device-side validation bits (0 = the
 * batch was valid; non-zero = corrupt CSR, and Phi was left unchanged).
 *
 * Memory: calls no cudaMalloc, cudaFree or allocating library routine.  All
 * scratch is one file-scope __device__ array of 8 MiB that every GPU which
 * loads the library holds until the process exits.  Sizes whose scratch does
 * not fit are rejected with TLDA_ERR_OOM and a one-line message on stderr.
 * For example, V = 4096, D = K = 64 and n_docs = 2048 fit.
 * The batch may hold at most 8 MiB / 768 B = 10,922 documents, else
 * TLDA_ERR_INVALID.
 * Set-up: every call looks up that array's device address in the current
 * context (cudaGetSymbolAddress, which allocates nothing).  The address
 * belongs to the context that loaded the module, so it can change after a
 * device reset (cudaDeviceReset, or a reset of the primary context) or under
 * another context; looking it up per call keeps every call on the array of
 * the context that is current when the call is made.  The first call in a
 * context loads the module; make it before any stream capture.
 * Sharing: every call uses the same array.  The array keeps the last call's
 * contents, so each call clears what must start at zero.  Calls that overlap
 * on the GPU (on different streams, or from different host threads) race on
 * it.  Order them on one stream. */
tlda_status tlda_cp_step_noalloc(const tlda_csr *batch, const float *W, const float *m1,
                                 int32_t dim, int32_t k, double alpha0, float theta, float *Phi,
                                 float lr, float *grad_out, int32_t *err_out, void *cuda_stream);

/* ------------------------------------------------- document-topic VI */

/* Document-topic proportions by standard variational inference (section
 * "Input and Output": the recovered topic-word matrix and weights feed a VI
 * that gives the document-topic matrix; the per-document E-step of Blei, Ng
 * and Jordan 2003, section 5.2, with the topics fixed).  No context.
 *   docs: host struct of device CSR pointers (indptr absolute, as batches of
 *         tlda_cp_pass; V = docs->vocab);
 *   mu:   V x K FP32 device, row-major, column k = topic k (for example the
 *         output of tlda_unwhiten_topics in FP32);
 *   alpha: K FP32 device, the Dirichlet parameters (alpha0 times the learned
 *         weights).
 * Per document with length L: gamma = alpha + L/K, then n_iter rounds of
 *   phi_jk proportional to mu_{m_j k} exp(digamma(gamma_k)) over k,
 *   gamma_k = alpha_k + sum_j f_j phi_jk,
 * where a word whose mu row is all zero gets phi = 0.  theta_out (B x K FP32,
 * device) receives gamma / sum_k gamma_k; gamma_out (B x K FP32, device) may
 * be NULL.  FP32 arithmetic; digamma by its recurrence up to x >= 6 and its
 * asymptotic series.  err_out (one int32, device) may be NULL; bit 0 is set
 * for a document with a word outside [0, V), a count <= 0 or a decreasing
 * indptr, and that document's outputs are NaN.  K in [1, 512], n_iter >= 0,
 * else TLDA_ERR_INVALID.  Enqueued on cuda_stream (NULL: the default stream);
 * returns without waiting; allocates nothing. */
tlda_status tlda_doc_topics(const tlda_csr *docs, const float *mu, const float *alpha, int32_t K,
                            int32_t n_iter, float *theta_out, float *gamma_out, int32_t *err_out,
                            void *cuda_stream);

/* ------------------------------------------------- synthetic corpora */

/* On-device generation of documents doc0 .. doc0+n_docs-1 of a seeded
 * synthetic corpus: the simulation data-generating process of the paper's
 * appendix, defined exactly as the host generator of the test inputs, so the
 * CSR arrays are identical to the host's for the same arguments.
 *  - Philox4x32-10 (Salmon et al., SC'11): counter (document lo, document hi,
 *    token, tag | refill << 8), key = seed.
 *  - Document length: the first l with u < len_cdf[l] (u the first word of
 *    tag 1), clipped below at min_len.
 *  - Token topics: the Polya urn of Dirichlet(alpha0/K), alpha0 =
 *    a_num / a_den, with Lemire integer draws (tag 2).
 *  - Token words: the first w with u < topic_cdf[z][w].
 *  - Tokens sorted and merged into strictly ascending words with counts.
 * Arguments:
 *  - topic_cdf: K x V uint64, device; each row a 2^32-scaled cumulative
 *    table whose last entry is 2^32.
 *  - len_cdf: n_len uint64, device; a cumulative table of the same kind,
 *    n_len <= 1025, so documents have at most 1024 tokens.
 *  - Output, device: indptr_out (n_docs + 1 int32, relative: indptr[0] = 0),
 *    indices_out and counts_out (capacity nnz_cap int32 each).  With
 *    nnz_cap = 0 only indptr and *nnz_out are produced.
 *  - scratch: device, (n_docs + 1023) / 1024 + 2 int64 words.  The write pass
 *    is still queued on cuda_stream when the call returns and uses it: keep
 *    it unchanged until the stream has passed that point.
 *  - *nnz_out (host): the chunk's nonzeros.
 * Synchronises the stream once, to learn the nonzeros.  Errors:
 *  - TLDA_ERR_OOM if they exceed nnz_cap (indices not written) or 2^31 - 1;
 *  - TLDA_ERR_INVALID for bad arguments, or if K (a_num + 1024 a_den)
 *    reaches 2^32. */
tlda_status tlda_generate_docs(uint64_t seed, int32_t V, int32_t K, const uint64_t *topic_cdf,
                               uint32_t a_num, uint32_t a_den, const uint64_t *len_cdf, int32_t n_len,
                               int32_t min_len, int64_t doc0, int32_t n_docs, int32_t *indptr_out,
                               int32_t *indices_out, int32_t *counts_out, int64_t nnz_cap,
                               int64_t *scratch, int64_t *nnz_out, void *cuda_stream);

/* ------------------------------------------------------------ self-test */

/* Exercises the bounded grid barrier of the persistent kernels: a
 * cooperative launch of *blocks_out blocks (the pass kernel's grid) in which
 * block 0 never arrives.  Every block waits out its bound (about one second
 * of clock cycles) or sees the abort flag that the first one to give up
 * raises, and returns.  *gave_up_out counts the blocks that gave up.  The
 * expected result is TLDA_ERR_TIMEOUT with every block counted; any context
 * stays usable afterwards.  TLDA_ERR_UNIMPLEMENTED without cooperative
 * launch.  Synchronises cuda_stream (NULL: the default stream). */
tlda_status tlda_selftest_barrier(void *cuda_stream, int32_t *blocks_out, int32_t *gave_up_out);

/* ------------------------------------------------------------ profiling */

/* Per-kernel device time, from CUDA events recorded around each launch on
 * the stream it is launched on.  Kernels of one CP step, in launch order:
 *   0 scan_whiten  1 qy  2 rz  3 zh  4 g_reduce  5 reduce_update
 *   6 phi_gram  7 phi_terms (6 and 7 run on the context's side stream)
 *   8 fused (BF16 form with D, K in (64, 128]: replaces kernels 0-4)
 *   9 pass (the persistent kernel of tlda_cp_pass in that form: one launch
 *     runs every step of the pass, kernels 0-8 do not run).
 * tlda_profile sets the mask of bracketed kernels (bit i = kernel i; 0 turns
 * profiling off) and clears the totals.  tlda_profile_read synchronises and
 * returns the kernel's name (static string), launch count and summed
 * milliseconds since the last tlda_profile; TLDA_ERR_INVALID past the last id. */
tlda_status tlda_profile(tlda_ctx *ctx, uint32_t mask);
tlda_status tlda_profile_read(tlda_ctx *ctx, int32_t kernel, const char **name, int64_t *launches,
                              double *total_ms);

/* FP32 CUDA-core throughput probe (diagnostic; the paper has no counterpart:
 * it measures the peak against which the FP32 plain form's "alu" roofline is
 * reported).  Launches one kernel on cuda_stream (NULL: the default stream)
 * that fills every SM with resident 256-thread blocks, each thread running 8
 * independent FMA chains for iters x 16 steps, and returns at once.
 * *flops_out (host) receives the kernel's flop count (2 per FMA); time the
 * launch with CUDA events on the same stream.  sink: device buffer of at
 * least (SMs x resident blocks per SM) floats, never written in practice.
 * TLDA_ERR_INVALID for iters < 1 or NULL pointers. */
tlda_status tlda_ffma_probe(int32_t iters, float *sink, double *flops_out, void *cuda_stream);

/* --------------------------------------------------------------- state */

/* Checkpoint / resume of the fitted state (integer statistics, whitening,
 * eigenvalues) to a flat binary file with a version word and a CRC-32.
 * Synchronises.  tlda_load_state checks V, D and the CRC and returns
 * TLDA_ERR_INVALID on a mismatch. */
tlda_status tlda_save_state(const tlda_ctx *ctx, const char *path);
tlda_status tlda_load_state(tlda_ctx *ctx, const char *path);

#ifdef __cplusplus
}
#endif
#endif /* TLDA_H */
