/*
 * Seeded synthetic LDA corpora (the simulation data-generating process of the
 * paper's appendix "Simulation Data Generation Process"): per topic a word
 * distribution mu_k ~ Dirichlet(beta), per document topic proportions
 * theta_d ~ Dirichlet(alpha0/K), per token a topic z ~ theta_d and a word
 * w ~ mu_z.  This file holds NO arithmetic of the estimation method; it only
 * produces inputs (counts in CSR form, the ground-truth topics, initial
 * factors, minibatch sizes) that both the FP64 oracle and the GPU library read.
 *
 * Design (integer-exact, independent of thread count and machine):
 *  - Random numbers: counter-based Philox4x32-10 (Salmon, Moraes, Dror, Shaw,
 *    "Parallel random numbers: as easy as 1, 2, 3", SC'11).  Counter =
 *    (index lo, index hi, sub-index, stream tag | retry << 8), key = seed.
 *  - Topic-word Dirichlet: Gamma variates (Marsaglia & Tsang 2000, with the
 *    U^{1/a} boost for a < 1), normalised in FP64 and quantised to a 2^32-scaled
 *    cumulative table; the quantised probabilities are the ground truth.  A
 *    Zipf-shaped concentration is either shared by every topic or laid over
 *    each topic's own ordering of the vocabulary (a seeded Fisher-Yates
 *    shuffle with Lemire draws).
 *  - Lengths: Poisson(lambda) by inversion of a 2^32-scaled CDF table, clipped
 *    below at min_len.
 *  - Topics: the Polya urn that gives the exact Dirichlet-multinomial marginal
 *    of theta_d ~ Dir(alpha0/K) (alpha0 passed as a rational num/den), with
 *    integer uniforms drawn by Lemire's method (Lemire 2019, "Fast random
 *    integer generation in an interval").
 *  - Words: inversion of the topic's cumulative table (binary search).
 *  - CSR: each document's tokens sorted by word id and merged; indices strictly
 *    ascending, counts > 0.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define TAG_LEN 1u
#define TAG_TOK 2u
#define TAG_GAMMA 3u
#define TAG_BATCH 4u
#define TAG_GAUSS 5u
#define TAG_PERM 6u

/* ------------------------------------------------------------------ Philox */
typedef struct {
  uint32_t v[4];
} ctr4;

static inline uint32_t mulhi32(uint32_t a, uint32_t b, uint32_t *lo) {
  uint64_t p = (uint64_t)a * (uint64_t)b;
  *lo = (uint32_t)p;
  return (uint32_t)(p >> 32);
}

/* Philox4x32 with 10 rounds: S-box = two 32x32->64 multiplies, key schedule =
 * Weyl sequence; round r uses the key bumped r times. */
ctr4 tsyn_philox4x32_10(ctr4 c, uint32_t k0, uint32_t k1) {
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint32_t lo0, lo1;
    uint32_t hi0 = mulhi32(0xD2511F53u, c.v[0], &lo0);
    uint32_t hi1 = mulhi32(0xCD9E8D57u, c.v[2], &lo1);
    ctr4 n;
    n.v[0] = hi1 ^ c.v[1] ^ k0;
    n.v[1] = lo1;
    n.v[2] = hi0 ^ c.v[3] ^ k1;
    n.v[3] = lo0;
    c = n;
  }
  return c;
}

void tsyn_philox_block(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  ctr4 c = {{ctr[0], ctr[1], ctr[2], ctr[3]}};
  ctr4 r = tsyn_philox4x32_10(c, key[0], key[1]);
  memcpy(out, r.v, sizeof(r.v));
}

/* A little stream of 32-bit words for one (index, sub, tag) counter: each
 * refill bumps the retry field so the words never repeat. */
typedef struct {
  uint64_t seed;
  uint64_t idx;
  uint32_t sub, tag, retry, pos;
  uint32_t buf[4];
} rstream;

static void rs_init(rstream *s, uint64_t seed, uint64_t idx, uint32_t sub, uint32_t tag) {
  s->seed = seed;
  s->idx = idx;
  s->sub = sub;
  s->tag = tag;
  s->retry = 0;
  s->pos = 4;
}

static inline uint32_t rs_next(rstream *s) {
  if (s->pos == 4) {
    ctr4 c = {{(uint32_t)s->idx, (uint32_t)(s->idx >> 32), s->sub, s->tag | (s->retry << 8)}};
    ctr4 r = tsyn_philox4x32_10(c, (uint32_t)s->seed, (uint32_t)(s->seed >> 32));
    memcpy(s->buf, r.v, sizeof(r.v));
    s->retry++;
    s->pos = 0;
  }
  return s->buf[s->pos++];
}

/* Uniform integer in [0, n), n >= 1, Lemire's multiply-and-reject. */
static inline uint32_t rs_below(rstream *s, uint32_t n) {
  uint64_t m = (uint64_t)rs_next(s) * (uint64_t)n;
  uint32_t l = (uint32_t)m;
  if (l < n) {
    uint32_t t = (uint32_t)(-n) % n;
    while (l < t) {
      m = (uint64_t)rs_next(s) * (uint64_t)n;
      l = (uint32_t)m;
    }
  }
  return (uint32_t)(m >> 32);
}

/* Uniform double in (0, 1) from 53 random bits (never 0, never 1). */
static inline double rs_unit(rstream *s) {
  uint64_t a = rs_next(s) >> 5, b = rs_next(s) >> 6; /* 27 + 26 bits */
  double u = ((double)a * 67108864.0 + (double)b) / 9007199254740992.0;
  return u + 0.5 / 9007199254740992.0;
}

static double rs_normal(rstream *s) { /* Box-Muller, one of the pair */
  double u1 = rs_unit(s), u2 = rs_unit(s);
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586476925286766559 * u2);
}

/* Gamma(a, 1), Marsaglia & Tsang (2000); a < 1 via Gamma(a+1) * U^{1/a}. */
static double rs_gamma(rstream *s, double a) {
  double boost = 1.0;
  if (a < 1.0) {
    double u = rs_unit(s);
    boost = exp(log(u) / a);
    a += 1.0;
  }
  double d = a - 1.0 / 3.0, c = 1.0 / sqrt(9.0 * d);
  for (;;) {
    double x = rs_normal(s), v = 1.0 + c * x;
    if (v <= 0.0) continue;
    v = v * v * v;
    double u = rs_unit(s);
    if (log(u) < 0.5 * x * x + d - d * v + d * log(v)) return d * v * boost;
  }
}

/* ------------------------------------------------------- topic-word tables */
/* Dirichlet concentration per word: symmetric beta when zipf_s == 0, else
 * a_w = beta * V * z_w with z_w proportional to (w+1)^-zipf_s, sum z = 1. */
static void word_prior(int V, double beta, double zipf_s, double *a) {
  if (zipf_s == 0.0) {
    for (int w = 0; w < V; ++w) a[w] = beta;
    return;
  }
  double z = 0.0;
  for (int w = 0; w < V; ++w) z += pow((double)(w + 1), -zipf_s);
  for (int w = 0; w < V; ++w) a[w] = beta * (double)V * pow((double)(w + 1), -zipf_s) / z;
}

/* rank[w] = the Zipf rank of word w in topic k: a Fisher-Yates shuffle of
 * 0..V-1 on the topic's own stream. */
static void topic_ranks(uint64_t seed, int k, int V, int *rank) {
  for (int w = 0; w < V; ++w) rank[w] = w;
  rstream s;
  rs_init(&s, seed, (uint64_t)k, 0, TAG_PERM);
  for (int i = V - 1; i > 0; --i) {
    const int j = (int)rs_below(&s, (uint32_t)(i + 1));
    const int t = rank[i];
    rank[i] = rank[j];
    rank[j] = t;
  }
}

/* cdf: K x V uint64 (2^32-scaled cumulative, last entry exactly 2^32),
 * mu:  K x V double, the quantised topic-word probabilities (ground truth).
 * per_topic != 0 (with zipf_s != 0): topic k's word w has the concentration
 * of Zipf rank rank_k[w] (topic_ranks) instead of rank w. */
int tsyn_topics(uint64_t seed, int V, int K, double beta, double zipf_s, int per_topic, uint64_t *cdf,
                double *mu) {
  if (V < 1 || K < 1) return 1;
  double *a = (double *)malloc(sizeof(double) * (size_t)V);
  double *g = (double *)malloc(sizeof(double) * (size_t)V);
  int *rank = (int *)malloc(sizeof(int) * (size_t)V);
  if (!a || !g || !rank) {
    free(a);
    free(g);
    free(rank);
    return 2;
  }
  word_prior(V, beta, zipf_s, a);
  const int shuffle = per_topic && zipf_s != 0.0;
  for (int k = 0; k < K; ++k) {
    double tot = 0.0;
    if (shuffle) topic_ranks(seed, k, V, rank);
    for (int w = 0; w < V; ++w) {
      rstream s;
      rs_init(&s, seed, (uint64_t)k * (uint64_t)V + (uint64_t)w, 0, TAG_GAMMA);
      g[w] = rs_gamma(&s, a[shuffle ? rank[w] : w]);
      tot += g[w];
    }
    if (!(tot > 0.0)) { /* all gammas underflowed: put the mass on the first word */
      g[0] = 1.0;
      tot = 1.0;
    }
    uint64_t *row = cdf + (size_t)k * V;
    double run = 0.0;
    uint64_t prev = 0;
    for (int w = 0; w < V; ++w) {
      run += g[w] / tot;
      double q = run * 4294967296.0;
      uint64_t c = (q >= 4294967296.0) ? 4294967296ull : (uint64_t)llround(q);
      if (c < prev) c = prev;
      if (w == V - 1) c = 4294967296ull;
      row[w] = c;
      if (mu) mu[(size_t)k * V + w] = (double)(c - prev) / 4294967296.0;
      prev = c;
    }
  }
  free(a);
  free(g);
  free(rank);
  return 0;
}

/* ----------------------------------------------------------------- lengths */
#define LEN_TABLE_MAX 4096
typedef struct {
  int n;
  uint64_t cdf[LEN_TABLE_MAX];
} len_table;

static int build_len_table(double lam, len_table *t) {
  if (!(lam > 0.0)) return 1;
  int lmax = (int)(lam + 14.0 * sqrt(lam) + 40.0);
  if (lmax >= LEN_TABLE_MAX) return 1;
  double p = exp(-lam), run = 0.0;
  for (int l = 0; l <= lmax; ++l) {
    if (l > 0) p *= lam / (double)l;
    run += p;
    double q = run * 4294967296.0;
    t->cdf[l] = (q >= 4294967296.0) ? 4294967296ull : (uint64_t)llround(q);
  }
  t->cdf[lmax] = 4294967296ull;
  t->n = lmax + 1;
  return 0;
}

static inline int draw_len(const len_table *t, uint64_t seed, uint64_t doc, int min_len) {
  rstream s;
  rs_init(&s, seed, doc, 0, TAG_LEN);
  uint64_t u = rs_next(&s);
  int lo = 0, hi = t->n - 1; /* first l with u < cdf[l] */
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (u < t->cdf[mid]) hi = mid;
    else lo = mid + 1;
  }
  return lo < min_len ? min_len : lo;
}

/* ------------------------------------------------------------------ corpus */
typedef struct {
  uint64_t seed;
  int V, K;
  const uint64_t *cdf; /* K x V */
  uint32_t a_num, a_den; /* alpha0 = a_num / a_den */
  const len_table *lt;
  int min_len;
  int64_t doc0;
} corpus_cfg;

static inline int draw_word(const uint64_t *row, int V, uint32_t u32) {
  uint64_t u = u32;
  int lo = 0, hi = V - 1;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (u < row[mid]) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

static void sort_int(int *x, int n) { /* insertion sort: documents are short */
  for (int i = 1; i < n; ++i) {
    int v = x[i], j = i - 1;
    while (j >= 0 && x[j] > v) {
      x[j + 1] = x[j];
      --j;
    }
    x[j + 1] = v;
  }
}

static int cmp_int(const void *a, const void *b) {
  int x = *(const int *)a, y = *(const int *)b;
  return (x > y) - (x < y);
}

/* Generates document `doc` (global id) with length L into words[0..L) (sorted)
 * using z[0..L) as scratch; returns the number of distinct words. */
static int gen_doc(const corpus_cfg *c, int64_t doc, int L, int *words, int *z) {
  const uint32_t Ka = (uint32_t)c->K * c->a_num, s = (uint32_t)c->K * c->a_den;
  for (int t = 0; t < L; ++t) {
    rstream r;
    rs_init(&r, c->seed, (uint64_t)doc, (uint32_t)t, TAG_TOK);
    /* Polya urn: weight of topic i is a_num + K a_den n_i (n_i = earlier
     * tokens with topic i), i.e. proportional to alpha0/K + n_i. */
    uint32_t u = rs_below(&r, Ka + s * (uint32_t)t);
    int zt = (u < Ka) ? (int)(u / c->a_num) : z[(u - Ka) / s];
    z[t] = zt;
    words[t] = draw_word(c->cdf + (size_t)zt * c->V, c->V, rs_next(&r));
  }
  if (L <= 64) sort_int(words, L);
  else qsort(words, (size_t)L, sizeof(int), cmp_int);
  int u = 0;
  for (int t = 0; t < L; ++t)
    if (t == 0 || words[t] != words[t - 1]) ++u;
  return u;
}

typedef struct {
  const corpus_cfg *c;
  int64_t d_begin, d_end; /* local doc range */
  const int32_t *len;     /* local lengths */
  int64_t *row_nnz;       /* out: distinct words per doc (pass 1) */
  const int64_t *indptr;  /* pass 2: local offsets */
  int32_t *indices, *counts;
  int pass;
  int maxlen;
} worker_arg;

static void *worker(void *p) {
  worker_arg *w = (worker_arg *)p;
  int *words = (int *)malloc(sizeof(int) * (size_t)(w->maxlen + 1));
  int *z = (int *)malloc(sizeof(int) * (size_t)(w->maxlen + 1));
  for (int64_t d = w->d_begin; d < w->d_end; ++d) {
    int L = w->len[d];
    int u = gen_doc(w->c, w->c->doc0 + d, L, words, z);
    if (w->pass == 1) {
      w->row_nnz[d] = u;
    } else {
      int64_t o = w->indptr[d];
      int j = -1;
      for (int t = 0; t < L; ++t) {
        if (t == 0 || words[t] != words[t - 1]) {
          ++j;
          w->indices[o + j] = words[t];
          w->counts[o + j] = 0;
        }
        w->counts[o + j]++;
      }
    }
  }
  free(words);
  free(z);
  return NULL;
}

static int run_workers(worker_arg *base, int64_t n, int nthreads) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  if ((int64_t)nthreads > n) nthreads = n > 0 ? (int)n : 1;
  pthread_t th[256];
  worker_arg args[256];
  int64_t chunk = (n + nthreads - 1) / nthreads;
  for (int i = 0; i < nthreads; ++i) {
    args[i] = *base;
    args[i].d_begin = (int64_t)i * chunk < n ? (int64_t)i * chunk : n;
    args[i].d_end = (int64_t)(i + 1) * chunk < n ? (int64_t)(i + 1) * chunk : n;
    if (pthread_create(&th[i], NULL, worker, &args[i]) != 0) return 1;
  }
  for (int i = 0; i < nthreads; ++i) pthread_join(th[i], NULL);
  return 0;
}

/* Opaque corpus handle: the caller copies the arrays out and frees it. */
typedef struct {
  int64_t n_docs, nnz;
  int64_t *indptr;
  int32_t *indices, *counts, *lengths;
} tsyn_corpus;

void tsyn_corpus_free(tsyn_corpus *h) {
  if (!h) return;
  free(h->indptr);
  free(h->indices);
  free(h->counts);
  free(h->lengths);
  free(h);
}

/* Documents doc0 .. doc0+n_docs-1 of the corpus defined by (seed, cdf, alpha0,
 * lambda, min_len).  Returns NULL on bad arguments or allocation failure. */
tsyn_corpus *tsyn_corpus_make(uint64_t seed, int V, int K, const uint64_t *cdf, uint32_t a_num,
                              uint32_t a_den, double lam, int min_len, int64_t doc0, int64_t n_docs,
                              int nthreads) {
  if (V < 1 || K < 1 || !cdf || a_num == 0 || a_den == 0 || n_docs < 0 || min_len < 0) return NULL;
  /* the urn's integer total must fit in 32 bits for the longest document */
  len_table *lt = (len_table *)malloc(sizeof(len_table));
  if (!lt || build_len_table(lam, lt)) {
    free(lt);
    return NULL;
  }
  int maxlen = lt->n - 1 > min_len ? lt->n - 1 : min_len;
  if ((uint64_t)K * a_num + (uint64_t)K * a_den * (uint64_t)maxlen >= 4294967296ull) {
    free(lt);
    return NULL;
  }
  tsyn_corpus *h = (tsyn_corpus *)calloc(1, sizeof(tsyn_corpus));
  h->n_docs = n_docs;
  h->lengths = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n_docs + 1));
  h->indptr = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_docs + 1));
  int64_t *row_nnz = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_docs + 1));
  if (!h->lengths || !h->indptr || !row_nnz) {
    free(row_nnz);
    free(lt);
    tsyn_corpus_free(h);
    return NULL;
  }
  for (int64_t d = 0; d < n_docs; ++d) h->lengths[d] = draw_len(lt, seed, (uint64_t)(doc0 + d), min_len);
  corpus_cfg c = {seed, V, K, cdf, a_num, a_den, lt, min_len, doc0};
  worker_arg w;
  memset(&w, 0, sizeof(w));
  w.c = &c;
  w.len = h->lengths;
  w.row_nnz = row_nnz;
  w.maxlen = maxlen;
  w.pass = 1;
  if (run_workers(&w, n_docs, nthreads)) goto fail;
  h->indptr[0] = 0;
  for (int64_t d = 0; d < n_docs; ++d) h->indptr[d + 1] = h->indptr[d] + row_nnz[d];
  h->nnz = h->indptr[n_docs];
  h->indices = (int32_t *)malloc(sizeof(int32_t) * (size_t)(h->nnz + 1));
  h->counts = (int32_t *)malloc(sizeof(int32_t) * (size_t)(h->nnz + 1));
  if (!h->indices || !h->counts) goto fail;
  w.pass = 2;
  w.indptr = h->indptr;
  w.indices = h->indices;
  w.counts = h->counts;
  if (run_workers(&w, n_docs, nthreads)) goto fail;
  free(row_nnz);
  free(lt);
  return h;
fail:
  free(row_nnz);
  free(lt);
  tsyn_corpus_free(h);
  return NULL;
}

int64_t tsyn_corpus_n_docs(const tsyn_corpus *h) { return h->n_docs; }
int64_t tsyn_corpus_nnz(const tsyn_corpus *h) { return h->nnz; }

void tsyn_corpus_copy(const tsyn_corpus *h, int64_t *indptr, int32_t *indices, int32_t *counts,
                      int32_t *lengths) {
  if (indptr) memcpy(indptr, h->indptr, sizeof(int64_t) * (size_t)(h->n_docs + 1));
  if (indices) memcpy(indices, h->indices, sizeof(int32_t) * (size_t)h->nnz);
  if (counts) memcpy(counts, h->counts, sizeof(int32_t) * (size_t)h->nnz);
  if (lengths) memcpy(lengths, h->lengths, sizeof(int32_t) * (size_t)h->n_docs);
}

/* The length table of Poisson(lam) (2^32-scaled CDF, as drawn from by the
 * corpus generator), for generators elsewhere that must draw the same
 * lengths.  Writes up to cap entries; returns the table size, or -1. */
int tsyn_len_table(double lam, int cap, uint64_t *out) {
  len_table lt;
  if (build_len_table(lam, &lt) || lt.n > cap) return -1;
  memcpy(out, lt.cdf, sizeof(uint64_t) * (size_t)lt.n);
  return lt.n;
}

/* Raw token stream of one document (topics and words in draw order), for
 * tests of the sampler itself. Returns the length, or -1. */
int tsyn_doc_tokens(uint64_t seed, int V, int K, const uint64_t *cdf, uint32_t a_num, uint32_t a_den,
                    double lam, int min_len, int64_t doc, int cap, int32_t *topics, int32_t *words) {
  len_table lt;
  if (build_len_table(lam, &lt)) return -1;
  int L = draw_len(&lt, seed, (uint64_t)doc, min_len);
  if (L > cap) return -1;
  const uint32_t Ka = (uint32_t)K * a_num, s = (uint32_t)K * a_den;
  for (int t = 0; t < L; ++t) {
    rstream r;
    rs_init(&r, seed, (uint64_t)doc, (uint32_t)t, TAG_TOK);
    uint32_t u = rs_below(&r, Ka + s * (uint32_t)t);
    int zt = (u < Ka) ? (int)(u / a_num) : topics[(u - Ka) / s];
    topics[t] = zt;
    words[t] = draw_word(cdf + (size_t)zt * V, V, rs_next(&r));
  }
  return L;
}

/* Minibatch sizes drawn uniformly from [bmin, bmax] until n_docs are covered
 * (the last batch is truncated). Writes up to cap sizes; returns the count. */
int64_t tsyn_batch_sizes(uint64_t seed, int64_t n_docs, int32_t bmin, int32_t bmax, int64_t cap,
                         int32_t *sizes) {
  if (bmin < 1 || bmax < bmin) return -1;
  int64_t done = 0, nb = 0;
  while (done < n_docs) {
    rstream s;
    rs_init(&s, seed, (uint64_t)nb, 0, TAG_BATCH);
    int64_t b = bmin + (int64_t)rs_below(&s, (uint32_t)(bmax - bmin + 1));
    if (b > n_docs - done) b = n_docs - done;
    if (nb < cap && sizes) sizes[nb] = (int32_t)b;
    done += b;
    ++nb;
  }
  return nb;
}

/* n standard-normal variates (Box-Muller on Philox uniforms), stream `tag2`. */
void tsyn_gaussian(uint64_t seed, uint32_t tag2, int64_t n, double *out) {
  for (int64_t i = 0; i < n; ++i) {
    rstream s;
    rs_init(&s, seed, (uint64_t)i, tag2, TAG_GAUSS);
    out[i] = rs_normal(&s);
  }
}
