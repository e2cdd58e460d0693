"""Seeded synthetic LDA corpora: the input generator shared by the FP64 oracle
and the GPU library.

It follows the simulation data-generating process in the paper's appendix
("Simulation Data Generation Process"): topic-word distributions
mu_k ~ Dirichlet(beta), document-topic proportions theta_d ~ Dirichlet(alpha0/K),
per token a topic z ~ Mult(theta_d) and a word w ~ Mult(mu_z).  Documents with
fewer than three words are clipped to three (the paper drops such documents
in pre-processing, section "Recommendations for Data Pre-processing").

All sampling lives in ``synth.c`` (Philox4x32-10 counters, integer sampling);
this module compiles it, marshals arrays, and derives orthonormal starting
factors from the Gaussian ones by a QR factorisation.  It holds none of the
estimation method's arithmetic, so both sides of a parity test may use it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, replace
from fractions import Fraction

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "_lib")
_LIBPATH = os.path.join(_LIBDIR, "libtlda_synth.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile synth.c into a shared library next to this file."""
    src = os.path.join(_HERE, "synth.c")
    if (not force and os.path.exists(_LIBPATH)
            and os.path.getmtime(_LIBPATH) >= os.path.getmtime(src)):
        return _LIBPATH
    os.makedirs(_LIBDIR, exist_ok=True)
    tmp = _LIBPATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
           "-ffp-contract=off", "-fno-fast-math", src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIBPATH)
    return _LIBPATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIBPATH)
    c_u64p = ctypes.POINTER(ctypes.c_uint64)
    c_f64p = ctypes.POINTER(ctypes.c_double)
    c_i32p = ctypes.POINTER(ctypes.c_int32)
    c_i64p = ctypes.POINTER(ctypes.c_int64)
    c_u32p = ctypes.POINTER(ctypes.c_uint32)
    lib.tsyn_topics.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                ctypes.c_double, ctypes.c_int, c_u64p, c_f64p]
    lib.tsyn_topics.restype = ctypes.c_int
    lib.tsyn_corpus_make.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_int, c_u64p,
                                     ctypes.c_uint32, ctypes.c_uint32, ctypes.c_double, ctypes.c_int,
                                     ctypes.c_int64, ctypes.c_int64, ctypes.c_int]
    lib.tsyn_corpus_make.restype = ctypes.c_void_p
    lib.tsyn_corpus_free.argtypes = [ctypes.c_void_p]
    lib.tsyn_corpus_n_docs.argtypes = [ctypes.c_void_p]
    lib.tsyn_corpus_n_docs.restype = ctypes.c_int64
    lib.tsyn_corpus_nnz.argtypes = [ctypes.c_void_p]
    lib.tsyn_corpus_nnz.restype = ctypes.c_int64
    lib.tsyn_corpus_copy.argtypes = [ctypes.c_void_p, c_i64p, c_i32p, c_i32p, c_i32p]
    lib.tsyn_doc_tokens.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_int, c_u64p,
                                    ctypes.c_uint32, ctypes.c_uint32, ctypes.c_double, ctypes.c_int,
                                    ctypes.c_int64, ctypes.c_int, c_i32p, c_i32p]
    lib.tsyn_doc_tokens.restype = ctypes.c_int
    lib.tsyn_batch_sizes.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                     ctypes.c_int64, c_i32p]
    lib.tsyn_batch_sizes.restype = ctypes.c_int64
    lib.tsyn_gaussian.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int64, c_f64p]
    lib.tsyn_philox_block.argtypes = [c_u32p, c_u32p, c_u32p]
    lib.tsyn_len_table.argtypes = [ctypes.c_double, ctypes.c_int, c_u64p]
    lib.tsyn_len_table.restype = ctypes.c_int
    _lib = lib
    return lib


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


# --------------------------------------------------------------------------- specs
@dataclass(frozen=True)
class CorpusSpec:
    """One synthetic workload. alpha0 is kept exact as a fraction because the
    Polya-urn sampler works in integers."""
    name: str
    V: int
    K: int
    beta: float            # topic-word Dirichlet concentration (mean per word)
    zipf_s: float          # 0: symmetric prior; else Zipf(s)-shaped prior
    alpha0: Fraction       # document-topic Dirichlet(alpha0/K)
    lam: float             # Poisson mean document length
    min_len: int           # lengths clipped below at this value
    n_docs: int
    seed: int
    batch: tuple           # (bmin, bmax) minibatch sizes, drawn uniformly
    zipf_per_topic: bool = False  # Zipf ranks over each topic's own ordering of the words

    def with_docs(self, n_docs: int) -> "CorpusSpec":
        return replace(self, n_docs=int(n_docs))


_BASE_SEED = 0x544C4441

#: The five seeded workloads.  Shapes, priors and length laws follow the
#: workloads the method is evaluated on (tweets: short documents, Zipf vocabularies).
WORKLOADS = {
    "small_v500_k10": CorpusSpec("small_v500_k10", 500, 10, 0.1, 0.0, Fraction(1), 50.0, 3,
                                 10_000, _BASE_SEED + 0, (1000, 1000)),
    "tweet_v5k_k50": CorpusSpec("tweet_v5k_k50", 5_000, 50, 0.05, 1.1, Fraction(1), 30.0, 3,
                                1_000_000, _BASE_SEED + 1, (4096, 4096)),
    "stream_v20k_k100": CorpusSpec("stream_v20k_k100", 20_000, 100, 0.1, 0.0, Fraction(2), 12.0, 3,
                                   10_000_000, _BASE_SEED + 2, (512, 8192)),
    "scale_v50k_k200": CorpusSpec("scale_v50k_k200", 50_000, 200, 0.1, 0.0, Fraction(1), 20.0, 3,
                                  50_000_000, _BASE_SEED + 3, (8192, 8192)),
    # a "Zipf(1.07) vocabulary": each topic Zipf-shaped over its own ordering of
    # the words (shared head words would leave the topics' 300th eigenvalue of
    # M2 far below the sampling noise even at a billion documents)
    "billion_v100k_k300": CorpusSpec("billion_v100k_k300", 100_000, 300, 0.05, 1.07, Fraction(5),
                                     15.0, 3, 1_000_000_000, _BASE_SEED + 4, (65536, 65536), True),
}


def e1_spec(V: int, rep: int) -> CorpusSpec:
    """The simulation study's corpora (section "Parameter Recovery and
    Comparison to Previous TLDA Methods"): K = 2 topics, alpha0 = 0.01,
    20,000 documents, vocabulary V (500, 1000 or 1500 there), one seed per
    repetition.  The topic prior and the lengths are not stated there: the
    small workload's Dirichlet(0.1) and Poisson(50), at least 3 words."""
    return CorpusSpec(f"e1_v{V}_k2_rep{rep}", int(V), 2, 0.1, 0.0, Fraction(1, 100), 50.0, 3, 20_000,
                      _BASE_SEED + 0x100 + 16 * int(rep) + int(V) // 500, (1000, 1000))


# --------------------------------------------------------------------------- draws
def philox4x32_10(ctr, key) -> np.ndarray:
    """One Philox4x32-10 block (exposed for known-answer tests)."""
    lib = _load()
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.tsyn_philox_block(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32),
                          _ptr(out, ctypes.c_uint32))
    return out


def topics(spec: CorpusSpec):
    """Topic-word tables. Returns (cdf uint64 [K,V], mu float64 [K,V]); mu is
    the exact (quantised) distribution the corpus is drawn from."""
    lib = _load()
    cdf = np.zeros((spec.K, spec.V), dtype=np.uint64)
    mu = np.zeros((spec.K, spec.V), dtype=np.float64)
    rc = lib.tsyn_topics(spec.seed, spec.V, spec.K, spec.beta, spec.zipf_s, int(spec.zipf_per_topic),
                         _ptr(cdf, ctypes.c_uint64), _ptr(mu, ctypes.c_double))
    if rc != 0:
        raise RuntimeError(f"tsyn_topics failed ({rc})")
    return cdf, mu


@dataclass
class Corpus:
    """CSR counts of documents doc0 .. doc0+n_docs-1: row d has the distinct
    words indices[indptr[d]:indptr[d+1]] (strictly ascending) with counts."""
    indptr: np.ndarray   # int64 [n_docs+1], starts at 0
    indices: np.ndarray  # int32 [nnz]
    counts: np.ndarray   # int32 [nnz], > 0
    lengths: np.ndarray  # int32 [n_docs], row sums of counts
    V: int

    @property
    def n_docs(self) -> int:
        return len(self.indptr) - 1

    @property
    def nnz(self) -> int:
        return int(self.indptr[-1])

    def rows(self, d0: int, d1: int) -> "Corpus":
        """Documents d0..d1-1 as a standalone CSR (indptr rebased to 0)."""
        a, b = int(self.indptr[d0]), int(self.indptr[d1])
        return Corpus(self.indptr[d0:d1 + 1] - a, self.indices[a:b], self.counts[a:b],
                      self.lengths[d0:d1], self.V)

    def dense(self) -> np.ndarray:
        """Dense int64 count matrix (small corpora only)."""
        F = np.zeros((self.n_docs, self.V), dtype=np.int64)
        rows = np.repeat(np.arange(self.n_docs), np.diff(self.indptr))
        F[rows, self.indices] = self.counts
        return F


def len_table(spec: CorpusSpec) -> np.ndarray:
    """The Poisson length table the generator draws document lengths from
    (uint64, 2^32-scaled CDF; the last entry is 2^32)."""
    lib = _load()
    out = np.zeros(4096, dtype=np.uint64)
    n = lib.tsyn_len_table(float(spec.lam), 4096, _ptr(out, ctypes.c_uint64))
    if n < 0:
        raise ValueError("length table out of range")
    return out[:n].copy()


def corpus(spec: CorpusSpec, doc0: int = 0, n_docs: int | None = None, cdf=None,
           nthreads: int | None = None) -> Corpus:
    """Documents doc0 .. doc0+n_docs-1 of the workload (same documents whatever
    the range or thread count: each document has its own counter)."""
    lib = _load()
    if n_docs is None:
        n_docs = spec.n_docs - doc0
    if cdf is None:
        cdf, _ = topics(spec)
    cdf = np.ascontiguousarray(cdf, dtype=np.uint64)
    if nthreads is None:
        nthreads = max(1, min(os.cpu_count() or 1, 64))
    a = Fraction(spec.alpha0)
    h = lib.tsyn_corpus_make(spec.seed, spec.V, spec.K, _ptr(cdf, ctypes.c_uint64),
                             a.numerator, a.denominator, spec.lam, spec.min_len,
                             int(doc0), int(n_docs), int(nthreads))
    if not h:
        raise RuntimeError("tsyn_corpus_make failed")
    try:
        nd = lib.tsyn_corpus_n_docs(h)
        nnz = lib.tsyn_corpus_nnz(h)
        indptr = np.zeros(nd + 1, dtype=np.int64)
        indices = np.zeros(nnz, dtype=np.int32)
        counts = np.zeros(nnz, dtype=np.int32)
        lengths = np.zeros(nd, dtype=np.int32)
        lib.tsyn_corpus_copy(h, _ptr(indptr, ctypes.c_int64), _ptr(indices, ctypes.c_int32),
                             _ptr(counts, ctypes.c_int32), _ptr(lengths, ctypes.c_int32))
    finally:
        lib.tsyn_corpus_free(h)
    return Corpus(indptr, indices, counts, lengths, spec.V)


def doc_tokens(spec: CorpusSpec, doc: int, cdf=None):
    """(topics, words) of one document in draw order (sampler tests)."""
    lib = _load()
    if cdf is None:
        cdf, _ = topics(spec)
    cdf = np.ascontiguousarray(cdf, dtype=np.uint64)
    cap = 8192
    z = np.zeros(cap, dtype=np.int32)
    w = np.zeros(cap, dtype=np.int32)
    a = Fraction(spec.alpha0)
    L = lib.tsyn_doc_tokens(spec.seed, spec.V, spec.K, _ptr(cdf, ctypes.c_uint64), a.numerator,
                            a.denominator, spec.lam, spec.min_len, int(doc), cap,
                            _ptr(z, ctypes.c_int32), _ptr(w, ctypes.c_int32))
    if L < 0:
        raise RuntimeError("tsyn_doc_tokens failed")
    return z[:L].copy(), w[:L].copy()


def batch_sizes(spec: CorpusSpec, n_docs: int | None = None) -> np.ndarray:
    """Seeded minibatch sizes, uniform on [bmin, bmax], covering n_docs."""
    lib = _load()
    n = spec.n_docs if n_docs is None else int(n_docs)
    bmin, bmax = spec.batch
    nb = lib.tsyn_batch_sizes(spec.seed, n, bmin, bmax, 0, None)
    out = np.zeros(max(nb, 1), dtype=np.int32)
    lib.tsyn_batch_sizes(spec.seed, n, bmin, bmax, nb, _ptr(out, ctypes.c_int32))
    return out[:nb]


def gaussian(seed: int, tag: int, n: int) -> np.ndarray:
    """n standard normals from stream `tag` of `seed`."""
    lib = _load()
    out = np.zeros(int(n), dtype=np.float64)
    lib.tsyn_gaussian(int(seed), int(tag), int(n), _ptr(out, ctypes.c_double))
    return out


def signs(seed: int, tag: int, n: int) -> np.ndarray:
    """n random signs (+1.0 or -1.0, each with probability 1/2) from stream
    `tag` of `seed`: the signs of its standard normals."""
    return np.where(gaussian(seed, tag, n) < 0.0, -1.0, 1.0)


def initial_factors(seed: int, k: int, K: int) -> np.ndarray:
    """Initial CP factors Phi0 (k x K) with entries N(0, 1/k), as FP32 values
    held in a float64 array (so both sides start from identical numbers)."""
    g = gaussian(seed, 7, k * K).reshape(k, K) / np.sqrt(k)
    return g.astype(np.float32).astype(np.float64)


def orthonormal_factors(seed: int, k: int, K: int) -> np.ndarray:
    """Initial CP factors with orthonormal columns (K <= k): the Q factor of
    the Gaussian start initial_factors(seed, k, K), each column's sign fixed
    so that the diagonal of R is positive, as FP32 values held in a float64
    array.  A start whose columns point in distinct directions, as the
    whitened topics do."""
    g = initial_factors(seed, k, K)
    q, r = np.linalg.qr(g)
    q = q * np.sign(np.diag(r))[None, :]
    return q.astype(np.float32).astype(np.float64)
