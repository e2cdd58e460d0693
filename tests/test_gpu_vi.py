"""Document-topic variational inference (tlda_doc_topics) against the FP64
oracle (section "Input and Output"; the E-step of Blei, Ng and Jordan 2003):
theta and gamma on the small and the streaming workload's ground-truth
topics, K not a multiple of 32 and K up to 300, the degenerate cases (one
topic, zero iterations, an empty document, a word no topic uses) and a
corrupt document."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import tlda_synth as ts
from oracle import tlda_oracle as O

from . import _cases as C

pytestmark = pytest.mark.gpu
TOL = 1e-5


def _check(lib, c, V, mu, alpha, n_iter, tol=TOL):
    # the kernel reads FP32 topics and weights: the oracle gets the same values
    # (which rows are all zero, a decision of the precision, is then the same too)
    mu = np.asarray(mu).astype(np.float32).astype(np.float64)
    alpha = np.asarray(alpha).astype(np.float32).astype(np.float64)
    dev = lib.DeviceCSR.from_arrays(c.indptr, c.indices, c.counts, V)
    theta, gamma = lib.doc_topics(dev, mu, alpha, n_iter, want_gamma=True)
    th_o, ga_o = O.doc_topics(c.indptr, c.indices, c.counts, V, mu, alpha, n_iter)
    assert C.rel(theta.cpu().numpy(), th_o) < tol
    assert C.rel(gamma.cpu().numpy(), ga_o) < tol
    return theta.cpu().numpy(), th_o


@pytest.mark.parametrize("name,n_docs,n_iter", [("small_v500_k10", 2000, 20), ("stream_v20k_k100", 3000, 30)])
def test_doc_topics_match_oracle(lib, name, n_docs, n_iter):
    sp = ts.WORKLOADS[name]
    _, mu = C.topics(name)
    c = C.corpus(name, n_docs)
    alpha = np.full(sp.K, float(sp.alpha0) / sp.K)
    _check(lib, c, sp.V, mu.T.copy(), alpha, n_iter)


def test_doc_topics_wide_k_and_degenerate_cases(lib):
    rng = np.random.default_rng(5)
    V, K = 1000, 300
    mu = rng.dirichlet(np.full(V, 0.05), size=K).T.copy()
    mu[7] = 0.0                                     # a word no topic uses
    alpha = rng.uniform(0.01, 0.5, size=K)
    rows, idx, cnt = [0], [], []
    for d in range(200):
        L = 0 if d == 3 else int(rng.integers(1, 60))  # document 3 is empty
        w = np.sort(rng.choice(V, size=L, replace=False))
        if d == 5 and 7 not in w:
            w = np.sort(np.append(w, 7))
        idx += list(w)
        cnt += list(rng.integers(1, 4, size=len(w)))
        rows.append(len(idx))
    c = ts.Corpus(np.array(rows, dtype=np.int64), np.array(idx, dtype=np.int32), np.array(cnt, dtype=np.int32),
                  None, V)
    theta, _ = _check(lib, c, V, mu, alpha, 25)
    assert np.allclose(theta[3], alpha / alpha.sum(), rtol=1e-6)
    _check(lib, c, V, mu, alpha, 0)                 # n_iter = 0: theta from the initial gamma
    one, _ = _check(lib, c, V, mu[:, :1].copy(), alpha[:1], 5)
    assert np.allclose(one, 1.0, rtol=0, atol=1e-7)   # one topic


def test_doc_topics_flags_a_corrupt_document(lib):
    sp = ts.WORKLOADS["small_v500_k10"]
    _, mu = C.topics("small_v500_k10")
    c = C.corpus("small_v500_k10", 50)
    counts = c.counts.copy()
    counts[c.indptr[10] + 2] = 0
    dev = lib.DeviceCSR.from_arrays(c.indptr, c.indices, counts, sp.V)
    with pytest.raises(lib.TLDAError) as e:
        lib.doc_topics(dev, mu.T.copy(), np.full(sp.K, 0.1), 5)
    assert e.value.status == lib.ERR_INVALID
