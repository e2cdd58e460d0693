"""Pins of the oracle's document-topic variational inference (section "Input
and Output"; the E-step of Blei, Ng and Jordan 2003) against facts that do
not come from its update formulas: closed forms (one topic; topics with
disjoint word supports; an empty document), the evidence lower bound of the
paper's appendix A.3 equal to the exact log-evidence at K = 1 and below the
exact log-evidence (summed over every topic assignment) otherwise, and each
half of the update being a local maximum of that bound."""
from __future__ import annotations

import itertools
import math

import numpy as np
import scipy.special

from oracle import tlda_oracle as O


def _doc(rng, V, n):
    m = np.sort(rng.choice(V, size=n, replace=False))
    f = rng.integers(1, 4, size=n)
    return np.array([0, n]), m.astype(np.int32), f.astype(np.int32)


def test_single_topic_closed_form():
    rng = np.random.default_rng(1)
    V = 20
    mu = rng.dirichlet(np.ones(V))[:, None]
    indptr, m, f = _doc(rng, V, 6)
    theta, gamma = O.doc_topics(indptr, m, f, V, mu, np.array([0.7]), 5)
    assert theta[0, 0] == 1.0 and np.isclose(gamma[0, 0], 0.7 + f.sum(), rtol=1e-15)
    # K = 1: the bound is the exact log-evidence sum_j f_j log mu_{m_j}
    elbo = O.doc_elbo(f.astype(float), mu[m], np.array([0.7]), gamma[0], np.ones((len(m), 1)))
    assert np.isclose(elbo, float(f @ np.log(mu[m, 0])), rtol=1e-12)


def test_disjoint_topic_supports_closed_form():
    """Each word belongs to one topic: phi is that topic whatever gamma is, so
    gamma_k = alpha_k + the document's counts of topic k's words."""
    rng = np.random.default_rng(2)
    V, K = 30, 3
    owner = rng.integers(0, K, size=V)
    mu = np.zeros((V, K))
    for k in range(K):
        w = owner == k
        mu[w, k] = rng.dirichlet(np.ones(w.sum()))
    alpha = np.array([0.1, 0.5, 2.0])
    indptr = np.array([0, 7, 7, 12])
    idx = np.concatenate([np.sort(rng.choice(V, 7, replace=False)), np.sort(rng.choice(V, 5, replace=False))])
    cnt = rng.integers(1, 5, size=12)
    _, gamma = O.doc_topics(indptr, idx.astype(np.int32), cnt.astype(np.int32), V, mu, alpha, 3)
    for d, (lo, hi) in enumerate([(0, 7), (7, 7), (7, 12)]):
        want = alpha + np.bincount(owner[idx[lo:hi]], weights=cnt[lo:hi], minlength=K)
        assert np.allclose(gamma[d], want, rtol=1e-14)   # the empty document keeps alpha


def _log_evidence(tokens, mu, alpha):
    """log p(w | alpha, mu) by summing over every topic assignment (Dirichlet-
    multinomial marginal of the assignments)."""
    K, N = mu.shape[1], len(tokens)
    tot = -np.inf
    for z in itertools.product(range(K), repeat=N):
        n = np.bincount(z, minlength=K)
        lp = (math.lgamma(alpha.sum()) - math.lgamma(alpha.sum() + N)
              + sum(math.lgamma(alpha[k] + n[k]) - math.lgamma(alpha[k]) for k in range(K))
              + sum(math.log(mu[w, k]) for w, k in zip(tokens, z)))
        tot = np.logaddexp(tot, lp)
    return tot


def test_bound_below_exact_evidence_and_non_decreasing():
    rng = np.random.default_rng(3)
    V, K = 12, 2
    mu = rng.dirichlet(np.full(V, 0.5), size=K).T
    alpha = np.array([0.3, 0.8])
    m = np.array([1, 4, 7, 9])
    f = np.array([2, 1, 3, 1], dtype=float)
    tokens = np.repeat(m, f.astype(int))
    logp = _log_evidence(tokens, mu, alpha)
    rows = mu[m]
    g = alpha + f.sum() / K
    prev = -np.inf
    for _ in range(30):
        phi, g = O.vi_update(f, rows, alpha, g)
        b = O.doc_elbo(f, rows, alpha, g, phi)
        assert b >= prev - 1e-12 and b <= logp + 1e-12
        prev = b
    assert logp - prev < 0.5  # a tight bound for this short document


def test_each_half_update_is_a_local_maximum_of_the_bound():
    rng = np.random.default_rng(4)
    V, K = 15, 4
    mu = rng.dirichlet(np.full(V, 0.4), size=K).T
    alpha = rng.uniform(0.2, 1.5, size=K)
    m = np.array([0, 3, 5, 8, 13])
    f = np.array([1, 2, 1, 4, 1], dtype=float)
    rows = mu[m]
    g0 = alpha + f.sum() / K + rng.uniform(0, 1, size=K)
    phi, g1 = O.vi_update(f, rows, alpha, g0)
    base_phi = O.doc_elbo(f, rows, alpha, g0, phi)   # phi maximises the bound at gamma = g0
    base_g = O.doc_elbo(f, rows, alpha, g1, phi)     # g1 maximises it at this phi
    for _ in range(50):
        d = rng.normal(size=phi.shape)
        d -= d.mean(axis=1, keepdims=True)           # stays on each simplex
        p2 = phi + 1e-4 * d
        if (p2 > 0).all():
            assert O.doc_elbo(f, rows, alpha, g0, p2) <= base_phi + 1e-12
        g2 = g1 + 1e-4 * rng.normal(size=K)
        assert O.doc_elbo(f, rows, alpha, g2, phi) <= base_g + 1e-12
