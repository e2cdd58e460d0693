"""Pins of the oracle's batched mode (section "Batched Implementation Enables
Arbitrary Scaling"; reading R) and of the simulations' recovery score
(section "Parameter Recovery and Comparison to Previous TLDA Methods"),
against facts that do not come from the oracle: exhaustive search over
matchings with numpy's own correlation routine, the invariance of Pearson
correlation under positive affine maps, and the closed-form stationary point
Phi = 0 of the CP objective (zero gradient, zero loss)."""
from __future__ import annotations

import itertools

import numpy as np

import tlda_synth as ts
from oracle import tlda_oracle as O


def test_topic_correlation_equals_exhaustive_search():
    rng = np.random.default_rng(11)
    for K in (2, 3, 4):
        mu_true = rng.dirichlet(np.full(30, 0.3), size=K)             # K x V
        mu_est = rng.dirichlet(np.full(30, 0.3), size=K).T            # V x K
        best, best_perm = -np.inf, None
        for p in itertools.permutations(range(K)):
            tot = sum(np.corrcoef(mu_true[i], mu_est[:, p[i]])[0, 1] for i in range(K))
            if tot > best:
                best, best_perm = tot, p
        perm, corr = O.topic_correlation(mu_est, mu_true)
        assert tuple(perm) == best_perm
        ref = [np.corrcoef(mu_true[i], mu_est[:, best_perm[i]])[0, 1] for i in range(K)]
        assert np.allclose(corr, ref, rtol=0, atol=1e-12)


def test_topic_correlation_invariances():
    rng = np.random.default_rng(12)
    K, V = 3, 40
    mu_true = rng.dirichlet(np.full(V, 0.5), size=K)
    order = np.array([2, 0, 1])
    # learned column j = a_j * (true topic order[j]) + b_j with a_j > 0: correlation exactly 1
    a, b = np.array([0.5, 3.0, 1.7]), np.array([0.01, -0.2, 0.0])
    mu_est = (mu_true[order] * a[:, None] + b[:, None]).T
    perm, corr = O.topic_correlation(mu_est, mu_true)
    assert np.array_equal(order[perm], np.arange(K))
    assert np.allclose(corr, 1.0, atol=1e-12)
    # a constant learned column scores 0
    mu_est[:, 1] = 1.0 / V
    _, corr = O.topic_correlation(mu_est, mu_true)
    assert np.isclose(np.sort(corr)[0], 0.0, atol=1e-12)


def test_batched_fit_keeps_the_lowest_loss_start():
    """Starts: Phi = 0 (a stationary point: zero gradient, zero loss at every
    step), the population factors (negative loss) and a NaN matrix (never
    kept)."""
    sp = ts.e1_spec(60, 0).with_docs(3000)
    cdf, mu = ts.topics(sp)
    c = ts.corpus(sp, cdf=cdf)
    offs = [0, 1000, 2000, 3000]
    h = np.full(sp.K, 1.0 / sp.K)
    _, W, m1, _, _ = O.batched_fit(c.indptr, c.indices, c.counts, sp.V, offs[:2], 1, float(sp.alpha0), 0.0,
                                   0.0, [np.zeros((2, 2))], 2)
    P_pop = O.population_factors(mu, h, W)
    starts = [np.zeros((2, 2)), P_pop, np.full((2, 2), np.nan)]
    P, W2, _, means, finals = O.batched_fit(c.indptr, c.indices, c.counts, sp.V, offs, 2, float(sp.alpha0),
                                            0.0, 1e-3, starts, 2)
    assert np.array_equal(W2, W)
    assert means[0] == 0.0 and np.array_equal(finals[0], np.zeros((2, 2)))
    assert means[1] < 0.0 and np.isnan(means[2])
    assert np.array_equal(P, finals[1])
    _, corr = O.topic_correlation(O.unwhiten_cp(P, W)[0], mu)
    assert corr.min() > 0.95
