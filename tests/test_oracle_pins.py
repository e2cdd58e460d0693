"""Pins of the FP64 oracle against facts that do not come from the oracle
itself: brute-force enumeration of token pairs/triples, Theorem 1 at constant
document length, population closed forms, the orthogonal-tensor special case,
finite differences and estimator unbiasedness.  CPU only."""
import itertools
from fractions import Fraction

import numpy as np
import pytest

import tlda_synth as ts
from oracle import tlda_oracle as O


def _rand_csr(rng, B, V, maxlen, minlen=0):
    """Random tiny CSR built from explicit token lists (also returned)."""
    docs, indptr, indices, counts = [], [0], [], []
    for _ in range(B):
        L = int(rng.integers(minlen, maxlen + 1))
        toks = rng.integers(0, V, size=L)
        docs.append(list(toks))
        w, c = np.unique(toks, return_counts=True)
        indices += list(w)
        counts += list(c)
        indptr.append(len(indices))
    return (np.array(indptr, dtype=np.int64), np.array(indices, dtype=np.int32),
            np.array(counts, dtype=np.int32), docs)


def _rel(a, b):
    return np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


# ----------------------------------------------------------------------------- generator
def test_philox_known_answers():
    # Known-answer vectors published with Random123 (Salmon et al., SC'11).
    assert [hex(x) for x in ts.philox4x32_10([0, 0, 0, 0], [0, 0])] == \
        ["0x6627e8d5", "0xe169c58d", "0xbc57ac4c", "0x9b00dbd8"]
    assert [hex(x) for x in ts.philox4x32_10([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2)] == \
        ["0x408f276d", "0x41c83b0e", "0xa20bc7c6", "0x6d5451fd"]
    assert [hex(x) for x in ts.philox4x32_10([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344],
                                             [0xA4093822, 0x299F31D0])] == \
        ["0xd16cfe09", "0x94fdcceb", "0x5001e420", "0x24126ea1"]


def test_generator_csr_and_determinism():
    sp = ts.WORKLOADS["small_v500_k10"].with_docs(3000)
    cdf, mu = ts.topics(sp)
    assert np.allclose(mu.sum(axis=1), 1.0, atol=0, rtol=0) or np.all(np.abs(mu.sum(1) - 1) < 1e-12)
    c = ts.corpus(sp, cdf=cdf, nthreads=4)
    O.validate_csr(c.indptr, c.indices, c.counts, sp.V)
    assert c.lengths.min() >= 3
    st = O.ingest(c.indptr, c.indices, c.counts, sp.V)
    assert np.array_equal(st["L"], c.lengths.astype(np.int64))
    assert abs(c.lengths.mean() - sp.lam) < 4 * np.sqrt(sp.lam / sp.n_docs) + 0.01
    c1 = ts.corpus(sp, doc0=777, n_docs=100, cdf=cdf, nthreads=1)
    sub = c.rows(777, 877)
    assert np.array_equal(c1.indices, sub.indices) and np.array_equal(c1.counts, sub.counts)
    # the CSR is the merged token stream of each document
    z, w = ts.doc_tokens(sp, 778, cdf=cdf)
    wu, wc = np.unique(w, return_counts=True)
    r = c.rows(778, 779)
    assert np.array_equal(r.indices, wu) and np.array_equal(r.counts, wc)


def test_generator_topic_marginal_is_dirichlet_multinomial():
    # Polya urn with weights alpha0/K + n_i: E[n_i] = L/K and
    # Var[n_i] = L p (1-p) (L + alpha0) / (1 + alpha0), p = 1/K.
    sp = ts.CorpusSpec("urn", 50, 4, 0.5, 0.0, Fraction(1, 2), 1e-3, 10, 4000, 1234, (1, 1))
    cdf, _ = ts.topics(sp)
    n0 = np.array([np.sum(ts.doc_tokens(sp, d, cdf=cdf)[0] == 0) for d in range(sp.n_docs)])
    L, p, a0 = 10, 0.25, 0.5
    assert abs(n0.mean() - L * p) < 4 * np.sqrt(n0.var() / sp.n_docs)
    var = L * p * (1 - p) * (L + a0) / (1 + a0)
    assert abs(n0.var() / var - 1.0) < 0.1


# ----------------------------------------------------------------------------- ingest / pairs / triples
def test_ingest_and_pairs_brute_force():
    rng = np.random.default_rng(1)
    V = 6
    indptr, indices, counts, docs = _rand_csr(rng, 40, V, 8)
    st = O.ingest(indptr, indices, counts, V)
    P = O.pair_counts(indptr, indices, counts, V)
    Pb = np.zeros((V, V), dtype=np.int64)
    S2 = S3 = 0
    for toks in docs:
        L = len(toks)
        for a, b in itertools.permutations(range(L), 2):
            Pb[toks[a], toks[b]] += 1
            S2 += 1
        S3 += sum(1 for _ in itertools.permutations(range(L), 3))
    assert np.array_equal(P, Pb)
    assert st["S2"] == S2 and st["S3"] == S3
    assert st["T"] == sum(len(t) for t in docs)
    assert np.array_equal(st["C"], np.bincount(np.concatenate([t for t in docs if t] or [[]]).astype(int),
                                               minlength=V))


def test_centred_triples_brute_force():
    rng = np.random.default_rng(2)
    V, k = 7, 3
    indptr, indices, counts, docs = _rand_csr(rng, 25, V, 7)
    W = rng.standard_normal((V, k))
    m1 = rng.standard_normal(k)
    U = W - m1
    C3, S3 = O.centred_triples(indptr, indices, counts, V, W, m1)
    acc = np.zeros((k, k, k))
    n = 0
    for toks in docs:
        for a, b, c in itertools.permutations(range(len(toks)), 3):
            acc += O.sym3(U[toks[a]], U[toks[b]], U[toks[c]])
            n += 1
    assert n == S3
    assert _rel(C3, acc / n) < 1e-12


def test_short_documents_carry_no_triples():
    rng = np.random.default_rng(3)
    V, k = 9, 4
    indptr, indices, counts, _ = _rand_csr(rng, 30, V, 2)
    W = rng.standard_normal((V, k))
    m1 = rng.standard_normal(k)
    C3, S3 = O.centred_triples(indptr, indices, counts, V, W, m1)
    assert S3 == 0 and np.all(C3 == 0)
    Phi = rng.standard_normal((k, 3))
    g = O.cp_grad_implicit(indptr, indices, counts, V, W, m1, Phi, 1.0, 0.0)
    assert np.all(g["grad"] == 0) and g["loss"] == 0.0


def test_validate_rejects_corrupt_csr():
    V = 5
    ok = (np.array([0, 2, 3]), np.array([1, 3, 0]), np.array([1, 2, 1]))
    O.validate_csr(*ok, V)
    with pytest.raises(ValueError):
        O.validate_csr(np.array([0, 3, 2]), ok[1], ok[2], V)       # indptr decreasing
    with pytest.raises(ValueError):
        O.validate_csr(ok[0], np.array([1, 5, 0]), ok[2], V)       # index >= V
    with pytest.raises(ValueError):
        O.validate_csr(ok[0], np.array([3, 1, 0]), ok[2], V)       # not ascending
    with pytest.raises(ValueError):
        O.validate_csr(ok[0], ok[1], np.array([1, 0, 1]), V)       # count <= 0


# ----------------------------------------------------------------------------- Theorem 1
@pytest.mark.parametrize("alpha0", [Fraction(1), Fraction(2), Fraction(1, 100)])
def test_theorem1_centred_form_equals_uncentred_cumulant(alpha0):
    """At constant document length the centred batch tensor over the whole
    corpus equals the whitened uncentred cumulant (appendix M3 with the
    proof's alpha0 term) exactly, when W whitens the empirical M2."""
    sp = ts.CorpusSpec("const", 40, 4, 0.3, 0.0, alpha0, 1e-3, 6, 3000, 99, (1, 1))
    cdf, mu = ts.topics(sp)
    c = ts.corpus(sp, cdf=cdf)
    assert np.all(c.lengths == 6)
    a0 = float(alpha0)
    st = O.ingest(c.indptr, c.indices, c.counts, sp.V)
    M1 = O.first_moment(st["C"], st["T"])
    M2 = O.second_moment(O.pair_counts(c.indptr, c.indices, c.counts, sp.V), st["S2"], M1, a0)
    W, _, _ = O.whitening(M2, sp.K)
    assert _rel(W.T @ M2 @ W, np.eye(sp.K)) < 1e-12
    Tfull = O.whitened_third_moment(c.indptr, c.indices, c.counts, sp.V, W, M1, a0)
    TB = O.batch_tensor(c.indptr, c.indices, c.counts, sp.V, W, W.T @ M1, a0)
    assert _rel(TB, Tfull) < 1e-10


def test_population_moment_identities():
    """Theorem 1 / factorisation: with population moments, the centred
    cumulant sum_i h_i nu_i^(x)3 (nu = mu - M1) re-centred equals
    sum_i h_i mu_i^(x)3; and sum_i h_i nu_i = 0."""
    rng = np.random.default_rng(5)
    K, V = 4, 12
    mu = rng.dirichlet(np.full(V, 0.5), size=K)
    h = rng.dirichlet(np.ones(K))
    M1, M2 = O.population_moments(mu, h)
    nu = mu - M1[None, :]
    assert np.linalg.norm(h @ nu) < 1e-15
    lhs = np.einsum("k,ki,kj,kl->ijl", h, nu + M1, nu + M1, nu + M1)
    assert _rel(lhs, O.population_m3(mu, h)) < 1e-13
    assert _rel(M2, (mu.T * h) @ mu) < 1e-15


# ----------------------------------------------------------------------------- estimator
def test_estimators_are_unbiased():
    """Empirical M2 and whitened M3 converge to the population closed forms at
    the Monte-Carlo rate (4x documents -> about half the error).  A dropped or
    mis-scaled alpha0 term leaves a bias that does not shrink."""
    sp = ts.CorpusSpec("mc", 30, 3, 0.3, 0.0, Fraction(1), 20.0, 3, 160_000, 321, (1, 1))
    cdf, mu = ts.topics(sp)
    h = np.full(sp.K, 1.0 / sp.K)
    M1p, M2p = O.population_moments(mu, h)
    Wp, _ = O.population_whitening(mu, h)
    Tp = O.population_tensor(mu, h, Wp)
    errs = []
    for n in (10_000, 40_000, 160_000):
        c = ts.corpus(sp.with_docs(n), cdf=cdf)
        st = O.ingest(c.indptr, c.indices, c.counts, sp.V)
        M1 = O.first_moment(st["C"], st["T"])
        M2 = O.second_moment(O.pair_counts(c.indptr, c.indices, c.counts, sp.V), st["S2"], M1, 1.0)
        T = O.whitened_third_moment(c.indptr, c.indices, c.counts, sp.V, Wp, M1, 1.0)
        errs.append((_rel(M2, M2p), _rel(T, Tp)))
    e = np.array(errs)
    assert e[-1, 0] < 0.02 and e[-1, 1] < 0.05
    for j in range(2):
        assert e[1, j] < 0.75 * e[0, j], e   # 4x docs: ~1/2 the error
        assert e[2, j] < 0.40 * e[0, j], e   # 16x docs: ~1/4 the error


# ----------------------------------------------------------------------------- whitening
def test_whitening_invariants_and_library_cross_check():
    sp = ts.WORKLOADS["small_v500_k10"].with_docs(4000)
    cdf, _ = ts.topics(sp)
    c = ts.corpus(sp, cdf=cdf)
    st = O.ingest(c.indptr, c.indices, c.counts, sp.V)
    M1 = O.first_moment(st["C"], st["T"])
    M2 = O.second_moment(O.pair_counts(c.indptr, c.indices, c.counts, sp.V), st["S2"], M1, 1.0)
    W, Uk, lam = O.whitening(M2, sp.K)
    assert _rel(W.T @ M2 @ W, np.eye(sp.K)) < 1e-11
    assert np.all(np.diff(lam) <= 0)
    res = np.linalg.norm(M2 @ Uk - Uk * lam[None, :], axis=0)
    assert np.all(res <= 1e-10 * lam[0])
    assert _rel(Uk.T @ Uk, np.eye(sp.K)) < 1e-12


# ----------------------------------------------------------------------------- power method / recovery
def _population_case(K=5, V=60, seed=7):
    rng = np.random.default_rng(seed)
    mu = rng.dirichlet(np.full(V, 0.3), size=K)
    h = np.sort(rng.dirichlet(np.full(K, 3.0)))
    return mu, h


def test_power_method_recovers_population_topics():
    mu, h = _population_case()
    W, _ = O.population_whitening(mu, h)
    T = O.population_tensor(mu, h, W)
    lams, vecs = O.tensor_power_method(T, len(h), n_restarts=10, n_iters=60, seed=0)
    assert np.allclose(np.sort(lams), np.sort(h ** -0.5), rtol=1e-10)
    mu_est, h_est = O.unwhiten_power(lams, vecs, W)
    perm, l1, _ = O.match_topics(mu_est, mu)
    assert np.max(l1) < 1e-8
    assert np.allclose(h_est[perm], h, atol=1e-10)


def test_population_factors_are_stationary_and_unwhiten():
    mu, h = _population_case(K=4, V=40, seed=11)
    W, m1 = O.population_whitening(mu, h)
    T = O.population_tensor(mu, h, W)
    Phi = O.population_factors(mu, h, W)
    g = O.cp_grad_explicit(Phi, T, 0.0)
    assert np.linalg.norm(g) < 1e-10 * np.linalg.norm(Phi) ** 5
    assert np.allclose(np.linalg.norm(Phi, axis=0), h ** (-1 / 6), rtol=1e-12)
    mu_est, a = O.unwhiten_cp(Phi, W)
    assert _rel(mu_est, mu.T) < 1e-10
    assert np.allclose(a, h, rtol=1e-10)


# ----------------------------------------------------------------------------- gradient
def _grad_case(seed, V=25, k=5, K=4, B=30, maxlen=9):
    rng = np.random.default_rng(seed)
    indptr, indices, counts, _ = _rand_csr(rng, B, V, maxlen)
    W = rng.standard_normal((V, k))
    m1 = rng.standard_normal(k) * 0.3
    Phi = rng.standard_normal((k, K))
    return indptr, indices, counts, V, W, m1, Phi


@pytest.mark.parametrize("seed,k,K", [(0, 5, 4), (1, 4, 4), (2, 6, 2)])
@pytest.mark.parametrize("alpha0,theta", [(1.0, 0.0), (2.0, 0.5), (0.01, 0.0)])
def test_implicit_gradient_equals_explicit_tensor(seed, k, K, alpha0, theta):
    indptr, indices, counts, V, W, m1, Phi = _grad_case(seed, k=k, K=K)
    g = O.cp_grad_implicit(indptr, indices, counts, V, W, m1, Phi, alpha0, theta)
    TB = O.batch_tensor(indptr, indices, counts, V, W, m1, alpha0)
    assert _rel(g["grad"], O.cp_grad_explicit(Phi, TB, theta)) < 1e-12
    assert abs(g["loss"] - O.cp_loss_explicit(Phi, TB, theta)) < 1e-10 * max(1, abs(g["loss"]))


def test_implicit_gradient_without_same_token_terms():
    indptr, indices, counts, V, W, m1, Phi = _grad_case(4)
    a0 = 1.0
    g = O.cp_grad_implicit(indptr, indices, counts, V, W, m1, Phi, a0, 0.0, same_token=False)
    F = O.csr_matrix(indptr, indices, counts, V)
    X = F @ (W - m1)
    S3 = O.ingest(indptr, indices, counts, V)["S3"]
    k = W.shape[1]
    c3 = (a0 + 1) * (a0 + 2) / 2
    T = (c3 / S3 * np.einsum("di,dj,dl->ijl", X, X, X) + O.perm3(np.eye(k), m1)
         - 2 * O.sym3(m1, m1, m1))
    assert _rel(g["grad"], O.cp_grad_explicit(Phi, T, 0.0)) < 1e-12


def test_gradient_matches_finite_differences():
    indptr, indices, counts, V, W, m1, Phi = _grad_case(9)
    a0, theta = 1.5, 0.25
    g = O.cp_grad_implicit(indptr, indices, counts, V, W, m1, Phi, a0, theta)["grad"]
    eps = 1e-6
    fd = np.zeros_like(Phi)
    for i in range(Phi.shape[0]):
        for j in range(Phi.shape[1]):
            P1, P2 = Phi.copy(), Phi.copy()
            P1[i, j] += eps
            P2[i, j] -= eps
            l1 = O.cp_grad_implicit(indptr, indices, counts, V, W, m1, P1, a0, theta)["loss"]
            l2 = O.cp_grad_implicit(indptr, indices, counts, V, W, m1, P2, a0, theta)["loss"]
            fd[i, j] = (l1 - l2) / (2 * eps)
    assert _rel(fd, g) < 1e-6


def test_grad_is_sum_over_documents():
    """The data term is additive over documents (the basis of sharding a
    batch): G_data(A u B) S3(A u B) = G1G2(A) + G1G2(B) in the c3/S3 scaling."""
    indptr, indices, counts, V, W, m1, Phi = _grad_case(12, B=40)
    full = O.cp_grad_implicit(indptr, indices, counts, V, W, m1, Phi, 1.0, 0.0)
    h = 17
    a = O.cp_grad_implicit(indptr[:h + 1], indices, counts, V, W, m1, Phi, 1.0, 0.0)
    b = O.cp_grad_implicit(indptr[h:], indices, counts, V, W, m1, Phi, 1.0, 0.0)
    assert a["S3"] + b["S3"] == full["S3"]
    assert _rel(a["G1"] + a["G2"] + b["G1"] + b["G2"], full["G1"] + full["G2"]) < 1e-12


def test_chunked_third_moment_equals_einsum_form():
    """whitened_third_moment_chunked adds the same sums in chunks (ragged last
    chunk) and maps the pair counts through W without forming them: equal to
    whitened_third_moment to rounding, for a D > K whitening too."""
    sp = ts.WORKLOADS["small_v500_k10"]
    cdf, _ = ts.topics(sp)
    c = ts.corpus(sp.with_docs(2500), cdf=cdf)
    st = O.ingest(c.indptr, c.indices, c.counts, sp.V)
    M1 = O.first_moment(st["C"], st["T"])
    M2 = O.second_moment(O.pair_counts(c.indptr, c.indices, c.counts, sp.V), st["S2"], M1, 1.0)
    for k in (10, 13):
        W, _, _ = O.whitening(M2, k)
        T1 = O.whitened_third_moment(c.indptr, c.indices, c.counts, sp.V, W, M1, 1.0)
        T2 = O.whitened_third_moment_chunked(c.indptr, c.indices, c.counts, sp.V, W, M1, 1.0, chunk=333)
        assert np.abs(T1 - T2).max() <= 1e-12 * np.abs(T1).max()
