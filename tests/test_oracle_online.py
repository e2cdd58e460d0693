"""Pins of the oracle's fully online mode (section "Fully Online
Implementation"; readings P and Q): the one-pass sketch of the pair counts,
the whitening built from it, the carrying of factors into a new whitened
basis and the blocked online pass.  Each is tied to an independent fact:
dense pair counts (themselves pinned by brute force over token pairs),
exactness of the single-pass eigendecomposition for low-rank and fully
sketched (also indefinite) matrices, invariance of the recovered topics,
and reduction of the online pass to the batched pipeline when one block
covers everything."""
from __future__ import annotations

import numpy as np
import pytest

import tlda_synth as ts
from oracle import tlda_oracle as O

from .test_oracle_pins import _rand_csr, _rel


def _omega(V, r, tag=0):
    return ts.gaussian(0x5EED, 0x4F4D + tag, V * r).reshape(V, r)


def test_sketch_accumulates_the_pair_counts():
    rng = np.random.default_rng(3)
    V, r = 40, 9
    indptr, indices, counts, _ = _rand_csr(rng, 60, V, 12)
    Om = _omega(V, r)
    # two batches summed = the sketch of the whole corpus = dense P @ Omega
    Z = (O.sketch_accumulate(indptr[:31], indices, counts, V, Om)
         + O.sketch_accumulate(indptr[30:], indices, counts, V, Om))
    P = O.pair_counts(indptr, indices, counts, V)
    assert _rel(Z, P @ Om) < 1e-13


def test_sketch_with_a_sign_test_matrix_is_exact():
    """With entries of +-1 every sum of the sketch is an integer: the oracle's
    FP64 sketch equals the integer pair counts times Omega bit for bit (the
    premise of the device tests that compare the two for equality)."""
    rng = np.random.default_rng(5)
    V, r = 50, 12
    indptr, indices, counts, _ = _rand_csr(rng, 80, V, 15)
    Om = ts.signs(0x5EED, 0x4F4D, V * r).reshape(V, r)
    assert set(np.unique(Om)) == {-1.0, 1.0}
    Z = O.sketch_accumulate(indptr, indices, counts, V, Om)
    P = O.pair_counts(indptr, indices, counts, V).astype(np.int64)
    exact = P @ Om.astype(np.int64)
    assert np.array_equal(Z, exact.astype(np.float64))


def test_sketched_m2_equals_dense_m2_times_omega():
    rng = np.random.default_rng(4)
    V, r, a0 = 30, 7, 1.5
    indptr, indices, counts, _ = _rand_csr(rng, 50, V, 10, minlen=3)
    Om = _omega(V, r, 1)
    st = O.ingest(indptr, indices, counts, V)
    Z = O.sketch_accumulate(indptr, indices, counts, V, Om)
    M1 = O.first_moment(st["C"], st["T"])
    M2 = O.second_moment(O.pair_counts(indptr, indices, counts, V), st["S2"], M1, a0)
    Y = (a0 + 1.0) / st["S2"] * Z - a0 * np.outer(M1, M1 @ Om)
    assert _rel(Y, M2 @ Om) < 1e-12


@pytest.mark.parametrize("case", ["low_rank", "full_sketch"])
def test_sketch_eigenpairs_are_exact_when_the_sketch_captures_the_range(case):
    """Rank(A) <= r (population M2, rank K), or r = V for an indefinite A:
    the sketch's pairs are A's own top-k eigenpairs."""
    sp = ts.WORKLOADS["small_v500_k10"]
    _, mu = ts.topics(sp)
    K = sp.K
    h = np.full(K, 1.0 / K)
    if case == "low_rank":
        M1, A = O.population_moments(mu, h)
        r = K + 6
    else:
        rng = np.random.default_rng(5)
        V = 60
        X = rng.standard_normal((V, V))
        A = X @ X.T / V - 0.3 * np.eye(V)  # indefinite
        r, K = V, 8
    V = A.shape[0]
    Om = _omega(V, r, 2)
    U, lam = O.sketch_eigenpairs(A @ Om, Om, K)
    W, Ue, lam_e = O.whitening(A, K)
    assert np.allclose(lam, lam_e, rtol=1e-7)
    assert _rel(U @ U.T, Ue @ Ue.T) < 1e-6          # same subspace
    assert _rel(U, Ue) < 1e-6                        # same signed vectors (reading J)


def test_rotated_factors_encode_the_same_topics():
    rng = np.random.default_rng(6)
    V, k, K = 50, 6, 5
    W0 = rng.standard_normal((V, k))
    R, _ = np.linalg.qr(rng.standard_normal((k, k)))
    S = np.diag(rng.uniform(0.5, 2.0, k))
    W1 = W0 @ R @ S + 1e-3 * rng.standard_normal((V, k))   # a new basis, slightly different subspace
    Phi = rng.standard_normal((k, K))
    assert _rel(O.rotate_factors(Phi, W0, W0), Phi) < 1e-12
    # exactly the same subspace: the encoded topics (pinv(W^T) phi) are unchanged
    W2 = W0 @ R @ S
    P2 = O.rotate_factors(Phi, W0, W2)
    assert _rel(O.pinv_transpose(W2) @ P2, O.pinv_transpose(W0) @ Phi) < 1e-10
    # a different subspace: the topics move by their projection only
    P1 = O.rotate_factors(Phi, W0, W1)
    assert _rel(O.pinv_transpose(W1) @ P1, O.pinv_transpose(W0) @ Phi) < 1e-2


def test_online_pass_with_one_block_and_full_sketch_is_the_batched_pipeline():
    """every = all batches and r = V: the online pass whitens once, exactly
    (O3 + O4), then takes the CP steps in order."""
    rng = np.random.default_rng(7)
    V, k, a0, lr = 40, 4, 1.0, 0.01
    indptr, indices, counts, _ = _rand_csr(rng, 90, V, 14, minlen=3)
    offs = [0, 30, 55, 90]
    Om = _omega(V, V, 3)
    Phi0 = rng.standard_normal((k, k)) / np.sqrt(k)
    P_on, state, losses = O.online_pass(indptr, indices, counts, V, offs, Om, 3, a0, 0.0, lr, Phi0, k)
    st = O.ingest(indptr, indices, counts, V)
    M1 = O.first_moment(st["C"], st["T"])
    M2 = O.second_moment(O.pair_counts(indptr, indices, counts, V), st["S2"], M1, a0)
    W, _, _ = O.whitening(M2, k)
    m1 = W.T @ M1
    assert _rel(state["W"], W) < 1e-6
    P = Phi0.copy()
    for b in range(3):
        r = indptr[offs[b]:offs[b + 1] + 1]
        P, _ = O.cp_step(r, indices, counts, V, W, m1, P, lr, a0, 0.0)
    assert _rel(P_on, P) < 1e-5


def test_online_pass_blocks_compose():
    """Two calls of one block each, with the state carried, equal one call
    with blocks of one batch (the paper's per-batch order)."""
    rng = np.random.default_rng(8)
    V, k, a0, lr = 40, 4, 1.0, 0.01
    indptr, indices, counts, _ = _rand_csr(rng, 80, V, 14, minlen=3)
    offs = [0, 40, 80]
    Om = _omega(V, 12, 4)
    Phi0 = rng.standard_normal((k, k)) / np.sqrt(k)
    Pa, _, la = O.online_pass(indptr, indices, counts, V, offs, Om, 1, a0, 0.0, lr, Phi0, k)
    Pb, st, lb1 = O.online_pass(indptr, indices, counts, V, offs[:2], Om, 1, a0, 0.0, lr, Phi0, k)
    Pb, st, lb2 = O.online_pass(indptr, indices, counts, V, offs[1:], Om, 1, a0, 0.0, lr, Pb, k, state=st)
    assert _rel(Pa, Pb) < 1e-12
    assert np.allclose(la, np.concatenate([lb1, lb2]), rtol=1e-12)
