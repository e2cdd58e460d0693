"""Parity of the CUDA path (called through the C ABI) with the FP64 oracle, on
seeded synthetic corpora.  Tolerances: relative Frobenius error 1e-5 for the
FP32 form; integer statistics bit-exact."""
import numpy as np
import pytest
import torch

import tlda_synth as ts
from oracle import tlda_oracle as O
from tests import _cases as C

pytestmark = pytest.mark.gpu

TOL32 = 1e-5
TOL16 = 2e-2


def _ctx(lib, name, precision="fp32", same_token=True, dim=0, theta=0.0, max_batch=8192, W=None):
    sp = ts.WORKLOADS[name]
    t = lib.TLDA(sp.V, sp.K, dim=dim, alpha0=float(sp.alpha0), theta=theta, precision=precision,
                 same_token=same_token, max_batch=max_batch)
    if W is None:
        W, m1 = C.population_whitening(name)
    else:
        W, m1 = W
    t.set_whitening(torch.tensor(W, dtype=torch.float32), torch.tensor(m1, dtype=torch.float32))
    return t, W, m1


def _phi0(sp, D=None):
    D = D or sp.K
    return ts.initial_factors(sp.seed + 1, D, sp.K)


def _oracle_grad(batch, sp, W, m1, Phi, theta=0.0, same_token=True):
    return O.cp_grad_implicit(batch.indptr, batch.indices, batch.counts, sp.V, W, m1, Phi,
                              float(sp.alpha0), theta, same_token)


# ----------------------------------------------------------------------------- whitening
@pytest.mark.parametrize("name,n", [("small_v500_k10", 1000), ("stream_v20k_k100", 3001)])
def test_whiten_batch(lib, name, n):
    sp = ts.WORKLOADS[name]
    t, W, m1 = _ctx(lib, name)
    c = C.corpus(name, n)
    X = t.whiten_batch(lib.DeviceCSR.from_corpus(c)).cpu().numpy()
    F = O.csr_matrix(c.indptr, c.indices, c.counts, sp.V)
    Xo = F @ W - c.lengths[:, None].astype(np.float64) * m1[None, :]
    assert C.rel(X, Xo) < TOL32
    t.sync()


# ----------------------------------------------------------------------------- data term / step
@pytest.mark.parametrize("name,n", [("small_v500_k10", 1000), ("small_v500_k10", 37),
                                    ("tweet_v5k_k50", 2048), ("stream_v20k_k100", 4099)])
def test_data_term_fp32(lib, name, n):
    sp = ts.WORKLOADS[name]
    t, W, m1 = _ctx(lib, name)
    c = C.corpus(name, n)
    Phi = _phi0(sp)
    G, S3 = t.cp_data_term(lib.DeviceCSR.from_corpus(c), torch.tensor(Phi, dtype=torch.float32, device="cuda"))
    g = _oracle_grad(c, sp, W, m1, Phi)
    assert S3 == g["S3"]
    assert C.rel(G.cpu().numpy(), g["G_data"]) < TOL32


@pytest.mark.parametrize("theta", [0.0, 0.5])
@pytest.mark.parametrize("same_token", [True, False])
def test_cp_step_fp32(lib, theta, same_token):
    name = "small_v500_k10"
    sp = ts.WORKLOADS[name]
    t, W, m1 = _ctx(lib, name, theta=theta, same_token=same_token)
    c = C.corpus(name, 1000)
    Phi0 = _phi0(sp)
    Phi = torch.tensor(Phi0, dtype=torch.float32, device="cuda")
    grad = torch.empty_like(Phi)
    lr = 0.01
    loss = t.cp_step(lib.DeviceCSR.from_corpus(c), Phi, lr, grad=grad, want_loss=True)
    g = _oracle_grad(c, sp, W, m1, Phi0, theta, same_token)
    assert C.rel(grad.cpu().numpy(), g["grad"]) < TOL32
    assert C.rel(Phi.cpu().numpy(), Phi0 - lr * g["grad"]) < TOL32
    assert abs(loss - g["loss"]) <= TOL32 * abs(g["loss"])


def test_ragged_and_tiny_batches(lib):
    name = "tweet_v5k_k50"
    sp = ts.WORKLOADS[name]
    t, W, m1 = _ctx(lib, name, max_batch=600)
    c = C.corpus(name, 700)
    Phi0 = _phi0(sp)
    for d0, d1 in [(0, 1), (1, 8), (8, 137), (137, 737 - 137), (100, 600)]:
        b = c.rows(d0, min(d1, c.n_docs))
        G, S3 = t.cp_data_term(lib.DeviceCSR.from_corpus(b), torch.tensor(Phi0, dtype=torch.float32, device="cuda"))
        g = _oracle_grad(b, sp, W, m1, Phi0)
        assert S3 == g["S3"]
        assert C.rel(G.cpu().numpy(), g["G_data"]) < TOL32, (d0, d1)


def test_short_documents_and_empty_batch_are_noops(lib):
    name = "small_v500_k10"
    sp = ts.WORKLOADS[name]
    t, W, m1 = _ctx(lib, name)
    Phi0 = _phi0(sp)
    Phi = torch.tensor(Phi0, dtype=torch.float32, device="cuda")
    grad = torch.ones_like(Phi)
    short = lib.DeviceCSR.from_arrays([0, 1, 3, 3, 4], [5, 1, 7, 9], [2, 1, 1, 1], sp.V)  # L = 2,2,0,1
    loss = t.cp_step(short, Phi, 0.1, grad=grad, want_loss=True)
    assert loss == 0.0 and torch.all(grad == 0) and np.array_equal(Phi.cpu().numpy(), Phi0.astype(np.float32))
    empty = lib.DeviceCSR.from_arrays([0], [], [], sp.V)
    t.cp_step(empty, Phi, 0.1, want_loss=True)
    assert np.array_equal(Phi.cpu().numpy(), Phi0.astype(np.float32))


@pytest.mark.parametrize("corrupt", ["index_ge_V", "count_zero", "not_ascending", "indptr_decreasing"])
def test_corrupt_batch_is_rejected_and_phi_kept(lib, corrupt):
    name = "small_v500_k10"
    sp = ts.WORKLOADS[name]
    t, W, m1 = _ctx(lib, name)
    c = C.corpus(name, 50)
    indptr, indices, counts = c.indptr.copy(), c.indices.copy(), c.counts.copy()
    j = int(indptr[10]) + 1
    if corrupt == "index_ge_V":
        indices[j] = sp.V + 3
    elif corrupt == "count_zero":
        counts[j] = 0
    elif corrupt == "not_ascending":
        indices[j], indices[j + 1] = indices[j + 1], indices[j]
    else:
        indptr[11], indptr[12] = indptr[12], indptr[11]   # stays within [0, nnz]
    Phi0 = _phi0(sp)
    Phi = torch.tensor(Phi0, dtype=torch.float32, device="cuda")
    b = lib.DeviceCSR.from_arrays(indptr, indices, counts, sp.V)
    t.cp_step(b, Phi, 0.1)
    with pytest.raises(lib.TLDAError) as ei:
        t.sync()
    assert ei.value.status == lib.ERR_INVALID
    assert np.array_equal(Phi.cpu().numpy(), Phi0.astype(np.float32))
    # the error is cleared by the synchronising call; a good batch works again
    t.cp_step(lib.DeviceCSR.from_corpus(c), Phi, 0.1)
    t.sync()


def test_whitening_dimension_above_topics(lib):
    """D > K: the whitening of the empirical M2 of the small workload to D = 16."""
    name = "small_v500_k10"
    sp = ts.WORKLOADS[name]
    c = C.corpus(name, 4000)
    st = O.ingest(c.indptr, c.indices, c.counts, sp.V)
    M1 = O.first_moment(st["C"], st["T"])
    M2 = O.second_moment(O.pair_counts(c.indptr, c.indices, c.counts, sp.V), st["S2"], M1, 1.0)
    Wd, _, _ = O.whitening(M2, 16)
    W = Wd.astype(np.float32).astype(np.float64)
    m1 = (W.T @ M1).astype(np.float32).astype(np.float64)
    t, _, _ = _ctx(lib, name, dim=16, W=(W, m1))
    Phi0 = ts.initial_factors(7, 16, sp.K)
    b = c.rows(0, 1000)
    G, S3 = t.cp_data_term(lib.DeviceCSR.from_corpus(b), torch.tensor(Phi0, dtype=torch.float32, device="cuda"))
    g = O.cp_grad_implicit(b.indptr, b.indices, b.counts, sp.V, W, m1, Phi0, 1.0, 0.0)
    assert C.rel(G.cpu().numpy(), g["G_data"]) < TOL32


# ----------------------------------------------------------------------------- pass
@pytest.mark.parametrize("host_input", [False, True])
def test_pass_equals_sequential_oracle_steps(lib, host_input):
    name = "tweet_v5k_k50"
    sp = ts.WORKLOADS[name]
    t, W, m1 = _ctx(lib, name, max_batch=1024)
    c = C.corpus(name, 3000)
    offs = [0, 700, 1024 + 700, 1724, 2500, 3000]
    Phi0 = _phi0(sp)
    Phi = torch.tensor(Phi0, dtype=torch.float32, device="cuda")
    corpus = lib.DeviceCSR.from_corpus(c, device="cpu" if host_input else "cuda", pin=host_input)
    lr = 0.002
    losses = t.cp_pass(corpus, offs, Phi, lr, host_input=host_input, losses=True)
    P = Phi0.copy()
    for b in range(len(offs) - 1):
        r = c.rows(offs[b], offs[b + 1])
        P, g = O.cp_step(r.indptr, r.indices, r.counts, sp.V, W, m1, P, lr, float(sp.alpha0), 0.0)
        assert abs(losses[b] - g["loss"]) <= 1e-5 * abs(g["loss"]), b
    assert C.rel(Phi.cpu().numpy(), P) < TOL32


# ----------------------------------------------------------------------------- BF16 tensor-core form
@pytest.mark.parametrize("name,n", [("small_v500_k10", 1000), ("small_v500_k10", 37),
                                    ("tweet_v5k_k50", 2048), ("stream_v20k_k100", 4099),
                                    ("stream_v20k_k100", 8192), ("stream_v20k_k100", 1)])
def test_data_term_bf16(lib, name, n):
    sp = ts.WORKLOADS[name]
    t, W, m1 = _ctx(lib, name, precision="bf16")
    c = C.corpus(name, n)
    Phi = _phi0(sp)
    G, S3 = t.cp_data_term(lib.DeviceCSR.from_corpus(c), torch.tensor(Phi, dtype=torch.float32, device="cuda"))
    g = _oracle_grad(c, sp, W, m1, Phi)
    assert S3 == g["S3"]
    if n == 1:  # one document: its distinct-token triples cancel; the bar is the rounding-error scale
        M = C.data_term_magnitude(c, sp.V, W, m1, Phi, float(sp.alpha0))
        C.assert_bf16_parity_scaled(G.cpu().numpy(), g["G_data"], M, TOL16, f"G_data {name} B={n}")
    else:
        C.assert_bf16_parity(G.cpu().numpy(), g["G_data"], TOL16, f"G_data {name} B={n}")


@pytest.mark.parametrize("same_token", [True, False])
def test_cp_step_bf16(lib, same_token):
    name = "tweet_v5k_k50"
    sp = ts.WORKLOADS[name]
    t, W, m1 = _ctx(lib, name, precision="bf16", same_token=same_token)
    c = C.corpus(name, 3000)
    Phi0 = _phi0(sp)
    Phi = torch.tensor(Phi0, dtype=torch.float32, device="cuda")
    grad = torch.empty_like(Phi)
    lr = 0.002
    loss = t.cp_step(lib.DeviceCSR.from_corpus(c), Phi, lr, grad=grad, want_loss=True)
    g = _oracle_grad(c, sp, W, m1, Phi0, 0.0, same_token)
    C.assert_bf16_parity(grad.cpu().numpy(), g["grad"], TOL16, "grad")
    C.assert_bf16_parity(Phi.cpu().numpy() - Phi0, -lr * g["grad"], TOL16, "Phi update")
    assert abs(loss - g["loss"]) <= TOL16 * abs(g["loss"])


@pytest.mark.parametrize("fused", [True, False])
@pytest.mark.parametrize("same_token", [True, False])
def test_bf16_fused_and_unfused_forms(lib, monkeypatch, fused, same_token):
    """D = K = 100 (padded 128) runs the fused tensor-core kernel; with
    TLDA_NO_FUSED the same context size takes the multi-kernel BF16 path."""
    if not fused:
        monkeypatch.setenv("TLDA_NO_FUSED", "1")
    name = "stream_v20k_k100"
    sp = ts.WORKLOADS[name]
    t, W, m1 = _ctx(lib, name, precision="bf16", same_token=same_token)
    c = C.corpus(name, 6000)
    b = c.rows(17, 5017)
    Phi0 = _phi0(sp)
    Phi = torch.tensor(Phi0, dtype=torch.float32, device="cuda")
    grad = torch.empty_like(Phi)
    loss = t.cp_step(lib.DeviceCSR.from_corpus(b), Phi, 0.002, grad=grad, want_loss=True)
    g = _oracle_grad(b, sp, W, m1, Phi0, 0.0, same_token)
    C.assert_bf16_parity(grad.cpu().numpy(), g["grad"], TOL16, f"grad fused={fused}")
    assert abs(loss - g["loss"]) <= TOL16 * abs(g["loss"])
    G, S3 = t.cp_data_term(lib.DeviceCSR.from_corpus(b), torch.tensor(Phi0, dtype=torch.float32, device="cuda"))
    assert S3 == g["S3"]
    C.assert_bf16_parity(G.cpu().numpy(), g["G_data"], TOL16, f"G_data fused={fused}")


def test_pass_bf16_ragged(lib):
    name = "stream_v20k_k100"
    sp = ts.WORKLOADS[name]
    t, W, m1 = _ctx(lib, name, precision="bf16")
    c = C.corpus(name, 12000)
    offs = [0, 513, 8192 + 513, 9000, 9001, 12000]
    Phi0 = _phi0(sp)
    Phi = torch.tensor(Phi0, dtype=torch.float32, device="cuda")
    lr = 0.002
    losses = t.cp_pass(lib.DeviceCSR.from_corpus(c), offs, Phi, lr, losses=True)
    P, steps, scales = Phi0.copy(), [], []
    for b in range(len(offs) - 1):
        r = c.rows(offs[b], offs[b + 1])
        Pn, g = O.cp_step(r.indptr, r.indices, r.counts, sp.V, W, m1, P, lr, float(sp.alpha0), 0.0)
        # the one-document step: its rounding-error scale (3 lr times the data term's)
        scales.append(3.0 * lr * C.data_term_magnitude(r, sp.V, W, m1, P, float(sp.alpha0)).max(axis=0)
                      if r.n_docs == 1 else None)
        steps.append(Pn - P)
        P = Pn
        assert abs(losses[b] - g["loss"]) <= TOL16 * abs(g["loss"]), b
    C.assert_bf16_pass_parity(Phi.cpu().numpy() - Phi0, P - Phi0, steps, TOL16, "Phi change over the pass",
                              step_scales=scales)


# ----------------------------------------------------------------------------- moments
def test_fit_moments_small(lib):
    name = "small_v500_k10"
    sp = ts.WORKLOADS[name]
    c = C.corpus(name, sp.n_docs)
    t = lib.TLDA(sp.V, sp.K, alpha0=float(sp.alpha0), seed=3)
    for d0 in range(0, c.n_docs, 3000):
        t.fit_moments(lib.DeviceCSR.from_corpus(c.rows(d0, min(d0 + 3000, c.n_docs))), lib.ACCUMULATE)
    t.fit_moments(None, lib.FINALIZE)
    Cg, T, S2, S3 = t.get_counts()
    st = O.ingest(c.indptr, c.indices, c.counts, sp.V)
    assert np.array_equal(Cg, st["C"]) and (T, S2, S3) == (st["T"], st["S2"], st["S3"])
    Wg, m1g, lam_g = t.get_whitening()
    Wg = Wg.cpu().numpy().astype(np.float64)
    M1 = O.first_moment(st["C"], st["T"])
    M2 = O.second_moment(O.pair_counts(c.indptr, c.indices, c.counts, sp.V), st["S2"], M1, 1.0)
    Wo, Uo, lam_o = O.whitening(M2, sp.K)
    assert np.allclose(lam_g, lam_o, rtol=1e-6)
    assert C.rel(Wg.T @ M2 @ Wg, np.eye(sp.K)) < 1e-5
    # same subspace and same signed eigenvectors (eigengap here is well above 1e-6 lambda_1)
    assert C.rel(Wg, Wo) < 1e-4
    assert C.rel(m1g.cpu().numpy(), Wo.T @ M1) < 1e-4
    assert 1 <= t.eig_sweeps() < 40  # the Jacobi eigensolve converged before its sweep cap


def test_fit_moments_tweet_v5k_k50(lib):
    """The fit at the 5k-word workload (V = 5000, K = 50, Zipf-shaped topics),
    where the randomised subspace iteration does real work: 200,000 documents
    in four chunks, against the oracle's dense eigendecomposition of the same
    M2.  Exact integer statistics; eigenvalues to 1e-6; W^T M2 W = I to 1e-5;
    the spectral projector of the top-K eigenspace, U U^T, to 1e-4 of its norm
    (sqrt(K)) -- the subspace is what the CP step depends on (reading J)."""
    name = "tweet_v5k_k50"
    sp = ts.WORKLOADS[name]
    n = 200_000
    c = C.corpus(name, n)
    t = lib.TLDA(sp.V, sp.K, alpha0=float(sp.alpha0), seed=5)
    for d0 in range(0, n, 50_000):
        t.fit_moments(lib.DeviceCSR.from_corpus(c.rows(d0, d0 + 50_000)), lib.ACCUMULATE)
    t.fit_moments(None, lib.FINALIZE)
    Cg, T, S2, S3 = t.get_counts()
    st = O.ingest(c.indptr, c.indices, c.counts, sp.V)
    assert np.array_equal(Cg, st["C"]) and (T, S2, S3) == (st["T"], st["S2"], st["S3"])
    Wg, m1g, lam_g = t.get_whitening()
    Wg = Wg.cpu().numpy().astype(np.float64)
    M1 = O.first_moment(st["C"], st["T"])
    M2 = O.second_moment(O.pair_counts(c.indptr, c.indices, c.counts, sp.V), st["S2"], M1, float(sp.alpha0))
    Wo, Uo, lam_o = O.whitening(M2, sp.K)
    lam_err = float(np.max(np.abs(lam_g - lam_o) / lam_o))
    Ug = Wg * np.sqrt(lam_g)[None, :]
    proj = np.linalg.norm(Ug @ Ug.T - Uo @ Uo.T) / np.sqrt(sp.K)
    ident = C.rel(Wg.T @ M2 @ Wg, np.eye(sp.K))
    print(f"fit V=5000 K=50: eigenvalue rel err {lam_err:.2e}, W^T M2 W - I {ident:.2e}, "
          f"projector gap {proj:.2e}, lambda_K / lambda_1 {lam_o[-1] / lam_o[0]:.2e}")
    assert lam_err < 1e-6
    assert ident < 1e-5
    assert proj < 1e-4
    assert C.rel(m1g.cpu().numpy(), Wg.T @ M1) < 1e-5
    assert 1 <= t.eig_sweeps() < 40
    t.close()


def test_unwhiten_population_factors(lib):
    name = "small_v500_k10"
    sp = ts.WORKLOADS[name]
    _, mu = C.topics(name)
    h = np.full(sp.K, 1.0 / sp.K)
    t, W, m1 = _ctx(lib, name)
    Phi = O.population_factors(mu, h, W).astype(np.float32).astype(np.float64)
    mu_g, al_g = t.unwhiten_topics(torch.tensor(Phi, dtype=torch.float32, device="cuda"))
    mu_o, al_o = O.unwhiten_cp(Phi, W)
    mu_o, _ = O.clip_normalise(mu_o)
    assert C.rel(mu_g, mu_o) < 1e-6
    assert C.rel(al_g, al_o) < 1e-6
    perm, l1, _ = O.match_topics(mu_g, mu)
    assert l1.max() < 1e-3


def test_state_roundtrip(lib, tmp_path):
    name = "small_v500_k10"
    sp = ts.WORKLOADS[name]
    t, W, m1 = _ctx(lib, name)
    p = tmp_path / "state.bin"
    t.save_state(str(p))
    t2 = lib.TLDA(sp.V, sp.K, alpha0=float(sp.alpha0))
    t2.load_state(str(p))
    W2, m12, _ = t2.get_whitening()
    assert np.array_equal(W2.cpu().numpy(), W.astype(np.float32))
    raw = bytearray(p.read_bytes())
    raw[100] ^= 0xFF
    p.write_bytes(bytes(raw))
    with pytest.raises(lib.TLDAError):
        t2.load_state(str(p))


# ----------------------------------------------------------------------------- wide BF16
@pytest.mark.parametrize("K", [150, 200, 300, 350, 448, 500])
def test_data_term_bf16_wide(lib, K):
    """D = K up to 512 in the multi-kernel BF16 form: 64-row reduction chunks
    through the TMA ring with MN-major operands, N above 256 as a 256-wide MMA
    and one of K - 256 (K = 300, 350: 64 and 128 wide), feature tiles of 128
    (K = 150: the second tile's upper 64 features read past D as zero), and
    1500 documents, so the last chunk has zero-padded rows."""
    from dataclasses import replace
    sp = replace(ts.WORKLOADS["small_v500_k10"], name=f"wide_k{K}", V=1500, K=K, lam=60.0,
                 seed=ts.WORKLOADS["small_v500_k10"].seed + K)
    cdf, mu = ts.topics(sp)
    W, m1 = O.population_whitening(mu, np.full(K, 1.0 / K))
    W, m1 = W.astype(np.float32).astype(np.float64), m1.astype(np.float32).astype(np.float64)
    c = ts.corpus(sp.with_docs(1500), cdf=cdf)
    t = lib.TLDA(sp.V, K, alpha0=float(sp.alpha0), precision="bf16", max_batch=2048)
    t.set_whitening(torch.tensor(W, dtype=torch.float32), torch.tensor(m1, dtype=torch.float32))
    Phi0 = _phi0(sp)
    dev = lib.DeviceCSR.from_corpus(c)
    G, S3 = t.cp_data_term(dev, torch.tensor(Phi0, dtype=torch.float32, device="cuda"))
    g = _oracle_grad(c, sp, W, m1, Phi0)
    assert S3 == g["S3"]
    C.assert_bf16_parity(G.cpu().numpy(), g["G_data"], TOL16, f"G_data K={K}")
    Phi = torch.tensor(Phi0, dtype=torch.float32, device="cuda")
    grad = torch.empty_like(Phi)
    loss = t.cp_step(dev, Phi, 0.002, grad=grad, want_loss=True)
    C.assert_bf16_parity(grad.cpu().numpy(), g["grad"], TOL16, f"grad K={K}")
    assert abs(loss - g["loss"]) <= TOL16 * abs(g["loss"])
    t.close()
