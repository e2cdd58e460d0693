"""The fully online mode (section "Fully Online Implementation"; readings P
and Q) through the C ABI against the FP64 oracle: the sketched whitening,
the carrying of Phi into each new basis, and whole online passes in the FP32
form and in the BF16 form (persistent pass kernel)."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import tlda_synth as ts
from oracle import tlda_oracle as O

from . import _cases as C

pytestmark = pytest.mark.gpu


def _omega(sp, r):
    """A random sign test matrix: with it the sketch's FP32 products and sums
    are integers below 2^24, so the device's Z is exact."""
    return ts.signs(sp.seed, 0x4F4D, sp.V * r).reshape(sp.V, r)


def _setup(lib, name, n_docs, nb, precision, r=None):
    sp = ts.WORKLOADS[name]
    c = C.corpus(name, n_docs)
    offs = np.linspace(0, n_docs, nb + 1).astype(np.int64)
    r = r or sp.K + 16
    Om = _omega(sp, r)
    t = lib.TLDA(sp.V, sp.K, alpha0=float(sp.alpha0), precision=precision)
    t.online_begin(torch.tensor(Om))
    return sp, c, offs, Om, t


def test_online_whitening_matches_oracle_sketch(lib):
    sp, c, offs, Om, t = _setup(lib, "small_v500_k10", 10000, 10, "fp32")
    Phi0 = ts.initial_factors(sp.seed, sp.K, sp.K)
    Phi = torch.tensor(Phi0, dtype=torch.float32, device="cuda")
    t.online_pass(lib.DeviceCSR.from_corpus(c), offs, Phi, 0.0, rewhiten_every=10)
    W, m1, ev = t.get_whitening()
    st = O.ingest(c.indptr, c.indices, c.counts, sp.V)
    Z = O.sketch_accumulate(c.indptr, c.indices, c.counts, sp.V, Om)
    Wo, m1o, lam = O.sketch_whitening(Z, st["C"], st["T"], st["S2"], Om, float(sp.alpha0), sp.K)
    assert np.allclose(ev, lam, rtol=1e-7)
    assert C.rel(W.cpu().numpy(), Wo) < 1e-5
    assert C.rel(m1.cpu().numpy(), m1o) < 1e-5
    assert torch.equal(Phi.cpu(), torch.tensor(Phi0, dtype=torch.float32))  # one block: no rotation, lr = 0
    assert 1 <= t.eig_sweeps() < 40
    t.close()


def test_online_chunks_accumulated_then_whitened(lib):
    """The sketch of a corpus read in chunks (tlda_online_accumulate), then one
    whitening (tlda_online_whiten), equals the oracle's whitening of the whole
    corpus; a corrupt chunk is reported by the next whitening."""
    sp, c, offs, Om, t = _setup(lib, "small_v500_k10", 10000, 10, "fp32")
    for a, b in ((0, 3000), (3000, 3001), (3001, 10000)):
        t.online_accumulate(lib.DeviceCSR.from_corpus(c.rows(a, b)))
    t.online_whiten()
    W, m1, ev = t.get_whitening()
    st = O.ingest(c.indptr, c.indices, c.counts, sp.V)
    Z = O.sketch_accumulate(c.indptr, c.indices, c.counts, sp.V, Om)
    Wo, m1o, lam = O.sketch_whitening(Z, st["C"], st["T"], st["S2"], Om, float(sp.alpha0), sp.K)
    assert np.allclose(ev, lam, rtol=1e-7)
    assert C.rel(W.cpu().numpy(), Wo) < 1e-5
    assert C.rel(m1.cpu().numpy(), m1o) < 1e-5
    bad = c.rows(0, 100)
    counts = bad.counts.copy()
    counts[5] = 0
    t.online_accumulate(lib.DeviceCSR.from_arrays(bad.indptr, bad.indices, counts, sp.V))
    with pytest.raises(lib.TLDAError) as e:
        t.online_whiten()
    assert e.value.status == lib.ERR_INVALID
    t.close()


def test_online_rotations_match_oracle(lib):
    """lr = 0 and a new whitening every batch: Phi only moves by the basis changes."""
    sp, c, offs, Om, t = _setup(lib, "small_v500_k10", 10000, 10, "fp32")
    Phi0 = ts.initial_factors(sp.seed, sp.K, sp.K)
    Phi = torch.tensor(Phi0, dtype=torch.float32, device="cuda")
    t.online_pass(lib.DeviceCSR.from_corpus(c), offs, Phi, 0.0, rewhiten_every=1)
    P, _, _ = O.online_pass(c.indptr, c.indices, c.counts, sp.V, offs, Om, 1, float(sp.alpha0), 0.0, 0.0,
                            Phi0.astype(np.float64), sp.K)
    assert C.rel(Phi.cpu().numpy(), P) < 1e-4
    t.close()


@pytest.mark.parametrize("every", [1, 3])
def test_online_pass_fp32_matches_oracle(lib, every):
    sp, c, offs, Om, t = _setup(lib, "small_v500_k10", 10000, 10, "fp32")
    Phi0 = ts.initial_factors(sp.seed, sp.K, sp.K)
    Phi = torch.tensor(Phi0, dtype=torch.float32, device="cuda")
    lr = 0.02
    losses = t.online_pass(lib.DeviceCSR.from_corpus(c), offs, Phi, lr, rewhiten_every=every, losses=True)
    P, _, lo = O.online_pass(c.indptr, c.indices, c.counts, sp.V, offs, Om, every, float(sp.alpha0), 0.0, lr,
                             Phi0.astype(np.float64), sp.K)
    assert C.rel(Phi.cpu().numpy(), P) < 1e-4
    assert np.allclose(losses, lo, rtol=1e-4)
    t.close()


def test_online_pass_bf16_persistent_kernel(lib):
    """V = 20,000, K = D = 100: this model's M2 has no clear gap after its
    100th eigenvalue, so the sketch is wider (r = 216) and the first block
    larger (50,000 documents) than the minimum."""
    sp, c, offs, Om, t = _setup(lib, "stream_v20k_k100", 100000, 16, "bf16", r=216)
    Phi0 = ts.initial_factors(sp.seed, sp.K, sp.K)
    Phi = torch.tensor(Phi0, dtype=torch.float32, device="cuda")
    lr = 5e-4
    losses = t.online_pass(lib.DeviceCSR.from_corpus(c), offs, Phi, lr, rewhiten_every=8, losses=True)
    assert 1 <= t.eig_sweeps() < 40
    P, _, lo = O.online_pass(c.indptr, c.indices, c.counts, sp.V, offs, Om, 8, float(sp.alpha0), 0.0, lr,
                             Phi0.astype(np.float64), sp.K)
    C.assert_bf16_parity(Phi.cpu().numpy(), P, 2e-2, "Phi after the online pass")
    assert np.all(np.abs(losses - lo) <= 2e-2 * np.abs(lo))
    t.close()


def test_online_arguments(lib):
    sp = ts.WORKLOADS["small_v500_k10"]
    t = lib.TLDA(sp.V, sp.K, alpha0=float(sp.alpha0))
    c = C.corpus("small_v500_k10", 1000)
    Phi = torch.zeros((sp.K, sp.K), dtype=torch.float32, device="cuda")
    assert t.eig_sweeps() == 0
    with pytest.raises(lib.TLDAError) as e:
        t.online_pass(lib.DeviceCSR.from_corpus(c), [0, 1000], Phi, 0.01)
    assert e.value.status == lib.ERR_STATE
    with pytest.raises(lib.TLDAError) as e:
        t.online_sketch()
    assert e.value.status == lib.ERR_STATE
    with pytest.raises(lib.TLDAError) as e:
        t.online_accumulate(lib.DeviceCSR.from_corpus(c))
    assert e.value.status == lib.ERR_STATE
    for r in (sp.K - 2, sp.K + 3, 600):
        with pytest.raises(lib.TLDAError) as e:
            t.online_begin(torch.zeros((sp.V, r), dtype=torch.float64))
        assert e.value.status == lib.ERR_INVALID
    t.close()


def _sketch_check(lib, t, indptr, indices, counts, V, Om):
    """The context's sketch, counts and token statistics against the oracle's:
    all exact (a sign test matrix makes every sum an integer)."""
    Z, Cw, TS = t.online_sketch()
    st = O.ingest(indptr, indices, counts, V)
    Zo = O.sketch_accumulate(indptr, indices, counts, V, Om)
    assert np.array_equal(Cw.cpu().numpy(), np.asarray(st["C"], dtype=np.int64))
    assert TS.cpu().tolist() == [int(st["T"]), int(st["S2"]), int(st["S3"])]
    assert np.array_equal(Z.cpu().numpy(), Zo)
    return Z, Cw, TS


def test_online_sketch_matches_oracle(lib):
    """Z = P Omega, C, T, S2, S3 after chunked accumulation (reading P), at
    r = 26, 200 and 300 (the kernels of 4, 8 and 16 columns per lane)."""
    for r in (26, 200, 300):
        sp, c, offs, Om, t = _setup(lib, "small_v500_k10", 10000, 10, "fp32", r=r)
        for a, b in ((0, 4000), (4000, 4001), (4001, 4001), (4001, 10000)):
            t.online_accumulate(lib.DeviceCSR.from_corpus(c.rows(a, b)))
        _sketch_check(lib, t, c.indptr, c.indices, c.counts, sp.V, Om)
        t.close()


def test_online_sketch_many_pieces(lib):
    """600,000 documents: three pieces of the per-piece transpose (262,144
    documents each at most), against the oracle's sketch."""
    sp = ts.WORKLOADS["small_v500_k10"]
    c = C.corpus("small_v500_k10", 600_000)
    r = 16
    Om = _omega(sp, r)
    t = lib.TLDA(sp.V, sp.K, alpha0=float(sp.alpha0), precision="fp32")
    t.online_begin(torch.tensor(Om))
    t.online_accumulate(lib.DeviceCSR.from_corpus(c))
    _sketch_check(lib, t, c.indptr, c.indices, c.counts, sp.V, Om)
    t.close()


def _dense_docs(n_docs, V, per_doc):
    """n_docs documents of per_doc distinct words each (a fixed pattern)."""
    d = np.arange(n_docs, dtype=np.int64)[:, None]
    j = np.arange(per_doc, dtype=np.int64)[None, :]
    words = np.sort((d * 37 + j * (V // per_doc)) % V, axis=1).astype(np.int32)
    counts = (1 + (d + j) % 3).astype(np.int32)
    indptr = np.arange(n_docs + 1, dtype=np.int64) * per_doc
    return indptr, words.ravel(), counts.ravel()


def test_online_sketch_piece_halving(lib):
    """262,144 documents of 100 distinct words: 26.2M nonzeros exceed a piece's
    16M slots, so the piece is halved; the sketch still equals the oracle's."""
    V, r = 500, 16
    indptr, indices, counts = _dense_docs(262_144, V, 100)
    Om = ts.signs(7, 0x4F4D, V * r).reshape(V, r)
    t = lib.TLDA(V, 10, alpha0=1.0, precision="fp32")
    t.online_begin(torch.tensor(Om))
    t.online_accumulate(lib.DeviceCSR.from_arrays(indptr, indices, counts, V))
    _sketch_check(lib, t, indptr, indices, counts, V, Om)
    t.close()


def test_online_sketch_checkpoint_resume(lib):
    """Statistics saved after part of a corpus and restored into a new context
    continue to the same sketch and whitening as one uninterrupted run."""
    sp, c, offs, Om, t = _setup(lib, "small_v500_k10", 10000, 10, "fp32")
    t.online_accumulate(lib.DeviceCSR.from_corpus(c.rows(0, 6000)))
    saved = [x.cpu() for x in t.online_sketch()]
    t.close()
    t2 = lib.TLDA(sp.V, sp.K, alpha0=float(sp.alpha0), precision="fp32")
    t2.online_begin(torch.tensor(Om))
    t2.online_set_sketch(*saved)
    t2.online_accumulate(lib.DeviceCSR.from_corpus(c.rows(6000, 10000)))
    _sketch_check(lib, t2, c.indptr, c.indices, c.counts, sp.V, Om)
    t2.online_whiten()
    W, m1, ev = t2.get_whitening()
    st = O.ingest(c.indptr, c.indices, c.counts, sp.V)
    Z = O.sketch_accumulate(c.indptr, c.indices, c.counts, sp.V, Om)
    Wo, m1o, lam = O.sketch_whitening(Z, st["C"], st["T"], st["S2"], Om, float(sp.alpha0), sp.K)
    assert np.allclose(ev, lam, rtol=1e-7)
    assert C.rel(W.cpu().numpy(), Wo) < 1e-5
    t2.close()


def test_online_sketch_rejects_decreasing_indptr(lib):
    """A decreasing indptr inside a chunk is reported, and the other documents
    still add exactly their part."""
    sp, c, offs, Om, t = _setup(lib, "small_v500_k10", 2000, 2, "fp32")
    indptr = c.indptr.copy()
    indptr[50] = indptr[49] - 1  # document 49 ends before it starts
    t.online_accumulate(lib.DeviceCSR.from_arrays(indptr, c.indices, c.counts, sp.V))
    with pytest.raises(lib.TLDAError) as e:
        t.online_sketch()
    assert e.value.status == lib.ERR_INVALID
    t.close()


def test_online_sketch_gaussian_test_matrix(lib):
    """A Gaussian test matrix: the products use its FP32 values and sum in FP32
    within a document (s_d, L_d terms) and within a run of at most 128 slots,
    then in FP64.  First-order rounding bound, per entry:
    |dZ_mj| <= (L_max + 128 + 3) u sum_d f_dm (sum_m' f_dm' |O_m'j| + |O_mj|),
    u = 2^-24 (the 3: rounding of Omega, of s_d - Omega_m and of the product)."""
    sp, c, offs, _, t = _setup(lib, "small_v500_k10", 10000, 10, "fp32", r=26)
    Om = ts.gaussian(sp.seed, 0x4F4D, sp.V * 26).reshape(sp.V, 26)
    t.online_begin(torch.tensor(Om))
    t.online_accumulate(lib.DeviceCSR.from_corpus(c))
    Z, _, _ = t.online_sketch()
    Zo = O.sketch_accumulate(c.indptr, c.indices, c.counts, sp.V, Om)
    F = O.csr_matrix(c.indptr, c.indices, c.counts, sp.V)
    A = np.abs(Om)
    Zabs = F.T @ (F @ A) + np.asarray(F.sum(axis=0)).ravel()[:, None] * A
    L_max = int(np.max(np.diff(c.indptr)))
    bound = (L_max + 128 + 3) * 2.0 ** -24 * Zabs
    assert np.all(np.abs(Z.cpu().numpy() - Zo) <= bound)
    t.close()
