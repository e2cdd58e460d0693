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
    return ts.gaussian(sp.seed, 0x4F4D, sp.V * r).reshape(sp.V, r)


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
    assert C.rel(Phi.cpu().numpy(), P) < 2e-2
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
    for r in (sp.K - 2, sp.K + 3, 600):
        with pytest.raises(lib.TLDAError) as e:
            t.online_begin(torch.zeros((sp.V, r), dtype=torch.float64))
        assert e.value.status == lib.ERR_INVALID
    t.close()
