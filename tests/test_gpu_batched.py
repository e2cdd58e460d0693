"""The batched mode through the C ABI (tlda_fit_batched) against the FP64
oracle's batched_fit (section "Batched Implementation Enables Arbitrary
Scaling"; reading R), on a corpus of the simulation study (K = D = 2,
alpha0 = 0.01, 20,000 documents, V = 500): the whitening, every start's
factors after the epochs, the mean last-epoch losses, the kept start and the
recovery score; TLDA_REUSE_WHITENING; argument errors."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import tlda_synth as ts
from oracle import tlda_oracle as O

from . import _cases as C

pytestmark = pytest.mark.gpu
LR = 1e-2


def _e1(V=500, rep=0):
    sp = ts.e1_spec(V, rep)
    cdf, mu = ts.topics(sp)
    c = ts.corpus(sp, cdf=cdf)
    offs = np.arange(0, sp.n_docs + 1, 1000, dtype=np.int64)
    return sp, mu, c, offs


def _starts(sp, n):
    return np.stack([ts.initial_factors(sp.seed + s, sp.K, sp.K) for s in range(n)]).astype(np.float64)


def test_batched_fit_matches_oracle(lib):
    sp, mu, c, offs = _e1()
    starts = _starts(sp, 3)
    t = lib.TLDA(sp.V, sp.K, alpha0=float(sp.alpha0), precision="fp32")
    Ps = torch.tensor(starts, dtype=torch.float32, device="cuda")
    means = t.fit_batched(lib.DeviceCSR.from_corpus(c), offs, Ps, LR, epochs=5)
    P, W, m1, means_o, finals = O.batched_fit(c.indptr, c.indices, c.counts, sp.V, offs, 5, float(sp.alpha0),
                                              0.0, LR, starts, sp.K)
    Wg, m1g, _ = t.get_whitening()
    assert C.rel(Wg.cpu().numpy(), W) < 1e-4
    assert C.rel(m1g.cpu().numpy(), m1) < 1e-4
    assert np.allclose(means, means_o, rtol=1e-3)
    best = int(np.argmin(means_o))
    for s in range(1, 3):
        if s != best:
            assert C.rel(Ps[s].cpu().numpy(), finals[s]) < 1e-3, s
    assert C.rel(Ps[0].cpu().numpy(), P) < 1e-3  # the kept start, copied into the first slot
    mu_g, _ = t.unwhiten_topics(Ps[0])
    _, cg = O.topic_correlation(mu_g, mu)
    _, co = O.topic_correlation(O.clip_normalise(O.unwhiten_cp(P, W)[0])[0], mu)
    assert np.allclose(cg, co, atol=1e-3)
    t.close()


def test_batched_fit_reuses_whitening(lib):
    """With TLDA_REUSE_WHITENING only the epochs run: equal to the oracle's CP
    steps on the whitening installed in the context (the oracle's own, from
    the corpus's M2)."""
    sp, mu, c, offs = _e1(1000, 1)
    dev = lib.DeviceCSR.from_corpus(c)
    st = O.ingest(c.indptr, c.indices, c.counts, sp.V)
    M1 = O.first_moment(st["C"], st["T"])
    M2 = O.second_moment(O.pair_counts(c.indptr, c.indices, c.counts, sp.V), st["S2"], M1, float(sp.alpha0))
    Wo, _, _ = O.whitening(M2, sp.K)
    W = Wo.astype(np.float32).astype(np.float64)
    m1 = (W.T @ M1).astype(np.float32).astype(np.float64)
    t = lib.TLDA(sp.V, sp.K, alpha0=float(sp.alpha0), precision="fp32")
    t.set_whitening(torch.tensor(W, dtype=torch.float32), torch.tensor(m1, dtype=torch.float32))
    Wg, _, _ = t.get_whitening()
    starts = _starts(sp, 2)
    Ps = torch.tensor(starts, dtype=torch.float32, device="cuda")
    means = t.fit_batched(dev, offs, Ps, LR, epochs=2, reuse_whitening=True)
    Wg2, _, _ = t.get_whitening()
    assert torch.equal(Wg, Wg2)
    finals, means_o = [], []
    for s in range(2):
        P = starts[s].copy()
        for _ in range(2):
            losses = []
            for b in range(len(offs) - 1):
                r = c.rows(int(offs[b]), int(offs[b + 1]))
                P, g = O.cp_step(r.indptr, r.indices, r.counts, sp.V, W, m1, P, LR, float(sp.alpha0), 0.0)
                losses.append(g["loss"])
        finals.append(P)
        means_o.append(np.mean(losses))
    assert np.allclose(means, means_o, rtol=1e-4)
    assert C.rel(Ps[1].cpu().numpy(), finals[1]) < 1e-4
    assert C.rel(Ps[0].cpu().numpy(), finals[int(np.argmin(means_o))]) < 1e-4
    t.close()


def test_batched_fit_arguments(lib):
    sp, mu, c, offs = _e1()
    dev = lib.DeviceCSR.from_corpus(c)
    t = lib.TLDA(sp.V, sp.K, alpha0=float(sp.alpha0), precision="fp32")
    Ps = torch.zeros((1, sp.K, sp.K), dtype=torch.float32, device="cuda")
    with pytest.raises(lib.TLDAError) as e:
        t.fit_batched(dev, offs, Ps, LR, epochs=1, reuse_whitening=True)
    assert e.value.status == lib.ERR_STATE
    with pytest.raises(lib.TLDAError) as e:
        t.fit_batched(dev, offs, Ps, LR, epochs=0)
    assert e.value.status == lib.ERR_INVALID
    t.close()
