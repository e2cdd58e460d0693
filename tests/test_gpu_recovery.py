"""Topic recovery on the small workload (V = 500, K = 10, 10,000 documents,
10 minibatches x 5 epochs): the FP32 and BF16 forms follow the FP64
oracle's SGD trajectory and give the same per-topic l1 recovery error
(section "Recovering the Topic Model Parameters"; Hungarian matching).

The recovery bar itself is statistical.  Even the exact orthogonal
decomposition of this corpus's tensor, by the tensor power method, is
reported here beside SGD and is not asserted."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import tlda_synth as ts
from oracle import tlda_oracle as O

from . import _cases as C

pytestmark = pytest.mark.gpu
NAME = "small_v500_k10"
LR = 0.02
EPOCHS = 5


def _recovery(mu_est, mu):
    mu_c, _ = O.clip_normalise(mu_est)
    _, l1, _ = O.match_topics(mu_c, mu)
    return l1


def test_recovery_equal_across_forms_and_oracle(lib):
    sp = ts.WORKLOADS[NAME]
    _, mu = C.topics(NAME)
    c = C.corpus(NAME, sp.n_docs)
    dev = lib.DeviceCSR.from_corpus(c)
    # whitening fitted by the library (FP32 values used by every run below)
    fit = lib.TLDA(sp.V, sp.K, alpha0=float(sp.alpha0), precision="fp32")
    fit.fit([dev])
    W, m1, _ = fit.get_whitening()
    W64 = W.cpu().numpy().astype(np.float64)
    m164 = m1.cpu().numpy().astype(np.float64)
    offs = list(range(0, sp.n_docs + 1, 1000))
    Phi0 = ts.initial_factors(sp.seed + 1, sp.K, sp.K)

    l1 = {}
    Phis = {}
    for prec in ("fp32", "bf16"):
        t = lib.TLDA(sp.V, sp.K, alpha0=float(sp.alpha0), precision=prec)
        t.set_whitening(W, m1)
        Phi = torch.tensor(Phi0, dtype=torch.float32, device="cuda")
        for _ in range(EPOCHS):
            t.cp_pass(dev, offs, Phi, LR)
        mu_est, _ = t.unwhiten_topics(Phi)
        l1[prec] = _recovery(mu_est, mu)
        Phis[prec] = Phi.cpu().numpy()
        t.close()

    # the oracle's SGD trajectory on the same whitening
    P = Phi0.astype(np.float64)
    for _ in range(EPOCHS):
        for b in range(len(offs) - 1):
            r = c.rows(offs[b], offs[b + 1])
            P, _ = O.cp_step(r.indptr, r.indices, r.counts, sp.V, W64, m164, P, LR, float(sp.alpha0), 0.0)
    mu_o, _ = O.unwhiten_cp(P, W64)
    l1_o = _recovery(mu_o, mu)

    assert C.rel(Phis["fp32"], P) < 1e-3  # 50 steps of FP32 rounding
    assert C.rel(Phis["bf16"], P) < 5e-2  # 50 steps of BF16 operand rounding
    # equal recovery error: per topic, and on average
    assert np.max(np.abs(np.sort(l1["fp32"]) - np.sort(l1_o))) < 1e-3
    assert np.max(np.abs(np.sort(l1["bf16"]) - np.sort(l1_o))) < 2e-2
    assert abs(l1["bf16"].mean() - l1["fp32"].mean()) < 1e-2

    # context: the exact orthogonal decomposition of the corpus tensor
    st = O.ingest(c.indptr, c.indices, c.counts, sp.V)
    M1 = O.first_moment(st["C"], st["T"])
    T = O.whitened_third_moment(c.indptr, c.indices, c.counts, sp.V, W64, M1, float(sp.alpha0))
    lams, V = O.tensor_power_method(T, sp.K, n_restarts=10, n_iters=50, seed=0)
    mu_p, _ = O.unwhiten_power(lams, V, W64)
    l1_p = _recovery(mu_p, mu)
    print(f"recovery l1 mean/max: sgd fp32 {l1['fp32'].mean():.3f}/{l1['fp32'].max():.3f}, "
          f"bf16 {l1['bf16'].mean():.3f}/{l1['bf16'].max():.3f}, oracle sgd {l1_o.mean():.3f}/{l1_o.max():.3f}, "
          f"power method {l1_p.mean():.3f}/{l1_p.max():.3f}")
    fit.close()
