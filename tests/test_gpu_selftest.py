"""Failure detection without a GPU fault: the bounded grid barrier of the
persistent kernels gives up when a block never arrives (tlda_selftest_barrier:
block 0 skips its arrival), every block returns within about a second, the
host reads TLDA_ERR_TIMEOUT, and a persistent pass afterwards still matches
the oracle."""
from __future__ import annotations

import time

import numpy as np
import pytest
import torch

import tlda_synth as ts
from oracle import tlda_oracle as O

from . import _cases as C

pytestmark = pytest.mark.gpu


def test_bounded_grid_barrier_gives_up_and_the_gpu_stays_usable(lib):
    t0 = time.perf_counter()
    st, blocks, gave_up = lib.selftest_barrier()
    dt = time.perf_counter() - t0
    assert st == lib.ERR_TIMEOUT
    assert blocks >= 128 and gave_up == blocks
    assert dt < 10.0
    # a persistent pass right afterwards
    name = "stream_v20k_k100"
    sp = ts.WORKLOADS[name]
    W, m1 = C.population_whitening(name)
    t = lib.TLDA(sp.V, sp.K, alpha0=float(sp.alpha0), precision="bf16")
    t.set_whitening(torch.tensor(W, dtype=torch.float32), torch.tensor(m1, dtype=torch.float32))
    t.autotune(fixed=18)
    c = C.corpus(name, 6000)
    offs = [0, 2500, 6000]
    P0 = ts.initial_factors(sp.seed + 1, sp.K, sp.K)
    Phi = torch.tensor(P0, dtype=torch.float32, device="cuda")
    t.cp_pass(lib.DeviceCSR.from_corpus(c), offs, Phi, 0.002)
    P, steps = P0.astype(np.float64), []
    for b in range(2):
        r = c.rows(offs[b], offs[b + 1])
        Pn, _ = O.cp_step(r.indptr, r.indices, r.counts, sp.V, W, m1, P, 0.002, float(sp.alpha0), 0.0)
        steps.append(Pn - P)
        P = Pn
    C.assert_bf16_pass_parity(Phi.cpu().numpy() - P0, P - P0, steps, 2e-2, "Phi change after the self-test")
    t.close()
