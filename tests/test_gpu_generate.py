"""The on-device corpus generator (tlda_generate_docs) against the host
generator of the test inputs, which follows the same definition: for the
same documents the CSR arrays are identical, bit for bit, on workloads with
integer and fractional alpha0, symmetric and Zipf-shaped topic priors, and
documents from the start and deep into the corpus; the count-only call and
the capacity check."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import tlda_synth as ts

pytestmark = pytest.mark.gpu


def _gen(lib, sp, cdf):
    a = sp.alpha0
    return lib.DeviceGenerator(sp.seed, sp.V, sp.K, cdf, a.numerator, a.denominator, ts.len_table(sp), sp.min_len)


@pytest.mark.parametrize("spec,doc0,n", [
    (ts.WORKLOADS["small_v500_k10"], 0, 3000),
    (ts.WORKLOADS["stream_v20k_k100"], 7_000_000, 20000),
    (ts.e1_spec(1000, 3), 123, 5000),
    (ts.WORKLOADS["billion_v100k_k300"], 987_654_321, 20000),
])
def test_device_generator_equals_host(lib, spec, doc0, n):
    cdf, _ = ts.topics(spec)
    g = _gen(lib, spec, cdf)
    dev = g.generate(doc0, n)
    host = ts.corpus(spec.with_docs(doc0 + n), doc0=doc0, n_docs=n, cdf=cdf)
    assert np.array_equal(dev.indptr.cpu().numpy().astype(np.int64), host.indptr)
    assert np.array_equal(dev.indices.cpu().numpy(), host.indices)
    assert np.array_equal(dev.counts.cpu().numpy(), host.counts)


def test_device_generator_capacity_and_reuse(lib):
    sp = ts.WORKLOADS["small_v500_k10"]
    cdf, _ = ts.topics(sp)
    g = _gen(lib, sp, cdf)
    first = g.generate(0, 1000)
    nnz = first.indices.numel()
    # a buffer too small for the next chunk: regenerated into fresh arrays
    small = lib.DeviceCSR(torch.empty(1001, dtype=torch.int32, device="cuda"),
                          torch.empty(nnz // 2, dtype=torch.int32, device="cuda"),
                          torch.empty(nnz // 2, dtype=torch.int32, device="cuda"), sp.V)
    again = g.generate(0, 1000, out=small)
    assert torch.equal(again.indices, first.indices) and torch.equal(again.counts, first.counts)
    big = lib.DeviceCSR(torch.empty(1001, dtype=torch.int32, device="cuda"),
                        torch.empty(2 * nnz, dtype=torch.int32, device="cuda"),
                        torch.empty(2 * nnz, dtype=torch.int32, device="cuda"), sp.V)
    reused = g.generate(1000, 1000, out=big)
    host = ts.corpus(sp.with_docs(2000), doc0=1000, n_docs=1000, cdf=cdf)
    assert np.array_equal(reused.indices.cpu().numpy(), host.indices)
    assert reused.indices.data_ptr() == big.indices.data_ptr()
