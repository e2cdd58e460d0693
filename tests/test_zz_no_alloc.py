"""The allocation-free CP step (tlda_cp_step_noalloc), for callers that cannot
allocate device memory, against the context-based tlda_cp_step: same batches,
same starting factors, FP32 tolerance.  The calls share one static scratch
array that keeps the previous call's contents, so the cases run in a fixed
order: the largest documented size first, then a smaller layout on the stale
array, then a corrupt batch and a valid one after it.  This file is collected
last on purpose, so a run that stops at the first failure has already run
every other test."""
import ctypes
from dataclasses import replace

import numpy as np
import pytest
import torch

import tlda_synth as ts
from oracle import tlda_oracle as O
from tests import _cases as C

pytestmark = pytest.mark.gpu

TOL32 = 1e-5


def _noalloc(lib, b, Wd, m1d, D, K, a0, theta, Phi, lr, g, err):
    raw = lib.load()
    s = b.struct()
    return raw.tlda_cp_step_noalloc(ctypes.byref(s), Wd.data_ptr(), m1d.data_ptr(), D, K, a0, theta,
                                    Phi.data_ptr(), lr, g.data_ptr() if g is not None else None,
                                    err.data_ptr() if err is not None else None,
                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def _against_context(lib, V, K, a0, W, m1, Phi0, batches, lr=0.01, theta=0.0):
    """Two or more calls in a row, each compared with the context step."""
    ctx = lib.TLDA(V, K, alpha0=a0, theta=theta, max_batch=max(b.n_docs for b in batches))
    ctx.set_whitening(torch.tensor(W, dtype=torch.float32), torch.tensor(m1, dtype=torch.float32))
    Phi_ref = torch.tensor(Phi0, dtype=torch.float32, device="cuda")
    g_ref = torch.empty_like(Phi_ref)
    Wd = torch.tensor(W, dtype=torch.float32, device="cuda")
    m1d = torch.tensor(m1, dtype=torch.float32, device="cuda")
    Phi = torch.tensor(Phi0, dtype=torch.float32, device="cuda")
    g = torch.empty_like(Phi)
    err = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    for b in batches:
        ctx.cp_step(b, Phi_ref, lr, grad=g_ref)
        ctx.sync()
        assert _noalloc(lib, b, Wd, m1d, K, K, a0, theta, Phi, lr, g, err) == lib.OK
        torch.cuda.synchronize()
        assert int(err.item()) == 0
        assert C.rel(g.cpu().numpy(), g_ref.cpu().numpy()) < TOL32
        assert C.rel(Phi.cpu().numpy(), Phi_ref.cpu().numpy()) < TOL32
    ctx.close()


def test_noalloc_documented_size_then_smaller_layout(lib):
    """V = 4096, D = K = 64, 2048 documents (the size the header quotes as
    fitting), two calls; then the small workload (V = 500, K = 10), whose
    layout of the array differs, on the contents the larger calls left."""
    base = ts.WORKLOADS["small_v500_k10"]
    sp = replace(base, name="noalloc_v4096_k64", V=4096, K=64, lam=30.0, seed=base.seed + 4096)
    cdf, mu = ts.topics(sp)
    W, m1 = O.population_whitening(mu, np.full(sp.K, 1.0 / sp.K))
    W, m1 = W.astype(np.float32).astype(np.float64), m1.astype(np.float32).astype(np.float64)
    c = ts.corpus(sp.with_docs(4096), cdf=cdf)
    big = [lib.DeviceCSR.from_corpus(c.rows(0, 2048)), lib.DeviceCSR.from_corpus(c.rows(2048, 4096))]
    _against_context(lib, sp.V, sp.K, float(sp.alpha0), W, m1, ts.initial_factors(sp.seed + 1, sp.K, sp.K), big)

    name = "small_v500_k10"
    sp = ts.WORKLOADS[name]
    W, m1 = C.population_whitening(name)
    c = C.corpus(name, 2000)
    small = [lib.DeviceCSR.from_corpus(c.rows(0, 1000)), lib.DeviceCSR.from_corpus(c.rows(1000, 2000))]
    _against_context(lib, sp.V, sp.K, float(sp.alpha0), W, m1, ts.initial_factors(sp.seed + 1, sp.K, sp.K), small)


def test_noalloc_corrupt_batch_then_valid_batch(lib):
    """A word index outside [0, V): err_out is non-zero and Phi is left bit for
    bit as it was; the next valid call reports 0 and matches the context step."""
    name = "small_v500_k10"
    sp = ts.WORKLOADS[name]
    W, m1 = C.population_whitening(name)
    c = C.corpus(name, 200)
    indptr, indices, counts = c.indptr.copy(), c.indices.copy(), c.counts.copy()
    indices[int(indptr[7]) + 1] = sp.V + 11
    bad = lib.DeviceCSR.from_arrays(indptr, indices, counts, sp.V)
    Phi0 = ts.initial_factors(sp.seed + 1, sp.K, sp.K)
    Wd = torch.tensor(W, dtype=torch.float32, device="cuda")
    m1d = torch.tensor(m1, dtype=torch.float32, device="cuda")
    Phi = torch.tensor(Phi0, dtype=torch.float32, device="cuda")
    before = Phi.cpu().numpy().copy()
    err = torch.zeros((1,), dtype=torch.int32, device="cuda")
    assert _noalloc(lib, bad, Wd, m1d, sp.K, sp.K, float(sp.alpha0), 0.0, Phi, 0.01, None, err) == lib.OK
    torch.cuda.synchronize()
    assert int(err.item()) != 0
    assert np.array_equal(Phi.cpu().numpy(), before)
    _against_context(lib, sp.V, sp.K, float(sp.alpha0), W, m1, Phi0, [lib.DeviceCSR.from_corpus(c)])


def test_noalloc_rejects_sizes_beyond_its_scratch(lib):
    raw = lib.load()
    V, K = 100_000, 64
    b = lib.DeviceCSR.from_arrays([0, 1], [5], [3], V)
    s = b.struct()
    W = torch.zeros((V, K), dtype=torch.float32, device="cuda")
    m1 = torch.zeros(K, dtype=torch.float32, device="cuda")
    Phi = torch.zeros((K, K), dtype=torch.float32, device="cuda")
    st = raw.tlda_cp_step_noalloc(ctypes.byref(s), W.data_ptr(), m1.data_ptr(), K, K, 1.0, 0.0,
                                  Phi.data_ptr(), 0.1, None, None,
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == lib.ERR_OOM
    # a batch count beyond the bound is rejected before any size arithmetic
    s.n_docs = 2_000_000_000
    st = raw.tlda_cp_step_noalloc(ctypes.byref(s), W.data_ptr(), m1.data_ptr(), K, K, 1.0, 0.0,
                                  Phi.data_ptr(), 0.1, None, None,
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == lib.ERR_INVALID
