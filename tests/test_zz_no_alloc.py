"""The allocation-free CP step (tlda_cp_step_noalloc), for callers that cannot
allocate device memory, against the context-based tlda_cp_step: same batches,
same starting factors, two calls in a row, FP32 tolerance.  This file is
collected last on purpose, so a run that stops at the first failure has
already run every other test."""
import ctypes

import numpy as np
import pytest
import torch

import tlda_synth as ts
from tests import _cases as C

pytestmark = pytest.mark.gpu

TOL32 = 1e-5


def test_noalloc_step_matches_context_step_twice(lib):
    name = "small_v500_k10"
    sp = ts.WORKLOADS[name]
    W, m1 = C.population_whitening(name)
    c = C.corpus(name, 2000)
    batches = [lib.DeviceCSR.from_corpus(c.rows(0, 1000)), lib.DeviceCSR.from_corpus(c.rows(1000, 2000))]
    Phi0 = ts.initial_factors(sp.seed + 1, sp.K, sp.K)
    lr, a0, theta = 0.01, float(sp.alpha0), 0.0

    ctx = lib.TLDA(sp.V, sp.K, alpha0=a0, theta=theta)
    ctx.set_whitening(torch.tensor(W, dtype=torch.float32), torch.tensor(m1, dtype=torch.float32))
    Phi_ref = torch.tensor(Phi0, dtype=torch.float32, device="cuda")
    g_ref = torch.empty_like(Phi_ref)

    raw = lib.load()
    Wd = torch.tensor(W, dtype=torch.float32, device="cuda")
    m1d = torch.tensor(m1, dtype=torch.float32, device="cuda")
    Phi = torch.tensor(Phi0, dtype=torch.float32, device="cuda")
    g = torch.empty_like(Phi)
    err = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream

    for b in batches:
        ctx.cp_step(b, Phi_ref, lr, grad=g_ref)
        ctx.sync()
        s = b.struct()
        st = raw.tlda_cp_step_noalloc(ctypes.byref(s), Wd.data_ptr(), m1d.data_ptr(), sp.K, sp.K,
                                      a0, theta, Phi.data_ptr(), lr, g.data_ptr(), err.data_ptr(),
                                      ctypes.c_void_p(stream))
        assert st == lib.OK
        torch.cuda.synchronize()
        assert int(err.item()) == 0
        assert C.rel(g.cpu().numpy(), g_ref.cpu().numpy()) < TOL32
        assert C.rel(Phi.cpu().numpy(), Phi_ref.cpu().numpy()) < TOL32
    ctx.close()


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
