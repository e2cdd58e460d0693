"""The persistent pass kernel of tlda_cp_pass (BF16 form, D = K in (64, 128]):
every step of a pass in one cooperative launch, against the FP64 oracle's
sequential CP steps (section "Fully Online Implementation", eq. vec_deriv),
for several tile sizes; host-input staging in several segments against the
device-input pass; empty minibatches inside a pass; the tile tuner; a corrupt
batch in the middle of a pass."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import tlda_synth as ts
from oracle import tlda_oracle as O

from . import _cases as C

pytestmark = pytest.mark.gpu
TOL16 = 2e-2
NAME = "stream_v20k_k100"


def _ctx(lib, max_batch=8192):
    sp = ts.WORKLOADS[NAME]
    W, m1 = C.population_whitening(NAME)
    t = lib.TLDA(sp.V, sp.K, alpha0=float(sp.alpha0), precision="bf16", max_batch=max_batch)
    t.set_whitening(torch.tensor(W, dtype=torch.float32), torch.tensor(m1, dtype=torch.float32))
    return t, W, m1


def _phi0(sp):
    return ts.initial_factors(sp.seed, sp.K, sp.K).astype(np.float64)


def _oracle_pass(c, offs, sp, W, m1, Phi0, lr, same_token=True, scales=None):
    """The oracle's sequential steps: final Phi, losses and per-step updates.
    With a list `scales`, appends per step the rounding-error scale of a
    one-document step (3 lr times its data term's) or None."""
    P, losses, steps = Phi0.copy(), [], []
    for b in range(len(offs) - 1):
        r = c.rows(offs[b], offs[b + 1])
        Pn, g = O.cp_step(r.indptr, r.indices, r.counts, sp.V, W, m1, P, lr, float(sp.alpha0), 0.0,
                          same_token=same_token)
        if scales is not None:
            scales.append(3.0 * lr * C.data_term_magnitude(r, sp.V, W, m1, P, float(sp.alpha0)).max(axis=0)
                          if r.n_docs == 1 else None)
        steps.append(Pn - P)
        P = Pn
        losses.append(g["loss"])
    return P, np.array(losses), steps


@pytest.mark.parametrize("cap", [1, 8, 32])
def test_pass_tile_sizes_match_oracle(lib, cap):
    sp = ts.WORKLOADS[NAME]
    t, W, m1 = _ctx(lib)
    assert t.autotune(fixed=cap) == cap
    c = C.corpus(NAME, 14000)
    # ragged sizes: below and above one tile per SM, one document, an exact 8192
    offs = [0, 700, 701, 700 + 4099, 700 + 4099 + 8192, 14000]
    Phi0 = _phi0(sp)
    Phi = torch.tensor(Phi0, dtype=torch.float32, device="cuda")
    lr = 0.002
    losses = t.cp_pass(lib.DeviceCSR.from_corpus(c), offs, Phi, lr, losses=True)
    scales = []
    P, lo, steps = _oracle_pass(c, offs, sp, W, m1, Phi0, lr, scales=scales)
    assert np.all(np.abs(losses - lo) <= TOL16 * np.abs(lo))
    C.assert_bf16_pass_parity(Phi.cpu().numpy() - Phi0, P - Phi0, steps, TOL16, f"Phi change, cap {cap}",
                              step_scales=scales)
    t.close()


def test_pass_without_same_token_correction(lib):
    """same_token_correction = 0 (the data term of eq. vec_deriv alone) in the
    persistent kernel, against the oracle's steps of the same form."""
    sp = ts.WORKLOADS[NAME]
    W, m1 = C.population_whitening(NAME)
    t = lib.TLDA(sp.V, sp.K, alpha0=float(sp.alpha0), precision="bf16", same_token=False)
    t.set_whitening(torch.tensor(W, dtype=torch.float32), torch.tensor(m1, dtype=torch.float32))
    t.autotune(fixed=18)
    c = C.corpus(NAME, 12000)
    offs = [0, 900, 4000, 9100, 12000]
    Phi0 = _phi0(sp)
    Phi = torch.tensor(Phi0, dtype=torch.float32, device="cuda")
    losses = t.cp_pass(lib.DeviceCSR.from_corpus(c), offs, Phi, 0.002, losses=True)
    P, lo, steps = _oracle_pass(c, offs, sp, W, m1, Phi0, 0.002, same_token=False)
    assert np.all(np.abs(losses - lo) <= TOL16 * np.abs(lo))
    C.assert_bf16_pass_parity(Phi.cpu().numpy() - Phi0, P - Phi0, steps, TOL16, "Phi change, correction off")
    t.close()


def test_pass_host_segments_equal_device_pass(lib):
    """A host-input pass large enough to be staged in several segments gives
    the device-input pass's Phi bit for bit (same kernel, same tiles)."""
    sp = ts.WORKLOADS[NAME]
    t, W, m1 = _ctx(lib)
    t.autotune(fixed=32)
    n = 1_500_000  # ~18M nonzeros: ~37M staged words, more than four 8M-word segments
    c = C.corpus(NAME, n)
    sizes = ts.batch_sizes(sp.with_docs(n))
    offs = np.concatenate([[0], np.cumsum(sizes)])
    offs = offs[offs <= n]
    if offs[-1] != n:
        offs = np.append(offs, n)
    Phi0 = torch.tensor(_phi0(sp), dtype=torch.float32, device="cuda")
    Pd, Ph = Phi0.clone(), Phi0.clone()
    ld = t.cp_pass(lib.DeviceCSR.from_corpus(c), offs, Pd, 1e-3, losses=True)
    lh = t.cp_pass(lib.DeviceCSR.from_corpus(c, device="cpu", pin=True), offs, Ph, 1e-3,
                   host_input=True, losses=True)
    assert torch.equal(Pd, Ph)
    assert np.allclose(ld, lh, rtol=1e-9, atol=0)
    assert np.isfinite(Pd.cpu().numpy()).all()
    t.close()


@pytest.mark.parametrize("host", [False, True])
def test_pass_with_empty_batches_equals_pass_without(lib, host):
    """Empty minibatches in a persistent pass: first, two in a row in the
    middle, and last.  An empty batch has S3 = 0, so its step leaves Phi as it
    is and its loss is 0.  With those steps taken out the pass is the same,
    bit for bit (fixed tile size, so both passes run the same tiles), and a
    pass of empty minibatches only changes nothing."""
    sp = ts.WORKLOADS[NAME]
    c = C.corpus(NAME, 9000)
    dev = lib.DeviceCSR.from_corpus(c, device="cpu", pin=True) if host else lib.DeviceCSR.from_corpus(c)
    with_empty = [0, 0, 700, 700, 700, 4800, 4801, 9000, 9000]
    without = [0, 700, 4800, 4801, 9000]
    t, W, m1 = _ctx(lib)
    t.autotune(fixed=32)
    Phi0 = torch.tensor(_phi0(sp), dtype=torch.float32, device="cuda")
    Pa, Pb, Pe = Phi0.clone(), Phi0.clone(), Phi0.clone()
    la = t.cp_pass(dev, with_empty, Pa, 2e-3, host_input=host, losses=True)
    lb = t.cp_pass(dev, without, Pb, 2e-3, host_input=host, losses=True)
    t.cp_pass(dev, [0, 0, 0, 0], Pe, 2e-3, host_input=host)
    assert torch.equal(Pa, Pb)
    assert not torch.equal(Pb, Phi0)
    assert torch.equal(Pe, Phi0)
    assert la[0] == 0.0 and la[2] == 0.0 and la[3] == 0.0 and la[-1] == 0.0
    assert np.allclose(la[[1, 4, 5, 6]], lb, rtol=1e-9, atol=0)  # block sums in atomic order
    t.close()


def test_pass_and_graph_path_agree(lib, monkeypatch):
    """The persistent kernel and the per-step graph path of the same form."""
    sp = ts.WORKLOADS[NAME]
    c = C.corpus(NAME, 20000)
    offs = [0, 512, 4000, 12192, 20000]
    Phi0 = _phi0(sp)
    out = []
    for no_pass in (False, True):
        if no_pass:
            monkeypatch.setenv("TLDA_NO_PASS", "1")
        t, W, m1 = _ctx(lib)
        Phi = torch.tensor(Phi0, dtype=torch.float32, device="cuda")
        t.cp_pass(lib.DeviceCSR.from_corpus(c), offs, Phi, 0.002)
        out.append(Phi.cpu().numpy())
        t.close()
    P, _, steps = _oracle_pass(c, offs, sp, W, m1, Phi0, 0.002)
    for o in out:
        C.assert_bf16_pass_parity(o - Phi0, P - Phi0, steps, TOL16, "Phi change")


def test_autotune_leaves_phi_and_state(lib, tmp_path):
    sp = ts.WORKLOADS[NAME]
    t, W, m1 = _ctx(lib)
    c = C.corpus(NAME, 30000)
    offs = np.arange(0, 30001, 3000)
    dev = lib.DeviceCSR.from_corpus(c)
    Phi = torch.tensor(_phi0(sp), dtype=torch.float32, device="cuda")
    before = Phi.clone()
    t.save_state(tmp_path / "a.tlda")
    cap = t.autotune(dev, offs, Phi)
    assert cap in (8, 14, 16, 18, 20, 24, 28, 32)
    assert torch.equal(Phi, before)
    t.save_state(tmp_path / "b.tlda")
    assert (tmp_path / "a.tlda").read_bytes() == (tmp_path / "b.tlda").read_bytes()
    # the pass then runs with that size: equal to a context fixed to it
    t.cp_pass(dev, offs, Phi, 0.002)
    t2, _, _ = _ctx(lib)
    t2.autotune(fixed=cap)
    P2 = before.clone()
    t2.cp_pass(dev, offs, P2, 0.002)
    assert torch.equal(Phi, P2)
    t.close()
    t2.close()


def test_corrupt_batch_stops_updates_from_that_step(lib):
    sp = ts.WORKLOADS[NAME]
    t, W, m1 = _ctx(lib)
    c = C.corpus(NAME, 12000)
    offs = [0, 3000, 6000, 9000, 12000]
    counts = c.counts.copy()
    counts[c.indptr[7000] + 1] = 0  # inside batch 2
    dev = lib.DeviceCSR.from_arrays(c.indptr, c.indices, counts, sp.V)
    Phi0 = _phi0(sp)
    Phi = torch.tensor(Phi0, dtype=torch.float32, device="cuda")
    with pytest.raises(lib.TLDAError) as e:
        t.cp_pass(dev, offs, Phi, 0.002)
    assert e.value.status == lib.ERR_INVALID
    P, _, steps = _oracle_pass(c, offs[:3], sp, W, m1, Phi0, 0.002)
    C.assert_bf16_pass_parity(Phi.cpu().numpy() - Phi0, P - Phi0, steps, TOL16, "Phi change up to the corrupt batch")
    # the error was taken: the next pass on valid data runs
    t.cp_pass(lib.DeviceCSR.from_corpus(c), offs[:2], Phi, 0.002)
    t.close()


def test_bench_sized_pass_sampled_steps(lib):
    """The bench's configuration: the streaming workload's seeded minibatch
    sequence (512..8192 documents), the persistent kernel with the tuned tile
    size.  Steps sampled deep into a 400-step pass are checked against the
    oracle's step from the GPU's own Phi before it: the update
    Phi_{t+1} - Phi_t = -lr grad and the loss."""
    sp = ts.WORKLOADS[NAME]
    sizes = ts.batch_sizes(sp)[:400]
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    n = int(offs[-1])
    c = C.corpus(NAME, n)
    t, W, m1 = _ctx(lib)
    dev = lib.DeviceCSR.from_corpus(c)
    lr = 5e-4  # with this whitening, SGD at 2e-3 leaves the basin after ~250 steps (the oracle too)
    Phi = torch.tensor(_phi0(sp), dtype=torch.float32, device="cuda")
    cap = t.autotune(dev, offs[:65], Phi)
    assert cap in (8, 14, 16, 18, 20, 24, 28, 32)
    prev = 0
    for s_ in (137, 283, 399):
        t.cp_pass(dev, offs[prev:s_ + 1], Phi, lr)  # steps prev .. s_-1
        before = Phi.cpu().numpy().astype(np.float64)
        loss = t.cp_pass(dev, offs[s_:s_ + 2], Phi, lr, losses=True)[0]  # step s_
        r = c.rows(int(offs[s_]), int(offs[s_ + 1]))
        ref, g = O.cp_step(r.indptr, r.indices, r.counts, sp.V, W, m1, before, lr, float(sp.alpha0), 0.0)
        step_gpu = Phi.cpu().numpy().astype(np.float64) - before
        C.assert_bf16_parity(step_gpu, ref - before, TOL16, f"update of step {s_}")
        assert abs(loss - g["loss"]) <= TOL16 * abs(g["loss"]), s_
        prev = s_ + 1
    t.close()


def test_no_wait_pass_equals_waiting_pass(lib):
    """tlda_cp_pass with TLDA_NO_WAIT returns once the pass is enqueued: the
    same Phi bit for bit, the same step losses (in device memory; the loss
    sums are double atomics, so equal to rounding), and a corrupt batch is
    reported by the next sync instead of by the call.  Host input cannot
    skip the wait."""
    import ctypes
    sp = ts.WORKLOADS[NAME]
    t, W, m1 = _ctx(lib)
    t.autotune(fixed=16)
    c = C.corpus(NAME, 12000)
    offs = [0, 3000, 3001, 6000, 6000, 9000, 12000]  # a one-document and an empty batch
    nb = len(offs) - 1
    dev = lib.DeviceCSR.from_corpus(c)
    Phi0 = torch.tensor(_phi0(sp), dtype=torch.float32, device="cuda")
    P1 = Phi0.clone()
    l1 = t.cp_pass(dev, offs, P1, 0.002, losses=True)
    P2 = Phi0.clone()
    dl = torch.full((nb,), float("nan"), dtype=torch.float64, device="cuda")
    assert t.cp_pass(dev, offs, P2, 0.002, wait=False, device_losses=dl) is None
    t.sync()
    assert torch.equal(P1, P2)
    np.testing.assert_allclose(dl.cpu().numpy(), l1, rtol=1e-12, atol=0.0)
    assert dl[3].item() == 0.0  # the empty batch
    P3 = Phi0.clone()
    t.cp_pass(dev, offs, P3, 0.002, wait=False)  # no losses asked for
    t.sync()
    assert torch.equal(P1, P3)
    # a corrupt batch (inside batch 4): the waiting call raises, the no-wait
    # call returns and the next sync raises; Phi the same either way
    counts = c.counts.copy()
    counts[c.indptr[7000] + 1] = 0
    bad = lib.DeviceCSR.from_arrays(c.indptr, c.indices, counts, sp.V)
    P4 = Phi0.clone()
    with pytest.raises(lib.TLDAError) as e:
        t.cp_pass(bad, offs, P4, 0.002)
    assert e.value.status == lib.ERR_INVALID
    P5 = Phi0.clone()
    t.cp_pass(bad, offs, P5, 0.002, wait=False)
    with pytest.raises(lib.TLDAError) as e:
        t.sync()
    assert e.value.status == lib.ERR_INVALID
    assert torch.equal(P4, P5)
    t.sync()  # taken: nothing pending
    host = lib.DeviceCSR.from_corpus(c, device="cpu", pin=True)
    s = host.struct()
    off = np.asarray(offs, dtype=np.int64)
    st = t.lib.tlda_cp_pass(t.h, ctypes.byref(s), off.ctypes.data, nb, P5.data_ptr(), ctypes.c_float(0.002),
                            lib.HOST_INPUT | lib.NO_WAIT, None)
    assert st == lib.ERR_INVALID
    t.close()
