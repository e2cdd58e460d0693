"""The CP objective as an autograd function: the implicit gradient (eq.
vec_deriv with the centred batch tensor of Theorem 1) against torch autograd
of the explicit k^3 objective at k = 16 and 32, and the GPU TLDALoss against
the same explicit objective and against finite differences of its own loss.

The explicit objective is written here from the section "Stochastic Tensor
Gradient Descent":  L(Phi) = (1+theta)/2 sum_ij (phi_i.phi_j)^3
                           - sum_i T_B(phi_i, phi_i, phi_i),
with T_B the oracle's explicit k x k x k batch tensor (pinned separately by
brute force over token triples and by Theorem 1)."""
from __future__ import annotations

from dataclasses import replace

import numpy as np
import pytest
import torch

import tlda_synth as ts
from oracle import tlda_oracle as O

from ._cases import corpus, population_whitening, rel


def _explicit_loss(Phi: torch.Tensor, T: torch.Tensor, theta: float) -> torch.Tensor:
    G = Phi.T @ Phi
    return (1 + theta) / 2 * (G ** 3).sum() - torch.einsum("ijl,ia,ja,la->", T, Phi, Phi, Phi)


def _case(k: int, n_docs: int = 400):
    """A V = 500 corpus from a k-topic model, its population whitening (FP32
    values) and the oracle's explicit batch tensor."""
    sp = replace(ts.WORKLOADS["small_v500_k10"], K=k, name=f"small_v500_k{k}").with_docs(n_docs)
    cdf, mu = ts.topics(sp)
    c = ts.corpus(sp, cdf=cdf)
    W, m1 = O.population_whitening(mu, np.full(k, 1.0 / k))
    W = W.astype(np.float32).astype(np.float64)
    m1 = m1.astype(np.float32).astype(np.float64)
    a0 = float(sp.alpha0)
    T = O.batch_tensor(c.indptr, c.indices, c.counts, sp.V, W, m1, a0)
    Phi0 = ts.initial_factors(sp.seed, k, k).astype(np.float64)
    return sp, c, W, m1, a0, T, Phi0


@pytest.mark.parametrize("k", [16, 32])
@pytest.mark.parametrize("theta", [0.0, 0.5])
def test_implicit_gradient_matches_autograd_of_explicit_objective(k, theta):
    sp, c, W, m1, a0, T, Phi0 = _case(k)
    P = torch.tensor(Phi0, dtype=torch.float64, requires_grad=True)
    loss = _explicit_loss(P, torch.tensor(T), theta)
    loss.backward()
    g = O.cp_grad_implicit(c.indptr, c.indices, c.counts, sp.V, W, m1, Phi0, a0, theta)
    assert rel(g["grad"], P.grad.numpy()) < 1e-12
    assert abs(g["loss"] - loss.item()) <= 1e-12 * max(1.0, abs(loss.item()))


# ----------------------------------------------------------------------------- GPU
def _model(V, k, W, m1, a0, theta=0.0, max_batch=8192):
    from paper_2511_07809_gb300 import tlda
    m = tlda.TLDA(V, k, alpha0=a0, theta=theta, precision="fp32", max_batch=max_batch)
    m.set_whitening(torch.tensor(W, dtype=torch.float32), torch.tensor(m1, dtype=torch.float32))
    return m


@pytest.mark.gpu
@pytest.mark.parametrize("k", [16, 32])
def test_tlda_loss_matches_explicit_autograd(lib, k):
    from paper_2511_07809_gb300 import tlda
    theta = 0.25
    sp, c, W, m1, a0, T, Phi0 = _case(k)
    model = _model(sp.V, k, W, m1, a0, theta)
    batch = tlda.DeviceCSR.from_corpus(c)
    Phi = torch.tensor(Phi0, dtype=torch.float32, device="cuda", requires_grad=True)
    loss = tlda.tlda_loss(Phi, model, batch)
    loss.backward()

    Pr = torch.tensor(Phi0, dtype=torch.float64, requires_grad=True)
    ref = _explicit_loss(Pr, torch.tensor(T), theta)
    ref.backward()
    # FP32 rounding acts on the orthogonality term and on the data term
    # separately; the tolerance is 1e-5 of their sizes, not of their difference.
    with torch.no_grad():
        orth = 3 * (1 + theta) * Pr @ ((Pr.T @ Pr) ** 2)
    g_ref = Pr.grad.numpy()
    scale = (np.linalg.norm(orth.numpy()) + np.linalg.norm(g_ref - orth.numpy())) / np.linalg.norm(g_ref)
    assert rel(Phi.grad.cpu().numpy(), g_ref) < 1e-5 * scale
    assert abs(loss.item() - ref.item()) <= 1e-5 * max(1.0, abs(ref.item()))
    assert torch.equal(Phi.detach().cpu(), torch.tensor(Phi0, dtype=torch.float32))  # lr = 0: unchanged
    model.close()


@pytest.mark.gpu
def test_tlda_loss_drives_torch_sgd_like_cp_step(lib):
    """A torch.optim.SGD step on TLDALoss equals tlda_cp_step with the same lr."""
    from paper_2511_07809_gb300 import tlda
    sp, c, W, m1, a0, T, Phi0 = _case(16)
    model = _model(sp.V, 16, W, m1, a0)
    batch = tlda.DeviceCSR.from_corpus(c)
    lr = 1e-2
    Phi = torch.tensor(Phi0, dtype=torch.float32, device="cuda", requires_grad=True)
    opt = torch.optim.SGD([Phi], lr=lr)
    opt.zero_grad()
    tlda.tlda_loss(Phi, model, batch).backward()
    opt.step()
    ref = torch.tensor(Phi0, dtype=torch.float32, device="cuda")
    model.cp_step(batch, ref, lr)
    assert rel(Phi.detach().cpu().numpy(), ref.cpu().numpy()) < 1e-6
    model.close()


@pytest.mark.gpu
def test_tlda_loss_finite_differences_at_scale(lib):
    """Directional derivatives of the GPU FP32 loss against its gradient at
    V = 50,000, K = D = 200 and a full 8,192-document minibatch.  Along a
    line the loss is a polynomial of degree 6, so a degree-6 fit through 7
    points gives the derivative without truncation error; what is left is
    FP32 rounding of the loss."""
    from paper_2511_07809_gb300 import tlda
    name = "scale_v50k_k200"
    sp = ts.WORKLOADS[name]
    W, m1 = population_whitening(name)
    c = corpus(name, 8192)
    model = _model(sp.V, sp.K, W, m1, float(sp.alpha0))
    batch = tlda.DeviceCSR.from_corpus(c)
    Phi0 = torch.tensor(ts.initial_factors(sp.seed, sp.K, sp.K), dtype=torch.float32, device="cuda")
    G = torch.empty_like(Phi0)
    model.cp_step(batch, Phi0.clone(), 0.0, grad=G)
    g = G.double()
    gn = g.norm().item()
    dirs = [g / gn]
    for tag in (1, 2):
        d = torch.tensor(ts.gaussian(sp.seed, 0x4644 + tag, sp.K * sp.K), dtype=torch.float64,
                         device="cuda").reshape(sp.K, sp.K)
        dirs.append(d / d.norm())
    h = 0.1
    ts_ = np.arange(-3, 4) * h
    A = np.vander(ts_, 7, increasing=True)
    for d in dirs:
        ls = []
        for t in ts_:
            P = (Phi0.double() + t * d).float().contiguous()
            ls.append(model.cp_step(batch, P, 0.0, want_loss=True))
        coef = np.linalg.solve(A, np.array(ls))
        fd = coef[1]
        exact = float((g * d).sum().item())
        assert abs(fd - exact) <= 1e-3 * gn, (fd, exact, gn)
    model.close()
