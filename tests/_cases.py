"""Seeded test inputs shared by the GPU parity tests: corpora from the
generator, whitenings and expected values from the FP64 oracle only."""
from __future__ import annotations

import functools

import numpy as np

import tlda_synth as ts
from oracle import tlda_oracle as O


@functools.lru_cache(maxsize=8)
def topics(name):
    return ts.topics(ts.WORKLOADS[name])


@functools.lru_cache(maxsize=8)
def corpus(name, n_docs):
    sp = ts.WORKLOADS[name]
    cdf, _ = topics(name)
    return ts.corpus(sp.with_docs(n_docs), cdf=cdf)


@functools.lru_cache(maxsize=8)
def population_whitening(name):
    """(W, m1) whitening the population M2 of the workload (oracle), FP32-rounded."""
    sp = ts.WORKLOADS[name]
    _, mu = topics(name)
    h = np.full(sp.K, 1.0 / sp.K)
    W, m1 = O.population_whitening(mu, h)
    return W.astype(np.float32).astype(np.float64), m1.astype(np.float32).astype(np.float64)


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def col_rel(a, b):
    """Largest per-column max-norm error: max over columns n of
    max_i |a_in - b_in| / max_i |b_in|.  Unlike the relative Frobenius error
    of the whole matrix, it fails when one column (a padded or edge topic
    column, or one wrong entry) is off while the rest are right."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if a.ndim == 1:
        a, b = a[:, None], b[:, None]
    scale = np.abs(b).max(axis=0)
    err = np.abs(a - b).max(axis=0)
    return float((err / np.maximum(scale, 1e-300)).max())


def assert_bf16_parity(a, b, tol, what=""):
    """The BF16 form's parity bar: relative Frobenius error and per-column
    max-norm error (col_rel) both within tol."""
    fr, cr = rel(a, b), col_rel(a, b)
    print(f"parity {what}: frobenius {fr:.3e}, worst column {cr:.3e}")
    assert fr < tol, (what, "frobenius", fr)
    assert cr < tol, (what, "worst column", cr)


def data_term_magnitude(batch, V, W, m1, Phi, alpha0):
    """Scale of the rounding error of the BF16 form's data term on one batch
    (D x K): c3/S3 sum_j |u_j| bbar_j^T over the batch's nonzeros j (word m,
    count f, document d), with q_j = u_m Phi, ybar_d = sum_{j in d} f_j |q_j|,
    r_d = sum_{j in d} f_j q_j^2 and
      bbar_j = f_j (ybar_d^2 + r_d + 2 q_j^2 + 2 |q_j| ybar_d),
    the magnitudes of the terms of b''_j = f_j (y_d^2 - r_d + 2 q_j^2 - 2 q_j y_d)
    that the BF16 form rounds (reading O: each operand rounded once, FP32
    sums).  A first-order rounding error of every entry is a small multiple
    of the BF16 unit roundoff times this scale.  When a batch's triples
    cancel (one document: z = y^2 - r is a small difference of large terms),
    the scale is far above the result itself."""
    indptr = np.asarray(batch.indptr, dtype=np.int64)
    idx = np.asarray(batch.indices, dtype=np.int64)
    f = np.asarray(batch.counts, dtype=np.float64)
    U = np.asarray(W, dtype=np.float64) - np.asarray(m1, dtype=np.float64)[None, :]
    q = U[idx] @ np.asarray(Phi, dtype=np.float64)
    doc = np.repeat(np.arange(len(indptr) - 1), np.diff(indptr))
    nd = len(indptr) - 1
    ybar = np.zeros((nd, q.shape[1]))
    r = np.zeros((nd, q.shape[1]))
    np.add.at(ybar, doc, f[:, None] * np.abs(q))
    np.add.at(r, doc, f[:, None] * q * q)
    yb, rd = ybar[doc], r[doc]
    bbar = f[:, None] * (yb * yb + rd + 2.0 * q * q + 2.0 * np.abs(q) * yb)
    Ld = np.zeros(nd)
    np.add.at(Ld, doc, f)
    S3 = float(np.sum(Ld * (Ld - 1) * (Ld - 2)))
    c3 = (alpha0 + 1.0) * (alpha0 + 2.0) / 2.0
    return c3 / S3 * (np.abs(U[idx]).T @ bbar)


def assert_bf16_parity_scaled(a, b, magnitude, tol, what=""):
    """The BF16 bar for a one-document batch: per column, the largest error
    relative to the column's largest rounding-error scale (data_term_magnitude,
    times 3 for the gradient), plus the relative Frobenius error."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    cr = float((np.abs(a - b).max(axis=0) / np.maximum(np.asarray(magnitude).max(axis=0), 1e-300)).max())
    print(f"parity {what}: worst column (of the rounding-error scale) {cr:.3e}, "
          f"worst column (of the result) {col_rel(a, b):.3e}")
    assert cr < tol, (what, "worst column of the scale", cr)


def assert_bf16_pass_parity(change, change_ref, steps_ref, tol, what="", step_scales=None):
    """The BF16 bar for the change of Phi over a pass of several steps:
    relative Frobenius error of the change, and per column the largest error
    of the change relative to that column's summed step sizes,
    sum_t max_i |step_t[i, n]| (steps_ref: the reference's per-step updates).
    Each step's rounding error scales with that step, and a pass adds them;
    when one step is much larger than the net change of a column, the summed
    step sizes, not the net change, are the column's scale.  step_scales
    (optional, per step: a per-column scale or None) replaces a step's size by
    its rounding-error scale, for one-document steps (data_term_magnitude)."""
    a = np.asarray(change, dtype=np.float64)
    b = np.asarray(change_ref, dtype=np.float64)
    per = []
    for t, st in enumerate(steps_ref):
        sz = np.abs(np.asarray(st, dtype=np.float64)).max(axis=0)
        if step_scales is not None and step_scales[t] is not None:
            sz = np.maximum(sz, step_scales[t])
        per.append(sz)
    scale = np.sum(per, axis=0)
    fr = rel(a, b)
    cr = float((np.abs(a - b).max(axis=0) / np.maximum(scale, 1e-300)).max())
    print(f"parity {what}: frobenius {fr:.3e}, worst column (of summed steps) {cr:.3e}")
    assert fr < tol, (what, "frobenius", fr)
    assert cr < tol, (what, "worst column", cr)
