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
