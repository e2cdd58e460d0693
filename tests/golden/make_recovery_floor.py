"""Writes recovery_floor_stream_v20k_k100.txt: the oracle's topic-recovery
floor on the stream workload (V = 20,000, K = 100, alpha0 = 2, Poisson(12)
lengths, Dirichlet(0.1) topics) with the population whitening.

Oracle only: the population whitening W (FP32 values) of the generator's
topics, the whitened third moment T = M3(W, W, W) of the first N documents
(whitened_third_moment_chunked), the tensor power method with deflation, the
unwhitening of its eigenpairs, clipping, and the Hungarian matching on
per-topic l1 (section "Recovering the Topic Model Parameters").  Nothing here
runs on the GPU.

  python tests/golden/make_recovery_floor.py [N]     (default N = 1,000,000)
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import tlda_synth as ts  # noqa: E402
from oracle import tlda_oracle as O  # noqa: E402


def main():
    n = int(sys.argv[1]) if len(sys.argv) > 1 else 1_000_000
    sp = ts.WORKLOADS["stream_v20k_k100"]
    cdf, mu = ts.topics(sp)
    h = np.full(sp.K, 1.0 / sp.K)
    W, _ = O.population_whitening(mu, h)
    W = W.astype(np.float32).astype(np.float64)
    t0 = time.time()
    c = ts.corpus(sp.with_docs(n), n_docs=n, cdf=cdf)
    st = O.ingest(c.indptr, c.indices, c.counts, sp.V)
    M1 = O.first_moment(st["C"], st["T"])
    T = O.whitened_third_moment_chunked(c.indptr, c.indices, c.counts, sp.V, W, M1, float(sp.alpha0))
    t1 = time.time()
    lams, V = O.tensor_power_method(T, sp.K, n_restarts=10, n_iters=30, seed=0)
    mu_p, _ = O.unwhiten_power(lams, V, W)
    _, l1, _ = O.match_topics(O.clip_normalise(mu_p)[0], mu)
    t2 = time.time()
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "recovery_floor_stream_v20k_k100.txt")
    with open(out, "w") as f:
        f.write("# Oracle topic-recovery floor, workload stream_v20k_k100 (V=20000, K=100, alpha0=2), written by\n")
        f.write(f"# tests/golden/make_recovery_floor.py {n}: population whitening (FP32 values), T = M3(W,W,W)\n")
        f.write(f"# of the first {n} documents, tensor power method (10 restarts x 30 iterations per\n")
        f.write("# component, deflation), unwhitened, clipped, Hungarian matching on per-topic l1.\n")
        f.write(f"docs {n}\n")
        f.write(f"l1_mean {l1.mean():.6f}\nl1_median {np.median(l1):.6f}\nl1_max {l1.max():.6f}\n")
        f.write(f"topics_above_1 {(l1 > 1.0).sum()}\n")
    print(f"T in {t1 - t0:.0f} s, power method in {t2 - t1:.0f} s: l1 mean {l1.mean():.4f} median "
          f"{np.median(l1):.4f} max {l1.max():.4f}")


if __name__ == "__main__":
    main()
