"""The N > 1 path of bench.py on CPU ranks (gloo, world size 2): each rank
runs an independent replica on its own document shard, with no exchange in
the data path; the job's throughput is every rank's documents over the
slowest rank's time.  Also checks that the replicas' shards are disjoint
slices of one seeded document stream and that a rank's replica step does not
depend on the other rank."""
from __future__ import annotations

import os
import socket

import numpy as np
import torch.multiprocessing as mp

import tlda_synth as ts
from oracle import tlda_oracle as O

from ._cases import population_whitening


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        name = "small_v500_k10"
        sp = ts.WORKLOADS[name]
        n = 300
        cdf, _ = ts.topics(sp)
        d0 = bench.shard_first_doc(rank, sp)
        c = ts.corpus(sp.with_docs(d0 + n), doc0=d0, n_docs=n, cdf=cdf)
        W, m1 = population_whitening(name)
        Phi0 = ts.initial_factors(sp.seed, sp.K, sp.K)
        Phi1, g = O.cp_step(c.indptr, c.indices, c.counts, sp.V, W, m1, Phi0, 1e-3, float(sp.alpha0), 0.0)
        ms = 10.0 * (rank + 1)
        value, ms_max, docs_all = bench.replica_throughput(ms, float(n), world, device="cpu")
        out[rank] = (d0, c.indptr.copy(), c.indices.copy(), c.counts.copy(), Phi1, value, ms_max, docs_all)
    finally:
        dist.destroy_process_group()


def test_two_replicas_over_gloo():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    sp = ts.WORKLOADS["small_v500_k10"]
    n = 300
    # aggregation: every rank sees the same whole-job figures
    for r in range(world):
        _, _, _, _, _, value, ms_max, docs_all = res[r]
        assert ms_max == 20.0 and docs_all == 2.0 * n
        assert value == docs_all / (ms_max / 1e3)
    # shards: rank r holds documents [r n_docs, r n_docs + n) of the stream
    assert res[0][0] == 0 and res[1][0] == sp.n_docs
    cdf, _ = ts.topics(sp)
    for r in range(world):
        d0, indptr, indices, counts, Phi1, *_ = res[r]
        ref = ts.corpus(sp.with_docs(d0 + n), doc0=d0, n_docs=n, cdf=cdf)
        assert np.array_equal(indptr, ref.indptr) and np.array_equal(indices, ref.indices)
        assert np.array_equal(counts, ref.counts)
        # the replica's step is computed from its own shard alone
        W, m1 = population_whitening("small_v500_k10")
        Phi0 = ts.initial_factors(sp.seed, sp.K, sp.K)
        P, _ = O.cp_step(ref.indptr, ref.indices, ref.counts, sp.V, W, m1, Phi0, 1e-3, float(sp.alpha0), 0.0)
        assert np.array_equal(P, Phi1)
    assert not np.array_equal(res[0][2][:50], res[1][2][:50])
