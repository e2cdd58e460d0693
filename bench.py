#!/usr/bin/env python3
"""Throughput of the online Tensor LDA hot path: docs/sec of one online pass
(one CP-SGD step per minibatch, W fixed) on the streaming workload
V = 20,000, K = D = 100, alpha0 = 2, Poisson(12) document lengths, minibatch
sizes uniform on 512..8192 (seeded synthetic LDA corpus).

A step is one pass of the whole hot path over one minibatch: CSR scan and
validation, demean + whiten (SpMM), Y = X Phi, Q = U Phi, the same-token terms,
the data-term contraction, the Dirichlet/M1 corrections, the orthogonality
term and the SGD update.  `value` is device-resident throughput (corpus
already in HBM): the timed calls are the library's no-wait passes, which
return once the pass is enqueued, so the timed region ends with the pass's
last kernel (the device status is read after it).  `e2e` goes through the
host-input pass of the public API, which waits (every step's CSR copied
host->device inside the timed region, every step's loss read back).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
  python bench.py --online [--online-every E] [--online-r R]   (fully online mode)
  python bench.py --e1 [--e1-reps N]   (the simulation study's shape check, batched mode)
  python bench.py --vi [--vi-docs N] [--vi-iters I]   (document-topic VI)
  python bench.py --billion [--billion-docs N]   (V = 100k, K = 300, on-device generation)
  python bench.py --billion --stream-workload scale_v50k_k200 --billion-docs 50000000

With N > 1 (torchrun) each rank runs an independent replica on its own shard
of documents (replicas: no exchange step between ranks); value = docs of
all ranks / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "stream_v20k_k100"
METRIC = "docs/sec per online TLDA pass at k=100,V=20k: BF16 TC form vs FP32 plain"
UNIT = "docs/s"
LR = 2e-3
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
# Nominal FP32 CUDA-core peak (152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz),
# reported beside the measured one; the "alu" fractions use the measurement.
FP32_ALU_NOMINAL_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
_ALU_PEAK = None


def alu_peak():
    """FP32 CUDA-core peak measured on this GPU by the library's FFMA probe
    (tlda_ffma_probe, timed by CUDA events), measured once per process."""
    global _ALU_PEAK
    if _ALU_PEAK is None:
        from paper_2511_07809_gb300 import tlda
        _ALU_PEAK = {"tflops": tlda.ffma_peak_tflops(), "source": "measured: tlda_ffma_probe (FFMA, CUDA events)",
                     "nominal_tflops": FP32_ALU_NOMINAL_TFLOPS}
    return _ALU_PEAK


def flush_l2():
    """Writes a 256 MB buffer (about twice the 129 MB L2) so a timed region
    starts with none of its inputs in L2."""
    import torch
    buf = torch.empty(64 << 20, dtype=torch.float32, device="cuda")
    buf.fill_(1.0)
    del buf


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["auto", "bf16", "fp32"], default="auto")
    ap.add_argument("--fit-docs", type=int, default=1_000_000)
    ap.add_argument("--tile-cap", type=int, default=0,
                    help="fix the persistent pass's tile size (documents per tile) instead of tuning it")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-compare", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--online", action="store_true",
                    help="time the fully online mode (sketched whitening rebuilt every E minibatches)")
    ap.add_argument("--online-every", type=int, default=256)
    ap.add_argument("--online-r", type=int, default=216)
    ap.add_argument("--e1", action="store_true",
                    help="the simulation study's recovery check with the batched mode")
    ap.add_argument("--e1-reps", type=int, default=10)
    ap.add_argument("--e1-epochs", type=int, default=30)
    ap.add_argument("--e1-starts", type=int, default=8)
    ap.add_argument("--batch-sweep", action="store_true",
                    help="the pass at fixed minibatch sizes 512..8192: step time against batch size")
    ap.add_argument("--vi", action="store_true", help="time document-topic variational inference")
    ap.add_argument("--vi-docs", type=int, default=2_000_000)
    ap.add_argument("--vi-iters", type=int, default=20)
    ap.add_argument("--vi-reps", type=int, default=5)
    ap.add_argument("--billion", action="store_true",
                    help="the billion-document workload: chunks generated on the device, one-pass sketch, CP pass")
    ap.add_argument("--billion-docs", type=int, default=16_000_000)
    ap.add_argument("--billion-chunk", type=int, default=1_000_000)
    ap.add_argument("--billion-r", type=int, default=512)
    ap.add_argument("--recovery", action="store_true",
                    help="topic recovery of one full streamed pass (10M documents) in both forms, "
                         "warm-started by the batched mode on a slice")
    ap.add_argument("--recovery-docs", type=int, default=10_000_000)
    ap.add_argument("--recovery-lr", type=float, default=1e-4)
    ap.add_argument("--stream-workload", default="billion_v100k_k300",
                    help="workload of the chunked pipeline (billion_v100k_k300, scale_v50k_k200)")
    return ap.parse_args()


# ----------------------------------------------------------------------------- helpers
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return dict(PEAKS_FALLBACK), "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while a region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu)], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        # nvidia-smi's start-up (driver queries) would otherwise overlap a
        # short timed region: wait for its first sample (at most 3 s), then
        # a quarter second (measured: a 20-step region right after the start
        # drew 0.17-0.19 ms outside the kernel, 0.09 ms half a second later)
        t_end = time.time() + 3.0
        while self.proc is not None and time.time() < t_end and self.proc.poll() is None:
            if os.path.getsize(self.f.name) > 0:
                time.sleep(0.25)
                break
            time.sleep(0.01)
        return self

    def stop(self):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip() == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def shard_first_doc(rank: int, sp) -> int:
    """First document of a rank's replica shard: rank r generates documents
    [r n_docs, r n_docs + n) of the workload's seeded stream, so shards are
    disjoint and each is the same whichever world size runs it."""
    return int(rank) * int(sp.n_docs)


def reduce_over_ranks(x: float, op: str, world: int, device: str = "cuda") -> float:
    """One float reduced over the process group ("max" or "sum")."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def replica_throughput(ms: float, docs: float, world: int, device: str = "cuda"):
    """Whole-job docs/s of N independent replicas: the documents of every
    rank over the slowest rank's time.  Returns (value, ms_max, docs_all)."""
    ms_max = reduce_over_ranks(ms, "max", world, device)
    docs_all = reduce_over_ranks(docs, "sum", world, device)
    return docs_all / (ms_max / 1e3), ms_max, docs_all


def recovery_l1(ctx, Phi, mu, steps):
    """Per-topic l1 distance of the recovered topics to the generator's, after
    Hungarian matching (a sanity figure: one SGD pass is far from converged)."""
    try:
        from scipy.optimize import linear_sum_assignment
        mu_e, _ = ctx.unwhiten_topics(Phi)
        Dm = np.abs(mu[:, :, None] - mu_e[None, :, :]).sum(axis=1)
        r_, c_ = linear_sum_assignment(Dm)
        l1 = Dm[r_, c_]
        return {"l1_mean": float(l1.mean()), "l1_median": float(np.median(l1)), "l1_max": float(l1.max()),
                "topics_above_1": int((l1 > 1.0).sum()), "after_steps": steps}
    except Exception as e:  # noqa: BLE001
        return {"error": str(e)[:80]}


def col_rel(a, b):
    """Largest per-column max-norm error max_n max_i |a_in - b_in| / max_i |b_in|."""
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float((np.abs(a - b).max(axis=0) / np.maximum(np.abs(b).max(axis=0), 1e-300)).max())


def step_parity(make_ctx, dev, first):
    """Error against the oracle's first step (`first`, from the CPU baseline)
    of the same step taken by a fresh context of one form through its pass
    entry point (the kernel the timed region runs), on the same documents
    from the same Phi and whitening: the update Phi_1 - Phi_0 against
    -lr grad (relative Frobenius and worst column) and the loss."""
    import torch
    ctx = make_ctx()
    ctx.set_whitening(torch.tensor(first["W"], dtype=torch.float32), torch.tensor(first["m1"], dtype=torch.float32))
    P0 = torch.tensor(first["Phi0"], dtype=torch.float32, device="cuda")
    P = P0.clone()
    a, b = first["docs"]
    loss = float(ctx.cp_pass(dev, [int(a), int(b)], P, LR, losses=True)[0])
    ctx.close()
    upd = (P - P0).cpu().numpy().astype(np.float64)
    ref = -LR * first["grad"]
    rel = float(np.linalg.norm(upd - ref) / np.linalg.norm(ref))
    return {"update_rel_frobenius": rel, "update_worst_column": col_rel(upd, ref),
            "loss_rel": abs(loss - first["loss"]) / abs(first["loss"]), "docs": int(b - a)}


def batch_plan(ts, sp, n_steps):
    """Seeded minibatch sizes (uniform 512..8192) for n_steps, and the document
    count they cover within one pass of the corpus."""
    sizes = ts.batch_sizes(sp)
    seq = np.array([sizes[i % len(sizes)] for i in range(n_steps)], dtype=np.int64)
    return seq


def segments(seq, n_docs, first):
    """Split consecutive batches into monotone offset lists (a new list when
    the next batch would run past the corpus end: the pass wraps around)."""
    segs, cur, off = [], [first], first
    for b in seq:
        if off + b > n_docs:
            segs.append(cur)
            cur, off = [0], 0
        off += int(b)
        cur.append(off)
    segs.append(cur)
    # int64 arrays: what the binding passes through without a conversion
    return [np.asarray(s, dtype=np.int64) for s in segs if len(s) > 1]


def distinct_words(c, offs):
    """Distinct words of each batch of a segment (algorithmic row count of the
    Q = U Phi product and of the U^T Zc reduction)."""
    out = []
    for a, b in zip(offs[:-1], offs[1:]):
        lo, hi = int(c.indptr[a]), int(c.indptr[b])
        out.append(len(np.unique(c.indices[lo:hi])))
    return np.array(out, dtype=np.int64)


def src_sha(path):
    with open(path, "rb") as f:
        return hashlib.sha1(f.read()).hexdigest()[:12]


# ----------------------------------------------------------------------------- CPU baseline
def cpu_baseline(ts, sp, cdf, mu, seconds, shard0=0):
    """The FP64 oracle's implicit CP step (as it stands) over consecutive
    minibatches of the same workload, for about `seconds` of CPU time, with
    the population whitening (FP32-rounded) and Phi0.  Also returns the
    oracle's first step (inputs and outputs), which the bench compares with
    each form's first step on the same inputs."""
    from oracle import tlda_oracle as O
    h = np.full(sp.K, 1.0 / sp.K)
    W, m1 = O.population_whitening(mu, h)
    W = W.astype(np.float32).astype(np.float64)
    m1 = m1.astype(np.float32).astype(np.float64)
    Phi = ts.initial_factors(sp.seed + 1, sp.K, sp.K)
    first = None
    sizes = ts.batch_sizes(sp)
    n_need = int(sizes[:64].sum())
    c = ts.corpus(sp.with_docs(shard0 + n_need), doc0=shard0, n_docs=n_need, cdf=cdf)
    docs, steps, off = 0, 0, 0
    t0 = time.perf_counter()
    while steps < 64:
        b = int(sizes[steps])
        r = c.rows(off, off + b)
        Phi_next, g = O.cp_step(r.indptr, r.indices, r.counts, sp.V, W, m1, Phi, LR, float(sp.alpha0), 0.0)
        if first is None:
            first = {"docs": (off, off + b), "W": W, "m1": m1, "Phi0": Phi, "grad": g["grad"], "loss": g["loss"]}
        Phi = Phi_next
        docs += b
        off += b
        steps += 1
        if time.perf_counter() - t0 > seconds and steps >= 2:
            break
    dt = time.perf_counter() - t0
    return ({"value": docs / dt, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
             "sample": f"{steps} minibatches ({docs} docs) of {WORKLOAD}, FP64 numpy/scipy oracle "
                       f"implicit CP step, {dt:.1f} s"}, first)


def reference_arm(args):
    """`--impl reference`: the FP64 oracle timed on the host cores for the same
    metric, each step one minibatch (prefix-sampled so the run stays within a
    few minutes)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import tlda_synth as ts
    from oracle import tlda_oracle as O
    sp = ts.WORKLOADS[WORKLOAD]
    cdf, mu = ts.topics(sp)
    h = np.full(sp.K, 1.0 / sp.K)
    W, m1 = O.population_whitening(mu, h)
    seq = batch_plan(ts, sp, args.warmup + args.steps)
    budget = 150.0
    # calibrate on one full first batch: per-step cost = a + b * docs
    c = ts.corpus(sp.with_docs(int(seq[0]) + 4096), n_docs=int(seq[0]) + 4096, cdf=cdf)
    Phi = ts.initial_factors(sp.seed + 1, sp.K, sp.K)
    t = []
    for n in (256, int(seq[0])):
        r = c.rows(0, n)
        t0 = time.perf_counter()
        O.cp_step(r.indptr, r.indices, r.counts, sp.V, W, m1, Phi, LR, float(sp.alpha0), 0.0)
        t.append(time.perf_counter() - t0)
    per_doc = max((t[1] - t[0]) / max(int(seq[0]) - 256, 1), 1e-9)
    fixed = max(t[0] - 256 * per_doc, 0.0)
    total = args.warmup + args.steps
    cap = int(max(64, min(8192, (budget / total - fixed) / per_doc)))
    sample = [min(int(b), cap) for b in seq]
    need = sum(sample)
    c = ts.corpus(sp.with_docs(need), n_docs=need, cdf=cdf)
    off = 0
    docs = 0
    t0 = None
    for i, b in enumerate(sample):
        if i == args.warmup:
            t0 = time.perf_counter()
            docs = 0
        r = c.rows(off, off + b)
        Phi, _ = O.cp_step(r.indptr, r.indices, r.counts, sp.V, W, m1, Phi, LR, float(sp.alpha0), 0.0)
        off += b
        docs += b
    dt = time.perf_counter() - (t0 if t0 is not None else time.perf_counter())
    value = docs / dt if dt > 0 else 0.0
    capped = "full minibatches" if cap >= 8192 else f"first {cap} docs of each minibatch"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "V": sp.V, "K": sp.K, "D": sp.K,
                                            "alpha0": float(sp.alpha0), "batch": "U{512..8192}"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"{args.steps} timed steps, {capped} ({docs} docs)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- our arm
def online_main(args):
    """`--online`: docs/s of the fully online mode on the streaming workload
    (BF16 form).  Per block of E minibatches: the block's statistics go into
    the one-pass sketch, the whitening is rebuilt from it, Phi is carried into
    the new basis, then the block's CP steps run.  The warm-up pass builds the
    first whitening; the timed pass covers the next `steps` minibatches with
    the corpus resident in HBM.  Also times a plain pass over the same batches
    with the final whitening, so the rebuild cost per block follows."""
    import torch
    import tlda_synth as ts
    from paper_2511_07809_gb300 import tlda

    sp = ts.WORKLOADS[WORKLOAD]
    cdf, _ = ts.topics(sp)
    seq = batch_plan(ts, sp, args.warmup + args.steps)
    n_docs = int(seq.sum())
    corpus = ts.corpus(sp.with_docs(n_docs), n_docs=n_docs, cdf=cdf)
    dev = tlda.DeviceCSR.from_corpus(corpus)
    offs = np.concatenate([[0], np.cumsum(seq)]).astype(np.int64)
    r, every, lr = args.online_r, args.online_every, 5e-4
    Om = torch.tensor(ts.signs(sp.seed, 0x4F4D, sp.V * r).reshape(sp.V, r))
    ctx = tlda.TLDA(sp.V, sp.K, alpha0=float(sp.alpha0), precision="bf16", max_batch=8192, seed=1)
    ctx.online_begin(Om)
    Phi = torch.tensor(ts.initial_factors(sp.seed + 1, sp.K, sp.K), dtype=torch.float32, device="cuda")
    ctx.online_pass(dev, offs[:args.warmup + 1], Phi, lr, rewhiten_every=args.warmup)
    torch.cuda.synchronize()
    timed_offs = offs[args.warmup:]
    n_timed = int(timed_offs[-1] - timed_offs[0])
    sampler = ClockSampler(0).start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    ctx.online_pass(dev, timed_offs, Phi, lr, rewhiten_every=every)
    e1.record()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    sweeps = ctx.eig_sweeps()
    # the same minibatches as plain CP steps with the last whitening
    Phi2 = Phi.clone()
    e0.record()
    ctx.cp_pass(dev, timed_offs, Phi2, lr)
    e1.record()
    torch.cuda.synchronize()
    ms_pass = e0.elapsed_time(e1)
    n_blocks = (args.steps + every - 1) // every
    line = {
        "metric": "docs/sec of the fully online TLDA mode at k=100,V=20k (sketched whitening "
                  f"rebuilt every {every} minibatches)",
        "value": n_timed / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
        "data": "synthetic: seeded LDA corpus (Dirichlet(0.1) topics, Poisson(12) lengths)",
        "config": {"workload": WORKLOAD, "V": sp.V, "K": sp.K, "D": sp.K, "sketch_r": r,
                   "rewhiten_every": every, "rebuilds": n_blocks, "docs": n_timed, "lr": lr,
                   "l2": "inputs larger than L2: a "
                         f"{(corpus.nnz * 8 + corpus.n_docs * 4) / 1e9:.2f} GB device-resident corpus"},
        "plain_pass_docs_s": n_timed / (ms_pass / 1e3),
        "ms_per_rebuild": (ms - ms_pass) / n_blocks,
        "jacobi_sweeps_last": sweeps,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def topic_correlation(mu_est, mu_true):
    """Pearson correlation of each true topic (row of mu_true) with its
    learned match (column of mu_est) under the matching of largest total
    correlation: the simulation study's score."""
    from scipy.optimize import linear_sum_assignment
    K = mu_true.shape[0]
    Cm = np.nan_to_num(np.corrcoef(np.vstack([mu_true, mu_est.T]))[:K, K:])
    r_, c_ = linear_sum_assignment(-Cm)
    return Cm[r_, c_]


def e1_main(args):
    """`--e1`: the simulation study as a shape check (section "Parameter
    Recovery and Comparison to Previous TLDA Methods"): K = 2, alpha0 = 0.01,
    whitening size 2, 20,000 documents, V in {500, 1000, 1500}, N seeded
    corpora each.  Per corpus: the batched mode (moments and whitening, then
    `epochs` passes of 1000-document batches from each Gaussian start, the
    start with the lowest last-epoch loss kept), the topics, and their
    correlation with the generator's.  Also the first start alone.  Device
    time per fit by CUDA events; the paper's figures are context only."""
    import torch
    import tlda_synth as ts
    from paper_2511_07809_gb300 import tlda

    paper = {500: 0.943, 1000: 0.930, 1500: 0.873}
    per_v = {}
    for V in (500, 1000, 1500):
        best, single, ms_fit = [], [], []
        for rep in range(args.e1_reps):
            sp = ts.e1_spec(V, rep)
            cdf, mu = ts.topics(sp)
            c = ts.corpus(sp, cdf=cdf)
            dev = tlda.DeviceCSR.from_corpus(c)
            offs = np.arange(0, sp.n_docs + 1, 1000, dtype=np.int64)
            starts = np.stack([ts.initial_factors(sp.seed + s, sp.K, sp.K) for s in range(args.e1_starts)])
            t = tlda.TLDA(sp.V, sp.K, alpha0=float(sp.alpha0), precision="fp32")
            Ps = torch.tensor(starts, dtype=torch.float32, device="cuda")
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            t.fit_batched(dev, offs, Ps, 1e-2, epochs=args.e1_epochs)
            e1.record()
            torch.cuda.synchronize()
            ms_fit.append(e0.elapsed_time(e1))
            best.append(float(topic_correlation(t.unwhiten_topics(Ps[0])[0], mu).mean()))
            P1 = torch.tensor(starts[:1], dtype=torch.float32, device="cuda")
            t.fit_batched(dev, offs, P1, 1e-2, epochs=args.e1_epochs, reuse_whitening=True)
            single.append(float(topic_correlation(t.unwhiten_topics(P1[0])[0], mu).mean()))
            t.close()
        per_v[str(V)] = {"corr_mean": float(np.mean(best)), "corr_std": float(np.std(best)),
                         "single_start_corr_mean": float(np.mean(single)),
                         "single_start_corr_std": float(np.std(single)),
                         "ms_per_fit_mean": float(np.mean(ms_fit)), "paper_corr_mean": paper[V]}
    line = {
        "metric": "simulation study shape check: mean topic correlation (K=2, alpha0=0.01, D=2, "
                  "20k docs, batched mode)",
        "value": float(np.mean([v["corr_mean"] for v in per_v.values()])), "unit": "pearson r",
        "n_gpus": 1, "higher_is_better": True, "dtype": "f32",
        "data": "synthetic: seeded LDA corpora (Dirichlet(0.1) topics, Poisson(50) lengths)",
        "config": {"workload": "e1_v{500,1000,1500}_k2", "reps": args.e1_reps, "epochs": args.e1_epochs,
                   "starts": args.e1_starts, "batch": 1000, "lr": 1e-2},
        "per_V": per_v,
    }
    print(json.dumps(line), flush=True)
    return 0


def restart_duplicate_factors(P, rng, thr=0.5):
    """Warm-start step of the recovery run (reading R): among the columns of
    the factors P (D x K), every pair whose directions have |cosine| above
    thr is taken for two components on one topic (a spurious stationary
    point of the unconstrained objective); the shorter of the pair is
    replaced by a random direction orthogonal to the kept columns, at the
    median column norm.  Uses the factors alone (no ground truth).  Returns
    (new P, number of columns replaced)."""
    P = np.array(P, dtype=np.float64)
    n = np.linalg.norm(P, axis=0)
    U = P / np.maximum(n, 1e-300)
    G = U.T @ U
    np.fill_diagonal(G, 0.0)
    bad = set()
    for i in range(P.shape[1]):
        for j in range(i + 1, P.shape[1]):
            if abs(G[i, j]) > thr and i not in bad and j not in bad:
                bad.add(j if n[j] < n[i] else i)
    keep = [i for i in range(P.shape[1]) if i not in bad]
    for b in sorted(bad):
        Q, _ = np.linalg.qr(P[:, keep])
        v = rng.standard_normal(P.shape[0])
        v -= Q @ (Q.T @ v)
        P[:, b] = v / np.linalg.norm(v) * np.median(n)
        keep.append(b)
    return P, len(bad)


def warm_start(ctx, dev, slice_docs, starts, lr, epochs=20, rounds=6, seed=0):
    """The batched mode on documents [0, slice_docs) in batches of 4096 from
    the given starts (the lowest-loss start kept), then rounds of duplicate
    restarts each followed by 10 more epochs, until no pair is duplicated.
    Returns (factors, mean last-epoch losses of the starts, restarts per round)."""
    import torch
    so = np.arange(0, slice_docs + 1, 4096)
    so[-1] = slice_docs
    Ps = torch.tensor(starts, dtype=torch.float32, device="cuda")
    means = ctx.fit_batched(dev, so, Ps, lr, epochs=epochs, reuse_whitening=True)
    P = Ps[0].cpu().numpy()
    rng = np.random.default_rng(seed)
    hist = []
    for _ in range(rounds):
        P, nb = restart_duplicate_factors(P, rng)
        hist.append(nb)
        if nb == 0:
            break
        Pt = torch.tensor(P[None], dtype=torch.float32, device="cuda")
        ctx.fit_batched(dev, so, Pt, lr, epochs=10, reuse_whitening=True)
        P = Pt[0].cpu().numpy()
    return torch.tensor(P, dtype=torch.float32, device="cuda"), means, hist


def recovery_main(args):
    """`--recovery`: topic recovery at the stream workload through the
    library alone, as a user would run it (section "Fully Online
    Implementation": initial factors from the batched mode run to convergence
    on a small portion of the data, then one CP step per minibatch):
      1. the moments and the whitening from all N documents (tlda_fit_moments);
      2. a warm start: the batched mode (reading R) on the first 1M documents,
         batches of 4096, 20 epochs, from 8 orthonormal starts, the start with
         the lowest mean last-epoch loss kept, then rounds of restarts of
         duplicated components (warm_start);
      3. one streamed pass over all N documents (the seeded 512..8192
         minibatch sizes, about 2300 steps) in the BF16 form and, from the
         same W and warm start, in the FP32 form.
    Reported per stage: per-topic l1 to the generator's topics (Hungarian
    matching) as mean, median, max and the count above 1 (a collapsed or
    missing topic), and each form's docs/s over the pass.  The oracle's
    power-method floor (tests/golden/recovery_floor_stream_v20k_k100.txt,
    written by an oracle-only script with the population whitening) is quoted
    as context."""
    import torch
    import tlda_synth as ts
    from paper_2511_07809_gb300 import tlda

    sp = ts.WORKLOADS[WORKLOAD]
    cdf, mu = ts.topics(sp)
    N = int(args.recovery_docs)
    t0 = time.perf_counter()
    c = ts.corpus(sp.with_docs(N), n_docs=N, cdf=cdf)
    gen_s = time.perf_counter() - t0
    dev = tlda.DeviceCSR.from_corpus(c)
    sizes = ts.batch_sizes(sp.with_docs(N))
    offs = np.concatenate([[0], np.cumsum(sizes)])
    offs = offs[offs <= N]
    if offs[-1] != N:
        offs = np.append(offs, N)
    fit = tlda.TLDA(sp.V, sp.K, alpha0=float(sp.alpha0), precision="fp32", max_batch=8192, seed=1)
    t0 = time.perf_counter()
    for d0 in range(0, N, 1_000_000):
        fit.fit_moments(tlda.DeviceCSR.from_corpus(c.rows(d0, min(d0 + 1_000_000, N))), tlda.ACCUMULATE)
    fit.fit_moments(None, tlda.FINALIZE)
    W, m1, ev = fit.get_whitening()
    fit_s = time.perf_counter() - t0
    slice_docs = min(1_000_000, N)
    starts = np.stack([ts.orthonormal_factors(sp.seed + 1 + s, sp.K, sp.K) for s in range(8)])
    Pw, means, restarts = warm_start(fit, dev, slice_docs, starts, LR)
    warm = recovery_l1(fit, Pw, mu, 0)
    fit.close()
    res = {}
    for prec in ("bf16", "fp32"):
        t = tlda.TLDA(sp.V, sp.K, alpha0=float(sp.alpha0), precision=prec, max_batch=8192, seed=1)
        t.set_whitening(W, m1)
        P = Pw.clone()
        t.cp_pass(dev, offs[:65], P.clone(), args.recovery_lr)  # tile tuning, on a copy
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        t.cp_pass(dev, offs, P, args.recovery_lr)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        res[prec] = {"recovery": recovery_l1(t, P, mu, len(offs) - 1), "docs_s": N / (ms / 1e3)}
        t.close()
    floor = None
    fpath = os.path.join(ROOT, "tests", "golden", "recovery_floor_stream_v20k_k100.txt")
    if os.path.exists(fpath):
        floor = {}
        for ln in open(fpath):
            if ln.strip() and not ln.startswith("#"):
                k, v = ln.split()
                floor[k] = float(v)
        floor["source"] = "oracle tensor power method, population whitening (tests/golden)"
    line = {
        "metric": "per-topic l1 recovery after one streamed online pass at k=100,V=20k (BF16 and FP32 forms)",
        "value": res["bf16"]["recovery"]["l1_mean"], "unit": "l1", "higher_is_better": False, "n_gpus": 1,
        "dtype": "bf16", "data": "synthetic: seeded LDA corpus (Dirichlet(0.1) topics, Poisson(12) lengths)",
        "config": {"workload": WORKLOAD, "docs": N, "steps": int(len(offs) - 1), "stream_lr": args.recovery_lr,
                   "whitening": f"tlda_fit_moments on all {N} documents", "warm_start":
                   f"batched mode, first {slice_docs} documents, batches of 4096, 20 epochs, 8 orthonormal "
                   f"starts, lr {LR}, then restarts of duplicated components", "gen_s": round(gen_s, 1),
                   "fit_s": round(fit_s, 2)},
        "warm_start_restarts_per_round": restarts,
        "eigenvalues": {"lambda_1": float(ev[0]), "lambda_K": float(ev[-1])},
        "warm_start": warm, "warm_start_mean_losses": [float(x) for x in np.sort(means)],
        "bf16": res["bf16"], "fp32": res["fp32"],
        "l1_mean_diff_bf16_fp32": abs(res["bf16"]["recovery"]["l1_mean"] - res["fp32"]["recovery"]["l1_mean"]),
        "oracle_floor": floor,
    }
    print(json.dumps(line), flush=True)
    return 0


def sweep_main(args):
    """`--batch-sweep`: the persistent BF16 pass over minibatches of one fixed
    size B (512, 1024, 2048, 4096, 8192 documents) of the streaming workload,
    with the whitening fitted on its first 1M documents and the tile size
    tuned per B.  Reported per B: ms per step and docs/s; and the least-squares
    line ms = t0 + b B, whose t0 is the per-step cost that does not scale with
    the batch (barriers, the update, the Phi image, pipeline fill) and whose
    1/b is the throughput the pass would approach with unbounded batches."""
    import torch
    import tlda_synth as ts
    from paper_2511_07809_gb300 import tlda

    sp = ts.WORKLOADS[WORKLOAD]
    cdf, _ = ts.topics(sp)
    n_docs = 4_000_000
    corpus = ts.corpus(sp.with_docs(n_docs), n_docs=n_docs, cdf=cdf)
    dev = tlda.DeviceCSR.from_corpus(corpus)
    Phi0 = torch.tensor(ts.initial_factors(sp.seed + 1, sp.K, sp.K), dtype=torch.float32, device="cuda")
    sizes, rows = (512, 1024, 2048, 4096, 8192), []
    sampler = ClockSampler(0).start()
    for B in sizes:
        ctx = tlda.TLDA(sp.V, sp.K, alpha0=float(sp.alpha0), precision="bf16", max_batch=8192, seed=1)
        ctx.fit_moments(tlda.DeviceCSR.from_corpus(corpus.rows(0, 1_000_000)), tlda.ACCUMULATE)
        ctx.fit_moments(None, tlda.FINALIZE)
        steps = min(2000, n_docs // B)
        offs = [i * B for i in range(steps + 1)]
        Phi = Phi0.clone()
        ctx.cp_pass(dev, offs[:65], Phi, LR)  # tile tuning and warm-up
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ctx.cp_pass(dev, offs, Phi, LR)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        rows.append({"batch": B, "steps": steps, "ms_per_step": ms, "docs_s": B / (ms / 1e3)})
        ctx.close()
    clocks = sampler.stop()
    x = np.array([r["batch"] for r in rows], dtype=np.float64)
    y = np.array([r["ms_per_step"] for r in rows])
    b, t0 = np.polyfit(x, y, 1)
    line = {
        "metric": "ms per CP step of the persistent BF16 pass at k=100,V=20k against the minibatch size",
        "value": None, "unit": "ms", "n_gpus": 1, "higher_is_better": False, "dtype": "bf16",
        "data": "synthetic: seeded LDA corpus (Dirichlet(0.1) topics, Poisson(12) lengths)",
        "config": {"workload": sp.name, "V": sp.V, "K": sp.K, "docs": n_docs,
                   "l2": "inputs larger than L2: a 0.4 GB device-resident corpus"},
        "rows": rows, "fit": {"t0_us": t0 * 1e3, "ns_per_doc": b * 1e6, "asymptotic_docs_s": 1e3 / b},
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    return 0


def vi_main(args):
    """`--vi`: docs/s of document-topic variational inference
    (tlda_doc_topics) over the first N documents of the streaming workload,
    with its ground-truth topics and alpha = alpha0/K, `vi_reps` timed
    repetitions after two untimed ones (each repetition one call over all N
    documents; the CSR and theta exceed L2).  The oracle's E-step on a
    sample of the same documents is timed beside it; e2e adds the host->device
    copy of the CSR and the device->host copy of theta."""
    import torch
    import tlda_synth as ts
    from paper_2511_07809_gb300 import tlda

    sp = ts.WORKLOADS[WORKLOAD]
    cdf, mu = ts.topics(sp)
    n = args.vi_docs
    c = ts.corpus(sp.with_docs(n), n_docs=n, cdf=cdf)
    dev = tlda.DeviceCSR.from_corpus(c)
    mu_d = torch.tensor(mu.T.copy(), dtype=torch.float32, device="cuda")
    al = np.full(sp.K, float(sp.alpha0) / sp.K)
    al_d = torch.tensor(al, dtype=torch.float32, device="cuda")
    for _ in range(2):
        theta = tlda.doc_topics(dev, mu_d, al_d, args.vi_iters)
    torch.cuda.synchronize()
    sampler = ClockSampler(0).start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.vi_reps):
        theta = tlda.doc_topics(dev, mu_d, al_d, args.vi_iters)
    e1.record()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / args.vi_reps
    # end to end: host CSR in, theta out
    host = tlda.DeviceCSR.from_corpus(c, device="cpu", pin=True)
    out = torch.empty((n, sp.K), dtype=torch.float32, pin_memory=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    d2 = tlda.DeviceCSR(host.indptr.to("cuda", non_blocking=True), host.indices.to("cuda", non_blocking=True),
                        host.counts.to("cuda", non_blocking=True), sp.V)
    out.copy_(tlda.doc_topics(d2, mu_d, al_d, args.vi_iters), non_blocking=True)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    nnz = c.nnz
    byts = 8.0 * nnz + 4.0 * (n + 1) + 4.0 * n * sp.K           # CSR stream + theta written
    flops = 4.0 * sp.K * nnz * args.vi_iters
    peaks, src = measured_peaks()
    hbm = peaks.get("hbm_gbs", PEAKS_FALLBACK["hbm_gbs"])
    ach = byts / (ms / 1e3) / 1e9
    # the oracle on a bounded sample
    from oracle import tlda_oracle as O
    ns = 1500
    r = c.rows(0, ns)
    t0 = time.perf_counter()
    O.doc_topics(r.indptr, r.indices, r.counts, sp.V, mu.T, al, args.vi_iters)
    cpu_s = time.perf_counter() - t0
    line = {
        "metric": "docs/sec of document-topic variational inference at k=100,V=20k "
                  f"({args.vi_iters} E-step rounds per document)",
        "value": n / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.vi_reps, "warmup": 2,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic: seeded LDA corpus (Dirichlet(0.1) topics, Poisson(12) lengths), true topics",
        "config": {"workload": WORKLOAD, "V": sp.V, "K": sp.K, "docs": n, "nnz": nnz, "iters": args.vi_iters,
                   "l2": f"inputs larger than L2: {(8 * nnz + 4 * n) / 1e9:.2f} GB CSR, "
                         f"{4 * n * sp.K / 1e9:.2f} GB theta written per call"},
        "roofline": {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                     "algorithmic_bytes_per_call": byts, "peak_source": src,
                     "fp32_tflops": flops / (ms / 1e3) / 1e12,
                     "fp32_frac": flops / (ms / 1e3) / 1e12 / alu_peak()["tflops"], "traffic": None},
        "cpu_baseline": {"value": ns / cpu_s, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"first {ns} documents, FP64 numpy/scipy E-step, {cpu_s:.1f} s"},
        "e2e": {"value": n / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 8.0 * nnz + 4.0 * (n + 1),
                "d2h_bytes_per_step": 4.0 * n * sp.K},
        "gpu_launches": args.vi_reps, "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    return 0


def billion_main(args):
    """`--billion`: the billion-document workload (V = 100,000, K = D = 300,
    Zipf(1.07)-shaped topics, alpha0 = 5, Poisson(15) lengths, minibatches of
    65,536) on the first N documents, in chunks generated on the device and
    never stored whole (with --stream-workload scale_v50k_k200: V = 50,000,
    K = D = 200, alpha0 = 1, Poisson(20) lengths, minibatches of 8192).  Pass 1: each chunk is generated and added to the
    one-pass sketch and the token statistics.  Then one whitening from the
    sketch (r = 512).  Pass 2: each chunk is generated again and its
    minibatches take CP steps in the BF16 tensor-core form; then the same
    pass 2 again in the FP32 form (same whitening, same starting factors),
    for the comparison.  Reported: docs/s of each pass (generation included)
    and of the whole job (pass 1, whitening, BF16 pass 2), the per-chunk
    times (linear scaling: flat), the whitening time."""
    import torch
    import tlda_synth as ts
    from paper_2511_07809_gb300 import tlda

    sp = ts.WORKLOADS[args.stream_workload]
    t0 = time.perf_counter()
    cdf, mu = ts.topics(sp)
    t_topics = time.perf_counter() - t0
    r = args.billion_r
    t0 = time.perf_counter()
    Om = torch.tensor(ts.signs(sp.seed, 0x4F4D, sp.V * r).reshape(sp.V, r))
    t_omega = time.perf_counter() - t0
    a = sp.alpha0
    gen = tlda.DeviceGenerator(sp.seed, sp.V, sp.K, cdf, a.numerator, a.denominator, ts.len_table(sp), sp.min_len)
    B = sp.batch[0]
    chunk = args.billion_chunk
    n_chunks = (args.billion_docs + chunk - 1) // chunk
    cap = chunk * 48
    buf = tlda.DeviceCSR(torch.empty(chunk + 1, dtype=torch.int32, device="cuda"),
                         torch.empty(cap, dtype=torch.int32, device="cuda"),
                         torch.empty(cap, dtype=torch.int32, device="cuda"), sp.V)
    ctx = tlda.TLDA(sp.V, sp.K, alpha0=float(sp.alpha0), precision="bf16", max_batch=B, seed=1)
    ctx.online_begin(Om)
    Phi0 = torch.tensor(ts.initial_factors(sp.seed + 1, sp.K, sp.K), dtype=torch.float32, device="cuda")
    Phi = Phi0.clone()
    sampler = ClockSampler(0).start()
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    marks1, marks2, nnz_tot, docs = [], [], 0, 0
    torch.cuda.synchronize()
    e_start = ev()
    e_start.record()
    for ci in range(n_chunks):
        n = min(chunk, args.billion_docs - ci * chunk)
        c = gen.generate(ci * chunk, n, out=buf)
        nnz_tot += c.indices.numel()
        docs += n
        ctx.online_accumulate(c)
        e = ev()
        e.record()
        marks1.append(e)
    e_w0 = ev()
    e_w0.record()
    ctx.online_whiten()
    e_w1 = ev()
    e_w1.record()
    lr = 1e-4

    def pass2(c_, P, start):
        marks = []
        for ci in range(n_chunks):
            n = min(chunk, args.billion_docs - ci * chunk)
            c = gen.generate(ci * chunk, n, out=buf)
            offs = list(range(0, n, B)) + [n]
            c_.cp_pass(c, offs, P, lr)
            e = ev()
            e.record()
            marks.append(e)
        torch.cuda.synchronize()
        return [(marks[i - 1] if i else start).elapsed_time(marks[i]) for i in range(n_chunks)], marks[-1]

    t2, e_end = pass2(ctx, Phi, e_w1)
    clocks = sampler.stop()

    def kernel_profile(c_, prec):
        """Per-kernel device times of one more pass over the first chunk (on a
        copy of Phi, after the timed region), and the roofline of the two
        dense contractions: [Q; Y] = [U; X] Phi, algorithmic 2 (n_t + B) D K
        flop (Q is needed for the n_t touched words only), and
        [X; U_t]^T [Z; Zc], 2 (B + n_t) D K flop."""
        n = min(chunk, args.billion_docs)
        c = gen.generate(0, n, out=buf)
        offs = list(range(0, n, B)) + [n]
        ip = c.indptr.cpu().numpy()
        bt, nt = [], []
        for a_, b_ in zip(offs[:-1], offs[1:]):
            bt.append(b_ - a_)
            nt.append(int(torch.unique(c.indices[int(ip[a_]):int(ip[b_])]).numel()))
        names = ("scan_whiten", "qy", "rz", "zh", "g_reduce", "reduce_update", "phi_gram", "phi_terms")
        P = Phi0.clone()
        c_.profile(names)
        c_.cp_pass(c, offs, P, lr)
        torch.cuda.synchronize()
        pr = c_.profile_read()
        c_.profile(())
        peaks, src = measured_peaks()
        if prec == "bf16":
            pk, bound = peaks.get("bf16_tflops_sustained", PEAKS_FALLBACK["bf16_tflops_sustained"]), "tensor"
        else:
            pk, bound = alu_peak()["tflops"], "alu"
        fl = 2.0 * float(np.sum(np.array(bt) + np.array(nt))) * sp.K * sp.K / len(bt)
        out = {"ms_per_step": {k: v[1] / v[0] for k, v in pr.items() if v[0] > 0}, "peak_source": src,
               "mean_touched_words": float(np.mean(nt))}
        for k in ("qy", "g_reduce"):
            if pr.get(k, (0, 0))[0] > 0:
                ach = fl / (pr[k][1] / pr[k][0] / 1e3) / 1e12
                out[k] = {"bound": bound, "achieved": ach, "peak": pk, "unit": "TFLOP/s", "frac": ach / pk,
                          "algorithmic_flop_per_launch": fl}
        return out

    prof_bf16 = kernel_profile(ctx, "bf16")
    t1 = [(marks1[i - 1] if i else e_start).elapsed_time(marks1[i]) for i in range(n_chunks)]
    ms_total = e_start.elapsed_time(e_end)
    w_ms = e_w0.elapsed_time(e_w1)
    finite = bool(torch.isfinite(Phi).all().item())
    # the FP32 form on the same chunks, whitening and starting factors
    W, m1, _ = ctx.get_whitening()
    c32 = tlda.TLDA(sp.V, sp.K, alpha0=float(sp.alpha0), precision="fp32", max_batch=B, seed=1)
    c32.set_whitening(W, m1)
    P32 = Phi0.clone()
    e32 = ev()
    e32.record()
    t2_32, _ = pass2(c32, P32, e32)
    rel32 = float((torch.linalg.norm(Phi - P32) / torch.linalg.norm(P32)).item())
    prof_fp32 = kernel_profile(c32, "fp32")
    c32.close()
    line = {
        "metric": f"docs/sec of the chunked streaming workload {sp.name} (V={sp.V}, K={sp.K}): on-device "
                  "generation, one-pass sketch, whitening, CP pass",
        "value": docs / (ms_total / 1e3), "unit": UNIT, "n_gpus": 1, "steps": n_chunks * ((chunk + B - 1) // B),
        "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
        "data": f"synthetic: generated on the device (Dirichlet({sp.beta}) topics"
                + (f", Zipf({sp.zipf_s})-shaped" if sp.zipf_s else "") + f", Poisson({sp.lam:g}) lengths)",
        "config": {"workload": sp.name, "V": sp.V, "K": sp.K, "D": sp.K, "docs": docs,
                   "nnz": nnz_tot, "chunk_docs": chunk, "batch": B, "sketch_r": r, "lr": lr,
                   "l2": "inputs larger than L2: each chunk (about 0.1 GB of CSR) is generated into HBM "
                         "and read once per pass"},
        "pass1_sketch_docs_s": docs / (sum(t1) / 1e3),
        "whiten_ms": w_ms,
        "pass2_cp_docs_s": docs / (sum(t2) / 1e3),
        "pass2_cp_docs_s_fp32": docs / (sum(t2_32) / 1e3),
        "phi_rel_diff_bf16_vs_fp32": rel32,
        "chunk_ms_pass1": {"mean": float(np.mean(t1)), "std": float(np.std(t1)), "first": t1[0], "last": t1[-1]},
        "chunk_ms_pass2": {"mean": float(np.mean(t2)), "std": float(np.std(t2)), "first": t2[0], "last": t2[-1]},
        "host_setup_s": {"topics": round(t_topics, 2), "omega": round(t_omega, 2)},
        "phi_finite": finite, "clocks": clocks,
        "pass2_kernels_bf16": prof_bf16, "pass2_kernels_fp32": prof_fp32,
    }
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    if args.billion:
        return billion_main(args)
    if args.batch_sweep:
        return sweep_main(args)
    if args.recovery:
        return recovery_main(args)
    if args.vi:
        return vi_main(args)
    if args.online:
        return online_main(args)
    if args.e1:
        return e1_main(args)
    import torch
    import torch.distributed as dist
    import tlda_synth as ts
    from paper_2511_07809_gb300 import tlda

    rank, world = int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()


    sp = ts.WORKLOADS[WORKLOAD]
    cdf, mu = ts.topics(sp)
    seq = batch_plan(ts, sp, args.warmup + args.steps)
    n_docs = int(min(seq.sum(), sp.n_docs))
    n_docs = max(n_docs, min(args.fit_docs, sp.n_docs))
    shard0 = shard_first_doc(rank, sp)
    t_gen = time.perf_counter()
    corpus = ts.corpus(sp.with_docs(shard0 + n_docs), doc0=shard0, n_docs=n_docs, cdf=cdf)
    t_gen = time.perf_counter() - t_gen
    dev = tlda.DeviceCSR.from_corpus(corpus)
    precs = [args.precision] if args.precision != "auto" else ["bf16", "fp32"]

    def make_ctx(prec, same_token=True):
        return tlda.TLDA(sp.V, sp.K, alpha0=float(sp.alpha0), precision=prec, max_batch=8192, seed=1,
                         same_token=same_token)

    # whitening fitted by the library on a prefix of the shard (outside the timed region)
    primary = None
    for p in precs:
        try:
            ctx = make_ctx(p)
            primary = p
            break
        except tlda.TLDAError as e:
            if e.status != tlda.ERR_UNIMPLEMENTED:
                raise
    n_fit = min(args.fit_docs, n_docs)
    t_fit = time.perf_counter()
    for d0 in range(0, n_fit, 1_000_000):
        ctx.fit_moments(tlda.DeviceCSR.from_corpus(corpus.rows(d0, min(d0 + 1_000_000, n_fit))),
                        tlda.ACCUMULATE)
    ctx.fit_moments(None, tlda.FINALIZE)
    t_fit = time.perf_counter() - t_fit
    W, m1, eig = ctx.get_whitening()
    Phi0 = torch.tensor(ts.initial_factors(sp.seed + 1, sp.K, sp.K), dtype=torch.float32, device="cuda")
    if args.tile_cap > 0 and primary == "bf16":
        ctx.autotune(fixed=args.tile_cap)

    warm_segs = segments(seq[:args.warmup], n_docs, 0)
    last_off = warm_segs[-1][-1] if warm_segs else 0
    timed_segs = segments(seq[args.warmup:], n_docs, last_off)
    n_timed_docs = int(seq[args.warmup:].sum())

    def timed(c, Phi, host=False, losses=False, profile=(), wait=True):
        # wait=False: the device-resident calls return once the pass is
        # enqueued (the library's no-wait mode); their status is read by
        # sync() after the timed region
        nonlocal dev_or_host
        dev_or_host = host_corpus if host else dev
        for s in warm_segs:  # the same calls as the timed ones (buffers sized before timing)
            c.cp_pass(dev_or_host, s, Phi, LR, host_input=host, losses=losses, wait=wait)
        torch.cuda.synchronize()
        c.sync()
        if profile:
            c.profile(profile)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        e1.record()  # both CUDA events exist before the timed region (created at first record)
        flush_l2()
        barrier()
        torch.cuda.synchronize()
        e0.record()
        for s in timed_segs:
            c.cp_pass(dev_or_host, s, Phi, LR, host_input=host, losses=losses, wait=wait)
        e1.record()
        torch.cuda.synchronize()
        c.sync()
        barrier()
        ms = e0.elapsed_time(e1)
        prof = c.profile_read() if profile else None
        if profile:
            c.profile(())
        return ms, prof

    dev_or_host = dev
    host_corpus = None
    # 1) which kernel dominates: the persistent pass kernel where the context
    # runs passes in one (its first pass also tunes the tile size), else a
    # short bracketed run of every kernel of the per-step chain
    probe_segs = segments(seq[args.warmup:args.warmup + min(200, args.steps)], n_docs, last_off)
    Phi = Phi0.clone()
    ctx.profile(("pass",))
    for s in probe_segs:
        ctx.cp_pass(dev, s, Phi, LR)
    shares = ctx.profile_read()
    ctx.profile(())
    persistent = shares["pass"][0] > 0
    if not persistent:
        Phi = Phi0.clone()
        ctx.profile(tlda.TLDA.KERNELS)
        for s in probe_segs:
            ctx.cp_pass(dev, s, Phi, LR)
        shares = ctx.profile_read()
        ctx.profile(())
    dominant = max((k for k in shares if shares[k][0] > 0), key=lambda k: shares[k][1])

    # 2) the timed region (device-resident corpus), dominant kernel bracketed by events
    sampler = ClockSampler(local).start()
    Phi = Phi0.clone()
    ms, prof = timed(ctx, Phi, profile=(dominant,), wait=False)
    clocks = sampler.stop()
    value, ms_max, docs_all = replica_throughput(ms, float(n_timed_docs), world)
    Phi_final = Phi.clone()

    # roofline of the dominant kernel
    peaks, peak_src = measured_peaks()
    launches, kms = prof[dominant]
    B_all = np.concatenate([np.diff(s) for s in timed_segs])
    nnz_all = np.concatenate([np.diff(corpus.indptr[np.array(s)]) for s in timed_segs])
    D = K = sp.K
    roof = None
    nt = np.concatenate([distinct_words(corpus, s) for s in timed_segs])
    # the method's algorithmic flops of every timed step (factored count,
    # unpadded D, K): X = F U, Y = X Phi, Q = U_t Phi, R = F (Q*Q), G1, H, G2,
    # and the Phi-only products Phi^T Phi and Phi (G * G)
    step_flops = float((2.0 * nnz_all * D + 4.0 * B_all * D * K + 4.0 * nt * D * K
                        + 4.0 * nnz_all * K + 4.0 * D * K * K).sum())
    if dominant in ("qy", "g_reduce", "fused", "pass") and launches:
        if dominant == "pass":
            # every step of the launches: the data-term contractions as for
            # "fused" below plus the Phi-only products Phi^T Phi and
            # Phi (G * G), over all timed steps, per launch
            flops = float((2.0 * nnz_all * D + 4.0 * B_all * D * K + 4.0 * nt * D * K
                           + 4.0 * nnz_all * K + 4.0 * D * K * K).sum()) / launches
        elif dominant == "fused":
            # the method's contractions this kernel performs (factored count,
            # unpadded D, K): X = F U, Y = X Phi, Q = U_t Phi, R = F (Q*Q),
            # G1 = X^T Z, H = F^T Y, G2 = U_t^T Zc
            flops = float((2.0 * nnz_all * D + 4.0 * B_all * D * K + 4.0 * nt * D * K
                           + 4.0 * nnz_all * K).sum()) / len(B_all)
        else:
            flops = 2.0 * float((B_all + nt).sum()) * D * K / len(B_all)
        ach = flops / (kms / launches / 1e3) / 1e12
        if primary == "bf16":
            pk, unit, bound = peaks.get("bf16_tflops_sustained", PEAKS_FALLBACK["bf16_tflops_sustained"]), "TFLOP/s", "tensor"
        else:
            pk, unit, bound = alu_peak()["tflops"], "TFLOP/s", "alu"
        roof = {"bound": bound, "achieved": ach, "peak": pk, "unit": unit, "frac": ach / pk,
                "algorithmic_flop_per_launch": flops}
    elif launches:
        # HBM-bound kernels: algorithmic bytes = the batch's CSR stream + X written
        xbytes = D * 4 if primary == "fp32" else D * 2 * 2
        byts = float(((B_all + 1) * 4 + nnz_all * 8 + B_all * xbytes).sum()) / len(B_all)
        ach = byts / (kms / launches / 1e3) / 1e9
        pk = peaks.get("hbm_gbs", PEAKS_FALLBACK["hbm_gbs"])
        roof = {"bound": "hbm", "achieved": ach, "peak": pk, "unit": "GB/s", "frac": ach / pk}
    if roof is not None:
        roof.update({"kernel": dominant, "peak_source": peak_src,
                     "kernel_ms_per_launch": kms / max(launches, 1),
                     "share_of_step": (shares[dominant][1] / sum(v[1] for v in shares.values())),
                     "traffic": None})
        tfile = os.path.join(ROOT, "profiles", "traffic.json")
        if os.path.exists(tfile):
            with open(tfile) as f:
                tr = json.load(f)
            key = f"{primary}:{dominant}"
            if key in tr and tr[key].get("src_sha") == src_sha(os.path.join(ROOT, tr[key]["src"])):
                if "bytes_per_doc" in tr[key]:
                    # DRAM bytes fitted on smaller captured launches (a fixed
                    # part per launch plus a part per document), evaluated at
                    # the documents one timed launch processes
                    roof["traffic"] = (tr[key].get("bytes_fixed_per_launch", 0.0)
                                       + tr[key]["bytes_per_doc"] * n_timed_docs / max(launches, 1))
                else:
                    roof["traffic"] = tr[key]["bytes_per_launch"]

    # 3) end to end through the public API: host CSR -> device inside the call, loss read back
    e2e = None
    if not args.no_e2e:
        host_corpus = tlda.DeviceCSR.from_corpus(corpus, device="cpu", pin=True)
        Phi = Phi0.clone()
        ms_e, _ = timed(ctx, Phi, host=True, losses=True)
        ms_e = reduce_over_ranks(ms_e, "max", world)
        h2d = float(((B_all + 1) * 4 + nnz_all * 8).mean())
        e2e = {"value": docs_all / (ms_e / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": 8}

    # 4) the other form on the same batches (BF16 TC vs FP32 plain)
    compare = None
    if not args.no_compare and len(precs) > 1:
        other = [p for p in precs if p != primary]
        try:
            c2 = make_ctx(other[0]) if other else None
        except tlda.TLDAError as e:
            if e.status != tlda.ERR_UNIMPLEMENTED:
                raise
            c2 = None
        if c2 is not None:
            c2.set_whitening(W, m1)
            Phi = Phi0.clone()
            ms2, _ = timed(c2, Phi)
            ms2 = reduce_over_ranks(ms2, "max", world)
            ach2 = step_flops / (ms2 / 1e3) / 1e12
            if other[0] == "fp32":
                pk2, b2, src2 = alu_peak()["tflops"], "alu", alu_peak()["source"]
            else:
                pk2, b2, src2 = peaks.get("bf16_tflops_sustained", PEAKS_FALLBACK["bf16_tflops_sustained"]), "tensor", peak_src
            compare = {"precision": other[0], "value": docs_all / (ms2 / 1e3),
                       "ms_per_step": ms2 / args.steps,
                       "roofline": {"bound": b2, "achieved": ach2, "peak": pk2, "unit": "TFLOP/s",
                                    "frac": ach2 / pk2, "kernel": "whole step (every kernel of the pass)",
                                    "peak_source": src2},
                       "recovery": recovery_l1(c2, Phi, mu, args.warmup + args.steps)}
            c2.close()
    # the same primary form with the same-token correction off (the data term
    # of eq. vec_deriv alone), on the same batches
    no_st = None
    if not args.no_compare:
        c3 = make_ctx(primary, same_token=False)
        c3.set_whitening(W, m1)
        Phi = Phi0.clone()
        ms3, _ = timed(c3, Phi)
        ms3 = reduce_over_ranks(ms3, "max", world)
        no_st = {"precision": primary, "same_token_correction": False, "value": docs_all / (ms3 / 1e3),
                 "ms_per_step": ms3 / args.steps,
                 "recovery": recovery_l1(c3, Phi, mu, args.warmup + args.steps)}
        c3.close()

    # recovery of the pass (per-topic l1 after Hungarian matching), as a sanity figure
    recovery = recovery_l1(ctx, Phi_final, mu, args.warmup + args.steps)

    cpu, parity = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu, first = cpu_baseline(ts, sp, cdf, mu, args.cpu_seconds)
        # each form's first step against the oracle's (same documents,
        # whitening and Phi0): the error of each result against the FP64 oracle
        parity = {"oracle": "FP64 implicit CP step (oracle/), population whitening (FP32 values), Phi0, "
                            "first minibatch", "tolerance": {"fp32": 1e-5, "bf16": 2e-2}}
        for p in precs:
            try:
                parity[p] = step_parity(lambda: make_ctx(p), dev, first)
            except tlda.TLDAError as e:
                if e.status != tlda.ERR_UNIMPLEMENTED:
                    raise

    if rank == 0:
        # kernels per step: fused BF16 form (D, K padded to 128): Phi-only x2,
        # fused, reduction, step end; otherwise Phi-only x2, scan/whiten, Q/Y,
        # R/Z/H, Zc, reduction over rows, reduction, step end
        fused = primary == "bf16" and sp.K <= 128 and sp.K > 64
        per_step_kernels = 5 if fused else 9
        # persistent form: per cp_pass call over a device-resident corpus, the
        # prologue kernel (split points, Phi^T image, control block) and one
        # pass kernel for all of its steps
        launches_timed = (2 * len(timed_segs) if persistent
                          else per_step_kernels * args.steps + len(timed_segs))
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16" if primary == "bf16" else "f32",
            "data": "synthetic: seeded LDA corpus (Dirichlet(0.1) topics, Poisson(12) lengths)",
            "config": {"workload": WORKLOAD, "V": sp.V, "K": sp.K, "D": sp.K, "alpha0": float(sp.alpha0),
                       "batch": "U{512..8192}", "docs_per_rank": n_timed_docs, "precision": primary,
                       "same_token_correction": True, "lr": LR,
                       "l2": "L2 flushed (256 MB written) before each timed pass; each step reads a fresh "
                             "minibatch of a "
                             f"{(corpus.nnz * 8 + corpus.n_docs * 4) / 1e9:.2f} GB device-resident corpus, "
                             "never re-read in the timed region; the whitening workspace (U) stays "
                             "L2-resident by design",
                       "parallelism": "replicas" if world > 1 else "single",
                       "fit_docs": n_fit, "fit_s": round(t_fit, 2), "gen_s": round(t_gen, 2)},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "parity": parity,
            "fp32_alu_peak": alu_peak(),
            "gpu_launches": launches_timed,
            "clocks": clocks, "compare": compare, "compare_same_token_off": no_st, "recovery": recovery,
            "kernel_shares": {k: round(v[1] / max(sum(x[1] for x in shares.values()), 1e-12), 4)
                              for k, v in shares.items() if v[0]},
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
