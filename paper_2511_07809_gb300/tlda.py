"""Python binding of libtlda (include/tlda.h): argument marshalling only.

Every step of the hot path runs in the library's CUDA kernels; this module
passes pointers of torch CUDA tensors (and numpy host arrays) through ctypes.
There is no fallback: if libtlda.so cannot be built or loaded, importing this
module raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np
import torch

from . import _build

# ---------------------------------------------------------------------------- library
_LIB = None

OK, ERR_INVALID, ERR_CUDA, ERR_NUMERIC, ERR_TIMEOUT, ERR_OOM, ERR_STATE, ERR_UNIMPLEMENTED = range(8)
FP32, BF16 = 0, 1
ACCUMULATE, FINALIZE = 1, 2
HOST_INPUT = 1
NO_WAIT = 4
HOST_OUTPUT = 1
REUSE_WHITENING = 2

STATUS_NAMES = {OK: "TLDA_OK", ERR_INVALID: "TLDA_ERR_INVALID", ERR_CUDA: "TLDA_ERR_CUDA",
                ERR_NUMERIC: "TLDA_ERR_NUMERIC", ERR_TIMEOUT: "TLDA_ERR_TIMEOUT",
                ERR_OOM: "TLDA_ERR_OOM", ERR_STATE: "TLDA_ERR_STATE",
                ERR_UNIMPLEMENTED: "TLDA_ERR_UNIMPLEMENTED"}

#: every entry point declared in include/tlda.h
ENTRY_POINTS = ("tlda_default_params", "tlda_create", "tlda_destroy", "tlda_last_error",
                "tlda_sync", "tlda_fit_moments", "tlda_get_whitening", "tlda_get_counts",
                "tlda_set_whitening", "tlda_whiten_batch", "tlda_cp_step",
                "tlda_cp_data_term", "tlda_cp_pass", "tlda_unwhiten_topics",
                "tlda_profile", "tlda_profile_read", "tlda_save_state", "tlda_load_state",
                "tlda_cp_step_noalloc", "tlda_autotune", "tlda_online_begin",
                "tlda_online_pass", "tlda_eig_sweeps", "tlda_fit_batched", "tlda_doc_topics",
                "tlda_generate_docs", "tlda_online_accumulate", "tlda_online_whiten",
                "tlda_selftest_barrier", "tlda_online_get_sketch", "tlda_online_set_sketch",
                "tlda_ffma_probe")


class Params(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("dim", ctypes.c_int32), ("alpha0", ctypes.c_double),
                ("theta", ctypes.c_float), ("precision", ctypes.c_int32),
                ("same_token_correction", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("max_batch", ctypes.c_int32)]


class CSR(ctypes.Structure):
    _fields_ = [("n_docs", ctypes.c_int32), ("vocab", ctypes.c_int32),
                ("indptr", ctypes.c_void_p), ("indices", ctypes.c_void_p),
                ("counts", ctypes.c_void_p)]


def library_path() -> str:
    return _build.LIB


def load(build: bool = True) -> ctypes.CDLL:
    """Builds (if stale) and loads libtlda.so; raises if either fails."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.build() if build else _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"libtlda.so not found at {path}; run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    vp, i32, i64, f32, f64, u32 = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64,
                                   ctypes.c_float, ctypes.c_double, ctypes.c_uint32)
    u64 = ctypes.c_uint64
    P = ctypes.POINTER
    sig = {
        "tlda_default_params": (None, [P(Params), i32]),
        "tlda_create": (i32, [P(vp), i32, P(Params), vp]),
        "tlda_destroy": (i32, [vp]),
        "tlda_last_error": (ctypes.c_char_p, [vp]),
        "tlda_eig_sweeps": (i32, [vp]),
        "tlda_sync": (i32, [vp]),
        "tlda_fit_moments": (i32, [vp, P(CSR), u32]),
        "tlda_get_whitening": (i32, [vp, vp, vp, vp]),
        "tlda_get_counts": (i32, [vp, vp, vp, vp, vp]),
        "tlda_set_whitening": (i32, [vp, vp, vp]),
        "tlda_whiten_batch": (i32, [vp, P(CSR), vp]),
        "tlda_cp_step": (i32, [vp, P(CSR), vp, f32, vp, vp]),
        "tlda_cp_data_term": (i32, [vp, P(CSR), vp, vp, vp]),
        "tlda_cp_pass": (i32, [vp, P(CSR), vp, i32, vp, f32, u32, vp]),
        "tlda_autotune": (i32, [vp, P(CSR), vp, i32, vp, i32, P(i32)]),
        "tlda_fit_batched": (i32, [vp, P(CSR), vp, i32, i32, i32, vp, f32, u32, vp]),
        "tlda_doc_topics": (i32, [P(CSR), vp, vp, i32, i32, vp, vp, vp, vp]),
        "tlda_generate_docs": (i32, [u64, i32, i32, vp, u32, u32, vp, i32, i32, i64, i32, vp, vp, vp, i64,
                                     vp, P(i64), vp]),
        "tlda_online_begin": (i32, [vp, vp, i32]),
        "tlda_online_pass": (i32, [vp, P(CSR), vp, i32, vp, f32, i32, vp]),
        "tlda_online_accumulate": (i32, [vp, P(CSR)]),
        "tlda_selftest_barrier": (i32, [vp, P(i32), P(i32)]),
        "tlda_online_whiten": (i32, [vp, vp]),
        "tlda_online_get_sketch": (i32, [vp, vp, vp, vp]),
        "tlda_online_set_sketch": (i32, [vp, vp, vp, vp]),
        "tlda_unwhiten_topics": (i32, [vp, vp, vp, vp, u32]),
        "tlda_cp_step_noalloc": (i32, [P(CSR), vp, vp, i32, i32, f64, f32, vp, f32, vp, vp, vp]),
        "tlda_ffma_probe": (i32, [i32, vp, P(f64), vp]),
        "tlda_profile": (i32, [vp, u32]),
        "tlda_profile_read": (i32, [vp, i32, P(ctypes.c_char_p), P(i64), P(f64)]),
        "tlda_save_state": (i32, [vp, ctypes.c_char_p]),
        "tlda_load_state": (i32, [vp, ctypes.c_char_p]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


class TLDAError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


# ---------------------------------------------------------------------------- data
@dataclass
class DeviceCSR:
    """A batch/corpus CSR whose arrays live in torch int32 tensors (CUDA, or
    pinned host memory for host-input passes)."""
    indptr: torch.Tensor
    indices: torch.Tensor
    counts: torch.Tensor
    vocab: int

    @property
    def n_docs(self) -> int:
        return self.indptr.numel() - 1

    @staticmethod
    def from_arrays(indptr, indices, counts, vocab, device="cuda", pin=False) -> "DeviceCSR":
        def t(a):
            x = torch.as_tensor(np.ascontiguousarray(np.asarray(a, dtype=np.int32)))
            if device == "cpu":
                return x.pin_memory() if pin else x
            return x.to(device)
        return DeviceCSR(t(indptr), t(indices), t(counts), int(vocab))

    @staticmethod
    def from_corpus(c, device="cuda", pin=False) -> "DeviceCSR":
        if int(c.indptr[-1]) >= 2 ** 31:
            raise ValueError("corpus too large for int32 offsets")
        return DeviceCSR.from_arrays(c.indptr, c.indices, c.counts, c.V, device=device, pin=pin)

    def struct(self) -> CSR:
        # built once per set of arrays (a call's marshalling is on the
        # critical path of a short pass)
        key = (id(self.indptr), id(self.indices), id(self.counts), self.vocab)
        cached = self.__dict__.get("_csr")
        if cached is None or cached[0] != key:
            cached = (key, CSR(self.n_docs, self.vocab, self.indptr.data_ptr(),
                               self.indices.data_ptr() if self.indices.numel() else 0,
                               self.counts.data_ptr() if self.counts.numel() else 0))
            self.__dict__["_csr"] = cached
        return cached[1]


def _ptr(t):
    return None if t is None else t.data_ptr()


# ---------------------------------------------------------------------------- context
class TLDA:
    """A libtlda context: vocabulary size V, K topics, whitening dimension D."""

    def __init__(self, vocab: int, k: int, dim: int = 0, alpha0: float = 1.0, theta: float = 0.0,
                 precision: str = "fp32", same_token: bool = True, seed: int = 0,
                 max_batch: int = 8192, stream: torch.cuda.Stream | None = None):
        self.lib = load()
        p = Params()
        self.lib.tlda_default_params(ctypes.byref(p), int(k))
        p.dim, p.alpha0, p.theta = int(dim), float(alpha0), float(theta)
        p.precision = BF16 if precision == "bf16" else FP32
        p.same_token_correction = 1 if same_token else 0
        p.seed, p.max_batch = int(seed), int(max_batch)
        self.params = p
        self.V, self.K = int(vocab), int(k)
        self.D = int(dim) if dim else int(k)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        st = self.lib.tlda_create(ctypes.byref(h), int(vocab), ctypes.byref(p),
                                  ctypes.c_void_p(self.stream.cuda_stream))
        if st != OK:
            raise TLDAError(st, "tlda_create failed")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.tlda_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int):
        if st != OK:
            raise TLDAError(st, self.lib.tlda_last_error(self.h).decode())

    # ------------------------------------------------------------ moments
    def fit_moments(self, chunk: DeviceCSR | None, flags: int):
        s = chunk.struct() if chunk is not None else None
        self._check(self.lib.tlda_fit_moments(self.h, ctypes.byref(s) if s is not None else None,
                                              int(flags)))

    def fit(self, chunks) -> None:
        for c in chunks:
            self.fit_moments(c, ACCUMULATE)
        self.fit_moments(None, FINALIZE)

    def get_whitening(self):
        W = torch.empty((self.V, self.D), dtype=torch.float32, device="cuda")
        m1 = torch.empty(self.D, dtype=torch.float32, device="cuda")
        ev = np.zeros(self.D, dtype=np.float64)
        self._check(self.lib.tlda_get_whitening(self.h, W.data_ptr(), m1.data_ptr(),
                                                ev.ctypes.data))
        return W, m1, ev

    def eig_sweeps(self) -> int:
        """Jacobi sweeps of the last whitening's eigensolve (diagnostic)."""
        return int(self.lib.tlda_eig_sweeps(self.h))

    def get_counts(self):
        C = np.zeros(self.V, dtype=np.int64)
        T, S2, S3 = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        self._check(self.lib.tlda_get_counts(self.h, C.ctypes.data, ctypes.byref(T),
                                             ctypes.byref(S2), ctypes.byref(S3)))
        return C, T.value, S2.value, S3.value

    def set_whitening(self, W: torch.Tensor, m1: torch.Tensor):
        W = W.to(device="cuda", dtype=torch.float32).contiguous()
        m1 = m1.to(device="cuda", dtype=torch.float32).contiguous()
        assert W.shape == (self.V, self.D) and m1.shape == (self.D,)
        self._check(self.lib.tlda_set_whitening(self.h, W.data_ptr(), m1.data_ptr()))
        self.stream.synchronize()

    # ------------------------------------------------------------ hot path
    def whiten_batch(self, batch: DeviceCSR, out: torch.Tensor | None = None) -> torch.Tensor:
        X = out if out is not None else torch.empty((batch.n_docs, self.D), dtype=torch.float32,
                                                    device="cuda")
        s = batch.struct()
        self._check(self.lib.tlda_whiten_batch(self.h, ctypes.byref(s), _ptr(X)))
        return X

    def cp_step(self, batch: DeviceCSR, Phi: torch.Tensor, lr: float, grad: torch.Tensor | None = None,
                want_loss: bool = False):
        """One CP-SGD step in place on Phi (D x K float32 CUDA). Returns the
        loss at the incoming Phi if want_loss (then the call synchronises)."""
        assert Phi.dtype == torch.float32 and Phi.is_cuda and Phi.is_contiguous()
        s = batch.struct()
        loss = ctypes.c_double()
        self._check(self.lib.tlda_cp_step(self.h, ctypes.byref(s), Phi.data_ptr(), float(lr),
                                          _ptr(grad), ctypes.byref(loss) if want_loss else None))
        return loss.value if want_loss else None

    def cp_data_term(self, batch: DeviceCSR, Phi: torch.Tensor):
        G = torch.empty((self.D, self.K), dtype=torch.float32, device="cuda")
        S3 = ctypes.c_int64()
        s = batch.struct()
        self._check(self.lib.tlda_cp_data_term(self.h, ctypes.byref(s), Phi.data_ptr(),
                                               G.data_ptr(), ctypes.byref(S3)))
        return G, S3.value

    def cp_pass(self, corpus: DeviceCSR, batch_offsets, Phi: torch.Tensor, lr: float,
                host_input: bool = False, losses: bool = False, wait: bool = True,
                device_losses: torch.Tensor | None = None):
        """One online pass (tlda_cp_pass).  wait=False (device input only)
        returns once the pass is enqueued; its status comes from the next
        sync().  The step losses then go, if asked for, to device_losses (a
        CUDA float64 tensor of at least one entry per batch)."""
        off = np.ascontiguousarray(np.asarray(batch_offsets, dtype=np.int64))
        nb = len(off) - 1
        s = corpus.struct()
        if not wait:
            assert not host_input and not losses
            lp = None
            if device_losses is not None:
                assert device_losses.is_cuda and device_losses.dtype == torch.float64
                assert device_losses.is_contiguous() and device_losses.numel() >= nb
                lp = device_losses.data_ptr()
            self._check(self.lib.tlda_cp_pass(self.h, ctypes.byref(s), off.ctypes.data, nb,
                                              Phi.data_ptr(), float(lr), NO_WAIT, lp))
            return None
        assert device_losses is None
        out = np.zeros(max(nb, 1), dtype=np.float64) if losses else None
        self._check(self.lib.tlda_cp_pass(self.h, ctypes.byref(s), off.ctypes.data, nb,
                                          Phi.data_ptr(), float(lr),
                                          HOST_INPUT if host_input else 0,
                                          out.ctypes.data if losses else None))
        return out[:nb] if losses else None

    def fit_batched(self, corpus: DeviceCSR, batch_offsets, Phi_starts: torch.Tensor, lr: float,
                    epochs: int, reuse_whitening: bool = False):
        """The batched mode: moments and whitening from `corpus` (unless
        reuse_whitening), then `epochs` passes from each start of Phi_starts
        (n_starts x D x K float32, CUDA, updated in place); the start with the
        lowest mean last-epoch loss ends up in Phi_starts[0].  Returns each
        start's mean last-epoch loss."""
        assert Phi_starts.dtype == torch.float32 and Phi_starts.is_cuda and Phi_starts.is_contiguous()
        assert Phi_starts.dim() == 3 and tuple(Phi_starts.shape[1:]) == (self.D, self.K)
        off = np.ascontiguousarray(np.asarray(batch_offsets, dtype=np.int64))
        n = int(Phi_starts.shape[0])
        out = np.zeros(n, dtype=np.float64)
        s = corpus.struct()
        self._check(self.lib.tlda_fit_batched(self.h, ctypes.byref(s), off.ctypes.data, len(off) - 1,
                                              int(epochs), n, Phi_starts.data_ptr(), float(lr),
                                              REUSE_WHITENING if reuse_whitening else 0,
                                              out.ctypes.data))
        return out

    def autotune(self, corpus: DeviceCSR | None = None, batch_offsets=None,
                 Phi: torch.Tensor | None = None, fixed: int = 0) -> int:
        """Tile size of the persistent pass kernel: set it (fixed > 0) or time
        the candidates on the first batches of `corpus` (Phi unchanged).
        Returns the size in use."""
        out = ctypes.c_int32()
        if fixed:
            self._check(self.lib.tlda_autotune(self.h, None, None, 0, None, int(fixed),
                                               ctypes.byref(out)))
            return out.value
        off = np.ascontiguousarray(np.asarray(batch_offsets, dtype=np.int64))
        s = corpus.struct()
        self._check(self.lib.tlda_autotune(self.h, ctypes.byref(s), off.ctypes.data, len(off) - 1,
                                           Phi.data_ptr(), 0, ctypes.byref(out)))
        return out.value

    # ------------------------------------------------------------ fully online mode
    def online_begin(self, Omega: torch.Tensor):
        """Start the fully online mode with the sketch test matrix Omega
        (V x r float64, any device; copied)."""
        Om = Omega.to(device="cuda", dtype=torch.float64).contiguous()
        assert Om.dim() == 2 and Om.shape[0] == self.V
        self._check(self.lib.tlda_online_begin(self.h, Om.data_ptr(), int(Om.shape[1])))
        self._online_r = int(Om.shape[1])

    def online_pass(self, corpus: DeviceCSR, batch_offsets, Phi: torch.Tensor, lr: float,
                    rewhiten_every: int = 1, losses: bool = False):
        """One fully online pass (blocks of `rewhiten_every` batches: statistics
        and whitening first, then the block's CP steps); Phi updated in place."""
        assert Phi.dtype == torch.float32 and Phi.is_cuda and Phi.is_contiguous()
        off = np.ascontiguousarray(np.asarray(batch_offsets, dtype=np.int64))
        nb = len(off) - 1
        out = np.zeros(max(nb, 1), dtype=np.float64) if losses else None
        s = corpus.struct()
        self._check(self.lib.tlda_online_pass(self.h, ctypes.byref(s), off.ctypes.data, nb,
                                              Phi.data_ptr(), float(lr), int(rewhiten_every),
                                              out.ctypes.data if losses else None))
        return out[:nb] if losses else None

    def online_accumulate(self, corpus: DeviceCSR):
        """Add a corpus chunk to the online statistics and sketch only."""
        s = corpus.struct()
        self._check(self.lib.tlda_online_accumulate(self.h, ctypes.byref(s)))

    def online_whiten(self, Phi: torch.Tensor | None = None):
        """Rebuild the whitening from the statistics so far; carry Phi."""
        self._check(self.lib.tlda_online_whiten(self.h, Phi.data_ptr() if Phi is not None else None))

    def online_sketch(self):
        """The online statistics as device tensors: (Z, C, TS) with Z = P Omega
        (V x r float64), C the word counts (V int64), TS = (T, S2, S3)."""
        r = getattr(self, "_online_r", 0)
        Z = torch.empty((self.V, r), dtype=torch.float64, device="cuda")
        Cw = torch.empty(self.V, dtype=torch.int64, device="cuda")
        TS = torch.empty(3, dtype=torch.int64, device="cuda")
        self._check(self.lib.tlda_online_get_sketch(self.h, Z.data_ptr(), Cw.data_ptr(), TS.data_ptr()))
        return Z, Cw, TS

    def online_set_sketch(self, Z: torch.Tensor, Cw: torch.Tensor, TS: torch.Tensor):
        """Replace the online statistics with saved ones (as online_sketch returns)."""
        Z = Z.to(device="cuda", dtype=torch.float64).contiguous()
        Cw = Cw.to(device="cuda", dtype=torch.int64).contiguous()
        TS = TS.to(device="cuda", dtype=torch.int64).contiguous()
        assert Z.shape == (self.V, getattr(self, "_online_r", 0)) and Cw.shape == (self.V,) and TS.shape == (3,)
        self._check(self.lib.tlda_online_set_sketch(self.h, Z.data_ptr(), Cw.data_ptr(), TS.data_ptr()))

    def sync(self):
        self._check(self.lib.tlda_sync(self.h))

    # ------------------------------------------------------------ profiling
    KERNELS = ("scan_whiten", "qy", "rz", "zh", "g_reduce", "reduce_update", "phi_gram",
               "phi_terms", "fused", "pass")

    def profile(self, kernels=()):
        """Bracket the named kernels with CUDA events from now on (empty: off)."""
        mask = 0
        for k in kernels:
            mask |= 1 << self.KERNELS.index(k)
        self._check(self.lib.tlda_profile(self.h, mask))

    def profile_read(self):
        """{kernel: (launches, total_ms)} since the last profile() call."""
        out = {}
        for i, _ in enumerate(self.KERNELS):
            name, n, ms = ctypes.c_char_p(), ctypes.c_int64(), ctypes.c_double()
            self._check(self.lib.tlda_profile_read(self.h, i, ctypes.byref(name), ctypes.byref(n),
                                                   ctypes.byref(ms)))
            out[name.value.decode()] = (n.value, ms.value)
        return out

    # ------------------------------------------------------------ recovery / state
    def unwhiten_topics(self, Phi: torch.Tensor):
        mu = np.zeros((self.V, self.K), dtype=np.float64)
        al = np.zeros(self.K, dtype=np.float64)
        self._check(self.lib.tlda_unwhiten_topics(self.h, Phi.data_ptr(), mu.ctypes.data,
                                                  al.ctypes.data, HOST_OUTPUT))
        return mu, al

    def save_state(self, path: str):
        self._check(self.lib.tlda_save_state(self.h, str(path).encode()))

    def load_state(self, path: str):
        self._check(self.lib.tlda_load_state(self.h, str(path).encode()))


# ---------------------------------------------------------------------------- self-test
def selftest_barrier():
    """Run tlda_selftest_barrier: (status, blocks, blocks that gave up)."""
    lib = load()
    nb, ng = ctypes.c_int32(), ctypes.c_int32()
    st = lib.tlda_selftest_barrier(None, ctypes.byref(nb), ctypes.byref(ng))
    return st, nb.value, ng.value


def ffma_peak_tflops(iters: int = 4096, reps: int = 5) -> float:
    """Measured FP32 CUDA-core throughput (TFLOP/s): the best of `reps`
    launches of tlda_ffma_probe after one warm-up, each timed by CUDA events
    on the current stream."""
    lib = load()
    stream = torch.cuda.current_stream()
    sink = torch.empty(1 << 16, dtype=torch.float32, device="cuda")
    flops = ctypes.c_double()
    best = float("inf")
    for r in range(reps + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = lib.tlda_ffma_probe(int(iters), sink.data_ptr(), ctypes.byref(flops), ctypes.c_void_p(stream.cuda_stream))
        e1.record(stream)
        if st != OK:
            raise TLDAError(st, "tlda_ffma_probe")
        stream.synchronize()
        if r:
            best = min(best, e0.elapsed_time(e1))
    return flops.value / (best / 1e3) / 1e12


# ---------------------------------------------------------------------------- synthetic corpora
class DeviceGenerator:
    """Documents of a seeded synthetic corpus generated on the device
    (tlda_generate_docs): topic_cdf K x V and len_cdf as the host generator
    builds them (uploaded once), alpha0 = a_num / a_den."""

    def __init__(self, seed: int, V: int, K: int, topic_cdf, a_num: int, a_den: int, len_cdf, min_len: int):
        self.lib = load()
        self.seed, self.V, self.K = int(seed), int(V), int(K)
        self.cdf = torch.as_tensor(np.ascontiguousarray(topic_cdf, dtype=np.uint64).view(np.int64)).to("cuda")
        self.len_cdf = torch.as_tensor(np.ascontiguousarray(len_cdf, dtype=np.uint64).view(np.int64)).to("cuda")
        self.a_num, self.a_den, self.min_len = int(a_num), int(a_den), int(min_len)
        self._scratch = None  # kept: the write pass still uses it after a call returns
        self._last_stream = None

    def _call(self, doc0, n_docs, indptr, indices, counts, cap, scratch, stream=None):
        nnz = ctypes.c_int64()
        st = self.lib.tlda_generate_docs(self.seed, self.V, self.K, self.cdf.data_ptr(), self.a_num, self.a_den,
                                         self.len_cdf.data_ptr(), int(self.len_cdf.numel()), self.min_len,
                                         int(doc0), int(n_docs), indptr.data_ptr(),
                                         indices.data_ptr() if indices is not None else None,
                                         counts.data_ptr() if counts is not None else None, int(cap),
                                         scratch.data_ptr(), ctypes.byref(nnz),
                                         ctypes.c_void_p(stream.cuda_stream) if stream is not None else None)
        return st, nnz.value

    def generate(self, doc0: int, n_docs: int, out: "DeviceCSR | None" = None,
                 stream: "torch.cuda.Stream | None" = None) -> DeviceCSR:
        """Documents doc0 .. doc0+n_docs-1 as a device CSR; `out` (with enough
        capacity in indices/counts) is reused when given.  The work runs on
        `stream` (default: the legacy default stream); the call returns once
        the row counts are known and the write pass is enqueued."""
        need = (n_docs + 1023) // 1024 + 2
        if self._scratch is None or self._scratch.numel() < need or stream is not self._last_stream:
            torch.cuda.synchronize()  # the previous call's write pass may still use the scratch
            if self._scratch is None or self._scratch.numel() < need:
                self._scratch = torch.empty(need, dtype=torch.int64, device="cuda")
            self._last_stream = stream
        scratch = self._scratch
        if out is not None and out.indptr.numel() >= n_docs + 1:
            indptr, indices, counts = out.indptr[:n_docs + 1], out.indices, out.counts
            st, nnz = self._call(doc0, n_docs, indptr, indices, counts, indices.numel(), scratch, stream)
            if st == OK:
                return DeviceCSR(indptr, indices[:nnz], counts[:nnz], self.V)
            if st != ERR_OOM:
                raise TLDAError(st, "tlda_generate_docs failed")
        indptr = torch.empty(n_docs + 1, dtype=torch.int32, device="cuda")
        st, nnz = self._call(doc0, n_docs, indptr, None, None, 0, scratch, stream)
        if st != OK:
            raise TLDAError(st, "tlda_generate_docs failed")
        indices = torch.empty(max(nnz, 1), dtype=torch.int32, device="cuda")
        counts = torch.empty_like(indices)
        st, nnz = self._call(doc0, n_docs, indptr, indices, counts, indices.numel(), scratch, stream)
        if st != OK:
            raise TLDAError(st, "tlda_generate_docs failed")
        return DeviceCSR(indptr, indices[:nnz], counts[:nnz], self.V)


# ---------------------------------------------------------------------------- document topics
def doc_topics(docs: DeviceCSR, mu, alpha, n_iter: int = 20, want_gamma: bool = False, stream=None):
    """Document-topic proportions by variational inference with the topics
    fixed (tlda_doc_topics): mu V x K (column k = topic k), alpha the K
    Dirichlet parameters; any device or dtype (copied to CUDA float32).
    Returns theta (B x K CUDA float32), and gamma if want_gamma; raises on a
    corrupt document."""
    lib = load()
    mu_d = torch.as_tensor(mu).to(device="cuda", dtype=torch.float32).contiguous()
    al_d = torch.as_tensor(alpha).to(device="cuda", dtype=torch.float32).contiguous()
    K = int(mu_d.shape[1])
    assert mu_d.dim() == 2 and int(mu_d.shape[0]) == docs.vocab and tuple(al_d.shape) == (K,)
    theta = torch.empty((docs.n_docs, K), dtype=torch.float32, device="cuda")
    gamma = torch.empty_like(theta) if want_gamma else None
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    s = docs.struct()
    st = lib.tlda_doc_topics(ctypes.byref(s), mu_d.data_ptr(), al_d.data_ptr(), K, int(n_iter),
                             theta.data_ptr(), gamma.data_ptr() if want_gamma else None, err.data_ptr(),
                             ctypes.c_void_p(stream.cuda_stream) if stream is not None else None)
    if st != OK:
        raise TLDAError(st, "tlda_doc_topics: bad arguments")
    if int(err.item()):
        raise TLDAError(ERR_INVALID, "tlda_doc_topics: corrupt document (outputs NaN)")
    return (theta, gamma) if want_gamma else theta


# ---------------------------------------------------------------------------- autograd
class TLDALoss(torch.autograd.Function):
    """The CP objective of one minibatch as a differentiable function of Phi.

    forward(Phi, model, batch) returns, as a 0-dim float64 tensor on Phi's
    device, the loss of tlda_cp_step at Phi (section "Stochastic Tensor
    Gradient Descent": (1+theta)/2 sum_ij (phi_i.phi_j)^3 minus
    sum_i T_B(phi_i, phi_i, phi_i)); backward returns grad_output times the
    gradient of eq. vec_deriv that the same call wrote.  Both come from one
    tlda_cp_step with lr = 0, which leaves Phi unchanged; the call
    synchronises because the loss is read on the host.
    """

    @staticmethod
    def forward(ctx, Phi: torch.Tensor, model: "TLDA", batch: DeviceCSR):
        P = Phi.detach()
        if P.dtype != torch.float32 or not P.is_cuda or not P.is_contiguous():
            raise TypeError("TLDALoss: Phi must be a contiguous float32 CUDA tensor")
        if tuple(P.shape) != (model.D, model.K):
            raise ValueError(f"TLDALoss: Phi must be {model.D} x {model.K}")
        G = torch.empty_like(P)
        loss = model.cp_step(batch, P, 0.0, grad=G, want_loss=True)
        ctx.save_for_backward(G)
        return torch.tensor(loss, dtype=torch.float64, device=P.device)

    @staticmethod
    def backward(ctx, grad_output):
        (G,) = ctx.saved_tensors
        return grad_output.to(G.dtype) * G, None, None


def tlda_loss(Phi: torch.Tensor, model: "TLDA", batch: DeviceCSR) -> torch.Tensor:
    """TLDALoss.apply(Phi, model, batch)."""
    return TLDALoss.apply(Phi, model, batch)
