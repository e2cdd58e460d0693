"""Checkpoint, kill and resume: a process runs the first batches of a
persistent BF16 pass, saves the context state (tlda_save_state) and Phi, and
exits without any cleanup, as a killed job would; a second process loads
both and runs the remaining batches.  Its Phi equals, bit for bit, that of
one uninterrupted pass over all batches (the kernels are deterministic for a
fixed tile size)."""
from __future__ import annotations

import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest
import torch

import tlda_synth as ts

from . import _cases as C

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent("""
    import os, sys
    import numpy as np, torch
    sys.path.insert(0, {root!r})
    import tlda_synth as ts
    from tests import _cases as C
    from paper_2511_07809_gb300 import tlda
    name, stage, d = "stream_v20k_k100", sys.argv[1], sys.argv[2]
    sp = ts.WORKLOADS[name]
    c = C.corpus(name, 20000)
    offs = [0, 1500, 5000, 9000, 12000, 16500, 20000]
    t = tlda.TLDA(sp.V, sp.K, alpha0=float(sp.alpha0), precision="bf16")
    t.autotune(fixed=18)
    dev = tlda.DeviceCSR.from_corpus(c)
    if stage == "first":
        W, m1 = C.population_whitening(name)
        t.set_whitening(torch.tensor(W, dtype=torch.float32), torch.tensor(m1, dtype=torch.float32))
        Phi = torch.tensor(ts.initial_factors(sp.seed + 1, sp.K, sp.K), dtype=torch.float32, device="cuda")
        t.cp_pass(dev, offs[:4], Phi, 0.002)
        t.save_state(os.path.join(d, "ctx.tlda"))
        np.save(os.path.join(d, "phi.npy"), Phi.cpu().numpy())
        os._exit(0)  # no cleanup: as if killed here
    t.load_state(os.path.join(d, "ctx.tlda"))
    Phi = torch.tensor(np.load(os.path.join(d, "phi.npy")), device="cuda")
    t.cp_pass(dev, offs[3:], Phi, 0.002)
    np.save(os.path.join(d, "phi_resumed.npy"), Phi.cpu().numpy())
""")


def test_resume_after_kill_gives_identical_phi(lib, tmp_path):
    script = tmp_path / "child.py"
    script.write_text(CHILD.format(root=ROOT))
    env = dict(os.environ, PYTHONPATH=ROOT)
    for stage in ("first", "second"):
        r = subprocess.run([sys.executable, str(script), stage, str(tmp_path)], cwd=ROOT, env=env,
                           capture_output=True, text=True, timeout=600)
        assert r.returncode == 0, r.stderr[-2000:]
    name = "stream_v20k_k100"
    sp = ts.WORKLOADS[name]
    W, m1 = C.population_whitening(name)
    t = lib.TLDA(sp.V, sp.K, alpha0=float(sp.alpha0), precision="bf16")
    t.set_whitening(torch.tensor(W, dtype=torch.float32), torch.tensor(m1, dtype=torch.float32))
    t.autotune(fixed=18)
    c = C.corpus(name, 20000)
    Phi = torch.tensor(ts.initial_factors(sp.seed + 1, sp.K, sp.K), dtype=torch.float32, device="cuda")
    t.cp_pass(lib.DeviceCSR.from_corpus(c), [0, 1500, 5000, 9000, 12000, 16500, 20000], Phi, 0.002)
    resumed = np.load(tmp_path / "phi_resumed.npy")
    assert np.array_equal(resumed, Phi.cpu().numpy())
    t.close()
