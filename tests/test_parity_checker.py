"""The per-column parity check of the BF16 tests (tests/_cases.col_rel) on
the CPU: it passes a matrix that carries BF16-sized rounding noise on every
entry, and fails a matrix whose one column, or one entry, is wrong although
the relative Frobenius error of the whole matrix stays below the tolerance."""
import numpy as np
import pytest

import tlda_synth as ts
from oracle import tlda_oracle as O
from tests import _cases as C

TOL16 = 2e-2


@pytest.fixture(scope="module")
def g_data():
    """An oracle data term at the metric shape (K = D = 100), 300 documents."""
    name = "stream_v20k_k100"
    sp = ts.WORKLOADS[name]
    W, m1 = C.population_whitening(name)
    c = C.corpus(name, 300)
    Phi = ts.initial_factors(sp.seed + 1, sp.K, sp.K)
    return O.cp_grad_implicit(c.indptr, c.indices, c.counts, sp.V, W, m1, Phi, float(sp.alpha0), 0.0)["G_data"]


def _noisy(G, seed=0):
    """G with an independent relative perturbation of one BF16 unit roundoff
    (2^-8) on every entry: the size of one rounding of a BF16 operand."""
    rng = np.random.default_rng(seed)
    return G * (1.0 + rng.uniform(-2.0 ** -8, 2.0 ** -8, size=G.shape))


def test_rounding_noise_passes(g_data):
    C.assert_bf16_parity(_noisy(g_data), g_data, TOL16, "noise")


@pytest.mark.parametrize("col", [0, 57, 99])
def test_one_wrong_column_fails(g_data, col):
    bad = _noisy(g_data)
    bad[:, col] *= 1.1
    assert C.rel(bad, g_data) < TOL16          # the Frobenius check alone misses it
    assert C.col_rel(bad, g_data) > TOL16
    with pytest.raises(AssertionError):
        C.assert_bf16_parity(bad, g_data, TOL16, "one column")


def test_one_wrong_entry_fails(g_data):
    """One entry off by 5% of its column's largest entry."""
    bad = _noisy(g_data)
    bad[13, 42] += 0.05 * np.abs(g_data[:, 42]).max()
    assert C.rel(bad, g_data) < TOL16
    with pytest.raises(AssertionError):
        C.assert_bf16_parity(bad, g_data, TOL16, "one entry")


def test_zeroed_last_column_fails(g_data):
    """A column left unwritten (the last real topic column before the padding
    of K = 100 to 128) reads as zero."""
    bad = _noisy(g_data)
    bad[:, -1] = 0.0
    with pytest.raises(AssertionError):
        C.assert_bf16_parity(bad, g_data, TOL16, "last column")


def test_pass_check_catches_a_wrong_column(g_data):
    """The pass form of the check (per column, relative to the summed step
    sizes): passes a change with BF16-sized noise, fails when one column of
    the change is off by a tenth of the column's summed step sizes."""
    rng = np.random.default_rng(3)
    steps = [-2e-3 * g_data * rng.uniform(0.5, 1.5) for _ in range(5)]
    change_ref = np.sum(steps, axis=0)
    noisy = change_ref * (1.0 + rng.uniform(-2.0 ** -8, 2.0 ** -8, size=change_ref.shape))
    C.assert_bf16_pass_parity(noisy, change_ref, steps, TOL16, "noisy pass")
    bad = noisy.copy()
    scale = np.sum([np.abs(s[:, 71]).max() for s in steps])
    bad[5, 71] += 0.1 * scale
    with pytest.raises(AssertionError):
        C.assert_bf16_pass_parity(bad, change_ref, steps, TOL16, "one column")
