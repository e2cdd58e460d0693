"""The printed setup of the paper's simulation study (tests/golden/
simulation_study.txt, transcribed from section "Parameter Recovery and
Comparison to Previous TLDA Methods") against the corpora the shape check
generates (tlda_synth.e1_spec): topics, alpha0 and corpus size as printed,
one corpus per vocabulary size and seed.  The paper prints no worked
numeric example of the method itself; its steps are pinned by closed forms
and brute force in the other oracle tests."""
from __future__ import annotations

import os
from fractions import Fraction

import tlda_synth as ts

HERE = os.path.dirname(os.path.abspath(__file__))


def _golden():
    setup, rows = {}, []
    with open(os.path.join(HERE, "golden", "simulation_study.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].split()
            if not line:
                continue
            if line[0] == "vocab":
                rows.append((int(line[1]), float(line[2]), float(line[3]), float(line[4])))
            else:
                setup[line[0]] = line[1]
    return setup, rows


def test_simulation_corpora_follow_the_printed_setup():
    setup, rows = _golden()
    assert [r[0] for r in rows] == [500, 1000, 1500]
    seeds = set()
    for V, corr, std, secs in rows:
        assert 0.0 < corr <= 1.0 and 0.0 < std < 1.0 and secs > 0.0
        for rep in range(int(setup["seeds"])):
            sp = ts.e1_spec(V, rep)
            assert sp.V == V and sp.K == int(setup["topics"])
            assert sp.alpha0 == Fraction(setup["alpha0"])
            assert sp.n_docs == int(setup["documents"])
            seeds.add(sp.seed)
    assert len(seeds) == 3 * int(setup["seeds"])  # one corpus per vocabulary size and seed
