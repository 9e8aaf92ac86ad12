"""The oracle's operation-counting build (CPU only).

The counting build (-DOR_COUNT_OPS) only adds counters: its trajectories equal
the plain build's bit for bit.  The deterministic categories follow closed
forms per bead-step: bond forces 12 - 12/N (two neighbours of an inner bead,
one of an end bead, a difference and a multiply-add per component), the
Euler update 6 (15 with a velocity gradient), a Philox block 58 per bead (10
rounds of two products and a three-input xor per word pair, key additions
after round 0) plus one block per created spring, the decoding 41 per bead
(two Box-Muller pairs of 16 and the 24-bit uniform of 9).  The stored counts
that bench.py uses (tests/golden/alg_ops.txt) agree with a fresh sample.
"""
import os
import sys

import numpy as np
import pytest

import oracle
import synth

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
import make_alg_ops  # noqa: E402


def test_counting_build_changes_no_result():
    p = oracle.Params(N=24, **synth.PAPER)
    k = synth.element_table(1, seed=3, n_kappa=1)[2][0, 0]
    out = []
    for counting in (False, True):
        e = oracle.Ensemble(p, seed=9, M=40, levels=6, counting=counting)
        e.init()
        e.set_flow(0, k)
        e.run(300, nthreads=1)
        out.append((e.get_state(), e.corr_sums()[0], e.counters()))
    for key in ("R", "Z", "S", "A"):
        assert np.array_equal(out[0][0][key], out[1][0][key]), key
    assert np.array_equal(out[0][1], out[1][1]) and out[0][2] == out[1][2]


@pytest.mark.parametrize("N,flow", [(16, False), (32, False), (24, True)])
def test_closed_form_categories(N, flow):
    p = oracle.Params(N=N, **synth.PAPER)
    kap = synth.element_table(1, seed=3, n_kappa=1)[2][0, 0] if flow else None
    M, steps = 32, 400
    c = oracle.op_counts(p, seed=3, M=M, steps=steps, levels=4, warm=50, kappa=kap)
    assert abs(c["bond"] - (12.0 - 12.0 / N)) < 1e-12
    assert abs(c["euler"] - (15.0 if flow else 6.0)) < 1e-12
    e = oracle.Ensemble(p, seed=3, M=M, levels=4)  # the plain build: creations in the same window
    e.init()
    if flow:
        e.set_flow(0, kap)
    e.run(50)
    c0 = e.counters()["created"]
    e.run(steps)
    created = (e.counters()["created"] - c0) / float(M * N * steps)
    assert abs(c["philox"] - 58.0 * (1.0 + created)) < 1e-9
    assert abs(c["decode"] - 41.0 * (1.0 + created)) < 1e-9
    assert (c["advect"] > 0) == flow


def test_stored_counts_match_a_fresh_sample():
    stored = make_alg_ops.load()
    for name, N, kappa, levels, log_every in make_alg_ops.workloads():
        if name not in ("lve", "flow_48"):
            continue
        c = make_alg_ops.measure(name, N, kappa, levels, log_every, M=64, steps=1000, warm=500)
        for k, v in c.items():
            assert abs(v - stored[name][k]) <= 0.03 * max(stored[name][k], 0.5), (name, k, v, stored[name][k])
        assert abs(sum(c.values()) - stored[name]["total"]) < 0.01 * stored[name]["total"]
