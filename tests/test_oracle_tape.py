"""Decision tape of the oracle (support for frozen-decision finite differences).

* Recording does not change the trajectory, and replaying the recorded tape at
  the same parameters reproduces it bit for bit.
* Replaying at other continuous parameters keeps every integer (Z, S) of the
  recorded trajectory while the positions move, and the bytes of the tape are
  the decision counts of the step (Sec. 3.1 items 2 and 3).
* The multiple-tau slot counts of the product's loss helper equal the oracle's.
"""
import numpy as np

import oracle
from oracle import Params


def _ens(p, M=24, seed=5):
    e = oracle.Ensemble(p, seed=seed, M=M, levels=6)
    e.init()
    return e


def test_record_is_transparent_and_replay_is_exact():
    p = Params(N=12)
    a, b = _ens(p), _ens(p)
    a.run(50)
    b.run(50)
    start = b.get_state()
    c0 = b.counters()
    tape = np.zeros((200, 24, 12), dtype=np.uint8)
    a.run(200)
    b.run_tape(200, tape, 1)
    sa, sb = a.get_state(), b.get_state()
    for k in ("R", "A", "Z", "S"):
        assert np.array_equal(sa[k], sb[k]), k
    c = _ens(p)
    c.set_state(start)
    c.step = 50
    c.run_tape(200, tape, 2)
    sc = c.get_state()
    for k in ("R", "A", "Z", "S"):
        assert np.array_equal(sa[k], sc[k]), k
    cnt = {k: v - c0[k] for k, v in b.counters().items()}
    bits = lambda m: int(np.count_nonzero(tape & m))
    assert bits(1) == cnt["hops_up"] and bits(2) == cnt["hops_down"]
    assert bits(4) + bits(8) == cnt["created"]
    assert bits(16) + bits(32) == cnt["destroyed"]
    assert not np.any(tape & 0xC0)


def test_replay_at_other_parameters_keeps_the_integers():
    p = Params(N=16)
    a = _ens(p, M=16, seed=8)
    a.run(30)
    start = a.get_state()
    tape = np.zeros((300, 16, 16), dtype=np.uint8)
    a.run_tape(300, tape, 1)
    ref = a.get_state()
    q = Params(N=16, k_b=3.3, k_s=5.0, zeta=1.2)
    b = _ens(q, M=16, seed=8)
    b.set_state(start)
    b.step = 30
    b.run_tape(300, tape, 2)
    got = b.get_state()
    assert np.array_equal(ref["Z"], got["Z"]) and np.array_equal(ref["S"], got["S"])
    assert not np.allclose(ref["R"], got["R"])
    # without the tape the other parameters change the decisions
    c = _ens(q, M=16, seed=8)
    c.set_state(start)
    c.step = 30
    c.run(300)
    free = c.get_state()
    assert not (np.array_equal(ref["Z"], free["Z"]) and np.array_equal(ref["S"], free["S"]))


def test_slot_counts_agree_with_oracle():
    from paper_1106_2899_gb300.adjoint import slot_counts, slot_lags
    for n in (0, 1, 7, 600, 10_000, 123_457):
        assert np.array_equal(slot_counts(n, 14), oracle.corr_counts(n, 14))
    assert np.array_equal(slot_lags(10), oracle.corr_lags(10))
