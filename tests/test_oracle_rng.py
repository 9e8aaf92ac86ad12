"""Pins of the oracle's random-number layer (CPU only).

* Philox4x32-10 against the published known-answer vectors (tests/golden).
* Box-Muller normals: moments and a Kolmogorov-Smirnov test against the
  standard normal; the 24-bit slot uniform: KS against U[0,1); the four
  normals and the uniform of one block are mutually uncorrelated.
* The inverse normal CDF against scipy's ndtri (a library routine).
"""
import os

import numpy as np
import pytest
from scipy import special, stats

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLD):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        w = [int(x, 16) for x in line.split()]
        rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,out", _kat())
def test_philox_known_answers(ctr, key, out):
    assert list(oracle.philox(ctr, key)) == out


def _blocks(n, seed=12345):
    key = [seed & 0xFFFFFFFF, 0]
    W = np.array([oracle.philox([i, 7, 1, 3], key) for i in range(n)], dtype=np.uint32)
    return W


def test_decode_normals_and_uniform():
    W = _blocks(20000)
    dec = [oracle.decode_block(w) for w in W]
    n = np.array([d[0] for d in dec])
    u = np.array([d[1] for d in dec])
    for c in range(4):
        x = n[:, c]
        assert abs(x.mean()) < 4 / np.sqrt(len(x))
        assert abs(x.var() - 1) < 5 * np.sqrt(2 / len(x))
        assert stats.kstest(x, "norm").pvalue > 1e-3
    assert stats.kstest(u, "uniform").pvalue > 1e-3
    assert np.all((u >= 0) & (u < 1))
    # 24-bit lattice: u * 2^24 is an integer
    assert np.all(np.floor(u * 2**24) == u * 2**24)
    # no correlation between the five draws of one block
    X = np.column_stack([n, u])
    cc = np.corrcoef(X.T)
    off = cc[~np.eye(5, dtype=bool)]
    assert np.max(np.abs(off)) < 5 / np.sqrt(len(u))


def test_norm_ppf_matches_library():
    for p in [1e-12, 1e-6, 0.01, 0.1, 0.3, 0.5, 0.77, 0.999]:
        assert oracle.norm_ppf(p) == pytest.approx(special.ndtri(p), rel=1e-12, abs=1e-13)
    assert oracle.norm_ppf(1.0) == np.inf
